"""Parity at the full size of the heterogeneous TTI workload: 512 x 512 nodes at 5 m (the 2560 m
square), 256 angles, 2801 TVD-RK3 steps, 10/20/40 Hz, run in the launch configuration of the timed
benchmark (persistent stencil over all SMs, autotuned theta chunk, 3-step rotations replayed from a
CUDA graph), 67 M phase-space cells, 1.3 GB per state buffer.

* Every cell's characteristic velocities against the FP64 oracle (Eqs. 3-12).
* Every cell's level sets after one 3-step rotation against the FP64 oracle's same 3 steps
  (Eqs. 16, 19, 20; the oracle's compiled loop runs at this size in seconds, its velocity planes
  come from a spawned process pool).
* The complete solve's arrivals (Eq. 35) against the Lagrangian ray shooter at a sample of
  receivers (every 8th node each way, beyond 4 r0 of the source): counts, first traveltimes and
  single-arrival amplitudes.  The shooter integrates the ray equations of the same Hamiltonian and
  computes each receiver's arrivals on its own, so it is an exact-solution check that holds at any
  size; its tolerances are those of the 40 m pin (discretisation error shrinks on this 5 m grid).
"""
import numpy as np
import pytest

import synthmedia
from tests.gpu_common import wrap

pytestmark = pytest.mark.gpu


def _problem():
    return synthmedia.tti_heterogeneous(n=512, h=5.0, n_theta=256, freqs=(10.0, 20.0, 40.0))


@pytest.fixture(scope='module')
def three_steps():
    from oracle import liouville as OL
    import paper_2006_11945_gb300 as egb
    p = _problem()
    vel_ref = OL.velocity_field_pooled(p, processes=16)
    S = OL.Setup(p, vel=vel_ref)
    _, st, dt = OL.evolve(p, steps=3, S=S)
    lab = OL.interior_state(st, S)
    del st
    with egb.Context(0) as ctx:
        m = ctx.medium_2d(p)
        s = ctx.source_2d(m, p)
        vel = ctx.read_velocity(s, p.n_theta, p.nz, p.nx)
        ctx.evolve(s, 3, p.cfl)
        state = ctx.read_state(s, p.n_theta, p.nz, p.nx)
        egb.egb_sync(ctx.h)
        info = egb.egb_get_solve_info(ctx.h, s)
    return p, S, lab, dt, vel, state, info


def test_full_size_velocities(three_steps):
    p, S, lab, dt, vel, state, info = three_steps
    rate = S.max_rate
    for i, key, h in ((0, 'Vx', S.hx), (1, 'Vz', S.hz), (2, 'thetadot', S.dth)):
        err = np.max(np.abs(vel[i] - S.vel[key])) / h / rate
        assert err < 1e-6, (key, err)
    assert np.max(np.abs(vel[3] - S.vel['v']) / S.vel['v']) < 1e-6
    assert abs(info['dt'] - dt) / dt < 1e-6


def test_full_size_three_steps(three_steps):
    p, S, lab, dt, vel, state, info = three_steps
    h = max(p.hx, p.hz)
    eb = np.max(np.abs(state[0] - lab['b'])) / h
    eq = np.max(np.abs(state[1] - lab['q']))
    et = np.max(np.abs(wrap(state[2] - lab['Th'])))
    etau = np.max(np.abs(state[3] - lab['tau'])) / np.max(np.abs(lab['tau']))
    print('full size, 3 steps: b err/h', eb, 'q', eq, 'angle', et, 'tau rel', etau,
          'theta chunk', info.get('tile_chunk'))
    assert eb < 2e-3 and eq < 2e-2 and et < 2e-4 and etau < 1e-6


def test_full_size_solve_against_ray_shooter():
    from oracle import shooter as SH
    import paper_2006_11945_gb300 as egb
    p = _problem()
    mask = np.zeros((p.nz, p.nx), bool)
    mask[4::8, 4::8] = True
    x = np.arange(p.nx) * p.hx - p.xs[0]
    z = np.arange(p.nz) * p.hz - p.xs[1]
    Z, X = np.meshgrid(z, x, indexing='ij')
    mask &= np.hypot(X, Z) > 4 * 2 * max(p.hx, p.hz)
    fan = SH.shoot(p, n_rays=2048, dt=5e-4)
    assert np.all(np.isfinite(fan['exit_time']))
    cnt, first, arr = SH.arrivals(p, fan, node_mask=mask)
    with egb.Context(0) as ctx:
        res, info = ctx.solve_problem(p)
    assert p.steps * info['dt'] > np.max(fan['exit_time'])
    agree = np.mean(res.count[mask] == cnt[mask])
    both = mask & (res.count >= 1) & (cnt >= 1)
    relT = np.abs(res.T[..., 0][both] - first[both]) / first[both]
    single = mask & (res.count == 1) & (cnt == 1)
    As = np.array([arr[(i, j)][0][1] for i, j in zip(*np.nonzero(single))])
    relA = np.abs(res.A[..., 0][single] - As) / As
    print('full size vs shooter: receivers', int(mask.sum()), 'count agreement', agree,
          'first T rel median', np.median(relT), 'p95', np.quantile(relT, 0.95),
          'single A rel median', np.median(relA), 'p90', np.quantile(relA, 0.9))
    assert agree > 0.99
    assert np.median(relT) < 5e-3 and np.quantile(relT, 0.95) < 3e-2
    assert np.median(relA) < 2e-2 and np.quantile(relA, 0.9) < 1.5e-1
