"""Parity of the 3-D CUDA path (through the C ABI) with the FP64 3-D oracle.

Cases: a homogeneous VTI cube and a heterogeneous triclinic medium (the 96^3 recipe at 16 nodes a
side and 30 m), plus a ragged triclinic sub-block
(13 x 11 x 15 nodes, odd nx so the last x pair has one cell).  Tolerances are the single-solve
bar: traveltime relative <= 1e-5, amplitude relative <= 1e-3, wavefield relative L2 <= 2e-3,
arrival counts bit-exact outside the ambiguous nodes (oracle decisions within rounding of a
triangle edge, of the q = 1/2 threshold or of the projected-zero bound); labels within 2e-3 h (b),
2e-4 (n0), 2e-2 (q), 1e-6 relative (tau); velocities within 2e-6 of the CFL rate.
"""
import dataclasses

import numpy as np
import pytest

import synthmedia
from oracle import liouville3d as L3
from oracle import superpose3d as S3

pytestmark = pytest.mark.gpu


def _ragged():
    p = synthmedia.triclinic_3d(n=16, n_theta=6, n_phi=12, length=480.0, freqs=(15.0, 25.0))
    c21 = np.asarray(p.c21).reshape(16, 16, 16, 21)[:15, :11, :13].reshape(-1, 21).copy()
    rho = np.asarray(p.rho).reshape(16, 16, 16)[:15, :11, :13].reshape(-1).copy()
    xs = (6 * p.hx, 5 * p.hy, 7 * p.hz)
    return synthmedia.Problem3D('triclinic_ragged', 13, 11, 15, p.hx, p.hy, p.hz, c21, rho, xs, 6, 12,
                                [15.0, 25.0], 50.0, 40)


def _vti_offset():
    """Homogeneous VTI with the source off the node lattice.  With the source on a node the grid's
    mirror symmetries put zeros of b exactly on triangle edges along symmetry planes, where rounding
    the labels to FP32 alone moves beam centres across flag boundaries (the oracle's own wavefield
    changes by 2 % when its labels are rounded to FP32); off the lattice no such ties exist."""
    p = synthmedia.vti_homogeneous_3d(n=16, n_theta=8, n_phi=16, freqs=[30.0])
    h = p.hx
    return dataclasses.replace(p, xs=(p.xs[0] + 0.37 * h, p.xs[1] + 0.21 * h, p.xs[2] + 0.13 * h))


def _cases():
    return {
        'vti_16': _vti_offset(),
        'triclinic_16': synthmedia.triclinic_3d(n=16, n_theta=8, n_phi=16, length=480.0, freqs=(15.0,)),
        'ragged': _ragged(),
    }


@pytest.fixture(scope='module', params=list(_cases().keys()))
def case(request):
    p = _cases()[request.param]
    S, st, dt = L3.evolve3d(p)
    lab = L3.interior_state3d(st)
    u = S3.green3d(S, lab, p.omegas, p.beam_width)
    cnt, T, A, over = S3.arrivals3d(S, lab)
    amb = S3.ambiguous_nodes3d(S, lab)
    import paper_2006_11945_gb300 as egb
    with egb.Context(0) as ctx:
        m = ctx.medium_3d(p)
        s = ctx.source_3d(m, p)
        vel = ctx.read_velocity_3d(s, p.n_phi, p.n_theta, p.nz, p.ny, p.nx)
        ctx.evolve(s, p.steps, p.cfl)
        res = ctx.superpose_3d(s, len(p.freqs), p.nz, p.ny, p.nx, 8)
        egb.egb_sync(ctx.h)
        state = ctx.read_state_3d(s, p.n_phi, p.n_theta, p.nz, p.ny, p.nx)
        info = egb.egb_get_solve_info(ctx.h, s)
    return request.param, p, S, lab, dt, dict(u=u, count=cnt, T=T, A=A, amb=amb), vel, state, res, info


def test_velocity_parity_3d(case):
    name, p, S, lab, dt, ref, vel, state, res, info = case
    rate = S.max_rate
    for i, key, h in ((0, 'Vx', S.hx), (1, 'Vy', S.hy), (2, 'Vz', S.hz), (3, 'thetadot', S.dth), (4, 'phidot', S.dph)):
        err = np.max(np.abs(vel[i] - S.vel[key])) / h / rate
        assert err < 2e-6, (name, key, err)
    assert np.max(np.abs(vel[5] - S.vel['v']) / S.vel['v']) < 1e-6
    assert abs(info['dt'] - dt) / dt < 1e-6 and info['dim'] == 3 and info['n_phi'] == p.n_phi


def test_state_parity_3d(case):
    name, p, S, lab, dt, ref, vel, state, res, info = case
    h = max(p.hx, p.hy, p.hz)
    eb = max(np.max(np.abs(state[i] - lab[f])) for i, f in enumerate(('bx', 'by', 'bz'))) / h
    en = max(np.max(np.abs(state[3 + i] - lab[f])) for i, f in enumerate(('n0x', 'n0y', 'n0z')))
    eq = np.max(np.abs(state[6] - lab['q']))
    et = np.max(np.abs(state[7] - lab['tau'])) / np.max(np.abs(lab['tau']))
    print(name, 'b err/h', eb, 'n0', en, 'q', eq, 'tau rel', et)
    assert eb < 2e-3 and en < 2e-4 and eq < 2e-2 and et < 1e-6, (name, eb, en, eq, et)


def test_output_parity_3d(case):
    name, p, S, lab, dt, ref, vel, state, res, info = case
    u = res.u.astype(np.complex128)
    eu = np.linalg.norm(u - ref['u']) / np.linalg.norm(ref['u'])
    ok = ~ref['amb']
    mism = int(np.sum((res.count != ref['count']) & ok))
    same = (res.count == ref['count']) & ok
    kk = np.arange(8)[None, None, None, :] < ref['count'][..., None]
    sel = same[..., None] & kk
    eT = np.max(np.abs(res.T[sel] - ref['T'][sel]) / ref['T'][sel])
    eA = np.max(np.abs(res.A[sel] - ref['A'][sel]) / ref['A'][sel])
    print(name, 'u rel L2', eu, 'count mismatch', mism, 'ambiguous', int(ref['amb'].sum()), 'arrivals',
          int(sel.sum()), 'T', eT, 'A', eA)
    assert eu < 2e-3 and mism == 0 and eT < 1e-5 and eA < 1e-3, (name, eu, mism, eT, eA)
