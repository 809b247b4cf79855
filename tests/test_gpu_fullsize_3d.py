"""Parity at the full size of the 3-D triclinic workload: 96^3 nodes at 10 m, 24 polar x 48 azimuth
angles (1.02e9 phase-space cells, 165 GB of device state), in the launch configuration of the timed
3-D benchmark.

* The characteristic velocities of every direction cell at 64 sampled nodes against the FP64
  oracle's (Eqs. 3-12, evaluated by the oracle at those nodes only).
* A homogeneous isotropic medium of the same size and angular sampling, solved for the workload's
  full 388 steps: at every node beyond 3 r0 reached by the source rays, one arrival with
  T = r / v and |u| = 1 / (4 pi r) (exact for straight rays), within the second-order error of the
  24 x 48 angular grid measured by the oracle's pins (4.3e-3 and 1.5 %).
"""
import math

import numpy as np
import pytest

import synthmedia
from oracle import christoffel as CH
from oracle import medium as MD

pytestmark = pytest.mark.gpu


def test_full_size_velocities_at_sampled_nodes_3d():
    import torch
    import paper_2006_11945_gb300 as egb
    p = synthmedia.triclinic_3d(n=96, h=10.0, n_theta=24, n_phi=48, freqs=(15.0,))
    rng = np.random.default_rng(3)
    nodes = rng.integers(0, 96, size=(64, 3))                  # (iz, iy, ix)
    a, dx, dy, dz, _ = MD.medium_3d(p)
    sel = (nodes[:, 0], nodes[:, 1], nodes[:, 2])
    sub = [f[sel].reshape(64, 1, 1, 3, 3, 3, 3) for f in (a, dx, dy, dz)]
    ref = CH.velocity_field_3d(*sub, 24, 48)                    # (48, 24, 64, 1, 1)
    with egb.Context(0) as ctx:
        m = ctx.medium_3d(p)
        s = ctx.source_3d(m, p)
        vel = torch.empty((9, 48, 24, 96, 96, 96), dtype=torch.float32, device='cuda')
        egb.egb_read_velocity(ctx.h, s, vel)
        idx = torch.as_tensor(nodes, device='cuda')
        got = vel[:, :, :, idx[:, 0], idx[:, 1], idx[:, 2]].cpu().numpy()   # (9, 48, 24, 64)
        info = egb.egb_get_solve_info(ctx.h, s)
        del vel
    torch.cuda.empty_cache()
    rate = info['max_rate']
    dth, dph = math.pi / 24, 2 * math.pi / 48
    for i, key, h in ((0, 'Vx', 10.0), (1, 'Vy', 10.0), (2, 'Vz', 10.0), (3, 'thetadot', dth), (4, 'phidot', dph)):
        err = np.max(np.abs(got[i] - ref[key][..., 0, 0])) / h / rate
        assert err < 2e-6, (key, err)
    assert np.max(np.abs(got[5] - ref['v'][..., 0, 0]) / ref['v'][..., 0, 0]) < 1e-6


def test_full_size_isotropic_arrivals_3d():
    import paper_2006_11945_gb300 as egb
    p = synthmedia.isotropic_homogeneous_3d(n=96, h=10.0, n_theta=24, n_phi=48, freqs=(15.0,))
    with egb.Context(0) as ctx:
        res, info = ctx.solve_problem_3d(p)
    v = p.meta['vp']
    o = np.arange(96) * 10.0 - p.xs[0]
    Z, Y, X = np.meshgrid(o, o, o, indexing='ij')
    r = np.sqrt(X ** 2 + Y ** 2 + Z ** 2)
    reached = (r > 3 * 20.0) & (r < v * p.steps * info['dt'] - 40.0)
    assert reached.sum() > 100000
    assert np.all(res.count[reached] == 1)
    eT = np.max(np.abs(res.T[..., 0][reached] - r[reached] / v) / (r[reached] / v))
    eA = np.max(np.abs(res.A[..., 0][reached] * 4 * math.pi * r[reached] - 1.0))
    print('full size 3-D isotropic: nodes', int(reached.sum()), 'T rel max', eT, 'A rel max', eA)
    assert eT < 5e-3 and eA < 2e-2
