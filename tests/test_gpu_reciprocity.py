"""Source-side against receiver-side (reciprocal) evaluation of the pseudo-time path, through the C ABI.

The qP Green's tensor is reciprocal, G_ij(r, s) = G_ji(s, r); the library's scalar output is
u = rho_s c_ref(s)^2 times its amplitude (c_ref the source medium's qP phase velocity along +z), so
u(r | s) / (rho_s c_s^2) = u(s | r) / (rho_r c_r^2), and the traveltimes agree.  The receiver-side
evaluation puts a source at every receiver (one batched evolution on the shared medium, which also
shares its characteristic velocities) and reads the arrivals at the true source; the source-side
evaluation is the usual solve.  The two use different sources, frozen manifolds, label fields and
beam families, so their agreement checks the arrival amplitudes (Eq. 26) and traveltimes
independently of the oracle.  Heterogeneous TTI medium, 128 x 128 at 20 m, 128 angles.
"""
import dataclasses

import numpy as np
import pytest

import synthmedia

pytestmark = pytest.mark.gpu


def test_receiver_side_arrivals_are_reciprocal():
    import paper_2006_11945_gb300 as egb
    p = synthmedia.tti_heterogeneous(n=128, n_theta=128, length=2560.0, freqs=(20.0,))
    h = p.hx
    src = (64, 64)                                        # (iz, ix)
    rng = np.random.default_rng(11)
    recv = []
    while len(recv) < 12:                                 # receivers 400-1000 m from the source
        iz, ix = rng.integers(12, 116, size=2)
        d = h * np.hypot(iz - src[0], ix - src[1])
        if 400.0 < d < 1000.0:
            recv.append((int(iz), int(ix)))
    rho = np.asarray(p.rho).reshape(p.nz, p.nx)
    kmax = 8
    with egb.Context(0) as ctx:
        m = ctx.medium_2d(p)
        fwd = dataclasses.replace(p, xs=(src[1] * h, src[0] * h))
        s0 = ctx.source_2d(m, fwd)
        ids = [ctx.source_2d(m, dataclasses.replace(p, xs=(ix * h, iz * h))) for iz, ix in recv]
        egb.egb_evolve_batch(ctx.h, [s0] + ids, [p.steps] * (1 + len(ids)), p.cfl)
        direct = ctx.superpose(s0, 1, p.nz, p.nx, kmax)
        c0 = egb.egb_get_solve_info(ctx.h, s0)['c_ref']
        back = []
        for s in ids:
            r = ctx.superpose(s, 1, p.nz, p.nx, kmax)
            back.append((r, egb.egb_get_solve_info(ctx.h, s)['c_ref']))
        egb.egb_sync(ctx.h)
    n0 = rho[src] * c0 ** 2
    eT, eA = [], []
    for (iz, ix), (r, cr) in zip(recv, back):
        assert direct.count[iz, ix] >= 1 and r.count[src] == direct.count[iz, ix]
        nr = rho[iz, ix] * cr ** 2
        Td, Tr = direct.T[iz, ix, 0], r.T[src][0]
        Ad, Ar = direct.A[iz, ix, 0] / n0, r.A[src][0] / nr
        eT.append(abs(Td - Tr) / Td)
        eA.append(abs(Ad - Ar) / Ad)
    eT, eA = np.array(eT), np.array(eA)
    print('reciprocity over', len(recv), 'pairs: T rel max', eT.max(), 'median', np.median(eT),
          '; normalised A rel max', eA.max(), 'median', np.median(eA))
    assert eT.max() < 2e-3 and np.median(eT) < 5e-4
    assert eA.max() < 1.5e-2 and np.median(eA) < 3e-3
