"""Parity of the CUDA depth march (egb_zmarch: Eqs. 13-20 with the same-row superposition of
Eqs. 25-28, 33-35) with the FP64 oracle, through the C ABI.

Bar (as for the pseudo-time path): wavefield relative L2 <= 2e-3, arrival counts exact outside the
nodes whose count hinges on a sign of X - x_s below 2e-4 h, traveltimes <= 1e-5 and amplitudes
<= 1e-3 relative where the counts agree.  Cases: homogeneous VTI, heterogeneous TTI, a focusing lens
(triplicated arrivals) and a wide lens at 100 and 200 Hz (a triplication zone past a caustic), a
ragged grid with the source off the centre column, sources on the top
row (no upgoing branch), on the bottom row (no march downward) and one row below the top; invalid
arguments; a medium where a branch's rays turn horizontal; the dynamic ray tracing advected with
the march (Eq. 21, drt = 1) against its own oracle.  Full size (the timed workload's
512 x 512 grid, 256 angles per branch, 5 m): homogeneous VTI against the closed-form traveltimes
and geometrical amplitudes of straight group rays at every node of the central cone.
"""
import dataclasses
import math

import numpy as np
import pytest

import synthmedia
from oracle import closed_forms as CF
from oracle import zmarch as ZM
from tests.test_oracle_zmarch import lens_problem, wide_lens_problem

pytestmark = pytest.mark.gpu

THETA_MAX = math.radians(60.0)


def _gpu(p, nth, theta_max=THETA_MAX, kmax=8):
    import paper_2006_11945_gb300 as egb
    with egb.Context(0) as ctx:
        m = ctx.medium_2d(p)
        return ctx.zmarch(m, p, nth, theta_max, 0.5, kmax)


def _compare(res, ref, p, parts):
    out = {}
    u, ur = res.u.astype(np.complex128), ref['u']
    out['u_rel_l2'] = float(np.linalg.norm(u - ur) / np.linalg.norm(ur))
    amb = ZM.ambiguous_nodes(p, parts, 2e-4 * max(p.hx, p.hz))
    ok = ~amb
    out['count_mismatch'] = int(np.sum((res.count != ref['count']) & ok))
    same = (res.count == ref['count']) & ok
    kk = np.arange(res.T.shape[-1])[None, None, :] < ref['count'][..., None]
    sel = same[..., None] & kk
    Tr, Ar = ref['T'][sel], ref['A'][sel]
    out['T_rel_max'] = float(np.max(np.abs(res.T[sel] - Tr) / Tr)) if sel.any() else 0.0
    out['A_rel_max'] = float(np.max(np.abs(res.A[sel] - Ar) / Ar)) if sel.any() else 0.0
    out['arrivals'] = int(sel.sum())
    out['ambiguous'] = int(amb.sum())
    return out


def _ragged():
    """The first 41 rows and 53 columns of the 64 x 64 TTI medium, source at (25 h + 3.7 m, 17 h)."""
    full = synthmedia.tti_heterogeneous(n=64, n_theta=64, length=2560.0, steps=1, freqs=(10.0,))
    c21 = np.asarray(full.c21).reshape(64, 64, 21)[:41, :53].reshape(-1, 21).copy()
    rho = np.asarray(full.rho).reshape(64, 64)[:41, :53].reshape(-1).copy()
    return dataclasses.replace(full, nx=53, nz=41, c21=c21, rho=rho,
                               xs=(25 * full.hx + 3.7, 17 * full.hz))


def _case(name):
    if name == 'vti48':
        return synthmedia.vti_homogeneous(n=48, n_theta=32, steps=1, freqs=(15.0, 30.0)), 32
    if name == 'tti64':
        return synthmedia.tti_heterogeneous(n=64, n_theta=64, length=2560.0, steps=1, freqs=(10.0, 20.0)), 64
    if name == 'lens64':
        return lens_problem(), 96
    return _ragged(), 48


@pytest.mark.parametrize('name', ['vti48', 'tti64', 'lens64', 'ragged'])
def test_zmarch_matches_the_oracle(name):
    p, nth = _case(name)
    res = _gpu(p, nth)
    ref = ZM.solve(p, nth, THETA_MAX, 0.5)
    m = _compare(res, ref, p, ref['parts'])
    print(name, m)
    assert m['u_rel_l2'] < 2e-3, m
    assert m['count_mismatch'] == 0 and m['arrivals'] > 100, m
    assert m['T_rel_max'] < 1e-5 and m['A_rel_max'] < 1e-3, m
    if name == 'lens64':
        assert res.count.max() == 3


def test_zmarch_matches_the_oracle_behind_a_wide_lens_at_high_frequency():
    """The wide lens at 100 and 200 Hz (beam width 40 m, 128 angles): the triplication zone whose
    late arrival has passed a caustic, where the oracle's wavefield is pinned against the
    KMAH-shifted geometrical field; phases omega tau reach about 500 rad."""
    p = dataclasses.replace(wide_lens_problem(), freqs=[100.0, 200.0])
    res = _gpu(p, 128)
    ref = ZM.solve(p, 128, THETA_MAX, 0.5)
    m = _compare(res, ref, p, ref['parts'])
    print('wide lens', m)
    assert m['u_rel_l2'] < 2e-3, m
    assert m['count_mismatch'] == 0 and m['arrivals'] > 1000, m
    assert m['T_rel_max'] < 1e-5 and m['A_rel_max'] < 1e-3, m
    assert np.sum(res.count == 3) > 300
    for w in range(2):
        tri = ref['count'] == 3
        d = np.linalg.norm(res.u[w][tri] - ref['u'][w][tri]) / np.linalg.norm(ref['u'][w][tri])
        assert d < 2e-3, (w, d)


@pytest.mark.parametrize('row', [0, 1, 47])
def test_zmarch_sources_on_the_edge_rows(row):
    p = synthmedia.vti_homogeneous(n=48, n_theta=32, steps=1, freqs=(20.0,))
    p = dataclasses.replace(p, xs=(200.0 + 3.3, row * p.hz))
    res = _gpu(p, 32)
    ref = ZM.solve(p, 32, THETA_MAX, 0.5)
    m = _compare(res, ref, p, ref['parts'])
    print(row, m)
    assert m['u_rel_l2'] < 2e-3 and m['count_mismatch'] == 0, m
    assert m['T_rel_max'] < 1e-5 and m['A_rel_max'] < 1e-3, m


def test_zmarch_rejects_invalid_arguments_and_turning_rays():
    import paper_2006_11945_gb300 as egb
    p = synthmedia.tti_heterogeneous(n=32, n_theta=16, length=1280.0, steps=1, freqs=(10.0,))
    q = synthmedia.vti_homogeneous_3d(n=8, n_theta=4, n_phi=8)

    def status(fn):
        try:
            fn()
        except egb.EgbError as e:
            return e.status
        return egb.EGB_OK

    with egb.Context(0) as ctx:
        m = ctx.medium_2d(p)
        u = np.zeros((1, p.nz, p.nx), np.complex64)
        call = lambda xs=p.xs, nth=16, tm=1.0, cfl=0.5, mm=m: egb.egb_zmarch(
            ctx.h, mm, xs, p.omegas, 50.0, nth, tm, cfl, u_out=u)
        assert status(call) == egb.EGB_OK
        assert status(lambda: call(xs=(p.xs[0], p.xs[1] + 0.3 * p.hz))) == egb.EGB_E_INVALID
        assert status(lambda: call(xs=(-5.0, p.xs[1]))) == egb.EGB_E_INVALID
        assert status(lambda: call(nth=3)) == egb.EGB_E_INVALID
        assert status(lambda: call(tm=math.pi / 2)) == egb.EGB_E_INVALID
        assert status(lambda: call(cfl=1.5)) == egb.EGB_E_INVALID
        m3 = ctx.medium_3d(q)
        assert status(lambda: call(mm=m3)) == egb.EGB_E_INVALID
        # phase angles up to 1.55 rad: some group directions in the tilted medium cross the horizontal
        assert status(lambda: call(tm=1.55)) == egb.EGB_E_INVALID
        assert status(call) == egb.EGB_OK        # the context stays usable


@pytest.mark.parametrize('drt', [0, 1])
def test_zmarch_full_size_homogeneous_vti_against_straight_rays(drt):
    """The timed workload's grid and angle sampling (512 x 512 at 5 m, 256 angles per branch,
    theta_max 60 deg, source at the centre) in a homogeneous VTI medium: one arrival per node of
    the cone |group angle| < 45 deg beyond 20 m, with T = r / |V_g| and A = |u_GO| sqrt(omega) of
    the closed-form far field, for both dynamic ray tracing routes."""
    import paper_2006_11945_gb300 as egb
    p = synthmedia.vti_homogeneous(n=512, h=5.0, n_theta=256, steps=1, freqs=(20.0,))
    with egb.Context(0) as ctx:
        res = ctx.zmarch(ctx.medium_2d(p), p, 256, THETA_MAX, 0.5, 8, drt=drt)
    m_ = p.meta
    x = np.arange(p.nx) * p.hx - p.xs[0]
    z = np.arange(p.nz) * p.hz - p.xs[1]
    Zg, Xg = np.meshgrid(z, x, indexing='ij')
    r = np.hypot(Xg, Zg)
    ang = np.degrees(np.arctan2(np.abs(Xg), np.abs(Zg)))
    sel = (ang < 45) & (r > 20.0)
    rng = np.random.default_rng(5)
    idx = np.flatnonzero(sel)
    pick = rng.choice(idx, size=4000, replace=False)
    iz, ix = np.unravel_index(pick, sel.shape)
    assert np.all(res.count[sel] == 1)
    om = 2 * math.pi * 20.0
    v_of = lambda th: CF.thomsen_vti_phase_velocity(th, m_['vp0'], m_['vs0'], m_['eps'], m_['delta'])
    V_of = lambda th: CF.vti_group_velocity(th, m_['vp0'], m_['vs0'], m_['eps'], m_['delta'])[1:]
    ref, T, _ = CF.homogeneous_go_green(Xg[iz, ix], Zg[iz, ix], 0.0, 0.0, om, v_of, V_of, m_['vp0'])
    eT = np.abs(res.T[iz, ix, 0] - T) / T
    Aref = np.abs(ref) * math.sqrt(om)
    eA = np.abs(res.A[iz, ix, 0] - Aref) / Aref
    print('full-size z-march VTI: T rel max', eT.max(), 'A rel max', eA.max())
    assert eT.max() < 2e-4 and eA.max() < 2e-3
    assert np.all(np.isfinite(res.u))


def test_full_size_tti_depth_march_agrees_with_the_pseudo_time_solve():
    """The timed 512 x 512 TTI medium (256 angles): the pseudo-time solve (full angle range, 2801
    steps) and the depth march (256 angles per branch within 60 deg) trace the same rays with
    different numerics.  Below the source, within 30 deg of vertical and beyond 100 m, both must
    see one arrival per node with the same traveltime and geometrical amplitude up to their
    discretisation errors."""
    import paper_2006_11945_gb300 as egb
    p = synthmedia.tti_heterogeneous(n=512, h=5.0, n_theta=256, freqs=(10.0,))
    with egb.Context(0) as ctx:
        pt, _ = ctx.solve_problem(p)
        m = ctx.medium_2d(p)
        zm = ctx.zmarch(m, p, 256, THETA_MAX)
        zq = ctx.zmarch(m, p, 256, THETA_MAX, drt=1)
    x = np.arange(p.nx) * p.hx - p.xs[0]
    z = np.arange(p.nz) * p.hz - p.xs[1]
    Zg, Xg = np.meshgrid(z, x, indexing='ij')
    r = np.hypot(Xg, Zg)
    ang = np.degrees(np.arctan2(np.abs(Xg), np.abs(Zg)))
    sel = (ang < 30) & (r > 100.0) & (pt.count == 1)
    assert sel.sum() > 20000
    assert np.mean(zm.count[sel] == 1) > 0.999
    both = sel & (zm.count == 1)
    eT = np.abs(zm.T[..., 0][both] - pt.T[..., 0][both]) / pt.T[..., 0][both]
    eA = np.abs(zm.A[..., 0][both] - pt.A[..., 0][both]) / pt.A[..., 0][both]
    print('depth march vs pseudo-time, 512^2 TTI: nodes', int(both.sum()), 'T rel median / max',
          np.median(eT), eT.max(), 'A rel median / q99', np.median(eA), np.quantile(eA, 0.99))
    assert np.median(eT) < 2e-4 and eT.max() < 2e-3
    assert np.median(eA) < 1e-2 and np.quantile(eA, 0.99) < 5e-2
    # the advected point-source family's amplitudes (drt = 1) agree as well
    bq = both & (zq.count == 1)
    eQ = np.abs(zq.A[..., 0][bq] - pt.A[..., 0][bq]) / pt.A[..., 0][bq]
    print('advected DRT amplitudes vs pseudo-time: median', np.median(eQ), 'q99', np.quantile(eQ, 0.99))
    assert np.median(eQ) < 1e-2 and np.quantile(eQ, 0.99) < 5e-2


@pytest.mark.parametrize('name', ['vti48', 'tti64', 'lens64'])
def test_zmarch_advected_drt_matches_the_oracle(name):
    """drt = 1: the beams' and arrivals' dynamic ray tracing advected with the march (Eq. 21)
    against oracle/zmarch_drt.py, at the same bar."""
    from oracle import zmarch_drt as DR
    p, nth = _case(name)
    import paper_2006_11945_gb300 as egb
    with egb.Context(0) as ctx:
        res = ctx.zmarch(ctx.medium_2d(p), p, nth, THETA_MAX, 0.5, 8, drt=1)
    ref = DR.solve(p, nth, THETA_MAX, 0.5)
    m = _compare(res, ref, p, ref['parts'])
    print(name, 'drt', m)
    assert m['u_rel_l2'] < 2e-3, m
    assert m['count_mismatch'] == 0 and m['arrivals'] > 100, m
    assert m['T_rel_max'] < 1e-5 and m['A_rel_max'] < 1e-3, m


def test_zmarch_output_pointers_and_arrival_capacity():
    """Device outputs equal host outputs bit for bit; an arrivals-only call (no frequencies, no
    wavefield) gives the same arrivals; with capacity 1 the lens's triplicated nodes report
    EGB_E_ARRIVAL_OVERFLOW and keep their earliest arrival."""
    import torch
    import paper_2006_11945_gb300 as egb
    p = lens_problem()
    nz, nx = p.nz, p.nx
    with egb.Context(0) as ctx:
        m = ctx.medium_2d(p)
        host = ctx.zmarch(m, p, 96, THETA_MAX)
        u = torch.zeros((1, nz, nx, 2), dtype=torch.float32, device='cuda')
        cnt = torch.zeros((nz, nx), dtype=torch.uint8, device='cuda')
        T = torch.zeros((nz, nx, 8), dtype=torch.float64, device='cuda')
        A = torch.zeros((nz, nx, 8), dtype=torch.float32, device='cuda')
        egb.egb_zmarch(ctx.h, m, p.xs, p.omegas, p.beam_width, 96, THETA_MAX, 0.5, u, cnt, T, A, 8)
        assert np.array_equal(u.cpu().numpy().view(np.complex64)[..., 0], host.u)
        assert np.array_equal(cnt.cpu().numpy(), host.count)
        assert np.array_equal(T.cpu().numpy(), host.T) and np.array_equal(A.cpu().numpy(), host.A)
        c2 = np.zeros((nz, nx), np.uint8)
        T2 = np.zeros((nz, nx, 8))
        egb.egb_zmarch(ctx.h, m, p.xs, [], p.beam_width, 96, THETA_MAX, 0.5, None, c2, T2, None, 8)
        assert np.array_equal(c2, host.count) and np.array_equal(T2, host.T)
        c1 = np.zeros((nz, nx), np.uint8)
        T1 = np.zeros((nz, nx, 1))
        A1 = np.zeros((nz, nx, 1), np.float32)
        try:
            egb.egb_zmarch(ctx.h, m, p.xs, [], p.beam_width, 96, THETA_MAX, 0.5, None, c1, T1, A1, 1)
            status = egb.EGB_OK
        except egb.EgbError as e:
            status = e.status
    assert host.count.max() == 3 and status == egb.EGB_E_ARRIVAL_OVERFLOW
    assert np.array_equal(c1, np.minimum(host.count, 1))
    assert np.array_equal(T1[..., 0], host.T[..., 0]) and np.array_equal(A1[..., 0], host.A[..., 0])
