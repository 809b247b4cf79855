"""Pins for the oracle's paraxial depth march (Eqs. 13-20) and its same-row superposition (Eqs. 25-28,
33-35).

Checked against things the march does not compute itself:
* exactness on data linear in x and theta with depth-varying coefficients (third-order HJ-WENO is
  exact on linear data, the linear ghost extrapolation continues it, and TVD-RK3 integrates a
  right-hand side linear in depth exactly only if its stages sit at the right depths);
* the closed-form labels of a homogeneous VTI medium from Thomsen's exact phase velocity (straight
  group rays: X = x - (z - z_s) Vx/Vz, vartheta = theta, tau = (z - z_s)/Vz), both branches;
* homogeneous isotropic: (i/4) H0^(1)(kr) inside the angle cone with an error that falls as kr
  grows and does not depend on the beam width to that order; one arrival per node with T = r/v and
  A = sqrt(v / (8 pi r));
* homogeneous VTI: the far field of the exact plane-wave integral (stationary phase);
* a low-velocity lens: arrival counts (single and triplicated) and first-arrival traveltimes of the
  Lagrangian ray shooter;
* the source indicator against straight rays traced back to the source row (inflow through the
  x edges);
* behind a wide lens, the triplicated wavefield against the shooter's geometrical field with the
  KMAH phase shift of the arrival that has passed a caustic.
"""
import math
import types

import numpy as np
import pytest

import synthmedia
from oracle import closed_forms as CF
from oracle import shooter as SH
from oracle import zmarch as ZM

THETA_MAX = math.radians(60.0)


def _fake(nth, nx, nr, U, W, S, h=1.0, dth=0.05):
    Z = types.SimpleNamespace()
    Z.nth, Z.nx, Z.hx, Z.hz, Z.dth = nth, nx, h, h, dth
    Z.rows = np.arange(nr)
    Z.U, Z.W, Z.S = U, W, S
    Z.n_sub = 3
    Z.x = h * np.arange(nx)
    Z.theta = dth * (np.arange(nth) - nth / 2 + 0.5)
    Z.eps = {'X': 1e-6, 'Th': 1e-6, 'tau': 1e-6, 'q': 1e-6}
    return Z


def test_pad_continues_linear_data():
    rng = np.random.default_rng(1)
    a, b, c = rng.normal(size=3)
    k, i = np.meshgrid(np.arange(-2, 9), np.arange(-2, 13), indexing='ij')
    full = a * k + b * i + c
    p = ZM._pad(full[2:-2, 2:-2])
    G = ZM.GHOST
    assert np.allclose(p[G:-G, :], full[G:-G, :], atol=1e-12)
    assert np.allclose(p[:, G:-G], full[:, G:-G], atol=1e-12)
    assert np.all(np.isnan(p[:G, :G])) and np.all(np.isnan(p[-G:, -G:]))


def test_march_exact_on_linear_data_with_depth_varying_coefficients():
    """phi = alpha x + beta theta with U = U_r + gamma r (linear in depth), W constant: the exact
    solution moves by -alpha int U - beta W per row, tau gains int S."""
    nth, nx, nr = 9, 13, 6
    rows = np.arange(nr, dtype=float)
    U = np.broadcast_to((0.3 + 0.05 * rows)[None, :, None], (nth, nr, nx)).copy()
    W = np.full((nth, nr, nx), -0.02)
    S = np.broadcast_to((2.0 + 0.1 * rows)[None, :, None], (nth, nr, nx)).copy()
    Z = _fake(nth, nx, nr, U, W, S)
    H = ZM.march(Z)
    x, th = Z.x[None, :], Z.theta[:, None]
    for r in range(nr):
        intU = 0.3 * r + 0.05 * r * r / 2          # int_0^r (0.3 + 0.05 z) dz
        intS = 2.0 * r + 0.1 * r * r / 2
        assert np.allclose(H['X'][:, r], x - intU, atol=1e-12)
        assert np.allclose(H['Th'][:, r], th + 0.02 * r, atol=1e-12)
        assert np.allclose(H['tau'][:, r], intS, atol=1e-12)


@pytest.mark.parametrize('branch', [1, -1])
def test_homogeneous_vti_labels_match_straight_group_rays(branch):
    p = synthmedia.vti_homogeneous(n=48, n_theta=32, steps=1)
    m = p.meta
    Z = ZM.ZSetup(p, 32, THETA_MAX, branch, 0.5)
    H = ZM.march(Z)
    v, Vx, Vz = CF.vti_group_velocity(Z.theta, m['vp0'], m['vs0'], m['eps'], m['delta'])
    dz = (Z.rows * p.hz + p.origin[1] - p.xs[1])[None, :, None]
    Xc = Z.x[None, None, :] - dz * (Vx / Vz)[:, None, None]
    tc = dz / Vz[:, None, None]
    # the medium's stiffness is stored in FP32: velocities agree to ~1e-7 relative
    assert np.max(np.abs(H['X'] - Xc)) < 1e-6 * np.max(np.abs(dz)) + 1e-9
    assert np.max(np.abs(H['tau'] - tc)) < 1e-6 * np.max(np.abs(tc))
    assert np.max(np.abs(H['Th'] - Z.theta[:, None, None])) < 1e-12
    assert len(Z.rows) == (p.nz - Z.js if branch == 1 else Z.js + 1)


def _down(problem, nth):
    Z = ZM.ZSetup(problem, nth, THETA_MAX, 1, 0.5)
    H = ZM.march(Z)
    x = Z.x - problem.xs[0]
    z = Z.rows * problem.hz + problem.origin[1] - problem.xs[1]
    Zg, Xg = np.meshgrid(z, x, indexing='ij')
    return Z, H, Xg, Zg, np.hypot(Xg, Zg), np.degrees(np.arctan2(np.abs(Xg), np.abs(Zg)))


@pytest.fixture(scope='module')
def iso():
    p = synthmedia.isotropic_homogeneous(n=128, h=10.0, n_theta=64, freqs=[60.0])
    return (p,) + _down(p, 192)


def test_isotropic_hankel_convergence_in_the_cone(iso):
    p, Z, H, X, Zd, r, ang = iso
    om = 2 * math.pi * 60.0
    k = om / p.meta['vp']
    ref = CF.hankel_green_2d(k, np.where(r > 0, r, 1.0))
    u = ZM.green_rows(Z, H, [om], 100.0)[0]
    errs = []
    for lo, hi in ((10, 20), (20, 40), (40, 60)):
        m = (k * r >= lo) & (k * r < hi) & (ang < 30)
        errs.append(np.linalg.norm(u[m] - ref[m]) / np.linalg.norm(ref[m]))
    assert np.all(np.diff(errs) < 0), errs
    assert errs[-1] < 0.02, errs
    u2 = ZM.green_rows(Z, H, [om], 200.0)[0]
    m = (k * r >= 20) & (ang < 30)
    assert np.linalg.norm(u[m] - u2[m]) / np.linalg.norm(u2[m]) < 0.05


def test_isotropic_arrivals(iso):
    p, Z, H, X, Zd, r, ang = iso
    c = p.meta['vp']
    cnt, T, A, overflow = ZM.arrivals_rows(Z, H)
    m = (r > 60.0) & (ang < 45)
    assert not overflow and np.all(cnt[m] == 1)
    assert np.max(np.abs(T[..., 0][m] - r[m] / c) / (r[m] / c)) < 1e-4
    Aref = np.sqrt(c / (8 * math.pi * r[m]))
    assert np.max(np.abs(A[..., 0][m] - Aref) / Aref) < 5e-4


def test_vti_far_field_and_arrivals():
    p = synthmedia.vti_homogeneous(n=128, h=10.0, n_theta=64, freqs=[60.0])
    Z, H, X, Zd, r, ang = _down(p, 192)
    m_ = p.meta
    om = 2 * math.pi * 60.0
    v_of = lambda th: CF.thomsen_vti_phase_velocity(th, m_['vp0'], m_['vs0'], m_['eps'], m_['delta'])
    V_of = lambda th: CF.vti_group_velocity(th, m_['vp0'], m_['vs0'], m_['eps'], m_['delta'])[1:]
    sel = (ang < 30) & (r > 350.0)
    ref, Tr, _ = CF.homogeneous_go_green(X[sel], Zd[sel], 0.0, 0.0, om, v_of, V_of, m_['vp0'])
    u = ZM.green_rows(Z, H, [om], 100.0)[0][sel]
    assert np.linalg.norm(u - ref) / np.linalg.norm(ref) < 0.04
    cnt, T, A, _ = ZM.arrivals_rows(Z, H)
    assert np.all(cnt[sel] == 1)
    assert np.max(np.abs(T[..., 0][sel] - Tr) / Tr) < 1e-4
    Aref = np.abs(ref) * math.sqrt(om)
    assert np.max(np.abs(A[..., 0][sel] - Aref) / Aref) < 1e-3


def lens_problem(n=64, h=10.0):
    """Isotropic medium with a 35 % slow Gaussian lens (sigma 70 m) 320 m below the source: rays
    focus behind it and nodes there see three arrivals."""
    x = np.arange(n) * h
    Z, X = np.meshgrid(x, x, indexing='ij')
    vp = 3000.0 * (1.0 - 0.35 * np.exp(-((X - 320.0) ** 2 + (Z - 470.0) ** 2) / (2 * 70.0 ** 2)))
    vs, rho = vp / 1.8, 2300.0
    mu = rho * vs ** 2
    C = synthmedia.isotropic_voigt(rho * vp ** 2 - 2 * mu, mu)
    c21 = synthmedia.voigt_to_c21(C).reshape(-1, 21).astype(np.float32)
    return synthmedia.Problem2D('lens', n, n, h, h, c21, np.full(n * n, rho, np.float32), (320.0, 150.0),
                                64, [15.0], 50.0, 200)


def test_lens_late_arrivals_match_the_ray_shooter():
    p = lens_problem()
    fan = SH.shoot(p, n_rays=2048)
    sc, first, _ = SH.arrivals(p, fan)
    res = ZM.solve(p, 96, THETA_MAX, 0.5)
    x = np.arange(p.nx) * p.hx - p.xs[0]
    z = np.arange(p.nz) * p.hz - p.xs[1]
    Zg, Xg = np.meshgrid(z, x, indexing='ij')
    r = np.hypot(Xg, Zg)
    ang = np.degrees(np.arctan2(np.abs(Xg), np.abs(Zg)))
    m = (ang < 30) & (r > 80) & (Zg > 0)
    assert np.sum(m & (sc == 3)) >= 5                      # the lens triplicates arrivals
    assert np.array_equal(res['count'][m], sc[m])
    mm = m & (sc >= 1)
    rel = np.abs(res['T'][..., 0][mm] - first[mm]) / first[mm]
    assert np.median(rel) < 1e-3 and rel.max() < 1e-2


def test_source_indicator_marks_rays_entering_through_the_edges():
    """Homogeneous VTI: a cell's straight group ray traced back reaches the source row at
    x - (z - z_s) Vx/Vz; where that point lies more than 4 cells outside the grid the ray entered
    through an edge (q < 1/2), more than 4 cells inside it carries source-plane labels (q > 1/2)."""
    p = synthmedia.vti_homogeneous(n=48, n_theta=32, steps=1)
    m = p.meta
    Z = ZM.ZSetup(p, 32, THETA_MAX, 1, 0.5)
    H = ZM.march(Z)
    v, Vx, Vz = CF.vti_group_velocity(Z.theta, m['vp0'], m['vs0'], m['eps'], m['delta'])
    zeta = (Z.rows * p.hz + p.origin[1] - p.xs[1])[None, :, None]
    x0 = Z.x[None, None, :] - zeta * (Vx / Vz)[:, None, None]
    lo, hi, h = Z.x[0], Z.x[-1], p.hx
    outside = (x0 < lo - 4 * h) | (x0 > hi + 4 * h)
    inside = (x0 > lo + 4 * h) & (x0 < hi - 4 * h)
    assert outside.sum() > 1000 and inside.sum() > 1000
    assert np.all(H['q'][outside] < 0.5) and np.all(H['q'][inside] > 0.5)


def wide_lens_problem():
    """Isotropic 128 x 128 medium at 10 m with a 30 % slow Gaussian lens (sigma 120 m) 320 m below
    the source: behind it a cusp caustic opens a triplication zone several wavelengths wide at
    200 Hz, whose late arrival has passed one caustic."""
    n, h = 128, 10.0
    x = np.arange(n) * h
    Z, X = np.meshgrid(x, x, indexing='ij')
    vp = 3000.0 * (1.0 - 0.3 * np.exp(-((X - 640.0) ** 2 + (Z - 420.0) ** 2) / (2 * 120.0 ** 2)))
    vs, rho = vp / 1.8, 2300.0
    mu = rho * vs ** 2
    C = synthmedia.isotropic_voigt(rho * vp ** 2 - 2 * mu, mu)
    c21 = synthmedia.voigt_to_c21(C).reshape(-1, 21).astype(np.float32)
    return synthmedia.Problem2D('wide-lens', n, n, h, h, c21, np.full(n * n, rho, np.float32),
                                (640.0, 100.0), 64, [15.0], 40.0, 200)


@pytest.mark.slow
def test_triplicated_wavefield_carries_the_kmah_phase_shift():
    """Behind the wide lens, at triplicated nodes at least three cells from any change of the arrival
    count, the beam sum (Eqs. 25-28 with the amplitude's square root continued through the caustic)
    tends with frequency to the geometrical field sum_k A_k exp(i (omega T_k + pi/4 - m_k pi/2)) /
    sqrt(omega) of the Lagrangian shooter, m_k its KMAH index; without the -m_k pi/2 shift the two
    differ at order one."""
    from scipy import ndimage
    p = wide_lens_problem()
    x = np.arange(p.nx) * p.hx
    Z, X = np.meshgrid(x, x, indexing='ij')
    box = (Z >= 700.0) & (np.abs(X - 640.0) <= 250.0)
    fan = SH.shoot(p, n_rays=2048, dt=1.5e-3)
    sc, first, arr = SH.arrivals(p, fan, node_mask=box)
    calm = ndimage.maximum_filter(sc, 7) == ndimage.minimum_filter(sc, 7)
    m = box & (sc == 3) & calm
    assert m.sum() >= 30
    assert all([a[3] for a in arr[key]] == [0, 0, 1] for key in zip(*np.nonzero(m)))
    freqs = (50.0, 100.0, 200.0)
    res = ZM.solve(p, 128, THETA_MAX, 0.5, omegas=[2 * math.pi * f for f in freqs], beam_width=40.0)
    assert np.array_equal(res['count'][box & calm], sc[box & calm])
    err = {}
    for w, f in enumerate(freqs):
        om = 2 * math.pi * f
        go = np.zeros(sc.shape, complex)
        go0 = np.zeros(sc.shape, complex)
        for key in zip(*np.nonzero(m)):
            for T, A, _, mk in arr[key]:
                g = A / math.sqrt(om) * np.exp(1j * (om * T + math.pi / 4))
                go[key] += g * (-1j) ** mk
                go0[key] += g
        u = res['u'][w][m]
        e = np.abs(u - go[m]) / np.abs(go[m])
        err[f] = np.median(e)
        if f == 200.0:
            assert err[f] < 0.06 and np.quantile(e, 0.9) < 0.1, (err[f], np.quantile(e, 0.9))
            assert np.median(np.abs(u - go0[m]) / np.abs(go0[m])) > 0.5
    assert err[50.0] > err[100.0] > 2 * err[200.0], err
