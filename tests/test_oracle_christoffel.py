"""Pins for the oracle's medium and Christoffel layer (Eqs. 3-5, 7 and the ray velocities).

Each check compares the oracle with something other than itself: closed-form velocities of
isotropic and VTI media (Thomsen's exact qP formula), the slowness-shell identity p . V = 1 that the
Hamiltonian normalisation implies, the eigen-equation residual, and finite differences of the phase
velocity for the ray-velocity components.
"""
import math

import numpy as np
import pytest

import synthmedia
from oracle import christoffel as CH
from oracle import closed_forms as CF
from oracle import medium as MD


def _a(C, rho):
    return MD.density_normalised(synthmedia.voigt_to_c21(C), rho)


def test_isotropic_velocity_every_direction():
    lam, mu, rho = 1.2e10, 6.6e9, 2300.0
    a = _a(synthmedia.isotropic_voigt(lam, mu), rho)
    th = np.linspace(0, 2 * np.pi, 73)
    v, V, Vn, g = CH.source_quantities(a, th)
    ref = CF.isotropic_velocity(lam, mu, rho)
    assert np.allclose(v, ref, rtol=1e-13)
    assert np.allclose(Vn, ref, rtol=1e-12)
    # group direction equals the phase direction in an isotropic medium
    assert np.allclose(g[:, 0], np.sin(th), atol=1e-12)
    assert np.allclose(g[:, 1], np.cos(th), atol=1e-12)


@pytest.mark.parametrize('eps,delta', [(0.2, 0.1), (0.25, -0.05), (0.0, 0.15)])
def test_vti_phase_velocity_matches_thomsen_exact(eps, delta):
    vp0, vs0, rho = 3000.0, 1500.0, 2200.0
    a = _a(synthmedia.thomsen_vti_voigt(vp0, vs0, eps, delta, rho), rho)
    th = np.linspace(0, 2 * np.pi, 181)
    v, V, Vn, g = CH.source_quantities(a, th)
    ref = CF.thomsen_vti_phase_velocity(th, vp0, vs0, eps, delta)
    assert np.allclose(v, ref, rtol=1e-12)
    _, Vx, Vz = CF.vti_group_velocity(th, vp0, vs0, eps, delta)
    assert np.allclose(V[:, 0], Vx, rtol=1e-10, atol=1e-7)
    assert np.allclose(V[:, 1], Vz, rtol=1e-10, atol=1e-7)


def test_vti_reference_numbers():
    """VTI medium of the 64x64 case: v(0) = 3000, v(45) = 3229.33, v(90) = 3549.65 m/s and a 45 deg
    phase direction carries energy along 55.25 deg at 3281.70 m/s (Thomsen exact formula)."""
    a = _a(synthmedia.thomsen_vti_voigt(3000, 1500, 0.2, 0.1, 2200), 2200.0)
    v, V, Vn, g = CH.source_quantities(a, np.radians([0.0, 45.0, 90.0]))
    assert np.allclose(v, [3000.0, 3229.3349, 3549.6479], atol=1e-3)
    assert abs(Vn[1] - 3281.6993) < 1e-3
    assert abs(math.degrees(math.atan2(V[1, 0], V[1, 1])) - 55.2491) < 1e-3


def _random_pd_media(rng, count):
    base = synthmedia.isotropic_voigt(1.3e10, 6.0e9)
    out = []
    while len(out) < count:
        P = rng.normal(size=(6, 6)) * 1.2e9
        C = base + 0.5 * (P + P.T)
        if np.linalg.eigvalsh(C).min() > 1e8:
            out.append(C)
    return np.array(out)


def test_shell_identity_and_eigen_residual_triclinic():
    """p . V = 1 (H = 0 on the slowness shell, dT/dt = 1) and |Gamma g - lambda g| ~ 0."""
    rng = np.random.default_rng(11)
    C = _random_pd_media(rng, 40)
    a = MD.density_normalised(synthmedia.voigt_to_c21(C), np.full(40, 2400.0))
    phi = rng.uniform(0, 2 * np.pi, 40)
    cth = rng.uniform(-1, 1, 40)
    sth = np.sqrt(1 - cth ** 2)
    n = np.stack([sth * np.cos(phi), sth * np.sin(phi), cth], -1)
    v, g, V, _ = CH.ray_velocity(a, [], n)
    p = n / v[:, None]
    assert np.allclose(np.einsum('ni,ni->n', p, V), 1.0, rtol=1e-12)
    G = CH.christoffel(a, n)
    res = np.einsum('nik,nk->ni', G, g) - (v ** 2)[:, None] * g
    assert np.max(np.abs(res)) < 1e-6 * np.max(v ** 2)
    # qP is the largest of the three eigenvalues
    assert np.all(np.linalg.eigvalsh(G)[:, -1] <= v ** 2 * (1 + 1e-14))


def test_pdot_is_minus_grad_log_v():
    """dp/dt = -grad v / v at fixed phase direction; checked against finite differences of v."""
    n_nodes = 9
    h = 7.0
    x = np.arange(n_nodes) * h
    lam = 1.1e10 * (1 + 0.01 * x)
    mu = 5.5e9 * (1 + 0.004 * x)
    C = synthmedia.isotropic_voigt(lam, mu)
    rho = 2300.0 * (1 + 0.002 * x)
    a = MD.density_normalised(synthmedia.voigt_to_c21(C), rho)
    da = np.gradient(a, h, axis=0, edge_order=2)
    th = 0.7
    n = np.broadcast_to(CH.direction_2d(th), (n_nodes, 3))
    v, g, V, (pdx,) = CH.ray_velocity(a, [da], n)
    dv = np.gradient(v, h, edge_order=2)
    assert np.allclose(pdx[2:-2], -dv[2:-2] / v[2:-2], rtol=2e-3)


def test_medium_gradient_second_order_one_sided_edges():
    nz, nx, h = 5, 6, 3.0
    xs = np.arange(nx) * h
    zs = np.arange(nz) * h
    Z, X = np.meshgrid(zs, xs, indexing='ij')
    field = (1e10 + 3e6 * X ** 2 + 2e6 * Z ** 2)[..., None] * np.ones(21)
    prob = synthmedia.Problem2D('t', nx, nz, h, h, field.reshape(-1, 21), np.ones(nz * nx), (0, 0),
                                4, [1.0], 1.0, 1)
    a, ddx, ddz, rho = MD.medium_2d(prob)
    # second-order formulas are exact for quadratics, edges included
    assert np.allclose(ddx[..., 0, 0, 0, 0], 6e6 * X, rtol=1e-12, atol=1e-3)
    assert np.allclose(ddz[..., 0, 0, 0, 0], 4e6 * Z, rtol=1e-12, atol=1e-3)


def test_positive_definite_check():
    good = synthmedia.voigt_to_c21(synthmedia.isotropic_voigt(1e10, 5e9))
    bad = good.copy()
    bad[synthmedia.voigt21_index(3, 3)] = -1.0
    assert MD.is_positive_definite(np.stack([good, bad])).tolist() == [True, False]


def test_near_degenerate_medium_has_the_stated_gap():
    """The input of the GPU test on the FP64 polish: positive definite, and the two largest
    Christoffel eigenvalues come within 6.8e-5 (relative) at theta = 0 and pi, not elsewhere."""
    import synthmedia
    from oracle import medium as MD
    p = synthmedia.triclinic_near_degenerate()
    assert MD.is_positive_definite(p.c21[:1].astype(np.float64)).all()
    a = MD.density_normalised(p.c21[0].astype(np.float64), float(p.rho[0]))
    th = 2 * np.pi * np.arange(p.n_theta) / p.n_theta
    n = np.stack([np.sin(th), np.zeros_like(th), np.cos(th)], -1)
    w = np.linalg.eigvalsh(CH.christoffel(a, n))
    gap = (w[:, -1] - w[:, -2]) / w[:, -1]
    assert abs(gap[0] - 6.8e-5) < 1e-6 and abs(gap[p.n_theta // 2] - 6.8e-5) < 1e-6
    assert np.sort(gap)[2] > 1e-3


def test_near_degenerate_cube_has_the_gap_on_a_grid_direction():
    """The 3-D version: the gap of 6.8e-5 lies on the direction (first polar cell centre, phi = 0)
    of the 3-D angle grid and its antipode, every other grid direction at least 1e-2."""
    import synthmedia
    from oracle import medium as MD
    p = synthmedia.triclinic_near_degenerate_3d()
    a = MD.density_normalised(p.c21[0].astype(np.float64), float(p.rho[0]))
    th, ph = CH.angle_grid_3d(p.n_theta, p.n_phi)
    gaps = {}
    for k in range(p.n_phi):
        for j in range(p.n_theta):
            w = np.linalg.eigvalsh(CH.christoffel(a, CH.direction_3d(th[j], ph[k])))
            gaps[(j, k)] = (w[-1] - w[-2]) / w[-1]
    assert abs(gaps[(0, 0)] - 6.8e-5) < 1e-6 and abs(gaps[(p.n_theta - 1, p.n_phi // 2)] - 6.8e-5) < 1e-6
    assert sorted(gaps.values())[2] > 1e-2
