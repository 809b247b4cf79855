"""Pins for the 3-D oracle (5-D phase space (x, y, z, theta, phi)).

* Velocities: the direction-angle rates equal the time derivatives of the angles of p along the
  Hamiltonian flow (finite differences of p + pdot dt); in a y-symmetric medium the phi = 0 cells
  reduce to the 2-D oracle's; isotropic homogeneous: V = v n and no turning; p . V = 1.
* Stepping: third-order WENO across the poles on smooth data on the sphere; C loop = numpy;
  homogeneous steady state = straight-ray closed form.
* Arrivals (closed-form labels): one arrival per node; T = r/v and |u| = 1/(4 pi r) (isotropic),
  T = r/|V| and |u| = c_ref^2/(4 pi sqrt(K) |V| r) with K the Gaussian curvature of the VTI slowness
  surface (Thomsen's exact phase velocity); errors second order in the angular spacing.
* Superposition: equals the continuous Gaussian-beam integral of analytic beams (independent
  quadrature) and tends to exp(ikr)/(4 pi r) as kr grows; VTI far field within a few per cent of
  the GO Green's function.
"""
import math

import numpy as np
import pytest

import synthmedia
from oracle import christoffel as CH
from oracle import closed_forms as CF
from oracle import liouville3d as L3
from oracle import medium as MD
from oracle import superpose3d as S3


def _homogeneous_vel(p):
    """velocity_field_3d of a homogeneous medium, evaluated at one node and broadcast to the grid."""
    a = MD.density_normalised(np.asarray(p.c21[:1], np.float64), np.asarray(p.rho[:1], np.float64))
    a = a.reshape(1, 1, 1, 3, 3, 3, 3)
    z = np.zeros_like(a)
    vel = CH.velocity_field_3d(a, z, z, z, p.n_theta, p.n_phi)
    shape = (p.n_phi, p.n_theta, p.nz, p.ny, p.nx)
    return {k: np.broadcast_to(v, shape) for k, v in vel.items()}


def _exact(p):
    S = L3.Setup3D(p, vel=_homogeneous_vel(p))
    lab = CF.homogeneous_labels_3d(S)
    o = np.arange(p.nx) * p.hx - p.xs[0]
    Z, Y, X = np.meshgrid(o, o, o, indexing='ij')
    return S, lab, X, Y, Z


# ---------------------------------------------------------------------------------- velocities

def test_angle_rates_are_the_hamiltonian_flow_of_the_direction():
    p = synthmedia.triclinic_3d(n=10, n_theta=6, n_phi=8, length=600.0, steps=1)
    a, dx, dy, dz, _ = MD.medium_3d(p)
    vel = CH.velocity_field_3d(a, dx, dy, dz, p.n_theta, p.n_phi)
    th, ph = CH.angle_grid_3d(p.n_theta, p.n_phi)
    rng = np.random.default_rng(1)
    for _ in range(20):
        k, j = rng.integers(p.n_phi), rng.integers(p.n_theta)
        c = (k, j) + tuple(rng.integers(1, 9, size=3))
        pvec = CH.direction_3d(th[j], ph[k]) / vel['v'][c]
        pdot = np.array([vel['pdx'][c], vel['pdy'][c], vel['pdz'][c]])
        dt = 1e-4

        def angles(q):
            return math.acos(q[2] / np.linalg.norm(q)), math.atan2(q[1], q[0])
        (tp, pp), (tm, pm) = angles(pvec + dt * pdot), angles(pvec - dt * pdot)
        dph = (pp - pm + math.pi) % (2 * math.pi) - math.pi
        assert abs((tp - tm) / (2 * dt) - vel['thetadot'][c]) < 1e-6 * (1 + abs(vel['thetadot'][c]))
        assert abs(dph / (2 * dt) - vel['phidot'][c]) < 1e-6 * (1 + abs(vel['phidot'][c]))
        V = np.array([vel['Vx'][c], vel['Vy'][c], vel['Vz'][c]])
        assert abs(pvec @ V - 1.0) < 1e-12


def test_xz_plane_reduces_to_the_2d_velocities():
    """A medium extruded along y with y-mirror symmetry (TTI tilted in the x-z plane): the 3-D cells
    with phi = 0 carry the 2-D velocities (theta_j = (j + 1/2) pi / n_theta is 2-D angle 2j + 1 of
    4 n_theta), no y motion and no azimuth turning."""
    p2 = synthmedia.tti_heterogeneous(n=12, n_theta=16, length=600.0, steps=1)
    c21 = np.repeat(np.asarray(p2.c21).reshape(12, 1, 12, 21), 5, axis=1).reshape(-1, 21)
    rho = np.repeat(np.asarray(p2.rho).reshape(12, 1, 12), 5, axis=1).reshape(-1)
    p3 = synthmedia.Problem3D('ext', 12, 5, 12, p2.hx, p2.hx, p2.hz, c21, rho, (0, 0, 0), 4, 4, [10.0], 50.0, 1)
    a, dx, dy, dz, _ = MD.medium_3d(p3)
    v3 = CH.velocity_field_3d(a, dx, dy, dz, 4, 4)
    a2, dx2, dz2, _ = MD.medium_2d(p2)
    v2 = CH.velocity_field_2d(a2, dx2, dz2, 16)
    for j in range(4):
        for key in ('Vx', 'Vz', 'thetadot', 'v'):
            np.testing.assert_allclose(v3[key][0, j, :, 2, :], v2[key][2 * j + 1], rtol=1e-10, atol=1e-9)
        assert np.max(np.abs(v3['Vy'][0, j])) < 1e-8 and np.max(np.abs(v3['phidot'][0, j])) < 1e-10


def test_isotropic_homogeneous_rays_are_straight():
    p = synthmedia.isotropic_homogeneous_3d(n=6, n_theta=6, n_phi=8)
    vel = _homogeneous_vel(p)
    th, ph = CH.angle_grid_3d(6, 8)
    n = CH.direction_3d(th[None, :], ph[:, None])
    for c, key in enumerate(('Vx', 'Vy', 'Vz')):
        np.testing.assert_allclose(vel[key][:, :, 0, 0, 0], p.meta['vp'] * n[..., c], atol=1e-9)
    assert np.max(np.abs(vel['thetadot'])) < 1e-12 and np.max(np.abs(vel['phidot'])) < 1e-12


# ---------------------------------------------------------------------------------- stepping

def test_weno_across_the_poles_is_third_order():
    """theta derivative of a smooth function on the sphere at the polar rows, with the stencil
    continued across the pole onto the opposite azimuth."""
    errs = []
    for nth in (16, 32, 64):
        nph = 2 * nth
        th, ph = CH.angle_grid_3d(nth, nph)
        n = CH.direction_3d(th[None, :], ph[:, None])
        c = np.array([0.3, -0.5, 0.8])
        f = np.exp(n @ c)                                         # smooth on the sphere
        n_th = np.stack([np.cos(th)[None, :] * np.cos(ph)[:, None], np.cos(th)[None, :] * np.sin(ph)[:, None],
                         -np.sin(th)[None, :] * np.ones_like(ph)[:, None]], -1)
        dfdth = f * (n_th @ c)
        S = type('S', (), {})()
        S.nx = S.ny = S.nz = 1
        S.nth, S.nph, S.hx, S.hy, S.hz = nth, nph, 1.0, 1.0, 1.0
        S.dth, S.dph = math.pi / nth, 2 * math.pi / nph
        z = np.zeros((nph, nth, 1, 1, 1))
        S.vel = {'Vx': z, 'Vy': z, 'Vz': z, 'thetadot': np.ones_like(z), 'phidot': z}
        u = np.pad(f[:, :, None, None, None], ((0, 0), (0, 0), (2, 2), (2, 2), (2, 2)), mode='edge')
        ut = L3.upwind_derivatives_3d(u, S, 1e-12)[3][:, :, 0, 0, 0]
        polar = np.r_[0:2, nth - 2:nth]
        errs.append(np.max(np.abs(ut[:, polar] - dfdth[:, polar])))
    orders = np.log2(np.array(errs[:-1]) / np.array(errs[1:]))
    assert np.all(orders > 2.5), (errs, orders)


def test_c_loop_equals_array_code_3d():
    p = synthmedia.triclinic_3d(n=10, n_theta=6, n_phi=10, length=400.0, steps=3)
    S = L3.Setup3D(p)
    st0 = S.initial_state()
    _, a, _ = L3.evolve3d(p, S=S, state={k: v.copy() for k, v in st0.items()}, backend='numpy')
    _, b, _ = L3.evolve3d(p, S=S, state={k: v.copy() for k, v in st0.items()}, backend='c')
    for f in L3.FIELDS3:
        assert np.array_equal(a[f], b[f]), f
    assert not np.array_equal(a['q'], st0['q']) and not np.array_equal(a['bx'], st0['bx'])


def test_homogeneous_steady_state_closed_form_3d():
    p = synthmedia.vti_homogeneous_3d(n=16, n_theta=8, n_phi=16, steps=40)
    S, st, dt = L3.evolve3d(p)
    lab = L3.interior_state3d(st)
    ref = CF.homogeneous_labels_3d(S)
    h = p.hx
    for f in ('bx', 'by', 'bz'):
        assert np.max(np.abs(lab[f] - ref[f])) < 1e-9 * h
    for f in ('n0x', 'n0y', 'n0z', 'tau'):
        assert np.max(np.abs(lab[f] - ref[f])) < 1e-12
    # the indicator front has passed every interior cell: away from its discontinuities (the tube
    # edge |b| = R_Sigma, the upstream face of the frozen disc |d| = R_Sigma, and the cells whose
    # stencil reaches the q = 0 ghosts) it is 1 on source rays and 0 elsewhere
    bn = np.sqrt(ref['bx'] ** 2 + ref['by'] ** 2 + ref['bz'] ** 2)
    o = np.arange(p.nx) * h - p.xs[0]
    Z, Y, X = np.meshgrid(o, o, o, indexing='ij')
    d = np.sqrt(X ** 2 + Y ** 2 + Z ** 2)
    L = sum(c[None, None] * S.gs[..., i][:, :, None, None, None] for i, c in enumerate((X, Y, Z)))
    inner = np.zeros((p.nz, p.ny, p.nx), bool)
    inner[3:-3, 3:-3, 3:-3] = True
    away = (inner[None, None] & (np.abs(bn - S.R_sigma) > 3 * h)
            & ~((L < 0) & (np.abs(d - S.R_sigma)[None, None] < 3 * h)))
    assert away.sum() > 1000
    assert np.max(np.abs(lab['q'] - ref['q'])[away]) < 0.05


# ---------------------------------------------------------------------------------- arrivals

def _arrival_errors(S, lab, X, Y, Z, Tref, Aref):
    cnt, T, A, over = S3.arrivals3d(S, lab)
    r = np.sqrt(X ** 2 + Y ** 2 + Z ** 2)
    m = r > 3 * S.r0
    assert not over and np.all(cnt[m] == 1)
    return (np.max(np.abs(T[..., 0][m] - Tref[m]) / Tref[m]),
            np.max(np.abs(A[..., 0][m] - Aref[m]) / Aref[m]))


def test_isotropic_arrivals_3d():
    errs = []
    for nth in (12, 24):
        S, lab, X, Y, Z = _exact(synthmedia.isotropic_homogeneous_3d(n=16, n_theta=nth, n_phi=2 * nth))
        v = S.p.meta['vp']
        r = np.sqrt(X ** 2 + Y ** 2 + Z ** 2)
        rr = np.where(r > 0, r, 1.0)
        errs.append(_arrival_errors(S, lab, X, Y, Z, rr / v, 1.0 / (4 * math.pi * rr)))
    (t1, a1), (t2, a2) = errs
    assert t2 < 5e-3 and a2 < 2e-2, errs
    # halving the angular spacing divides both errors by about four (second order)
    assert t1 / t2 > 3.0 and a1 / a2 > 3.0, errs


def test_vti_slowness_curvature_matches_the_ellipsoid():
    """Elliptical VTI (eps = delta): the qP slowness surface is the ellipsoid
    p_h^2 / a^2 + p_z^2 / c^2 = 1 (a = 1/(Vp0 sqrt(1 + 2 eps)), c = 1/Vp0) with Gaussian curvature
    1 / (a^4 c^2 (p_h^2/a^4 + p_z^2/c^4)^2)."""
    vp0, vs0, eps = 3000.0, 1500.0, 0.2
    th = np.linspace(0.05, 1.5, 9)
    K = CF.vti_slowness_gaussian_curvature(th, vp0, vs0, eps, eps)
    v = CF.thomsen_vti_phase_velocity(th, vp0, vs0, eps, eps)
    ph_, pz = np.sin(th) / v, np.cos(th) / v
    a, c = 1.0 / (vp0 * math.sqrt(1 + 2 * eps)), 1.0 / vp0
    Kell = 1.0 / (a ** 4 * c ** 2 * (ph_ ** 2 / a ** 4 + pz ** 2 / c ** 4) ** 2)
    np.testing.assert_allclose(K, Kell, rtol=1e-7)
    np.testing.assert_allclose(CF.vti_slowness_gaussian_curvature(th, vp0, vs0, 0.0, 0.0), vp0 ** 2, rtol=1e-7)


@pytest.fixture(scope='module')
def vti_fine():
    return _exact(synthmedia.vti_homogeneous_3d(n=24, n_theta=24, n_phi=48, freqs=[400.0], beam_width=20.0))


def test_vti_arrivals_3d(vti_fine):
    S, lab, X, Y, Z = vti_fine
    m = S.p.meta
    r = np.sqrt(X ** 2 + Y ** 2 + Z ** 2)
    with np.errstate(divide='ignore', invalid='ignore'):
        _, Tref, Aref = CF.homogeneous_go_green_3d_vti(X, Y, Z, 1.0, m['vp0'], m['vs0'], m['eps'], m['delta'])
    et, ea = _arrival_errors(S, lab, X, Y, Z, np.where(r > 0, Tref, 1.0), np.where(r > 0, Aref, 1.0))
    assert et < 5e-3 and ea < 3e-2, (et, ea)


# ---------------------------------------------------------------------------------- superposition

def test_isotropic_beam_sum_equals_the_beam_integral():
    p = synthmedia.isotropic_homogeneous_3d(n=24, n_theta=24, n_phi=48, freqs=[400.0], beam_width=20.0)
    S, lab, X, Y, Z = _exact(p)
    om = 2 * math.pi * 400.0
    u = S3.green3d(S, lab, [om], 20.0)[0]
    v = p.meta['vp']
    k = om / v
    r = np.sqrt(X ** 2 + Y ** 2 + Z ** 2)
    edge = np.minimum.reduce([X - X.min(), X.max() - X, Y - Y.min(), Y.max() - Y, Z - Z.min(), Z.max() - Z])
    box = ((X.min(),) * 3, (X.max(),) * 3)
    rng = np.random.default_rng(0)
    out = []
    for lo, hi in ((20, 40), (40, 60), (60, 80)):
        idx = np.flatnonzero((edge >= 0.25 * p.nx * p.hx) & (k * r >= lo) & (k * r < hi))
        idx = rng.choice(idx, size=min(30, idx.size), replace=False)
        ref = CF.isotropic_beam_integral_3d(X.ravel()[idx], Y.ravel()[idx], Z.ravel()[idx], om, 20.0, v,
                                            S.r0, box=box)
        exact = np.exp(1j * k * r.ravel()[idx]) / (4 * math.pi * r.ravel()[idx])
        uu = u.ravel()[idx]
        out.append((np.linalg.norm(uu - ref) / np.linalg.norm(ref),
                    np.linalg.norm(uu - exact) / np.linalg.norm(exact)))
    (_, e20), (i40, e40), (i60, e60) = out
    assert i40 < 3e-2 and i60 < 2e-2, out
    assert e20 > e40 > e60 and e60 < 3e-2, out


def test_vti_beam_sum_far_field(vti_fine):
    S, lab, X, Y, Z = vti_fine
    m = S.p.meta
    om = 2 * math.pi * 400.0
    u = S3.green3d(S, lab, [om], 20.0)[0]
    r = np.sqrt(X ** 2 + Y ** 2 + Z ** 2)
    k = om / m['vp0']
    edge = np.minimum.reduce([X - X.min(), X.max() - X, Y - Y.min(), Y.max() - Y, Z - Z.min(), Z.max() - Z])
    sel = (edge >= 0.2 * 24 * 10.0) & (k * r >= 40) & (k * r < 80)
    ref, _, _ = CF.homogeneous_go_green_3d_vti(X[sel], Y[sel], Z[sel], om, m['vp0'], m['vs0'], m['eps'], m['delta'])
    assert np.linalg.norm(u[sel] - ref) / np.linalg.norm(ref) < 5e-2
