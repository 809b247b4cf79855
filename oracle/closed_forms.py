"""Exact references that pin the oracle (test infrastructure only).

None of these routines shares arithmetic with the Eulerian oracle they check:
* qP phase velocity of an isotropic medium: sqrt((lambda + 2 mu)/rho);
* qP phase velocity of a VTI medium in Thomsen's parameters (exact formula, Tsvankin 1996), its
  group velocity V = v n + (dv/dtheta) n_theta by complex-step differentiation;
* the 2-D Helmholtz Green's function (i/4) H0^(1)(k r) (scipy's Hankel function);
* the steady-state labels of a homogeneous medium (straight rays from the source);
* the geometrical-optics Green's function of a homogeneous anisotropic medium, from the stationary
  phase evaluation of its plane-wave (Fourier) representation;
* 3-D: the steady-state labels of a homogeneous medium, the Gaussian curvature of the VTI slowness
  surface (from Thomsen's exact phase velocity) and the GO Green's function built on it, and the
  continuous Gaussian-beam integral of analytic beams in a homogeneous isotropic medium.
"""
from __future__ import annotations

import math

import numpy as np


def isotropic_velocity(lam, mu, rho):
    return np.sqrt((lam + 2.0 * mu) / rho)


def thomsen_vti_phase_velocity(theta, vp0, vs0, eps, delta):
    """Exact qP phase velocity of a VTI medium (theta from the symmetry axis):
    v^2/Vp0^2 = 1 + eps s^2 - f/2 + f/2 sqrt((1 + 2 eps s^2 / f)^2 - 2 (eps - delta) sin^2(2 theta)/f),
    f = 1 - Vs0^2/Vp0^2, s = sin theta.  Works for complex theta (complex-step derivatives)."""
    s2 = np.sin(theta) ** 2
    f = 1.0 - (vs0 / vp0) ** 2
    root = np.sqrt((1.0 + 2.0 * eps * s2 / f) ** 2 - 2.0 * (eps - delta) * np.sin(2.0 * theta) ** 2 / f)
    return vp0 * np.sqrt(1.0 + eps * s2 - 0.5 * f + 0.5 * f * root)


def vti_group_velocity(theta, vp0, vs0, eps, delta):
    """Group velocity (x, z components) at phase angle theta: V = v n + v_theta n_theta,
    n = (sin, cos), n_theta = (cos, -sin); v_theta by complex-step differentiation."""
    theta = np.asarray(theta, np.float64)
    hstep = 1e-30
    v = thomsen_vti_phase_velocity(theta, vp0, vs0, eps, delta)
    vt = np.imag(thomsen_vti_phase_velocity(theta + 1j * hstep, vp0, vs0, eps, delta)) / hstep
    Vx = v * np.sin(theta) + vt * np.cos(theta)
    Vz = v * np.cos(theta) - vt * np.sin(theta)
    return v, Vx, Vz


def hankel_green_2d(k, r):
    """(i/4) H0^(1)(k r): outgoing 2-D Green's function of (Laplacian + k^2) u = -delta."""
    from scipy.special import hankel1
    return 0.25j * hankel1(0, k * r)


def group_angle_inverse(psi_target, phase_to_group, n_grid=20001):
    """Phase angle whose group direction is psi_target (monotone map, bracketed + bisection)."""
    psi_target = np.atleast_1d(np.asarray(psi_target, np.float64))
    th = np.linspace(-math.pi, math.pi, n_grid)
    g = phase_to_group(th)
    g = np.unwrap(g)
    out = np.empty_like(psi_target)
    for i, t in enumerate(psi_target):
        tt = (t - g[0]) % (2 * math.pi) + g[0]
        j = np.searchsorted(g, tt)
        j = min(max(j, 1), n_grid - 1)
        lo, hi = th[j - 1], th[j]
        for _ in range(60):
            mid = 0.5 * (lo + hi)
            gm = (phase_to_group(np.array([mid]))[0] - tt + math.pi) % (2 * math.pi) - math.pi
            if gm < 0:
                lo = mid
            else:
                hi = mid
        out[i] = 0.5 * (lo + hi)
    return out


def homogeneous_go_green(x, z, xs, zs, omega, v_of, V_of, c_ref):
    """Geometrical-optics Green's function of a homogeneous anisotropic medium (acoustic scaling).

    The plane-wave integral int d^2k e^{i k.x} c_ref^2 / (lambda(k) - omega^2) / (2 pi)^2 has the
    far field c_ref^2 e^{i pi/4} e^{i omega T} / (v(psi*) sqrt(8 pi omega J_t)), where psi* is the
    phase angle whose group velocity points at the receiver, T = |x - x_s| / |V(psi*)| and
    J_t = T (dV/dpsi x V) is the ray Jacobian in (take-off angle, traveltime).
    v_of(theta) -> phase velocity; V_of(theta) -> (Vx, Vz).
    """
    dx, dz = x - xs, z - zs
    r = np.hypot(dx, dz)
    psi_g = np.arctan2(dx, dz)
    phase_to_group = lambda th: np.arctan2(*V_of(th))
    th = group_angle_inverse(psi_g.ravel(), phase_to_group).reshape(np.shape(psi_g))
    Vx, Vz = V_of(th)
    Vn = np.hypot(Vx, Vz)
    T = r / Vn
    e = 1e-6
    Vxp, Vzp = V_of(th + e)
    Vxm, Vzm = V_of(th - e)
    dVx, dVz = (Vxp - Vxm) / (2 * e), (Vzp - Vzm) / (2 * e)
    beta = dVx * Vz - dVz * Vx
    Jt = T * beta
    return c_ref ** 2 * np.exp(1j * (omega * T + math.pi / 4)) / (v_of(th) * np.sqrt(8 * math.pi * omega * Jt)), T, th


def homogeneous_labels(theta, X, Z, ghat, p, R_sigma):
    """Steady-state labels of a homogeneous medium with the source at the origin.

    theta: (nth,) phase angles; X, Z: node offsets from the source (nz, nx); ghat (nth, 2) unit
    group directions; p (nth, 2) slownesses; R_sigma the radius of the source manifold's disc.
    A ray through (x, theta) is the straight line along ghat(theta): b = x x ghat (its distance from
    the source at closest approach), Th = theta, tau = p(theta) . x, and q = 1 when it passed its
    closest approach within R_sigma of the source (|b| <= R_sigma, x downstream of the foot point).
    """
    gx = ghat[:, 0][:, None, None]
    gz = ghat[:, 1][:, None, None]
    L = X[None] * gx + Z[None] * gz
    b = X[None] * gz - Z[None] * gx
    q = ((np.abs(b) <= R_sigma) & (L >= 0)).astype(np.float64)
    tau = p[:, 0][:, None, None] * X[None] + p[:, 1][:, None, None] * Z[None]
    Th = np.broadcast_to(theta[:, None, None], tau.shape).copy()
    return dict(b=b, q=q, Th=Th, tau=tau)


# ------------------------------------------------------------------------------------------------
# 3-D

def homogeneous_labels_3d(S):
    """Steady-state labels of a homogeneous medium on every cell of a Setup3D: straight rays along
    the source group direction g(n) of each direction cell, b = d - (d . g) g, n0 = n, tau = p . d,
    q = 1 on the frozen manifold and on rays that passed their closest approach within R_Sigma
    (|b| <= R_Sigma and not approaching, with the frozen manifold's rule for d . g at rounding
    level)."""
    from .christoffel import source_quantities_3d
    o = S.p.origin
    X = (np.arange(S.nx) * S.hx + o[0] - S.xs[0])[None, None, None, None, :]
    Y = (np.arange(S.ny) * S.hy + o[1] - S.xs[1])[None, None, None, :, None]
    Z = (np.arange(S.nz) * S.hz + o[2] - S.xs[2])[None, None, :, None, None]
    g = [S.gs[..., c][:, :, None, None, None] for c in range(3)]
    n = [S.n[..., c][:, :, None, None, None] for c in range(3)]
    v = source_quantities_3d(S.a_s, S.n)[0][:, :, None, None, None]
    L = X * g[0] + Y * g[1] + Z * g[2]
    b = [X - L * g[0], Y - L * g[1], Z - L * g[2]]
    bn = np.sqrt(b[0] ** 2 + b[1] ** 2 + b[2] ** 2)
    shape = np.broadcast(X, Y, Z, g[0]).shape
    r2 = Z * Z + Y * Y + X * X
    approach = (L < 0) & (L * L > 1e-24 * r2)   # the frozen manifold's tie rule
    q = (S.frozen | ((bn <= S.R_sigma) & ~approach)).astype(np.float64)
    out = {'bx': np.broadcast_to(b[0], shape).copy(), 'by': np.broadcast_to(b[1], shape).copy(),
           'bz': np.broadcast_to(b[2], shape).copy(), 'q': q,
           'tau': np.broadcast_to((n[0] * X + n[1] * Y + n[2] * Z) / v, shape).copy()}
    for c, f in enumerate(('n0x', 'n0y', 'n0z')):
        out[f] = np.broadcast_to(n[c], shape).copy()
    return out


def vti_slowness_gaussian_curvature(theta, vp0, vs0, eps, delta):
    """Gaussian curvature of the qP slowness surface of a VTI medium at polar phase angle theta.

    The surface is one of revolution about z with the meridian r(theta) = 1/v(theta) (polar form,
    Thomsen's exact v); its curvatures are the meridian's, |r^2 + 2 r'^2 - r r''| / (r^2 + r'^2)^1.5,
    and the parallel's, g_h / p_h (horizontal component of the unit normal, i.e. of the group
    direction, over the distance from the axis; equal to the meridian's on the axis)."""
    theta = np.asarray(theta, np.float64)
    hstep = 1e-30
    r_of = lambda t: 1.0 / thomsen_vti_phase_velocity(t, vp0, vs0, eps, delta)
    r = r_of(theta)
    d1 = lambda t: np.imag(r_of(t + 1j * hstep)) / hstep
    r1 = d1(theta)
    e = 1e-5
    r2 = (d1(theta + e) - d1(theta - e)) / (2 * e)
    km = np.abs(r ** 2 + 2 * r1 ** 2 - r * r2) / (r ** 2 + r1 ** 2) ** 1.5
    v, Vx, Vz = vti_group_velocity(theta, vp0, vs0, eps, delta)
    gh = np.abs(Vx) / np.hypot(Vx, Vz)
    ph = np.abs(np.sin(theta)) / v
    with np.errstate(divide='ignore', invalid='ignore'):
        kp = np.where(ph > 1e-12, gh / ph, km)
    return km * kp


def homogeneous_go_green_3d_vti(X, Y, Z, omega, vp0, vs0, eps, delta):
    """Geometrical-optics Green's function of a homogeneous VTI medium, acoustic scaling, source at
    the origin: the stationary-phase evaluation of the plane-wave integral,
        u = c_ref^2 exp(i omega T) / (4 pi sqrt(K) |V| r),  T = r / |V|,
    with p* the slowness whose group velocity V points at the receiver and K the Gaussian curvature
    of the slowness surface there (c_ref = vp0).  Returns u, T and |u|."""
    rho_h = np.hypot(X, Y)
    r = np.sqrt(X ** 2 + Y ** 2 + Z ** 2)
    psi = np.arctan2(rho_h, Z)
    phase_to_group = lambda th: np.arctan2(*vti_group_velocity(th, vp0, vs0, eps, delta)[1:])
    th = group_angle_inverse(psi.ravel(), phase_to_group).reshape(np.shape(psi))
    _, Vx, Vz = vti_group_velocity(th, vp0, vs0, eps, delta)
    Vn = np.hypot(Vx, Vz)
    K = vti_slowness_gaussian_curvature(th, vp0, vs0, eps, delta)
    T = r / Vn
    amp = vp0 ** 2 / (4 * math.pi * np.sqrt(K) * Vn * r)
    return amp * np.exp(1j * omega * T), T, amp


def isotropic_beam_integral_3d(X, Y, Z, omega, w0, v, r_min, n_theta=240, n_phi=480, box=None):
    """The continuous Gaussian-beam integral of the 3-D superposition in a homogeneous isotropic
    medium (source at the origin), by direct quadrature over take-off directions n (midpoint rule,
    n_theta x n_phi cells), for receivers (X, Y, Z) (1-D arrays).

    Each grid-plane family a (normal e_a) contributes, for every ray that crosses the receiver's
    plane outward at s = (x . e_a)/(n . e_a) > r_min, the analytic paraxial beam of that ray
        W (n . e_a)^2 exp(i omega (s/v + n . delta / v + m(s) (|delta|^2 - (n . delta)^2) / 2)) / (1 + v s M0)
    with delta = x - s n, M0 = 2 i/(omega w0^2), m(s) = M0 / (1 + v s M0) (the wavefront Hessian of
    a beam of 1/e half-width w0 at the source), W = i omega / (8 pi^2 v).  As omega grows with
    omega w0^2 fixed relative to the distance this tends to exp(i k r)/(4 pi r).  box = (lo, hi)
    (3-vectors) keeps only beams whose centre s n lies inside the box (a finite grid)."""
    th = (np.arange(n_theta) + 0.5) * np.pi / n_theta
    ph = (np.arange(n_phi) + 0.5) * 2 * np.pi / n_phi
    TH, PH = np.meshgrid(th, ph, indexing='ij')
    n = np.stack([np.sin(TH) * np.cos(PH), np.sin(TH) * np.sin(PH), np.cos(TH)], -1).reshape(-1, 3)
    dW = (np.sin(TH) * (np.pi / n_theta) * (2 * np.pi / n_phi)).reshape(-1)
    M0 = 2j / (omega * w0 ** 2)
    W = 1j * omega / (8 * np.pi ** 2 * v)
    xr = np.stack([np.ravel(X), np.ravel(Y), np.ravel(Z)], -1)
    out = np.zeros(len(xr), np.complex128)
    for i, x in enumerate(xr):
        acc = 0.0
        for a in range(3):
            na = n[:, a]
            with np.errstate(divide='ignore', invalid='ignore'):
                s = x[a] / na
            ok = np.isfinite(s) & (s > r_min)
            if box is not None:
                xc = np.where(ok[:, None], s[:, None] * n, 0.0)
                ok &= np.all((xc >= np.asarray(box[0]) - 1e-9) & (xc <= np.asarray(box[1]) + 1e-9), axis=-1)
            nn, sa, dw = n[ok], s[ok], dW[ok]
            d = x[None, :] - sa[:, None] * nn
            nd = np.einsum('ij,ij->i', nn, d)
            m = M0 / (1 + v * sa * M0)
            ph_ = omega * (sa / v + nd / v + 0.5 * m * (np.einsum('ij,ij->i', d, d) - nd ** 2))
            acc = acc + np.sum(dw * nn[:, a] ** 2 * W * np.exp(1j * ph_) / (1 + v * sa * M0))
        out[i] = acc
    return out.reshape(np.shape(X))
