"""Exact references that pin the oracle (test infrastructure only).

None of these routines shares arithmetic with the Eulerian oracle they check:
* qP phase velocity of an isotropic medium: sqrt((lambda + 2 mu)/rho);
* qP phase velocity of a VTI medium in Thomsen's parameters (exact formula, Tsvankin 1996), its
  group velocity V = v n + (dv/dtheta) n_theta by complex-step differentiation;
* the 2-D Helmholtz Green's function (i/4) H0^(1)(k r) (scipy's Hankel function);
* the steady-state labels of a homogeneous medium (straight rays from the source);
* the geometrical-optics Green's function of a homogeneous anisotropic medium, from the stationary
  phase evaluation of its plane-wave (Fourier) representation.
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
