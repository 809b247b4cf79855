"""Christoffel matrix, qP eigenpair and ray velocities (oracle, float64).  Test infrastructure only.

Eq. 4: Gamma_ik(x, p) = a_ijkl p_j p_l.  Eq. 3: (Gamma_ik - delta_ik) U_k = 0, i.e. on the slowness
surface the qP eigenvalue of Gamma(x, p) equals 1.  Eq. 7 parametrises the slowness by the phase
angle theta measured from +z: p = n(theta) / v(x, theta) with n = (sin theta, 0, cos theta), so
v^2 = lambda_max(Gamma(x, n)) and the eigenvector g is the qP polarisation.

The ray system of Eqs. 8-12 is taken in its Hamiltonian form with H(x, p) = (lambda_qP(Gamma(x, p))
- 1) / 2, for which the parameter is the traveltime (dT/dt = p . dH/dp = 1):
    dx_i/dt = V_i = a_ijkl p_l g_j g_k                     (group velocity)
    dp_i/dt = -1/2 (d_i a_jkln) p_k p_n g_j g_l
and the phase angle moves as dtheta/dt = v (cos theta dp_x/dt - sin theta dp_z/dt), which follows
from theta = atan2(p_x, p_z) and |p| = 1/v.  (Eq. 11 as printed has a sign slip in its second line
and Eq. 12 drops an argument; the Hamiltonian form above is the one used.)
"""
from __future__ import annotations

import numpy as np


def direction_2d(theta):
    """n(theta) = (sin theta, 0, cos theta) for phase angles measured from +z toward +x (Eq. 7)."""
    theta = np.asarray(theta, np.float64)
    return np.stack([np.sin(theta), np.zeros_like(theta), np.cos(theta)], axis=-1)


def christoffel(a, n):
    """Eq. 4 with a unit direction: Gamma_ik = a_ijkl n_j n_l (broadcast over leading axes)."""
    return np.einsum('...ijkl,...j,...l->...ik', a, n, n, optimize=True)


def qp_eigen(gamma):
    """Largest eigenvalue and its unit eigenvector of the symmetric 3x3 Christoffel matrix (Eq. 3).

    The sign of g is fixed by g . (largest-|component| axis) >= 0; velocities are quadratic in g.
    """
    w, vec = np.linalg.eigh(gamma)
    lam = w[..., -1]
    g = vec[..., :, -1]
    k = np.argmax(np.abs(g), axis=-1)
    s = np.sign(np.take_along_axis(g, k[..., None], axis=-1))
    s[s == 0] = 1.0
    return lam, g * s


def phase_velocity(a, n):
    """v(x, n) = sqrt(lambda_qP(Gamma(x, n)))."""
    lam, _ = qp_eigen(christoffel(a, n))
    return np.sqrt(lam)


def ray_velocity(a, da, n):
    """Group velocity V (3-vector) and dp/dt (one entry per gradient direction) at direction n.

    a: (..., 3,3,3,3); da: list of gradient tensors [d a / d x_d]; n: (..., 3) unit directions.
    Returns v, g, V, [dp_d/dt].
    """
    lam, g = qp_eigen(christoffel(a, n))
    v = np.sqrt(lam)
    p = n / v[..., None]
    ap = np.einsum('...ijkl,...l->...ijk', a, p)
    V = np.einsum('...ijk,...j,...k->...i', ap, g, g)
    # dp_i/dt = -1/2 g_j (d_i a_jkln p_k p_n) g_l = -1/2 g . Gamma(d_i a, p) . g
    pdot = [-0.5 * np.einsum('...jl,...j,...l->...', christoffel(d, p), g, g) for d in da]
    return v, g, V, pdot


def velocity_field_2d(a, da_dx, da_dz, n_theta):
    """Characteristic velocities of the reduced phase space (x, z, theta) on every cell.

    Returns dict of arrays shaped (n_theta, nz, nx): Vx, Vz, thetadot, v (phase velocity),
    pdx, pdz (dp/dt components).
    """
    nz, nx = a.shape[:2]
    out = {k: np.empty((n_theta, nz, nx)) for k in ('Vx', 'Vz', 'thetadot', 'v', 'pdx', 'pdz')}
    for k in range(n_theta):
        th = 2.0 * np.pi * k / n_theta
        n = np.broadcast_to(direction_2d(th), (nz, nx, 3))
        v, g, V, (pdx, pdz) = ray_velocity(a, [da_dx, da_dz], n)
        out['Vx'][k] = V[..., 0]
        out['Vz'][k] = V[..., 2]
        out['v'][k] = v
        out['pdx'][k] = pdx
        out['pdz'][k] = pdz
        out['thetadot'][k] = v * (np.cos(th) * pdx - np.sin(th) * pdz)
    return out


def source_quantities(a_s, theta):
    """Source-medium phase velocity, group velocity and unit group direction at phase angles theta.

    a_s: (3,3,3,3) moduli at the source; theta: array of angles.  Returns v (..), V (.., 2: x, z),
    |V| (..), ghat (.., 2).
    """
    theta = np.asarray(theta, np.float64)
    n = direction_2d(theta)
    lam, g = qp_eigen(christoffel(a_s, n))
    v = np.sqrt(lam)
    p = n / v[..., None]
    V = np.einsum('ijkl,...l,...j,...k->...i', a_s, p, g, g)
    V2 = np.stack([V[..., 0], V[..., 2]], axis=-1)
    Vn = np.linalg.norm(V2, axis=-1)
    return v, V2, Vn, V2 / Vn[..., None]
