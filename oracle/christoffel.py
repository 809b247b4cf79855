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


def velocity_field_2d(a, da_dx, da_dz, n_theta, ks=None):
    """Characteristic velocities of the reduced phase space (x, z, theta) on every cell.

    Returns dict of arrays shaped (n_theta, nz, nx): Vx, Vz, thetadot, v (phase velocity),
    pdx, pdz (dp/dt components).  With ks (a sequence of angle indices) only those planes are
    computed and the arrays are shaped (len(ks), nz, nx); planes are independent of each other.
    """
    nz, nx = a.shape[:2]
    ks = range(n_theta) if ks is None else list(ks)
    out = {k: np.empty((len(ks), nz, nx)) for k in ('Vx', 'Vz', 'thetadot', 'v', 'pdx', 'pdz')}
    for j, k in enumerate(ks):
        th = 2.0 * np.pi * k / n_theta
        n = np.broadcast_to(direction_2d(th), (nz, nx, 3))
        v, g, V, (pdx, pdz) = ray_velocity(a, [da_dx, da_dz], n)
        out['Vx'][j] = V[..., 0]
        out['Vz'][j] = V[..., 2]
        out['v'][j] = v
        out['pdx'][j] = pdx
        out['pdz'][j] = pdz
        out['thetadot'][j] = v * (np.cos(th) * pdx - np.sin(th) * pdz)
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


# ----------------------------------------------------------------------------------------------
# 3-D: phase directions n = (sin th cos ph, sin th sin ph, cos th).  With dn/dt = v (I - n n^T) dp/dt
# (p = n / v on the slowness surface), the direction angles move as
#   dth/dt = v n_th . dp/dt,   dph/dt = v e_ph . dp/dt / sin th,
# n_th = (cos th cos ph, cos th sin ph, -sin th), e_ph = (-sin ph, cos ph, 0).

def direction_3d(theta, phi):
    theta = np.asarray(theta, np.float64)
    phi = np.asarray(phi, np.float64)
    return np.stack([np.sin(theta) * np.cos(phi), np.sin(theta) * np.sin(phi),
                     np.cos(theta) * np.ones_like(phi)], axis=-1)


def angle_grid_3d(n_theta, n_phi):
    """Polar angles at cell centres th_j = (j + 1/2) pi / n_theta; azimuths ph_k = 2 pi k / n_phi."""
    return (np.arange(n_theta) + 0.5) * np.pi / n_theta, 2.0 * np.pi * np.arange(n_phi) / n_phi


def velocity_field_3d(a, da_dx, da_dy, da_dz, n_theta, n_phi):
    """Characteristic velocities of the 5-D phase space (x, y, z, th, ph) on every cell.

    Returns dict of arrays shaped (n_phi, n_theta, nz, ny, nx): Vx, Vy, Vz, thetadot, phidot,
    v (phase velocity), pdx, pdy, pdz (dp/dt components).
    """
    spatial = a.shape[:3]
    th, ph = angle_grid_3d(n_theta, n_phi)
    keys = ('Vx', 'Vy', 'Vz', 'thetadot', 'phidot', 'v', 'pdx', 'pdy', 'pdz')
    out = {k: np.empty((n_phi, n_theta) + spatial) for k in keys}
    for k in range(n_phi):
        for j in range(n_theta):
            n = np.broadcast_to(direction_3d(th[j], ph[k]), spatial + (3,))
            v, g, V, pd = ray_velocity(a, [da_dx, da_dy, da_dz], n)
            n_th = np.array([np.cos(th[j]) * np.cos(ph[k]), np.cos(th[j]) * np.sin(ph[k]), -np.sin(th[j])])
            e_ph = np.array([-np.sin(ph[k]), np.cos(ph[k]), 0.0])
            out['Vx'][k, j] = V[..., 0]
            out['Vy'][k, j] = V[..., 1]
            out['Vz'][k, j] = V[..., 2]
            out['v'][k, j] = v
            out['pdx'][k, j], out['pdy'][k, j], out['pdz'][k, j] = pd
            out['thetadot'][k, j] = v * (n_th[0] * pd[0] + n_th[1] * pd[1] + n_th[2] * pd[2])
            out['phidot'][k, j] = v * (e_ph[0] * pd[0] + e_ph[1] * pd[1]) / np.sin(th[j])
    return out


def source_quantities_3d(a_s, n):
    """Source-medium phase velocity v, group velocity V (.., 3), |V| and unit group direction at
    unit phase directions n (.., 3)."""
    lam, g = qp_eigen(christoffel(a_s, n))
    v = np.sqrt(lam)
    p = n / v[..., None]
    V = np.einsum('ijkl,...l,...j,...k->...i', a_s, p, g, g)
    Vn = np.linalg.norm(V, axis=-1)
    return v, V, Vn, V / Vn[..., None]
