"""Medium preparation (oracle, float64).  Test infrastructure only.

Eq. 5 defines the density-normalised elastic moduli a_ijkl = c_ijkl / rho.  The ray velocities need
their spatial gradient, taken here with numpy's second-order central differences (second-order
one-sided at the grid edges).
"""
from __future__ import annotations

import numpy as np

_VOIGT = np.array(((0, 5, 4), (5, 1, 3), (4, 3, 2)))


def voigt_matrix(c21):
    """(..., 21) upper-triangle Voigt list -> (..., 6, 6) symmetric stiffness matrix."""
    c21 = np.asarray(c21, np.float64)
    C = np.zeros(c21.shape[:-1] + (6, 6))
    iu = np.triu_indices(6)
    C[..., iu[0], iu[1]] = c21
    C[..., iu[1], iu[0]] = c21
    return C


def stiffness_tensor(c21):
    """(..., 21) Voigt list -> c_ijkl with shape (..., 3, 3, 3, 3)."""
    C = voigt_matrix(c21)
    return C[..., _VOIGT[:, :, None, None], _VOIGT[None, None, :, :]]


def is_positive_definite(c21):
    """Strain-energy positivity: every eigenvalue of the 6x6 Voigt matrix is > 0 (per node)."""
    return np.linalg.eigvalsh(voigt_matrix(c21)).min(axis=-1) > 0.0


def density_normalised(c21, rho):
    """Eq. 5: a_ijkl = c_ijkl / rho, per node."""
    rho = np.asarray(rho, np.float64)
    return stiffness_tensor(c21) / rho[..., None, None, None, None]


def medium_2d(problem):
    """a (nz, nx, 3,3,3,3), da/dx and da/dz (same shape), rho (nz, nx) for a 2-D problem."""
    nz, nx = problem.nz, problem.nx
    c21 = np.asarray(problem.c21, np.float64).reshape(nz, nx, 21)
    rho = np.asarray(problem.rho, np.float64).reshape(nz, nx)
    a = density_normalised(c21, rho)
    da_dz = np.gradient(a, problem.hz, axis=0, edge_order=2) if nz >= 3 else np.zeros_like(a)
    da_dx = np.gradient(a, problem.hx, axis=1, edge_order=2) if nx >= 3 else np.zeros_like(a)
    return a, da_dx, da_dz, rho


def bilinear_at(field, problem, x, z):
    """Bilinear interpolation of a node field (nz, nx, ...) at the point (x, z)."""
    fx = (x - problem.origin[0]) / problem.hx
    fz = (z - problem.origin[1]) / problem.hz
    ix = int(np.clip(np.floor(fx), 0, problem.nx - 2))
    iz = int(np.clip(np.floor(fz), 0, problem.nz - 2))
    tx = fx - ix
    tz = fz - iz
    return ((1 - tz) * ((1 - tx) * field[iz, ix] + tx * field[iz, ix + 1])
            + tz * ((1 - tx) * field[iz + 1, ix] + tx * field[iz + 1, ix + 1]))


def medium_3d(problem):
    """a (nz, ny, nx, 3,3,3,3), da/dx, da/dy, da/dz (same shape), rho (nz, ny, nx) for a 3-D problem
    (second-order central differences, second-order one-sided at the edges)."""
    nz, ny, nx = problem.nz, problem.ny, problem.nx
    c21 = np.asarray(problem.c21, np.float64).reshape(nz, ny, nx, 21)
    rho = np.asarray(problem.rho, np.float64).reshape(nz, ny, nx)
    a = density_normalised(c21, rho)
    da_dz = np.gradient(a, problem.hz, axis=0, edge_order=2)
    da_dy = np.gradient(a, problem.hy, axis=1, edge_order=2)
    da_dx = np.gradient(a, problem.hx, axis=2, edge_order=2)
    return a, da_dx, da_dy, da_dz, rho


def trilinear_at(field, problem, x, y, z):
    """Trilinear interpolation of a node field (nz, ny, nx, ...) at the point (x, y, z)."""
    o = problem.origin
    f = [(x - o[0]) / problem.hx, (y - o[1]) / problem.hy, (z - o[2]) / problem.hz]
    n = [problem.nx, problem.ny, problem.nz]
    i = [int(np.clip(np.floor(f[d]), 0, n[d] - 2)) for d in range(3)]
    t = [f[d] - i[d] for d in range(3)]
    out = 0.0
    for dz in (0, 1):
        for dy in (0, 1):
            for dx in (0, 1):
                w = ((t[0] if dx else 1 - t[0]) * (t[1] if dy else 1 - t[1]) * (t[2] if dz else 1 - t[2]))
                out = out + w * field[i[2] + dz, i[1] + dy, i[0] + dx]
    return out
