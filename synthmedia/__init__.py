"""Seeded synthetic media and workloads for the anisotropic Eulerian Gaussian beam solver.

This module builds INPUTS only: elastic stiffness fields c_IJ(x) (21 Voigt constants per node,
upper triangle row by row: C11 C12 C13 C14 C15 C16 C22 C23 C24 C25 C26 C33 C34 C35 C36 C44 C45
C46 C55 C56 C66, in Pa), densities rho(x) (kg/m^3), grids, source positions, angular sampling,
frequencies and step counts.  It holds none of the method's arithmetic (no Christoffel solve, no
ray or level-set computation), so both the CUDA library and the independent FP64 oracle can take
their inputs from here.

Coordinates: x is the horizontal axis, z points down (depth); nodes sit at origin + i*h.  2-D grids
are stored z-major with x fastest (node index = iz*nx + ix).

Workloads (all synthetic, seeded with numpy PCG64):
  * ``vti_homogeneous``    homogeneous VTI medium from Thomsen parameters (the 64x64x64 case)
  * ``tti_heterogeneous``  2-D TTI medium: Vp0 = 2000 + z with two Gaussian +-15 % anomalies,
                           Vs0 = Vp0/1.8, scalar epsilon/delta drawn once per medium, tilt from
                           Gaussian-filtered noise scaled to +-30 deg, Gardner density
  * ``isotropic_homogeneous``  Lame medium (closed-form pins)
  * ``batched_instances``  uneven TTI instances (sizes, angle counts, frequencies drawn per instance)
  * ``request_stream``     Poisson arrival stream of solve requests
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field
from typing import List, Optional, Tuple

import numpy as np

# Voigt index of the tensor index pair (i, j), 0-based: 11->0 22->1 33->2 23->3 13->4 12->5
_VOIGT = ((0, 5, 4), (5, 1, 3), (4, 3, 2))


def voigt21_index(I: int, J: int) -> int:
    """Position of C_IJ (0-based Voigt indices, any order) in the 21-entry upper-triangle list."""
    if I > J:
        I, J = J, I
    return I * 6 - I * (I - 1) // 2 + (J - I)


def thomsen_vti_voigt(vp0, vs0, eps, delta, rho, gamma=0.0):
    """Stiffness (6x6 Voigt, Pa) of a VTI medium from Thomsen's parameters (Thomsen 1986).

    c33 = rho Vp0^2, c55 = c44 = rho Vs0^2, c11 = c33 (1 + 2 eps), c66 = c44 (1 + 2 gamma),
    (c13 + c55)^2 = (c33 - c55) (c33 (1 + 2 delta) - c55), c12 = c11 - 2 c66.
    Broadcasts over array arguments; returns shape (..., 6, 6).
    """
    vp0, vs0, eps, delta, rho, gamma = np.broadcast_arrays(
        *[np.asarray(a, dtype=np.float64) for a in (vp0, vs0, eps, delta, rho, gamma)])
    c33 = rho * vp0 ** 2
    c55 = rho * vs0 ** 2
    c11 = c33 * (1.0 + 2.0 * eps)
    c66 = c55 * (1.0 + 2.0 * gamma)
    c13 = np.sqrt((c33 - c55) * (c33 * (1.0 + 2.0 * delta) - c55)) - c55
    c12 = c11 - 2.0 * c66
    C = np.zeros(vp0.shape + (6, 6))
    C[..., 0, 0] = C[..., 1, 1] = c11
    C[..., 2, 2] = c33
    C[..., 0, 1] = C[..., 1, 0] = c12
    C[..., 0, 2] = C[..., 2, 0] = C[..., 1, 2] = C[..., 2, 1] = c13
    C[..., 3, 3] = C[..., 4, 4] = c55
    C[..., 5, 5] = c66
    return C


def isotropic_voigt(lam, mu):
    """Stiffness (6x6 Voigt) of an isotropic medium from the Lame constants."""
    lam, mu = np.broadcast_arrays(np.asarray(lam, np.float64), np.asarray(mu, np.float64))
    C = np.zeros(lam.shape + (6, 6))
    for i in range(3):
        for j in range(3):
            C[..., i, j] = lam
        C[..., i, i] = lam + 2 * mu
        C[..., 3 + i, 3 + i] = mu
    return C


def _voigt_to_tensor(C):
    c = np.empty(C.shape[:-2] + (3, 3, 3, 3))
    for i in range(3):
        for j in range(3):
            for k in range(3):
                for l in range(3):
                    c[..., i, j, k, l] = C[..., _VOIGT[i][j], _VOIGT[k][l]]
    return c


def _tensor_to_voigt(c):
    C = np.empty(c.shape[:-4] + (6, 6))
    for i in range(3):
        for j in range(3):
            for k in range(3):
                for l in range(3):
                    C[..., _VOIGT[i][j], _VOIGT[k][l]] = c[..., i, j, k, l]
    return C


def rotate_voigt_about_y(C, tilt):
    """Rotate a stiffness so that its z symmetry axis tilts by ``tilt`` (rad) from +z toward +x."""
    tilt = np.asarray(tilt, np.float64)
    ct, st = np.cos(tilt), np.sin(tilt)
    R = np.zeros(tilt.shape + (3, 3))
    R[..., 0, 0] = ct
    R[..., 0, 2] = st
    R[..., 1, 1] = 1.0
    R[..., 2, 0] = -st
    R[..., 2, 2] = ct
    # Bond's 6x6 form of c'_ijkl = R_ip R_jq R_kr R_ls c_pqrs: C' = M C M^T with the stress
    # transformation M_IJ = R_ik R_jl + R_il R_jk (k != l) or R_ik R_jk (k = l), I ~ (i, j), J ~ (k, l)
    pairs = [(0, 0), (1, 1), (2, 2), (1, 2), (0, 2), (0, 1)]
    M = np.empty(tilt.shape + (6, 6))
    for I, (i, j) in enumerate(pairs):
        for J, (k, l) in enumerate(pairs):
            M[..., I, J] = R[..., i, k] * R[..., j, l]
            if k != l:
                M[..., I, J] += R[..., i, l] * R[..., j, k]
    C = np.broadcast_to(np.asarray(C, np.float64), tilt.shape + (6, 6))
    MC = sum(M[..., :, j, None] * C[..., None, j, :] for j in range(6))
    return sum(MC[..., :, k, None] * M[..., None, :, k] for k in range(6))


def voigt_to_c21(C):
    """(..., 6, 6) symmetric Voigt matrix -> (..., 21) upper triangle, row by row."""
    iu = np.triu_indices(6)
    return C[..., iu[0], iu[1]]


def c21_to_voigt(c21):
    """(..., 21) upper triangle -> (..., 6, 6) symmetric Voigt matrix."""
    c21 = np.asarray(c21, np.float64)
    C = np.zeros(c21.shape[:-1] + (6, 6))
    iu = np.triu_indices(6)
    C[..., iu[0], iu[1]] = c21
    C[..., iu[1], iu[0]] = c21
    return C


def gardner_density(vp):
    """Gardner's relation rho = 310 Vp^0.25 (kg/m^3, Vp in m/s)."""
    return 310.0 * np.asarray(vp, np.float64) ** 0.25


def _gaussian_filter(a, sigma_cells):
    from scipy.ndimage import gaussian_filter
    return gaussian_filter(a, sigma=sigma_cells, mode='reflect')


def _smooth_uniform(rng, n, sigma_cells, lo, hi):
    """An n x n smooth random field with values spread uniformly over [lo, hi]: white noise filtered
    by a Gaussian, standardised, and mapped through the standard normal distribution function."""
    from scipy.special import ndtr
    f = _gaussian_filter(rng.standard_normal((n, n)), sigma_cells)
    f = (f - f.mean()) / f.std()
    return lo + (hi - lo) * ndtr(f)


@dataclass
class Problem2D:
    """One 2-D solve request: medium on an nz x nx node grid plus the source description."""
    name: str
    nx: int
    nz: int
    hx: float
    hz: float
    c21: np.ndarray           # (nz*nx, 21) float32, Pa
    rho: np.ndarray           # (nz*nx,) float32, kg/m^3
    xs: Tuple[float, float]   # source (x, z), m
    n_theta: int
    freqs: List[float]        # Hz
    beam_width: float         # m
    steps: int
    cfl: float = 0.5
    r0: Optional[float] = None   # frozen source-ball radius (m); default 2*max(hx, hz)
    origin: Tuple[float, float] = (0.0, 0.0)
    R_sigma: Optional[float] = None   # closest-approach disc radius (m); default max(4 r0, min(L)/8)
    meta: dict = field(default_factory=dict)

    @property
    def omegas(self):
        return [2.0 * math.pi * f for f in self.freqs]

    @property
    def ball_radius(self):
        return self.r0 if self.r0 is not None else 2.0 * max(self.hx, self.hz)

    @property
    def cells(self):
        return self.nx * self.nz * self.n_theta


def _pack(C, rho):
    c21 = voigt_to_c21(C).reshape(-1, 21).astype(np.float32)
    return c21, np.asarray(rho, np.float64).reshape(-1).astype(np.float32)


def vti_homogeneous(n=64, h=10.0, n_theta=64, steps=150, vp0=3000.0, vs0=1500.0, eps=0.20,
                    delta=0.10, rho=2200.0, freqs=(15.0,), beam_width=50.0, cfl=0.5):
    """Homogeneous VTI medium (Thomsen Vp0, Vs0, eps, delta, rho), source at node (n/2, n/2).

    Defaults give the 64x64 grid at 10 m x 64 angles, 150 TVD-RK3 steps at CFL 0.5, 15 Hz, 50 m.
    """
    C = thomsen_vti_voigt(vp0, vs0, eps, delta, rho)
    C = np.broadcast_to(C, (n, n, 6, 6))
    c21, r = _pack(C, np.full((n, n), rho))
    xs = ((n // 2) * h, (n // 2) * h)
    return Problem2D('vti_homogeneous', n, n, h, h, c21, r, xs, n_theta, list(freqs), beam_width,
                     steps, cfl, meta=dict(vp0=vp0, vs0=vs0, eps=eps, delta=delta, rho=rho))


def isotropic_homogeneous(n=64, h=10.0, n_theta=64, steps=150, vp=3000.0, vs=1700.0, rho=2300.0,
                          freqs=(15.0,), beam_width=50.0, cfl=0.5, xs=None):
    """Homogeneous isotropic medium with P and S speeds vp, vs; source at the grid centre node."""
    mu = rho * vs ** 2
    lam = rho * vp ** 2 - 2 * mu
    C = np.broadcast_to(isotropic_voigt(lam, mu), (n, n, 6, 6))
    c21, r = _pack(C, np.full((n, n), rho))
    if xs is None:
        xs = ((n // 2) * h, (n // 2) * h)
    return Problem2D('isotropic_homogeneous', n, n, h, h, c21, r, xs, n_theta, list(freqs),
                     beam_width, steps, cfl, meta=dict(vp=vp, vs=vs, rho=rho))


def v_channel(nx=128, nz=64, h=10.0, n_theta=256, gradient=0.002, smoothing=30.0, vp0=3000.0,
              freqs=(50.0, 100.0, 200.0), beam_width=40.0, steps=200, cfl=0.5, x_source=100.0):
    """Isotropic low-velocity channel: vp = vp0 (1 + g (sqrt((z - z_c)^2 + a^2) - a)) about the
    middle row z_c (a V-shaped profile rounded over a), vs = vp / 1.8, rho 2300; the source on the
    channel axis at x_source.  Rays within the trapping angle oscillate about the axis and touch a
    caustic every half period, so arrivals late in the channel have passed two caustics and more."""
    x = np.arange(nx) * h
    z = np.arange(nz) * h
    Z, _ = np.meshgrid(z, x, indexing='ij')
    zc = z[nz // 2]
    vp = vp0 * (1.0 + gradient * (np.sqrt((Z - zc) ** 2 + smoothing ** 2) - smoothing))
    vs, rho = vp / 1.8, 2300.0
    mu = rho * vs ** 2
    C = isotropic_voigt(rho * vp ** 2 - 2 * mu, mu)
    c21, r = _pack(C, np.full((nz, nx), rho))
    return Problem2D('v_channel', nx, nz, h, h, c21, r, (float(x_source), float(zc)), n_theta,
                     list(freqs), beam_width, steps, cfl,
                     meta=dict(vp0=vp0, gradient=gradient, smoothing=smoothing))


def tti_heterogeneous(n=512, h=5.0, n_theta=256, steps=None, freqs=(10.0, 20.0, 40.0),
                      beam_width=None, seed=2, cfl=0.5, length=None):
    """2-D heterogeneous TTI medium.

    Vp0 = (2000 + 1.0 z) (1 + 0.15 G1 - 0.15 G2), G_k Gaussians of sigma 300 m centred uniformly in
    the middle 60 % of the domain; Vs0 = Vp0/1.8; epsilon and delta smooth fields with uniform
    marginals on [0, 0.25] and [-0.05, 0.15]: white noise filtered by a Gaussian of sigma 300 m,
    standardised and mapped through the normal distribution function onto the interval; tilt =
    white noise filtered by a Gaussian of sigma 200 m, scaled to a maximum of 30 deg; Gardner
    density.  ``length`` (m) fixes the physical extent so reduced grids
    (coarser h) describe the same medium; default n*h.  Source at the centre node.
    """
    rng = np.random.Generator(np.random.PCG64(seed))
    L = n * h if length is None else float(length)
    h = L / n
    x = np.arange(n) * h
    z = np.arange(n) * h
    Z, X = np.meshgrid(z, x, indexing='ij')
    centres = rng.uniform(0.2 * L, 0.8 * L, size=(2, 2))
    sig = 300.0
    g = [np.exp(-((X - cx) ** 2 + (Z - cz) ** 2) / (2 * sig ** 2)) for cx, cz in centres]
    vp0 = (2000.0 + 1.0 * Z) * (1.0 + 0.15 * g[0] - 0.15 * g[1])
    vs0 = vp0 / 1.8
    # two uniform draws that once set constant epsilon and delta: kept, so that the tilt field and
    # the velocity anomalies are those of that earlier form of the medium
    rng.uniform(0.0, 0.25)
    rng.uniform(-0.05, 0.15)
    noise = rng.standard_normal((n, n))
    tilt = _gaussian_filter(noise, 200.0 / h)
    tilt = tilt / np.max(np.abs(tilt)) * math.radians(30.0)
    eps = _smooth_uniform(rng, n, 300.0 / h, 0.0, 0.25)
    delta = _smooth_uniform(rng, n, 300.0 / h, -0.05, 0.15)
    rho = gardner_density(vp0)
    C = thomsen_vti_voigt(vp0, vs0, eps, delta, rho)
    C = rotate_voigt_about_y(C, tilt)
    c21, r = _pack(C, rho)
    xs = ((n // 2) * h, (n // 2) * h)
    if steps is None:
        steps = tti_default_steps(n, h)
    if beam_width is None:
        beam_width = 50.0
    return Problem2D('tti_heterogeneous', n, n, h, h, c21, r, xs, n_theta, list(freqs), beam_width,
                     steps, cfl, meta=dict(seed=seed, eps_mean=float(eps.mean()), delta_mean=float(delta.mean()),
                                           centres=centres.tolist(), length=L))


def triclinic_near_degenerate(n=32, h=10.0, n_theta=64, steps=40, freqs=(15.0,), beam_width=50.0, cfl=0.5):
    """Homogeneous triclinic medium whose qP eigenvalue nearly meets the next one in the x-z plane.

    Voigt matrix C = B B^T + 0.05 I with B a 6 x 6 standard normal draw of PCG64 seed 39760, scaled
    to C33 = rho (3000 m/s)^2, rho = 2200 kg/m^3, then rotated about y by -0.0338158 rad.  The seed
    and the rotation come from a search over seeded draws with an FP64 eigen-solve (not part of
    this generator): in this medium the relative gap between the two largest eigenvalues of the
    Christoffel matrix is 6.8e-5 at the phase angles theta = 0 and pi of the x-z plane.
    """
    B = np.random.Generator(np.random.PCG64(39760)).standard_normal((6, 6))
    C = B @ B.T + 0.05 * np.eye(6)
    rho = 2200.0
    C = C * (rho * 3000.0 ** 2 / C[2, 2])
    C = rotate_voigt_about_y(np.broadcast_to(C, (n, n, 6, 6)), np.full((n, n), -0.0338158))
    c21, r = _pack(C, np.full((n, n), rho))
    xs = ((n // 2) * h, (n // 2) * h)
    return Problem2D('triclinic_near_degenerate', n, n, h, h, c21, r, xs, n_theta, list(freqs), beam_width,
                     steps, cfl, meta=dict(seed=39760, tilt=-0.0338158))


def tti_default_steps(n, h):
    """Pseudo-time steps for the TTI medium: 1.1 x (latest exit time of source rays) / dt.

    Estimates for this medium family on the 2560 m square: latest exit time 0.95 s and a CFL-0.5
    time step of 0.5 h / 6700 m/s; the count is fixed here so that every run of the workload
    advances the same number of steps (2801 at 512 x 512, 5 m).
    """
    t_exit = 0.95 * (n * h) / 2560.0
    dt = 0.5 * h / 6700.0  # CFL-0.5 step bound: max(|Vx| + |Vz|) <= 6700 m/s in this family
    return int(math.ceil(1.1 * t_exit / dt))


def batched_instances(count=64, seed=3, n_range=(256, 1024), nth_range=(128, 512),
                      f_range=(8.0, 40.0), h=5.0, size_scale=1.0):
    """Uneven batch: instance i draws (seed 3 + i) grid n, angle count, 1-4 frequencies, TTI medium.

    ``size_scale`` shrinks every drawn size (n and angle count) for reduced test versions.
    """
    out = []
    for i in range(count):
        rng = np.random.Generator(np.random.PCG64(seed + i))
        n = int(rng.integers(n_range[0], n_range[1] + 1))
        nth = int(rng.integers(nth_range[0], nth_range[1] + 1))
        nf = int(rng.integers(1, 5))
        freqs = sorted(float(f) for f in rng.uniform(f_range[0], f_range[1], size=nf))
        n = max(16, int(round(n * size_scale)) // 4 * 4)
        nth = max(16, int(round(nth * size_scale)) // 2 * 2)
        hh = h * (1.0 / size_scale if size_scale != 1.0 else 1.0)
        p = tti_heterogeneous(n=n, h=hh, n_theta=nth, freqs=freqs, seed=1000 + seed + i)
        p.name = f'batched_{i}'
        out.append(p)
    return out


def request_stream(rate=200.0, duration=60.0, seed=4, max_requests=None):
    """Poisson request stream: (arrival time s, kind, n_freq, freqs) with a 50/50 size mix."""
    rng = np.random.Generator(np.random.PCG64(seed))
    t = 0.0
    reqs = []
    while True:
        t += rng.exponential(1.0 / rate)
        if t >= duration:
            break
        kind = 'small' if rng.random() < 0.5 else 'large'
        nf = int(rng.integers(1, 9))
        freqs = sorted(float(f) for f in rng.uniform(8.0, 40.0, size=nf))
        reqs.append((t, kind, nf, freqs))
        if max_requests is not None and len(reqs) >= max_requests:
            break
    return reqs


# ---------------------------------------------------------------------------------------------
# 3-D workloads.  Grids are stored z-major, then y, with x fastest (node = (iz*ny + iy)*nx + ix).
# Phase directions n = (sin th cos ph, sin th sin ph, cos th): n_theta polar samples at cell
# centres th_j = (j + 1/2) pi / n_theta, n_phi azimuth samples ph_k = 2 pi k / n_phi (n_phi even).

@dataclass
class Problem3D:
    """One 3-D solve request: medium on an nz x ny x nx node grid plus the source description."""
    name: str
    nx: int
    ny: int
    nz: int
    hx: float
    hy: float
    hz: float
    c21: np.ndarray                  # (nz*ny*nx, 21) float32, Pa
    rho: np.ndarray                  # (nz*ny*nx,) float32, kg/m^3
    xs: Tuple[float, float, float]   # source (x, y, z), m
    n_theta: int                     # polar samples (cell centred)
    n_phi: int                       # azimuth samples (even)
    freqs: List[float]
    beam_width: float
    steps: int
    cfl: float = 0.5
    r0: Optional[float] = None
    origin: Tuple[float, float, float] = (0.0, 0.0, 0.0)
    meta: dict = field(default_factory=dict)

    @property
    def omegas(self):
        return [2.0 * math.pi * f for f in self.freqs]

    @property
    def ball_radius(self):
        return self.r0 if self.r0 is not None else 2.0 * max(self.hx, self.hy, self.hz)

    @property
    def cells(self):
        return self.nx * self.ny * self.nz * self.n_theta * self.n_phi


def default_steps_3d(n, h, vp=3000.0):
    """ceil(1.1 T / dt) for a cube of n nodes at spacing h with the source at the centre: T = the
    half diagonal over 0.9 vp (slowest qP speed of a +-10 % medium), dt = 0.5 h / (sqrt(3) 1.1 vp)
    (CFL 0.5 with every group-velocity component at its bound).  387 steps at 96^3, 10 m."""
    t_exit = math.sqrt(3.0) * 0.5 * n * h / (0.9 * vp)
    dt = 0.5 * h / (math.sqrt(3.0) * 1.1 * vp)
    return int(math.ceil(1.1 * t_exit / dt))


def _cube(C, rho, n):
    C = np.broadcast_to(C, (n, n, n, 6, 6))
    return _pack(C, np.broadcast_to(np.asarray(rho, np.float64), (n, n, n)))


def isotropic_homogeneous_3d(n=32, h=10.0, n_theta=12, n_phi=24, steps=None, vp=3000.0, vs=1700.0,
                             rho=2300.0, freqs=(15.0,), beam_width=50.0, cfl=0.5):
    """Homogeneous isotropic cube, source at the centre node."""
    mu = rho * vs ** 2
    lam = rho * vp ** 2 - 2 * mu
    c21, r = _cube(isotropic_voigt(lam, mu), rho, n)
    xs = ((n // 2) * h,) * 3
    steps = default_steps_3d(n, h, vp) if steps is None else steps
    return Problem3D('isotropic_homogeneous_3d', n, n, n, h, h, h, c21, r, xs, n_theta, n_phi,
                     list(freqs), beam_width, steps, cfl, meta=dict(vp=vp, vs=vs, rho=rho))


def vti_homogeneous_3d(n=32, h=10.0, n_theta=12, n_phi=24, steps=None, vp0=3000.0, vs0=1500.0,
                       eps=0.20, delta=0.10, rho=2200.0, freqs=(15.0,), beam_width=50.0, cfl=0.5):
    """Homogeneous VTI cube (Thomsen parameters), source at the centre node."""
    c21, r = _cube(thomsen_vti_voigt(vp0, vs0, eps, delta, rho), rho, n)
    xs = ((n // 2) * h,) * 3
    steps = default_steps_3d(n, h, vp0) if steps is None else steps
    return Problem3D('vti_homogeneous_3d', n, n, n, h, h, h, c21, r, xs, n_theta, n_phi,
                     list(freqs), beam_width, steps, cfl,
                     meta=dict(vp0=vp0, vs0=vs0, eps=eps, delta=delta, rho=rho))


def triclinic_near_degenerate_3d(n=8, h=10.0, n_theta=12, n_phi=24, steps=4, freqs=(15.0,), beam_width=50.0,
                                  cfl=0.5):
    """The stiffness of triclinic_near_degenerate in a homogeneous cube, rotated about y by a further
    pi / (2 n_theta), so that its near qP-qS degeneracy (relative gap 6.8e-5) lies along the grid
    direction theta = pi / (2 n_theta) (the first polar cell centre), phi = 0."""
    B = np.random.Generator(np.random.PCG64(39760)).standard_normal((6, 6))
    C = B @ B.T + 0.05 * np.eye(6)
    rho = 2200.0
    C = C * (rho * 3000.0 ** 2 / C[2, 2])
    C = rotate_voigt_about_y(C[None], np.array([-0.0338158 + np.pi / (2 * n_theta)]))[0]
    c21, r = _cube(C, rho, n)
    xs = ((n // 2) * h,) * 3
    return Problem3D('triclinic_near_degenerate_3d', n, n, n, h, h, h, c21, r, xs, n_theta, n_phi,
                     list(freqs), beam_width, steps, cfl, meta=dict(seed=39760))


def triclinic_3d(n=96, h=10.0, n_theta=24, n_phi=48, steps=None, freqs=(15.0,), beam_width=50.0,
                 seed=5, cfl=0.5, length=None, vp=3000.0, vs=1700.0, rho=2300.0, amplitude=0.10,
                 sigma=150.0):
    """3-D triclinic medium: isotropic background (vp, vs, rho) plus a smooth random perturbation of
    all 21 stiffness constants.

    Each of the 21 perturbation fields is seeded white noise filtered by a Gaussian of ``sigma`` m;
    the symmetric 6x6 perturbation is scaled so that its largest spectral norm over the grid is
    ``amplitude`` times the background's, and every node's matrix is made positive definite by
    flooring its eigenvalues at 1/10 of the background's smallest (with 10 % amplitude the floor is
    never reached).  ``length`` keeps the physical extent for reduced grids.  Source at the centre.
    """
    rng = np.random.Generator(np.random.PCG64(seed))
    L = n * h if length is None else float(length)
    h = L / n
    mu = rho * vs ** 2
    lam = rho * vp ** 2 - 2 * mu
    C0 = isotropic_voigt(lam, mu)
    iu = np.triu_indices(6)
    dC = np.zeros((n, n, n, 6, 6))
    for m in range(21):
        f = _gaussian_filter(rng.standard_normal((n, n, n)), sigma / h)
        dC[..., iu[0][m], iu[1][m]] = f
        dC[..., iu[1][m], iu[0][m]] = f
    norm0 = np.linalg.norm(C0, 2)
    dnorm = np.max(np.linalg.norm(dC.reshape(-1, 6, 6), ord=2, axis=(1, 2)))
    C = C0 + dC * (amplitude * norm0 / dnorm)
    w, Q = np.linalg.eigh(C)
    floor = 0.1 * np.min(np.linalg.eigvalsh(C0))
    C = np.einsum('...ij,...j,...kj->...ik', Q, np.maximum(w, floor), Q)
    c21, r = _pack(C, np.full((n, n, n), rho))
    xs = ((n // 2) * h,) * 3
    steps = default_steps_3d(n, h, vp) if steps is None else steps
    return Problem3D('triclinic_3d', n, n, n, h, h, h, c21, r, xs, n_theta, n_phi, list(freqs),
                     beam_width, steps, cfl, meta=dict(seed=seed, length=L, vp=vp, vs=vs, rho=rho,
                                                       amplitude=amplitude, sigma=sigma))
