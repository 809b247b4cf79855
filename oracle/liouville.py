"""Level-set advection through the phase-space Liouville equation (oracle, float64).

Test infrastructure only.

Eq. 16 states that every level-set function phi is constant along the bicharacteristics; Eq. 19
applies it to the position label X, the angle label vartheta and, with the source p_3 + p_1 dx/dz,
to the traveltime tau; Eq. 20 initialises the labels to the phase-space coordinates and tau to 0.

The paper marches in depth z, which limits it to rays with dz/dtau > 0 (Eq. 13).  Here the same
equations are taken in pseudo-time t on the full reduced phase space (x, z, theta), theta in [0, 2pi):
    d_t u + Vx d_x u + Vz d_z u + thetadot d_theta u = s_u,   s = 0 for labels, s = 1 for tau
(with H normalised so that t is traveltime, the tau source p.V equals 1; Eq. 19's source is this one
divided by dz/dt).

Labels: b, the impact parameter of the ray at the source (the full-angle counterpart of Eq. 20's
position label X - x_s: Gamma = {b = 0} is Eq. 35's {X = x_s}); q, an indicator that the ray's
labels come from the source manifold (1) rather than the domain boundary (0); Th, the angle label
vartheta; tau.  Eq. 20's initial surface (the plane z = z_s) is replaced by the closest-approach
manifold of the point source: every phase cell within R_Sigma of x_s whose ray is still approaching
the source ((x - x_s) . g_s(theta) < 0, g_s the source medium's unit group direction), and every
cell of a small ball |x - x_s| <= r0, is frozen at the
straight-ray data of its own medium
    b = (x - x_s) x g(x, theta),  q = 1,  Th = theta,  tau = p(x, theta) . (x - x_s)
(g the unit group direction, p = n / v the slowness, 2-D cross product a x b = a_x b_z - a_z b_x).
A ray leaves the frozen set where it passes closest to x_s, so downstream it carries the distance
and phase angle of its closest approach, and tau its traveltime from the source when b = 0.  The
source-manifold tube in phase space is then about 2 R_Sigma wide, so its edge (where q and b jump
to boundary data) stays far from Gamma.  Two ghost layers in x and z hold the same straight-ray
data (media clamped to the nearest node) with q = 0 (Dirichlet inflow); theta is periodic.
Angle-label differences are wrapped into [-pi, pi).

Discretisation: Jiang & Peng's third-order HJ-WENO in each of x, z, theta, upwinded by the sign of
the velocity component; Shu & Osher's TVD-RK3; dt = cfl / max_cells(|Vx|/hx + |Vz|/hz +
|thetadot|/dtheta).

Beside the labels the state carries alpha, the argument of the complex spreading continued through
the evolution (superpose.track_branch, Eq. 26's square root past caustics): set from the initial
data, re-lifted after every step whose count is a multiple of superpose.BRANCH_SAMPLE, and 'step',
the number of steps taken.
"""
from __future__ import annotations

import math

import numpy as np

from . import christoffel as _ch
from . import medium as _md
from . import superpose as _sp

FIELDS = ('b', 'q', 'Th', 'tau')
WENO_EPS_REL = 1e-6
GHOST = 2


def _wrap(d):
    return (d + np.pi) % (2.0 * np.pi) - np.pi


class Setup:
    """Everything the evolution needs for one 2-D problem (float64)."""

    def __init__(self, problem, vel=None):
        self.p = problem
        nx, nz, nth = problem.nx, problem.nz, problem.n_theta
        self.nx, self.nz, self.nth = nx, nz, nth
        self.hx, self.hz = float(problem.hx), float(problem.hz)
        self.dth = 2.0 * math.pi / nth
        self.a, self.da_dx, self.da_dz, self.rho = _md.medium_2d(problem)
        # vel: the same fields computed beforehand (e.g. by velocity_field_pooled)
        self.vel = _ch.velocity_field_2d(self.a, self.da_dx, self.da_dz, nth) if vel is None else vel
        self.xs = np.array(problem.xs, np.float64)
        self.a_s = _md.bilinear_at(self.a, problem, self.xs[0], self.xs[1])
        self.rho_s = float(_md.bilinear_at(self.rho, problem, self.xs[0], self.xs[1]))
        self.theta = self.dth * np.arange(nth)
        vs, _, _, _ = _ch.source_quantities(self.a_s, self.theta)
        self.ps = np.stack([np.sin(self.theta) / vs, np.cos(self.theta) / vs], axis=-1)
        self.c_ref = float(_ch.source_quantities(self.a_s, np.array([0.0]))[0][0])
        self.r0 = float(problem.ball_radius)
        self.R_sigma = source_disc_radius(problem, self.r0)
        # node coordinates including the ghost layers
        ox, oz = problem.origin
        self.xg = ox + self.hx * np.arange(-GHOST, nx + GHOST)
        self.zg = oz + self.hz * np.arange(-GHOST, nz + GHOST)
        dx = (self.xg[GHOST:-GHOST] - self.xs[0])[None, None, :]
        dz = (self.zg[GHOST:-GHOST] - self.xs[1])[None, :, None]
        r2 = dz * dz + dx * dx
        # approaching the source: (x - x_s) . g_s(theta) < 0 with the source medium's unit group
        # direction (the disc is small enough that the local direction differs by a few degrees,
        # which only moves the freeze point along rays with b != 0 by a second-order amount)
        _, _, _, gs = _ch.source_quantities(self.a_s, self.theta)
        self.gs = gs
        dot = dx * gs[:, 0][:, None, None] + dz * gs[:, 1][:, None, None]
        # a cell on the closest-approach line (d . g_s at rounding level, e.g. diagonal directions of
        # an isotropic source on a node) belongs to the leaving half, as in 3-D
        approach = (dot < 0.0) & (dot * dot > 1e-24 * r2)
        self.frozen = (r2 <= self.r0 * self.r0) | ((r2 <= self.R_sigma * self.R_sigma) & approach)
        rate = (np.abs(self.vel['Vx']) / self.hx + np.abs(self.vel['Vz']) / self.hz
                + np.abs(self.vel['thetadot']) / self.dth)
        self.max_rate = float(rate.max())
        h = max(self.hx, self.hz)
        self.eps = {'b': WENO_EPS_REL * h * h, 'q': WENO_EPS_REL,
                    'Th': WENO_EPS_REL * self.dth ** 2,
                    'tau': WENO_EPS_REL * (h / self.c_ref) ** 2}

    def dt(self, cfl):
        return cfl / self.max_rate

    def initial_state(self):
        """Straight-ray data of the local medium on every padded cell (media clamped at the
        edges); q = 1 on the frozen source manifold, 0 elsewhere."""
        pad = ((0, 0), (GHOST, GHOST), (GHOST, GHOST))
        Vx = np.pad(self.vel['Vx'], pad, mode='edge')
        Vz = np.pad(self.vel['Vz'], pad, mode='edge')
        v = np.pad(self.vel['v'], pad, mode='edge')
        Vn = np.hypot(Vx, Vz)
        X = (self.xg - self.xs[0])[None, None, :]
        Z = (self.zg - self.xs[1])[None, :, None]
        th = self.theta[:, None, None]
        b = X * (Vz / Vn) - Z * (Vx / Vn)
        tau = (np.sin(th) * X + np.cos(th) * Z) / v
        q = np.zeros_like(b)
        q[:, GHOST:-GHOST, GHOST:-GHOST][self.frozen] = 1.0
        st = {'b': b, 'q': q, 'Th': np.broadcast_to(th, b.shape).copy(), 'tau': tau}
        st['alpha'] = _sp.track_branch(self, interior_state(st, self))
        st['step'] = 0
        return st


def _velocity_planes(args):
    problem, ks = args
    a, da_dx, da_dz, _ = _md.medium_2d(problem)
    return ks, _ch.velocity_field_2d(a, da_dx, da_dz, problem.n_theta, ks)


def velocity_field_pooled(problem, processes=8):
    """velocity_field_2d of the problem's medium, its angle planes split over a pool of `processes`
    spawned worker processes (for large grids; the planes are computed exactly as in one process)."""
    import multiprocessing as mp
    nth = problem.n_theta
    parts = [list(range(i, nth, processes)) for i in range(processes) if i < nth]
    out = {k: np.empty((nth, problem.nz, problem.nx)) for k in ('Vx', 'Vz', 'thetadot', 'v', 'pdx', 'pdz')}
    with mp.get_context('spawn').Pool(len(parts)) as pool:
        for ks, vel in pool.imap_unordered(_velocity_planes, [(problem, ks) for ks in parts]):
            for key in out:
                out[key][ks] = vel[key]
    return out


def source_disc_radius(problem, r0):
    """R_Sigma, the radius of the closest-approach manifold's disc: the problem's own value when it
    sets one, else max(4 r0, min(Lx, Lz) / 8)."""
    if getattr(problem, 'R_sigma', None):
        return float(problem.R_sigma)
    Lx = (problem.nx - 1) * problem.hx
    Lz = (problem.nz - 1) * problem.hz
    return max(4.0 * r0, min(Lx, Lz) / 8.0)


def _weno3_pair(dm2, dm1, d0, dp1, eps):
    """Jiang-Peng third-order HJ-WENO one-sided derivatives from undivided first differences.

    d_j = u_{j+1} - u_j around cell i: dm2 = d_{i-2}, dm1 = d_{i-1}, d0 = d_i, dp1 = d_{i+1}.
    Left-biased:  u^- = (d_{i-1} + d_i)/2 - w^-/2 (d_{i-2} - 2 d_{i-1} + d_i),
                  w^- = 1/(1 + 2 r^2), r = (eps + (d_{i-1} - d_{i-2})^2) / (eps + (d_i - d_{i-1})^2)
    Right-biased: u^+ = (d_{i-1} + d_i)/2 - w^+/2 (d_{i+1} - 2 d_i + d_{i-1}),
                  w^+ = 1/(1 + 2 r^2), r = (eps + (d_{i+1} - d_i)^2) / (eps + (d_i - d_{i-1})^2)
    (both undivided; divide by the spacing).
    """
    centre = 0.5 * (dm1 + d0)
    rm = (eps + (dm1 - dm2) ** 2) / (eps + (d0 - dm1) ** 2)
    wm = 1.0 / (1.0 + 2.0 * rm * rm)
    um = centre - 0.5 * wm * (dm2 - 2.0 * dm1 + d0)
    rp = (eps + (dp1 - d0) ** 2) / (eps + (d0 - dm1) ** 2)
    wp = 1.0 / (1.0 + 2.0 * rp * rp)
    up = centre - 0.5 * wp * (dp1 - 2.0 * d0 + dm1)
    return um, up


def upwind_derivatives(u, S, eps, angle):
    """Upwind WENO3 derivatives (d_x u, d_z u, d_theta u) on the interior cells of padded u."""
    nz, nx, G = S.nz, S.nx, GHOST
    core = u[:, G:G + nz, G:G + nx]
    shifts = {
        'x': {k: u[:, G:G + nz, G + k:G + k + nx] for k in range(-2, 3)},
        'z': {k: u[:, G + k:G + k + nz, G:G + nx] for k in range(-2, 3)},
        'theta': {k: np.roll(core, -k, axis=0) for k in range(-2, 3)},
    }
    out = []
    for name, h, vel in (('x', S.hx, S.vel['Vx']), ('z', S.hz, S.vel['Vz']),
                         ('theta', S.dth, S.vel['thetadot'])):
        s = shifts[name]
        d = {j: s[j + 1] - s[j] for j in (-2, -1, 0, 1)}
        if angle:
            d = {j: _wrap(v) for j, v in d.items()}
        um, up = _weno3_pair(d[-2], d[-1], d[0], d[1], eps)
        out.append(np.where(vel > 0, um, up) / h)
    return out


def rhs(state, S):
    """L(u) = -(Vx u_x + Vz u_z + thetadot u_theta) + s_u on interior cells; 0 in the frozen ball."""
    out = {}
    for f in FIELDS:
        ux, uz, ut = upwind_derivatives(state[f], S, S.eps[f], angle=(f == 'Th'))
        L = -(S.vel['Vx'] * ux + S.vel['Vz'] * uz + S.vel['thetadot'] * ut)
        if f == 'tau':
            L = L + 1.0
        L[S.frozen] = 0.0
        out[f] = L
    return out


def _interior(u, S):
    return u[:, GHOST:GHOST + S.nz, GHOST:GHOST + S.nx]


def rk3_step(state, S, dt):
    """Shu-Osher TVD-RK3: u1 = u + dt L(u); u2 = 3/4 u + 1/4 (u1 + dt L(u1));
    u_new = 1/3 u + 2/3 (u2 + dt L(u2)).  Ghost layers and frozen cells keep their initial data bit
    for bit (they are copied, not recombined)."""
    def combine(a, u, b, v, L):
        w = {f: state[f].copy() for f in FIELDS}
        for f in FIELDS:
            _interior(w[f], S)[...] = a * _interior(u[f], S) + b * (_interior(v[f], S) + dt * L[f])
            _interior(w[f], S)[S.frozen] = _interior(state[f], S)[S.frozen]
        return w
    L0 = rhs(state, S)
    u1 = combine(0.0, state, 1.0, state, L0)
    L1 = rhs(u1, S)
    u2 = combine(0.75, state, 0.25, u1, L1)
    L2 = rhs(u2, S)
    return combine(1.0 / 3.0, state, 2.0 / 3.0, u2, L2)


def _evolve_c(S, state, dt, steps):
    """The same TVD-RK3 / WENO3 steps run by the compiled float64 loop in liouville_c.c."""
    import ctypes
    from .build import library
    lib = library()
    vel = [np.ascontiguousarray(S.vel[k], np.float64) for k in ('Vx', 'Vz', 'thetadot')]
    ball = np.ascontiguousarray(S.frozen, np.uint8)
    eps = np.array([S.eps[f] for f in FIELDS], np.float64)
    fields = [np.ascontiguousarray(state[f], np.float64).copy() for f in FIELDS]
    ptr = lambda a: a.ctypes.data_as(ctypes.c_void_p)
    rc = lib.oracle_rk3_steps(S.nth, S.nz, S.nx, S.hx, S.hz, S.dth, ptr(vel[0]), ptr(vel[1]),
                              ptr(vel[2]), ptr(ball), ptr(eps), dt, int(steps),
                              *[ptr(f) for f in fields])
    if rc != 0:
        raise MemoryError('oracle stepping could not allocate its stage buffers')
    return dict(zip(FIELDS, fields))


def evolve(problem, steps=None, cfl=None, S=None, state=None, backend='c'):
    """Advance the labels `steps` TVD-RK3 steps from Eq. 20's initial data.  Returns (S, state, dt).

    backend 'c' runs the compiled loop (liouville_c.c), 'numpy' the array code above; both compute
    the same float64 scheme.
    """
    if S is None:
        S = Setup(problem)
    steps = problem.steps if steps is None else steps
    cfl = problem.cfl if cfl is None else cfl
    dt = S.dt(cfl)
    if state is None:
        state = S.initial_state()
    fields = {f: state[f] for f in FIELDS}
    if 'alpha' in state:
        alpha, step = state['alpha'], int(state['step'])
    else:
        alpha, step = _sp.track_branch(S, interior_state(fields, S)), 0
    done = 0
    while done < steps:
        n = min(steps - done, _sp.BRANCH_SAMPLE - step % _sp.BRANCH_SAMPLE)
        if backend == 'c':
            fields = _evolve_c(S, fields, dt, n)
        else:
            for _ in range(n):
                fields = rk3_step(fields, S, dt)
        done += n
        step += n
        if step % _sp.BRANCH_SAMPLE == 0:
            alpha = _sp.track_branch(S, interior_state(fields, S), alpha)
    out = dict(fields)
    out['alpha'], out['step'] = alpha, step
    return S, out, dt


def interior_state(state, S):
    """Interior (unpadded) copies of the four fields, shape (n_theta, nz, nx), and of the continued
    spreading argument alpha when the state has one."""
    out = {f: _interior(state[f], S).copy() for f in FIELDS}
    if 'alpha' in state:
        out['alpha'] = state['alpha'].copy()
    return out
