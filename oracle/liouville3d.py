"""Level-set advection through the 3-D phase-space Liouville equation (oracle, float64).

Test infrastructure only.

The 3-D counterpart of the reduced phase space of Sec. 3: (x, y, z, theta, phi) with the phase
direction n = (sin th cos ph, sin th sin ph, cos th) and p = n / v(x, n).  Every label u obeys
Eqs. 16/19 in pseudo-time t (traveltime, H = (lambda_qP - 1)/2):
    d_t u + Vx d_x u + Vy d_y u + Vz d_z u + thetadot d_th u + phidot d_ph u = s_u,
s = 1 for tau, 0 otherwise (velocities from christoffel.velocity_field_3d).

Labels (the 3-D form of the 2-D closest-approach labels):
  b = (bx, by, bz)    the ray's offset from x_s at its closest approach; on the frozen manifold
                      b = d - (d . g) g for the straight ray of the local medium (d = x - x_s, g the
                      local unit group direction), so b is perpendicular to the ray and b = 0 is
                      Eq. 35's Gamma = {X = x_s}
  n0 = (n0x, n0y, n0z) the ray's phase direction at closest approach (take-off direction; on the
                      frozen manifold n0 = n)
  q                   1 on rays that carry source-manifold data, 0 on rays from the boundary
  tau                 traveltime since closest approach; p . d on the frozen manifold
Source manifold (Eq. 20 generalised as in 2-D): a cell is frozen when |d| <= r0, or |d| <= R_Sigma
and d . g_s(n) < 0 (g_s the source medium's unit group direction), R_Sigma = max(4 r0,
min(Lx, Ly, Lz) / 8, 2 dA r_far) (dA the angular spacing, r_far the farthest corner), r0 = 2 max(h).  The decision takes r^2 = (dz dz + dy dy) + dx dx and
d . g_s = (dx gx + dy gy) + dz gz, each product and sum rounded in that order; a cell counts as
approaching only when (d . g_s)^2 > 1e-24 r^2 as well (cells on the closest-approach plane, where
symmetric grids put d . g_s at rounding level with either sign, are leaving).

Grid: nodes at origin + i h with two ghost layers in x, y, z holding the straight-ray data (media
clamped to the nearest node), the indicator included: q = 1 where the straight ray passed its closest
approach within R_Sigma (outflow through the source-ray tube), 0 elsewhere (Dirichlet inflow).  theta is sampled at cell centres
th_j = (j + 1/2) pi / n_theta and continues across a pole onto the opposite azimuth (the point
(-th, ph) is (th, ph + pi), and (pi + th, ph) is (pi - th, ph + pi)); phi is periodic.

Discretisation: Jiang & Peng's third-order HJ-WENO in each of the five dimensions, upwinded by the
sign of the cell's velocity component; Shu & Osher's TVD-RK3; frozen cells and ghosts are copied;
dt = cfl / max_cells(|Vx|/hx + |Vy|/hy + |Vz|/hz + |thetadot|/dtheta + |phidot|/dphi).
"""
from __future__ import annotations

import math

import numpy as np

from . import christoffel as _ch
from . import medium as _md
from .liouville import _weno3_pair, WENO_EPS_REL

FIELDS3 = ('bx', 'by', 'bz', 'n0x', 'n0y', 'n0z', 'q', 'tau')
GHOST = 2


def source_disc_radius_3d(problem, r0):
    """R_Sigma = max(4 r0, min(Lx, Ly, Lz) / 8, 2 dA r_far): the last term keeps the source-ray
    tube, which subtends R_Sigma / r at distance r, wider than two angular cells at the farthest
    node (dA = max(pi / n_theta, 2 pi / n_phi), r_far the largest distance from x_s to a corner),
    so that every direction cell around an arrival carries source labels."""
    L = min((problem.nx - 1) * problem.hx, (problem.ny - 1) * problem.hy, (problem.nz - 1) * problem.hz)
    dA = max(math.pi / problem.n_theta, 2.0 * math.pi / problem.n_phi)
    far2 = 0.0
    for c, n, h, o in ((problem.xs[0], problem.nx, problem.hx, problem.origin[0]),
                       (problem.xs[1], problem.ny, problem.hy, problem.origin[1]),
                       (problem.xs[2], problem.nz, problem.hz, problem.origin[2])):
        far2 += max((c - o) ** 2, (o + (n - 1) * h - c) ** 2)
    return max(4.0 * r0, L / 8.0, 2.0 * dA * math.sqrt(far2))


class Setup3D:
    """Everything the 3-D evolution needs for one problem (float64).  Arrays over cells are shaped
    (n_phi, n_theta, nz, ny, nx)."""

    def __init__(self, problem, vel=None):
        self.p = problem
        self.nx, self.ny, self.nz = problem.nx, problem.ny, problem.nz
        self.nth, self.nph = problem.n_theta, problem.n_phi
        self.hx, self.hy, self.hz = float(problem.hx), float(problem.hy), float(problem.hz)
        self.dth, self.dph = math.pi / self.nth, 2.0 * math.pi / self.nph
        self.theta, self.phi = _ch.angle_grid_3d(self.nth, self.nph)
        self.a, self.da_dx, self.da_dy, self.da_dz, self.rho = _md.medium_3d(problem)
        self.vel = (_ch.velocity_field_3d(self.a, self.da_dx, self.da_dy, self.da_dz, self.nth, self.nph)
                    if vel is None else vel)
        self.xs = np.array(problem.xs, np.float64)
        self.a_s = _md.trilinear_at(self.a, problem, *self.xs)
        self.rho_s = float(_md.trilinear_at(self.rho, problem, *self.xs))
        self.n = _ch.direction_3d(self.theta[None, :], self.phi[:, None])      # (nph, nth, 3)
        _, _, _, self.gs = _ch.source_quantities_3d(self.a_s, self.n)
        self.c_ref = float(_ch.source_quantities_3d(self.a_s, np.array([0.0, 0.0, 1.0]))[0])
        self.r0 = float(problem.ball_radius)
        self.R_sigma = source_disc_radius_3d(problem, self.r0)
        o = problem.origin
        self.xg = o[0] + self.hx * np.arange(-GHOST, self.nx + GHOST)
        self.yg = o[1] + self.hy * np.arange(-GHOST, self.ny + GHOST)
        self.zg = o[2] + self.hz * np.arange(-GHOST, self.nz + GHOST)
        dx = (self.xg[GHOST:-GHOST] - self.xs[0])[None, None, None, None, :]
        dy = (self.yg[GHOST:-GHOST] - self.xs[1])[None, None, None, :, None]
        dz = (self.zg[GHOST:-GHOST] - self.xs[2])[None, None, :, None, None]
        r2 = dz * dz + dy * dy + dx * dx
        g = [self.gs[..., c][:, :, None, None, None] for c in range(3)]
        dot = dx * g[0] + dy * g[1] + dz * g[2]
        # approaching: d . g_s < 0 by more than 1e-12 |d| (a cell on the closest-approach plane, where
        # d . g_s is rounding noise of either sign, belongs to the leaving half)
        approach = (dot < 0.0) & (dot * dot > 1e-24 * r2)
        self.frozen = (r2 <= self.r0 * self.r0) | ((r2 <= self.R_sigma * self.R_sigma) & approach)
        v = self.vel
        rate = (np.abs(v['Vx']) / self.hx + np.abs(v['Vy']) / self.hy + np.abs(v['Vz']) / self.hz
                + np.abs(v['thetadot']) / self.dth + np.abs(v['phidot']) / self.dph)
        self.max_rate = float(rate.max())
        h = max(self.hx, self.hy, self.hz)
        self.eps = {f: WENO_EPS_REL * h * h for f in ('bx', 'by', 'bz')}
        self.eps.update({f: WENO_EPS_REL for f in ('n0x', 'n0y', 'n0z', 'q')})
        self.eps['tau'] = WENO_EPS_REL * (h / self.c_ref) ** 2

    def dt(self, cfl):
        return cfl / self.max_rate

    def initial_state(self):
        """Straight-ray data of the local medium on every padded cell; q = 1 on the frozen
        manifold, 0 elsewhere."""
        G = GHOST
        pad = ((0, 0), (0, 0), (G, G), (G, G), (G, G))
        V = [np.pad(self.vel[k], pad, mode='edge') for k in ('Vx', 'Vy', 'Vz')]
        v = np.pad(self.vel['v'], pad, mode='edge')
        Vn = np.sqrt(V[0] ** 2 + V[1] ** 2 + V[2] ** 2)
        g = [c / Vn for c in V]
        X = (self.xg - self.xs[0])[None, None, None, None, :]
        Y = (self.yg - self.xs[1])[None, None, None, :, None]
        Z = (self.zg - self.xs[2])[None, None, :, None, None]
        dg = X * g[0] + Y * g[1] + Z * g[2]
        n = [self.n[..., c][:, :, None, None, None] for c in range(3)]
        st = {'bx': X - dg * g[0], 'by': Y - dg * g[1], 'bz': Z - dg * g[2],
              'tau': (n[0] * X + n[1] * Y + n[2] * Z) / v}
        for c, f in enumerate(('n0x', 'n0y', 'n0z')):
            st[f] = np.broadcast_to(n[c], v.shape).copy()
        # indicator: the frozen manifold inside; on the ghost layers the straight-ray value, 1 on rays
        # that passed their closest approach within R_Sigma (|b| <= R_Sigma, not approaching) and 0
        # elsewhere, so that outflow ghosts continue the source-ray tube instead of cutting it
        bn = np.sqrt(st['bx'] ** 2 + st['by'] ** 2 + st['bz'] ** 2)
        r2 = Z * Z + Y * Y + X * X
        approach = (dg < 0.0) & (dg * dg > 1e-24 * r2)
        q = ((bn <= self.R_sigma) & ~approach).astype(np.float64)
        inner = q[:, :, G:-G, G:-G, G:-G]
        inner[...] = 0.0
        inner[self.frozen] = 1.0
        st['q'] = q
        return st


def _interior(u):
    G = GHOST
    return u[:, :, G:-G, G:-G, G:-G]


def _theta_extended(core, nph):
    """core (nph, nth, ...) -> (nph, nth + 4, ...) with two planes continued across each pole."""
    half = nph // 2
    over = lambda j: np.roll(core[:, j], -half, axis=0)   # (th_j, ph + pi)
    nth = core.shape[1]
    return np.concatenate([over(1)[:, None], over(0)[:, None], core,
                           over(nth - 1)[:, None], over(nth - 2)[:, None]], axis=1)


def upwind_derivatives_3d(u, S, eps):
    """Upwind WENO3 derivatives along x, y, z, theta, phi on the interior cells of padded u."""
    G = GHOST
    nx, ny, nz = S.nx, S.ny, S.nz
    core = _interior(u)
    ext = _theta_extended(core, S.nph)
    shifts = {
        'x': lambda k: u[:, :, G:G + nz, G:G + ny, G + k:G + k + nx],
        'y': lambda k: u[:, :, G:G + nz, G + k:G + k + ny, G:G + nx],
        'z': lambda k: u[:, :, G + k:G + k + nz, G:G + ny, G:G + nx],
        'theta': lambda k: ext[:, 2 + k:2 + k + S.nth],
        'phi': lambda k: np.roll(core, -k, axis=0),
    }
    out = []
    for name, h, vel in (('x', S.hx, S.vel['Vx']), ('y', S.hy, S.vel['Vy']), ('z', S.hz, S.vel['Vz']),
                         ('theta', S.dth, S.vel['thetadot']), ('phi', S.dph, S.vel['phidot'])):
        s = {k: shifts[name](k) for k in range(-2, 3)}
        d = {j: s[j + 1] - s[j] for j in (-2, -1, 0, 1)}
        um, up = _weno3_pair(d[-2], d[-1], d[0], d[1], eps)
        out.append(np.where(vel > 0, um, up) / h)
    return out


def rhs3d(state, S):
    """L(u) = -(V . grad_x u + thetadot u_th + phidot u_ph) + s_u on interior cells; 0 where frozen."""
    out = {}
    v = S.vel
    for f in FIELDS3:
        ux, uy, uz, ut, up = upwind_derivatives_3d(state[f], S, S.eps[f])
        L = -(v['Vx'] * ux + v['Vy'] * uy + v['Vz'] * uz + v['thetadot'] * ut + v['phidot'] * up)
        if f == 'tau':
            L = L + 1.0
        L[S.frozen] = 0.0
        out[f] = L
    return out


def rk3_step3d(state, S, dt):
    """Shu-Osher TVD-RK3; ghosts and frozen cells keep their initial data (copied)."""
    def combine(a, u, b, w, L):
        out = {f: state[f].copy() for f in FIELDS3}
        for f in FIELDS3:
            _interior(out[f])[...] = a * _interior(u[f]) + b * (_interior(w[f]) + dt * L[f])
            _interior(out[f])[S.frozen] = _interior(state[f])[S.frozen]
        return out
    u1 = combine(0.0, state, 1.0, state, rhs3d(state, S))
    u2 = combine(0.75, state, 0.25, u1, rhs3d(u1, S))
    return combine(1.0 / 3.0, state, 2.0 / 3.0, u2, rhs3d(u2, S))


def _evolve3d_c(S, state, dt, steps):
    """The same steps run by the compiled float64 loop in liouville3d_c.c."""
    import ctypes
    from .build import library
    lib = library()
    vel = [np.ascontiguousarray(S.vel[k], np.float64) for k in ('Vx', 'Vy', 'Vz', 'thetadot', 'phidot')]
    frozen = np.ascontiguousarray(S.frozen, np.uint8)
    eps = np.array([S.eps[f] for f in FIELDS3], np.float64)
    fields = [np.ascontiguousarray(state[f], np.float64).copy() for f in FIELDS3]
    ptrs = (ctypes.c_void_p * 8)(*[f.ctypes.data for f in fields])
    ptr = lambda a: a.ctypes.data_as(ctypes.c_void_p)
    rc = lib.oracle3d_rk3_steps(S.nph, S.nth, S.nz, S.ny, S.nx, S.hx, S.hy, S.hz, S.dth, S.dph,
                                *[ptr(v) for v in vel], ptr(frozen), ptr(eps), dt, int(steps),
                                ctypes.cast(ptrs, ctypes.c_void_p))
    if rc != 0:
        raise MemoryError('oracle stepping could not allocate its stage buffers')
    return dict(zip(FIELDS3, fields))


def evolve3d(problem, steps=None, cfl=None, S=None, state=None, backend='c'):
    """Advance the 3-D labels `steps` TVD-RK3 steps from the source-manifold data.  Returns
    (S, state, dt).  backend 'c' runs the compiled loop (liouville3d_c.c), 'numpy' the array code
    above; both compute the same float64 scheme."""
    if S is None:
        S = Setup3D(problem)
    steps = problem.steps if steps is None else steps
    cfl = problem.cfl if cfl is None else cfl
    dt = S.dt(cfl)
    if state is None:
        state = S.initial_state()
    if backend == 'c':
        return S, _evolve3d_c(S, state, dt, steps), dt
    for _ in range(steps):
        state = rk3_step3d(state, S, dt)
    return S, state, dt


def interior_state3d(state):
    """Interior (unpadded) copies of the eight fields, shape (n_phi, n_theta, nz, ny, nx)."""
    return {f: _interior(state[f]).copy() for f in FIELDS3}
