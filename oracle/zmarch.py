"""Paraxial depth march of the level sets: the paper's own formulation (oracle, float64).

Test infrastructure only.

Sec. 3-4 write the level-set equations with depth z as the evolution variable: along a ray with
dz/dtau > 0 (Eq. 13) the horizontal position and the phase angle move as dx/dz and dtheta/dz
(Eqs. 14-15, 17-18), every level-set function phi(z, x, theta) obeys phi_z + u phi_x + w phi_theta = 0
(Eq. 16), which applied to the position label X, the angle label vartheta and the traveltime tau
gives Eq. 19, started from the source plane with X = x, vartheta = theta, tau = 0 (Eq. 20).  The
Green's function on a depth row is the sum of the Gaussian beams centred where that row crosses
Gamma = {X = x_s} (Eqs. 25-28, 34-35), evaluated along the same row.

Readings taken here:
* u = dx/dz = Vx / Vz, w = dtheta/dz = thetadot / Vz and the tau source p_3 + p_1 dx/dz = (p . V) / Vz
  = 1 / Vz, with V the qP group velocity and thetadot the phase-angle rate of the pseudo-time
  system (Eqs. 8-12), so that the depth march and the pseudo-time form share their rays.
* Two-sided from the source plane z_s (a grid row): the downgoing branch marches z upward in index
  with phase angles theta_k = -theta_max + (k + 1/2) dtheta, dtheta = 2 theta_max / n_theta; the
  upgoing branch marches toward z = 0 with the angles theta_k + pi.  With the marching variable
  zeta = s (z - z_s) (s = +1 down, -1 up) every branch reads phi_zeta + U phi_x + W phi_theta = S_phi
  with U = s Vx / Vz, W = s thetadot / Vz, S_tau = s / Vz > 0 and S = 0 for the labels.  Every cell
  must have s Vz > 0 (the branch's rays keep their vertical direction, Eq. 13).
* Rows j_s, j_s + s, ... are reached through n_sub equal substeps of Shu-Osher TVD-RK3 each,
  n_sub = ceil(h_z R / cfl), R = max over the branch's cells of |U|/h_x + |W|/dtheta; inside a row
  interval the coefficients U, W, S are interpolated linearly in zeta between the two rows (stage
  positions zeta_n, zeta_n + dzeta, zeta_n + dzeta/2).
* Jiang & Peng's third-order HJ-WENO in x and theta, upwinded by the signs of U and W.  Two ghost
  cells on each side of x and of theta hold the linear extrapolation of the two outermost interior
  values (exact for fields linear in x or theta).
* A source indicator q is advected like the labels from q = 1 on the source row, its ghosts hold
  q = 0 (Dirichlet inflow): rays that enter through the x or theta boundaries carry no source-plane
  data (their labels are extrapolations), and only cells with q > 1/2 take part in beam centres and
  arrivals (the pseudo-time form's source indicator, for the same reason).
* Rows j >= j_s of the output come from the downgoing branch, rows j < j_s from the upgoing one.

Beams (same reading as the pseudo-time form's superposition, with the dynamic ray tracing taken
from the label gradients in (x, theta) at fixed depth instead of advecting Eq. 21):
* on each row and angle, every sign change of X - x_s between neighbouring nodes that both have
  q > 1/2 (sign(0) = +1) is a beam centre; quantities are interpolated linearly there;
* the perturbation (dx, dtheta) solves [[X_x, X_theta], [vartheta_x, vartheta_theta]] (dx, dtheta) =
  (1 / ghat_z, kappa), kappa = 2 i |V_s| / (omega w0^2), ghat_z and |V_s| the source medium's unit
  group direction and group speed at vartheta: at the source plane db/dX = ghat_z (b = (X - x_s)
  ghat_z is the impact parameter), so this is the pseudo-time form's perturbation with db = 1 and the
  initial transverse beam Hessian i 2 / (omega w0^2) (Eq. 24's complex initial data);
* M_xx = dp_x / dx with dp_x = p_x (pdot_x dx) + (dp_x/dtheta) dtheta (Eq. 25's M = B C^-1 along the
  row), J = dx Vz the complex spreading (Eq. 26's det C), amplitude sigma sqrt(rho_s |V_s| / (rho J))
  with sigma = -1 once arg J < -1e-3 (KMAH index 1);
* weight i c_ref^2 / (4 pi v_s(vartheta)^2) times the take-off measure
  |d vartheta_c / d theta| dtheta = |vartheta_theta X_x - vartheta_x X_theta| / |X_x| dtheta (Eq. 33's
  Psi_0, calibrated as in the pseudo-time form);
* arrivals at a node: sign changes of X - x_s between theta_k and theta_k+1 (both q > 1/2), T = tau
  interpolated,
  A = c_ref^2 sqrt(rho_s / rho_r) / (v_r sqrt(8 pi |V_s ghat_z| |X_theta|)) (|d_theta b| =
  |ghat_z X_theta| on Gamma), sorted by T then angle, at most kmax kept.
"""
from __future__ import annotations

import math

import numpy as np

from . import christoffel as _ch
from . import medium as _md
from . import superpose as _SP

GHOST = 2
WENO_EPS_REL = 1e-6
KMAH_ARG = 1e-3
FIELDS = ('X', 'Th', 'tau', 'q')


class ZSetup:
    """Grids, characteristic coefficients and steps of one branch (s = +1 down, -1 up)."""

    def __init__(self, problem, n_theta, theta_max, branch, cfl=0.5, medium=None):
        if branch not in (1, -1):
            raise ValueError('branch must be +1 (down) or -1 (up)')
        self.p = problem
        self.s = branch
        self.nx, self.nz, self.nth = problem.nx, problem.nz, int(n_theta)
        self.hx, self.hz = float(problem.hx), float(problem.hz)
        self.theta_max = float(theta_max)
        self.dth = 2.0 * self.theta_max / self.nth
        self.theta = (-self.theta_max + (np.arange(self.nth) + 0.5) * self.dth
                      + (0.0 if branch == 1 else math.pi))
        ox, oz = problem.origin
        self.xs = np.array(problem.xs, np.float64)
        js = (self.xs[1] - oz) / self.hz
        self.js = int(round(js))
        if abs(js - self.js) > 1e-9 or not 0 <= self.js < self.nz:
            raise ValueError('the source depth must lie on a grid row')
        self.rows = (np.arange(self.js, self.nz) if branch == 1 else np.arange(self.js, -1, -1))
        self.x = ox + self.hx * np.arange(self.nx)
        a, dax, daz, rho = _md.medium_2d(problem) if medium is None else medium
        self.rho = rho
        self.a_s = _md.bilinear_at(a, problem, self.xs[0], self.xs[1])
        self.rho_s = float(_md.bilinear_at(rho, problem, self.xs[0], self.xs[1]))
        self.c_ref = float(_ch.source_quantities(self.a_s, np.array([0.0]))[0][0])
        # characteristic velocities on every (theta, row, x) cell of the branch's rows
        nr = len(self.rows)
        self.vel = {k: np.empty((self.nth, nr, self.nx)) for k in ('Vx', 'Vz', 'thetadot', 'v', 'pdx', 'pdz')}
        sub = (a[self.rows], dax[self.rows], daz[self.rows])
        for k, th in enumerate(self.theta):
            n = np.broadcast_to(_ch.direction_2d(th), (nr, self.nx, 3))
            v, g, V, (pdx, pdz) = _ch.ray_velocity(sub[0], [sub[1], sub[2]], n)
            self.vel['Vx'][k] = V[..., 0]
            self.vel['Vz'][k] = V[..., 2]
            self.vel['v'][k] = v
            self.vel['pdx'][k] = pdx
            self.vel['pdz'][k] = pdz
            self.vel['thetadot'][k] = v * (math.cos(th) * pdx - math.sin(th) * pdz)
        Vz = self.vel['Vz']
        if not np.all(branch * Vz > 0.0):
            raise ValueError('rays of this branch turn horizontal: lower theta_max')
        self.U = branch * self.vel['Vx'] / Vz
        self.W = branch * self.vel['thetadot'] / Vz
        self.S = branch / Vz
        rate = np.abs(self.U) / self.hx + np.abs(self.W) / self.dth
        self.max_rate = float(rate.max())
        self.n_sub = max(1, int(math.ceil(self.hz * self.max_rate / cfl)))
        h = max(self.hx, self.hz)
        self.eps = {'X': WENO_EPS_REL * h * h, 'Th': WENO_EPS_REL * self.dth ** 2,
                    'tau': WENO_EPS_REL * (h / self.c_ref) ** 2, 'q': WENO_EPS_REL}


def _pad(u, dirichlet=None):
    """Two ghost cells per side in theta (axis 0) and x (axis 1) by linear extrapolation of the two
    outermost interior values, or holding the value `dirichlet`; the four corner blocks are never
    read and stay NaN."""
    nth, nx = u.shape
    G = GHOST
    p = np.full((nth + 2 * G, nx + 2 * G), np.nan)
    p[G:-G, G:-G] = u
    if dirichlet is not None:
        p[G:-G, :G] = p[G:-G, -G:] = dirichlet
        p[:G, G:-G] = p[-G:, G:-G] = dirichlet
        return p
    for k in (1, 2):
        p[G:-G, G - k] = (1 + k) * u[:, 0] - k * u[:, 1]
        p[G:-G, G + nx - 1 + k] = (1 + k) * u[:, -1] - k * u[:, -2]
        p[G - k, G:-G] = (1 + k) * u[0] - k * u[1]
        p[G + nth - 1 + k, G:-G] = (1 + k) * u[-1] - k * u[-2]
    return p


def _weno3(d, vel, eps):
    """Jiang-Peng third-order HJ-WENO derivative (undivided) from the differences d[j] = u_{i+j+1} -
    u_{i+j}, j = -2..1, upwinded by the sign of vel (left-biased for vel > 0)."""
    dm2, dm1, d0, dp1 = d[-2], d[-1], d[0], d[1]
    centre = 0.5 * (dm1 + d0)
    rm = (eps + (dm1 - dm2) ** 2) / (eps + (d0 - dm1) ** 2)
    um = centre - 0.5 / (1.0 + 2.0 * rm * rm) * (dm2 - 2.0 * dm1 + d0)
    rp = (eps + (dp1 - d0) ** 2) / (eps + (d0 - dm1) ** 2)
    up = centre - 0.5 / (1.0 + 2.0 * rp * rp) * (dp1 - 2.0 * d0 + dm1)
    return np.where(vel > 0, um, up)


def rhs(state, Z, U, W, S):
    """L(phi) = -(U phi_x + W phi_theta) + S_phi on the (theta, x) plane of one depth."""
    out = {}
    G = GHOST
    nth, nx = Z.nth, Z.nx
    for f in FIELDS:
        p = _pad(state[f], 0.0 if f == 'q' else None)
        sx = {m: p[G:G + nth, G + m:G + m + nx] for m in range(-2, 3)}
        st = {m: p[G + m:G + m + nth, G:G + nx] for m in range(-2, 3)}
        dx = {j: sx[j + 1] - sx[j] for j in (-2, -1, 0, 1)}
        dt = {j: st[j + 1] - st[j] for j in (-2, -1, 0, 1)}
        ux = _weno3(dx, U, Z.eps[f]) / Z.hx
        ut = _weno3(dt, W, Z.eps[f]) / Z.dth
        L = -(U * ux + W * ut)
        if f == 'tau':
            L = L + S
        out[f] = L
    return out


def march(Z):
    """Labels on every row of the branch: dict of (n_theta, n_rows, nx) arrays, row r at depth
    index Z.rows[r] (r = 0 is the source row, Eq. 20's initial data)."""
    nth, nx, nr = Z.nth, Z.nx, len(Z.rows)
    state = {'X': np.broadcast_to(Z.x[None, :], (nth, nx)).copy(),
             'Th': np.broadcast_to(Z.theta[:, None], (nth, nx)).copy(),
             'tau': np.zeros((nth, nx)), 'q': np.ones((nth, nx))}
    hist = {f: np.empty((nth, nr, nx)) for f in FIELDS}
    for f in FIELDS:
        hist[f][:, 0] = state[f]
    dz = 1.0 / Z.n_sub  # substep as a fraction of the row spacing
    h = Z.hz * dz
    for r in range(nr - 1):
        def coef(t):
            return ((1 - t) * Z.U[:, r] + t * Z.U[:, r + 1], (1 - t) * Z.W[:, r] + t * Z.W[:, r + 1],
                    (1 - t) * Z.S[:, r] + t * Z.S[:, r + 1])
        for n in range(Z.n_sub):
            t0 = n * dz
            L0 = rhs(state, Z, *coef(t0))
            u1 = {f: state[f] + h * L0[f] for f in FIELDS}
            L1 = rhs(u1, Z, *coef(t0 + dz))
            u2 = {f: 0.75 * state[f] + 0.25 * (u1[f] + h * L1[f]) for f in FIELDS}
            L2 = rhs(u2, Z, *coef(t0 + 0.5 * dz))
            state = {f: state[f] / 3.0 + 2.0 / 3.0 * (u2[f] + h * L2[f]) for f in FIELDS}
        for f in FIELDS:
            hist[f][:, r + 1] = state[f]
    return hist


def _grad_x(f, h):
    """Second-order centred difference along x (last axis), second-order one-sided at the edges."""
    out = np.empty_like(f)
    out[..., 1:-1] = (f[..., 2:] - f[..., :-2]) / (2 * h)
    out[..., 0] = (4 * (f[..., 1] - f[..., 0]) - (f[..., 2] - f[..., 0])) / (2 * h)
    out[..., -1] = (4 * (f[..., -1] - f[..., -2]) - (f[..., -1] - f[..., -3])) / (2 * h)
    return out


def _grad_t(f, h):
    """The same along theta (axis 0), one-sided at the two ends of the angle range."""
    return np.moveaxis(_grad_x(np.moveaxis(f, 0, -1), h), -1, 0)


def fields(Z, H):
    """Per-cell quantities of the superposition and of the arrivals on the branch's rows."""
    X, Th, tau = H['X'], H['Th'], H['tau']
    vs, Vs, Vsn, gs = _ch.source_quantities(Z.a_s, Th)
    return dict(X=X, Th=Th, tau=tau, vs=vs, Vsn=Vsn, gsz=gs[..., 1],
                Xx=_grad_x(X, Z.hx), Xt=_grad_t(X, Z.dth),
                Tx=_grad_x(Th, Z.hx), Tt=_grad_t(Th, Z.dth))


def _lin(a, c0, c1, t):
    return a[c0] + t * (a[c1] - a[c0])


def green_rows(Z, H, omegas, beam_width, F=None):
    """u(omega, r, x) complex128 on the branch's rows (Eqs. 25-28, 34-35)."""
    F = fields(Z, H) if F is None else F
    nth, nr, nx = F['X'].shape
    D = F['X'] - Z.xs[0]
    fl = H['q'] > 0.5  # rays carrying source-plane labels
    cross = fl[..., :-1] & fl[..., 1:] & ((D[..., :-1] >= 0) != (D[..., 1:] >= 0))
    k, r, i = np.nonzero(cross)
    c0, c1 = (k, r, i), (k, r, i + 1)
    t = D[c0] / (D[c0] - D[c1])
    q = {nm: _lin(F[nm], c0, c1, t) for nm in ('tau', 'Xx', 'Xt', 'Tx', 'Tt', 'Th')}
    for nm in ('Vx', 'Vz', 'pdx', 'v'):
        q[nm] = _lin(Z.vel[nm], c0, c1, t)
    rho = Z.rho[Z.rows]
    q['rho'] = rho[r, i] + t * (rho[r, i + 1] - rho[r, i])
    th = Z.theta[k]
    vs, _, Vsn, gs = _ch.source_quantities(Z.a_s, q['Th'])
    det = q['Xx'] * q['Tt'] - q['Xt'] * q['Tx']
    out = np.zeros((len(omegas), nr, nx), np.complex128)
    xc = Z.x[i] + t * Z.hx
    delta = Z.x[None, :] - xc[:, None]
    v = q['v']
    px = np.sin(th) / v
    v_th = np.cos(th) * q['Vx'] - np.sin(th) * q['Vz']
    dpx_dth = (np.cos(th) * v - np.sin(th) * v_th) / v ** 2
    wj = np.abs(q['Tt'] * q['Xx'] - q['Tx'] * q['Xt']) / np.abs(q['Xx'])
    weight = 1j * Z.c_ref ** 2 / (4 * np.pi * vs ** 2)
    for w, om in enumerate(omegas):
        kappa = 2j * Vsn / (om * beam_width ** 2)
        r0, r1 = 1.0 / gs[:, 1], kappa
        dx = (q['Tt'] * r0 - q['Xt'] * r1) / det
        dth = (-q['Tx'] * r0 + q['Xx'] * r1) / det
        dpx = px * q['pdx'] * dx + dpx_dth * dth
        M = dpx / dx
        J = dx * q['Vz']
        sigma = np.where(np.angle(J) < -KMAH_ARG, -1.0, 1.0)
        amp = sigma * np.sqrt(Z.rho_s * Vsn / (q['rho'] * J))
        coef = Z.dth * wj * weight * amp
        ok = np.isfinite(coef) & np.isfinite(M)
        coef = np.where(ok, coef, 0.0)
        M = np.where(ok, M, 0.0)
        Mc = M.real + 1j * np.maximum(M.imag, 0.0)
        ph = np.exp(1j * om * (q['tau'][:, None] + px[:, None] * delta + 0.5 * Mc[:, None] * delta ** 2))
        _SP._scatter_add(out[w], r[:, None] * nx + np.arange(nx)[None, :], coef[:, None] * ph)
    return out


def arrivals_rows(Z, H, kmax=8, F=None):
    """count (n_rows, nx) uint8, T and A (n_rows, nx, kmax), overflow flag, on the branch's rows."""
    F = fields(Z, H) if F is None else F
    rho_r = Z.rho[Z.rows][None]
    with np.errstate(divide='ignore'):  # X_theta = 0 only on the source row, which has no crossing
        Acell = Z.c_ref ** 2 * np.sqrt(Z.rho_s / rho_r) / (
            Z.vel['v'] * np.sqrt(8 * np.pi * np.abs(F['Vsn'] * F['gsz']) * np.abs(F['Xt'])))
    D = F['X'] - Z.xs[0]
    fl = H['q'] > 0.5
    cross = fl[:-1] & fl[1:] & ((D[:-1] >= 0) != (D[1:] >= 0))
    nth, nr, nx = D.shape
    ks, rs, ixs = np.nonzero(cross)
    t = D[ks, rs, ixs] / (D[ks, rs, ixs] - D[ks + 1, rs, ixs])
    tau = F['tau']
    Tval = tau[ks, rs, ixs] + t * (tau[ks + 1, rs, ixs] - tau[ks, rs, ixs])
    Aval = Acell[ks, rs, ixs] + t * (Acell[ks + 1, rs, ixs] - Acell[ks, rs, ixs])
    count = np.zeros((nr, nx), np.uint8)
    T = np.zeros((nr, nx, kmax))
    A = np.zeros((nr, nx, kmax))
    overflow = False
    order = np.lexsort((ks, Tval, ixs, rs))
    per = {}
    for j in order:
        per.setdefault((rs[j], ixs[j]), []).append(j)
    for (rr, ix), js in per.items():
        if len(js) > kmax:
            overflow = True
        js = js[:kmax]
        count[rr, ix] = len(js)
        T[rr, ix, :len(js)] = Tval[js]
        A[rr, ix, :len(js)] = Aval[js]
    return count, T, A, overflow


def solve(problem, n_theta, theta_max, cfl=0.5, kmax=8, omegas=None, beam_width=None):
    """Both branches on the full grid: u (n_omega, nz, nx), count, T, A (nz, nx[, kmax]), overflow,
    and the two branch setups and label histories."""
    omegas = problem.omegas if omegas is None else omegas
    w0 = problem.beam_width if beam_width is None else beam_width
    medium = _md.medium_2d(problem)
    nz, nx = problem.nz, problem.nx
    u = np.zeros((len(omegas), nz, nx), np.complex128)
    count = np.zeros((nz, nx), np.uint8)
    T = np.zeros((nz, nx, kmax))
    A = np.zeros((nz, nx, kmax))
    overflow = False
    parts = {}
    for s in (1, -1):
        Z = ZSetup(problem, n_theta, theta_max, s, cfl, medium)
        H = march(Z)
        F = fields(Z, H)
        ub = green_rows(Z, H, omegas, w0, F)
        cb, Tb, Ab, ob = arrivals_rows(Z, H, kmax, F)
        keep = Z.rows >= Z.js if s == 1 else Z.rows < Z.js
        rows = Z.rows[keep]
        u[:, rows] = ub[:, keep]
        count[rows] = cb[keep]
        T[rows] = Tb[keep]
        A[rows] = Ab[keep]
        overflow |= bool(ob)
        parts[s] = (Z, H)
    return dict(u=u, count=count, T=T, A=A, overflow=overflow, parts=parts)


def ambiguous_nodes(problem, parts, tol, q_band=0.05):
    """Nodes whose arrival count hinges on a decision below the rounding of an FP32 evaluation: a
    sign change of X - x_s along theta with min |X - x_s| < tol (m), or with a source indicator
    within q_band of the 1/2 threshold at either cell."""
    nz, nx = problem.nz, problem.nx
    amb = np.zeros((nz, nx), bool)
    for s, part in parts.items():
        Z, H = part[0], part[1]
        D = H['X'] - Z.xs[0]
        q = H['q']
        cross = (D[:-1] >= 0) != (D[1:] >= 0)
        near = cross & (np.minimum(np.abs(D[:-1]), np.abs(D[1:])) < tol)
        near |= cross & ((np.abs(q[:-1] - 0.5) < q_band) | (np.abs(q[1:] - 0.5) < q_band))
        keep = Z.rows >= Z.js if s == 1 else Z.rows < Z.js
        amb[Z.rows[keep]] |= near.any(axis=0)[keep]
    return amb
