"""Dynamic ray tracing advected with the depth march (Eq. 21), oracle float64.

Test infrastructure only.

Eq. 21 advects the dynamic ray tracing quantities B and C over the phase space of one depth with
the same characteristic velocities as the labels (Eq. 16), with right-hand sides linear in (B, C);
the coefficients printed in Eqs. 22-23 are the isotropic ones with only u_1 changed.  Reading taken
here (anisotropic, in the depth march's own variables): a ray perturbation Q = (dx, dtheta) at
fixed depth follows the linearised flow of (dx/dz, dtheta/dz), so as a field over (x, theta) it
obeys
    Q_zeta + U Q_x + W Q_theta = J Q,   J = [[U_x, U_theta], [W_x, W_theta]],
with U, W of the depth march (oracle/zmarch.py, zeta = s (z - z_s)).  J is the second-order
difference of the tabulated U, W (one-sided at the ends of x and theta), interpolated linearly in
zeta between rows like U and W.  C = dx and B = dp_x = p_x pdot_x dx + (dp_x/dtheta) dtheta (the
paper's B C^-1 = M, Eq. 25).  Two real families start on the source row:
    Q1 = (1 / ghat_z(theta), 0)   (the offset db = 1 of the impact parameter),
    Q2 = (0, 1)                    (a unit change of take-off angle);
the complex beam of the label-gradient reading (transverse Hessian i 2/(omega w0^2)) is
Q1 + kappa Q2, kappa = 2 i |V_s| / (omega w0^2), and Q2 alone is the point-source family, whose
spreading at fixed depth J_t = |dx_2 Vz| gives the geometrical amplitude
    A = c_ref^2 sqrt(rho_s / rho_r) / (v_s(vartheta) sqrt(8 pi J_t))
(the ray-tube form of the Lagrangian shooter).  Everything else (centres, weights, KMAH sign,
arrival detection) is the depth march's.  WENO epsilon: 1e-6 times the squared scale of each
field (dx_1: 1, dtheta_1: 1/h^2, dx_2: h^2, dtheta_2: 1).
"""
from __future__ import annotations

import numpy as np

from . import christoffel as _ch
from . import superpose as _SP
from . import zmarch as _zm

QFIELDS = ('x1', 't1', 'x2', 't2')


def jacobian(Z):
    """dU/dx, dU/dtheta, dW/dx, dW/dtheta on every (theta, row, x) cell of the branch."""
    return (_zm._grad_x(Z.U, Z.hx), _zm._grad_t(Z.U, Z.dth),
            _zm._grad_x(Z.W, Z.hx), _zm._grad_t(Z.W, Z.dth))


def _rhs(Q, Z, U, W, J, eps):
    G = _zm.GHOST
    nth, nx = Z.nth, Z.nx
    adv = {}
    for f in QFIELDS:
        p = _zm._pad(Q[f])
        sx = {m: p[G:G + nth, G + m:G + m + nx] for m in range(-2, 3)}
        st = {m: p[G + m:G + m + nth, G:G + nx] for m in range(-2, 3)}
        dx = {j: sx[j + 1] - sx[j] for j in (-2, -1, 0, 1)}
        dt = {j: st[j + 1] - st[j] for j in (-2, -1, 0, 1)}
        adv[f] = -(U * _zm._weno3(dx, U, eps[f]) / Z.hx + W * _zm._weno3(dt, W, eps[f]) / Z.dth)
    Ux, Ut, Wx, Wt = J
    out = {}
    for a, b in (('x1', 't1'), ('x2', 't2')):
        out[a] = adv[a] + Ux * Q[a] + Ut * Q[b]
        out[b] = adv[b] + Wx * Q[a] + Wt * Q[b]
    return out


def march_q(Z):
    """Q1 and Q2 on every row of the branch: dict of (n_theta, n_rows, nx) arrays."""
    nth, nx, nr = Z.nth, Z.nx, len(Z.rows)
    _, _, _, gs = _ch.source_quantities(Z.a_s, Z.theta)
    Q = {'x1': np.broadcast_to((1.0 / gs[:, 1])[:, None], (nth, nx)).copy(),
         't1': np.zeros((nth, nx)), 'x2': np.zeros((nth, nx)), 't2': np.ones((nth, nx))}
    h = max(Z.hx, Z.hz)
    eps = {'x1': 1e-6, 't1': 1e-6 / h ** 2, 'x2': 1e-6 * h ** 2, 't2': 1e-6}
    Jt = jacobian(Z)
    hist = {f: np.empty((nth, nr, nx)) for f in QFIELDS}
    for f in QFIELDS:
        hist[f][:, 0] = Q[f]
    dz = 1.0 / Z.n_sub
    hh = Z.hz * dz
    for r in range(nr - 1):
        def coef(t):
            lin = lambda a: (1 - t) * a[:, r] + t * a[:, r + 1]
            return lin(Z.U), lin(Z.W), tuple(lin(j) for j in Jt)
        for n in range(Z.n_sub):
            t0 = n * dz
            L0 = _rhs(Q, Z, *coef(t0), eps)
            u1 = {f: Q[f] + hh * L0[f] for f in QFIELDS}
            L1 = _rhs(u1, Z, *coef(t0 + dz), eps)
            u2 = {f: 0.75 * Q[f] + 0.25 * (u1[f] + hh * L1[f]) for f in QFIELDS}
            L2 = _rhs(u2, Z, *coef(t0 + 0.5 * dz), eps)
            Q = {f: Q[f] / 3.0 + 2.0 / 3.0 * (u2[f] + hh * L2[f]) for f in QFIELDS}
        for f in QFIELDS:
            hist[f][:, r + 1] = Q[f]
    return hist


def green_rows_q(Z, H, Qh, omegas, beam_width):
    """u(omega, r, x) on the branch's rows with the beams' dynamic ray tracing taken from the
    advected Q fields: (dx, dtheta) = Q1 + kappa Q2 at each centre; the take-off measure along a row
    |det J2| / |X_x| equals 1 / |dtheta_2| (the columns of J2^-1 are ghat_z Q1 and Q2)."""
    D = H['X'] - Z.xs[0]
    nth, nr, nx = D.shape
    fl = H['q'] > 0.5
    cross = fl[..., :-1] & fl[..., 1:] & ((D[..., :-1] >= 0) != (D[..., 1:] >= 0))
    k, r, i = np.nonzero(cross)
    c0, c1 = (k, r, i), (k, r, i + 1)
    t = D[c0] / (D[c0] - D[c1])
    L = _zm._lin
    q = {nm: L(H[nm], c0, c1, t) for nm in ('tau', 'Th')}
    for nm in QFIELDS:
        q[nm] = L(Qh[nm], c0, c1, t)
    for nm in ('Vx', 'Vz', 'pdx', 'v'):
        q[nm] = L(Z.vel[nm], c0, c1, t)
    rho = Z.rho[Z.rows]
    q['rho'] = rho[r, i] + t * (rho[r, i + 1] - rho[r, i])
    th = Z.theta[k]
    vs, _, Vsn, _ = _ch.source_quantities(Z.a_s, q['Th'])
    out = np.zeros((len(omegas), nr, nx), np.complex128)
    xc = Z.x[i] + t * Z.hx
    delta = Z.x[None, :] - xc[:, None]
    v = q['v']
    px = np.sin(th) / v
    v_th = np.cos(th) * q['Vx'] - np.sin(th) * q['Vz']
    dpx_dth = (np.cos(th) * v - np.sin(th) * v_th) / v ** 2
    wj = 1.0 / np.abs(q['t2'])
    weight = 1j * Z.c_ref ** 2 / (4 * np.pi * vs ** 2)
    for w, om in enumerate(omegas):
        kappa = 2j * Vsn / (om * beam_width ** 2)
        dx = q['x1'] + kappa * q['x2']
        dth = q['t1'] + kappa * q['t2']
        dpx = px * q['pdx'] * dx + dpx_dth * dth
        M = dpx / dx
        J = dx * q['Vz']
        sigma = np.where(np.angle(J) < -_zm.KMAH_ARG, -1.0, 1.0)
        amp = sigma * np.sqrt(Z.rho_s * Vsn / (q['rho'] * J))
        coef = Z.dth * wj * weight * amp
        ok = np.isfinite(coef) & np.isfinite(M)
        coef = np.where(ok, coef, 0.0)
        M = np.where(ok, M, 0.0)
        Mc = M.real + 1j * np.maximum(M.imag, 0.0)
        ph = np.exp(1j * om * (q['tau'][:, None] + px[:, None] * delta + 0.5 * Mc[:, None] * delta ** 2))
        _SP._scatter_add(out[w], r[:, None] * nx + np.arange(nx)[None, :], coef[:, None] * ph)
    return out


def arrivals_rows_q(Z, H, Qh, kmax=8):
    """Arrivals as in the depth march, amplitudes from the point-source family Q2:
    A = c_ref^2 sqrt(rho_s / rho_r) / (v_s(vartheta) sqrt(8 pi |dx_2 Vz|))."""
    vs, _, _, _ = _ch.source_quantities(Z.a_s, H['Th'])
    rho_r = Z.rho[Z.rows][None]
    with np.errstate(divide='ignore'):  # dx_2 = 0 only on the source row, which has no crossing
        Acell = Z.c_ref ** 2 * np.sqrt(Z.rho_s / rho_r) / (
            vs * np.sqrt(8 * np.pi * np.abs(Qh['x2'] * Z.vel['Vz'])))
    D = H['X'] - Z.xs[0]
    fl = H['q'] > 0.5
    cross = fl[:-1] & fl[1:] & ((D[:-1] >= 0) != (D[1:] >= 0))
    nth, nr, nx = D.shape
    ks, rs, ixs = np.nonzero(cross)
    t = D[ks, rs, ixs] / (D[ks, rs, ixs] - D[ks + 1, rs, ixs])
    tau = H['tau']
    Tval = tau[ks, rs, ixs] + t * (tau[ks + 1, rs, ixs] - tau[ks, rs, ixs])
    Aval = Acell[ks, rs, ixs] + t * (Acell[ks + 1, rs, ixs] - Acell[ks, rs, ixs])
    count = np.zeros((nr, nx), np.uint8)
    T = np.zeros((nr, nx, kmax))
    A = np.zeros((nr, nx, kmax))
    overflow = False
    per = {}
    for j in np.lexsort((ks, Tval, ixs, rs)):
        per.setdefault((rs[j], ixs[j]), []).append(j)
    for (rr, ix), js in per.items():
        overflow |= len(js) > kmax
        js = js[:kmax]
        count[rr, ix] = len(js)
        T[rr, ix, :len(js)] = Tval[js]
        A[rr, ix, :len(js)] = Aval[js]
    return count, T, A, overflow


def solve(problem, n_theta, theta_max, cfl=0.5, kmax=8, omegas=None, beam_width=None):
    """Both branches with the advected dynamic ray tracing; outputs as zmarch.solve."""
    from . import medium as _md
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
        Z = _zm.ZSetup(problem, n_theta, theta_max, s, cfl, medium)
        H = _zm.march(Z)
        Qh = march_q(Z)
        ub = green_rows_q(Z, H, Qh, omegas, w0)
        cb, Tb, Ab, ob = arrivals_rows_q(Z, H, Qh, kmax)
        keep = Z.rows >= Z.js if s == 1 else Z.rows < Z.js
        rows = Z.rows[keep]
        u[:, rows] = ub[:, keep]
        count[rows] = cb[keep]
        T[rows] = Tb[keep]
        A[rows] = Ab[keep]
        overflow |= bool(ob)
        parts[s] = (Z, H, Qh)
    return dict(u=u, count=count, T=T, A=A, overflow=overflow, parts=parts)
