"""3-D Gaussian-beam superposition and arrival extraction (oracle, float64).  Test infrastructure only.

The 3-D form of the 2-D reading (oracle/superpose.py) on the labels of liouville3d.py: b (offset
of the ray from x_s at closest approach), n0 (take-off phase direction), q, tau.  Gamma = {b = 0}
(Eq. 35).  Only flagged cells count: q > 1/2 and not frozen.

Zero search.  A 3-vector b that vanishes on a 2-parameter family is projected on a fixed frame
(e1, e2) and the origin is located in triangles of a 2-D grid (edge functions cross(Pa, Pb) of the
projected vertex values; a zero edge function is decided by the lexicographic sign of Pb - Pa, so
that a point on an edge shared by two triangles belongs to exactly one of them).  Barycentric
weights of the origin interpolate every per-cell quantity.  frame(u): a the axis with the smallest
|u_a| (the first on ties), e1 = (E_a - u_a u)/|.|, e2 = u x e1.
  * Arrivals at a node x: the (theta, phi) sphere of directions in triangles (each quad of the
    grid split along its (k, j)-(k+1, j+1) diagonal, each polar cap a fan), frame(r_hat),
    r_hat = (x - x_s)/|x - x_s|; a zero is accepted when |b . r_hat| <= |x - x_s| / 4 (b is
    perpendicular to the take-off group direction, so a projected zero with b along r_hat is not a
    ray through x_s).
  * Beam centres: for each direction cell (theta_j, phi_k) and each grid plane normal to axis a,
    the plane's node grid in triangles, frame(g_s(n_kj)) (g_s the source medium's unit group
    direction at the cell's current direction); accepted when |b . g_s| <= |x_c - x_s| / 4.

Dynamic ray tracing from the label gradients (3-D form of Eqs. 21-26).  Label gradients are
second-order centred differences in x, y, z (one-sided at the grid edges), theta (continued across
the poles) and phi (periodic); the angular part is carried as the ambient tangent vector
grad_n u = u_th n_th + (u_ph / sin th) e_ph, so that values from cells on both sides of a pole can
be interpolated.  A phase-space perturbation is (dx, a1, a2) with direction change
dn = a1 t1 + a2 t2, (t1, t2) = frame(n).  At a point with take-off direction n0 (normalised), source
phase velocity v_s and group velocity V_s (G0 = V_s/|V_s|), frames (e1, e2) = frame(G0) and
(f1, f2) = frame(n0), rows R = [e_k . grad b; f_l . grad n0; e_t] (e_t = (V, dn/dt), the null
direction of every label), and a perturbation d solves R d = r:
  * point-source family (arrivals): r_j = (0, 0, delta_1j, delta_2j, 0); J_ps = det[dx_1, dx_2, V];
    A = c_ref^2 sqrt(rho_s/rho_r) / (4 pi v_s^(3/2) sqrt|J_ps|) = |u| of that arrival (the 3-D
    Green's function carries no omega factor);
  * Gaussian beam (reading of Eq. 24): the source Hessian M0 = i (2/(omega w0^2)) Pi^T Pi with
    Pi = I - V_s n0^T / v_s (the beam's 1/e half-width is w0 along the wavefront); a unit offset
    e_j at the source needs the take-off rotation with dp = M0 e_j, i.e.
    r_j = (delta_1j, delta_2j, kappa (A^-1 Q)_1j, kappa (A^-1 Q)_2j, 0), kappa = 2 i/(omega w0^2),
    A_kl = (e_k . f_l)/v_s - (e_k . n0)(V_s . f_l)/v_s^2 (dp/dn0 in the frames),
    Q_kj = (Pi e_k) . (Pi e_j).  Then
    M [dx_1, dx_2, V] = [dp_1, dp_2, pdot] and J = det[dx_1, dx_2, V] (det C of Eq. 26), with
    dp = p (pdot . dx) + dn / v - n (V . dn) / v^2;
    amplitude sigma sqrt(rho_s |V_s| / (rho J)), sigma = -1 where arg J < -1e-3.
Superposition (Eq. 34): each centre in a plane normal to axis a adds to the receivers x_r of that
plane (delta = x_r - x_c, delta_a = 0)
    W dOmega w_a coef exp(i omega (tau + p . delta + Re(delta^T M delta)/2)) exp(-omega max(Im(.), 0)/2)
with dOmega = dth dph sin th the cell's solid angle, W = i omega c_ref^2 / (8 pi^2 v_s^3)
(calibrated by stationary phase so that a homogeneous isotropic medium gives exp(ikr)/(4 pi r)),
and the take-off measure times the plane blend
    w_a = |det B_a| |det J_a| / sum_a' det(B_a')^2,
B_a the 2x2 Jacobian of (e_k . b) in the plane's two coordinates, J_a the 4x4 Jacobian of
(e_k . b, f_l . n0) in (plane coordinates, a1, a2).  sum_a' det(B_a')^2 = det(K)^2 |t|^2 with t
the ray tangent, so w_a sums to the take-off measure over the three plane families.
"""
from __future__ import annotations

import numpy as np

from . import christoffel as _ch

KMAH_ARG = 1e-3


def frame(u):
    """Orthonormal (e1, e2) perpendicular to the unit vectors u (..., 3), right-handed with u."""
    u = np.asarray(u, np.float64)
    a = np.argmin(np.abs(u), axis=-1)
    E = np.eye(3)[a]
    ua = np.take_along_axis(u, a[..., None], axis=-1)
    e1 = E - ua * u
    e1 = e1 / np.linalg.norm(e1, axis=-1, keepdims=True)
    e2 = np.cross(u, e1)
    return e1, e2


def _cross2(P, Q):
    return P[..., 0] * Q[..., 1] - P[..., 1] * Q[..., 0]


def _edge_sign(Pa, Pb):
    """Sign of the edge function cross(Pa, Pb); a zero is decided by the lexicographic sign of
    Pb - Pa (antisymmetric in the edge's direction)."""
    E = _cross2(Pa, Pb)
    dx = Pb[..., 0] - Pa[..., 0]
    dy = Pb[..., 1] - Pa[..., 1]
    tie = np.where((dx > 0) | ((dx == 0) & (dy > 0)), 1.0, -1.0)
    return np.where(E > 0, 1.0, np.where(E < 0, -1.0, tie))


def origin_in_triangle(P0, P1, P2):
    """inside (bool), barycentric weights (w0, w1, w2) of the origin in the projected triangles."""
    area = _cross2(P1 - P0, P2 - P0)
    s0, s1, s2 = _edge_sign(P0, P1), _edge_sign(P1, P2), _edge_sign(P2, P0)
    sa = np.sign(area)
    inside = (area != 0) & (s0 == sa) & (s1 == sa) & (s2 == sa)
    with np.errstate(divide='ignore', invalid='ignore'):
        w0 = _cross2(P1, P2) / area
        w1 = _cross2(P2, P0) / area
        w2 = _cross2(P0, P1) / area
    return inside, (w0, w1, w2)


def sphere_triangles(nth, nph):
    """Triangles of the (phi_k, theta_j) direction grid as (k, j) index triples, consistently
    oriented: each quad split along its (k, j)-(k+1, j+1) diagonal, each polar cap a fan."""
    tri = []
    for j in range(nth - 1):
        for k in range(nph):
            k1 = (k + 1) % nph
            tri.append(((k, j), (k1, j), (k1, j + 1)))
            tri.append(((k, j), (k1, j + 1), (k, j + 1)))
    for k in range(1, nph - 1):
        tri.append(((0, 0), (k + 1, 0), (k, 0)))
        tri.append(((0, nth - 1), (k, nth - 1), (k + 1, nth - 1)))
    return np.array(tri, np.int64)


def grad5(S, f, k, j, iz, iy, ix):
    """Centred derivatives of the cell field f (nph, nth, nz, ny, nx) in (x, y, z, theta, phi) at the
    cells (k, j, iz, iy, ix) (arrays): second order, one-sided second order at spatial edges, theta
    continued across the poles, phi periodic.  Returns (..., 5)."""
    out = []
    for axis, idx, n, h in ((4, ix, S.nx, S.hx), (3, iy, S.ny, S.hy), (2, iz, S.nz, S.hz)):
        def at(m):
            c = [k, j, iz, iy, ix]
            c[axis] = m
            return f[tuple(c)]
        lo, hi = idx == 0, idx == n - 1
        cen = (at(np.clip(idx + 1, 0, n - 1)) - at(np.clip(idx - 1, 0, n - 1))) / (2 * h)
        fwd = (4 * (at(np.minimum(idx + 1, n - 1)) - at(idx)) - (at(np.minimum(idx + 2, n - 1)) - at(idx))) / (2 * h)
        bwd = (4 * (at(idx) - at(np.maximum(idx - 1, 0))) - (at(idx) - at(np.maximum(idx - 2, 0)))) / (2 * h)
        out.append(np.where(lo, fwd, np.where(hi, bwd, cen)))
    nth, nph = S.nth, S.nph

    def ang(kk, jj):
        over = (jj < 0) | (jj >= nth)
        jr = np.where(jj < 0, -1 - jj, np.where(jj >= nth, 2 * nth - 1 - jj, jj))
        kr = np.where(over, (kk + nph // 2) % nph, kk)
        return f[kr, jr, iz, iy, ix]
    out.append((ang(k, j + 1) - ang(k, j - 1)) / (2 * S.dth))
    out.append((f[(k + 1) % nph, j, iz, iy, ix] - f[(k - 1) % nph, j, iz, iy, ix]) / (2 * S.dph))
    return np.stack(out, -1)


def _tangents(S, k, j):
    th, ph = S.theta[j], S.phi[k]
    n_th = np.stack([np.cos(th) * np.cos(ph), np.cos(th) * np.sin(ph), -np.sin(th)], -1)
    e_ph = np.stack([-np.sin(ph), np.cos(ph), np.zeros_like(ph)], -1)
    return th, n_th, e_ph


def grad6(S, f, k, j, iz, iy, ix):
    """Chart-free form of grad5: (d_x, d_y, d_z) and the ambient angular gradient
    grad_n f = f_th n_th + (f_ph / sin th) e_ph (tangent to the unit sphere).  Returns (..., 6)."""
    g = grad5(S, f, k, j, iz, iy, ix)
    th, n_th, e_ph = _tangents(S, k, j)
    gn = g[..., 3:4] * n_th + (g[..., 4] / np.sin(th))[..., None] * e_ph
    return np.concatenate([g[..., :3], gn], -1)


def _flags(S, lab):
    return (lab['q'] > 0.5) & ~S.frozen


def _ndot(S, vel, c):
    """dn/dt = thetadot n_th + phidot sin th e_ph at the cells c (ambient 3-vectors)."""
    th, n_th, e_ph = _tangents(S, c[0], c[1])
    return vel['thetadot'][c][..., None] * n_th + (vel['phidot'][c] * np.sin(th))[..., None] * e_ph


def _gather(S, lab, cells, w):
    """Barycentric interpolation of the quantities the dynamic ray tracing needs at the points with
    vertex cells cells[v] = (k, j, iz, iy, ix) (v = 0, 1, 2) and weights w[v]."""
    vel = S.vel
    acc = {}
    for v in range(3):
        c = cells[v]
        vals = {
            'n0': np.stack([lab[f][c] for f in ('n0x', 'n0y', 'n0z')], -1),
            'tau': lab['tau'][c],
            'V': np.stack([vel['Vx'][c], vel['Vy'][c], vel['Vz'][c]], -1),
            'v': vel['v'][c],
            'pdot': np.stack([vel['pdx'][c], vel['pdy'][c], vel['pdz'][c]], -1),
            'rho': S.rho[c[2], c[3], c[4]],
            'gb': np.stack([grad6(S, lab[f], *c) for f in ('bx', 'by', 'bz')], -2),
            'gn': np.stack([grad6(S, lab[f], *c) for f in ('n0x', 'n0y', 'n0z')], -2),
            'n': _ch.direction_3d(S.theta[c[1]], S.phi[c[0]]),
            'ndot': _ndot(S, vel, c),
        }
        for key, val in vals.items():
            wv = w[v].reshape(w[v].shape + (1,) * (val.ndim - w[v].ndim))
            acc[key] = acc.get(key, 0.0) + wv * val
    return acc


def _source_frames(S, n0):
    n0 = n0 / np.linalg.norm(n0, axis=-1, keepdims=True)
    vs, Vs, Vsn, G0 = _ch.source_quantities_3d(S.a_s, n0)
    e1, e2 = frame(G0)
    f1, f2 = frame(n0)
    return n0, vs, Vs, Vsn, e1, e2, f1, f2


def _rows(gb, gn, e1, e2, f1, f2, V, ndot, t1, t2):
    """R = [e1 . grad b; e2 . grad b; f1 . grad n0; f2 . grad n0; e_t] (..., 5, 5) in the unknowns
    (dx, dy, dz, a1, a2) of a perturbation with direction change dn = a1 t1 + a2 t2."""
    def row(G):
        return np.concatenate([G[..., :3], np.einsum('...i,...i->...', G[..., 3:], t1)[..., None],
                               np.einsum('...i,...i->...', G[..., 3:], t2)[..., None]], -1)
    r = [row(np.einsum('...i,...ic->...c', e, gb)) for e in (e1, e2)]
    r += [row(np.einsum('...i,...ic->...c', f, gn)) for f in (f1, f2)]
    r.append(row(np.concatenate([V, ndot], -1)))
    return np.stack(r, -2)


def arrivals3d(S, lab, kmax=8):
    """count (nz, ny, nx) uint8, T (nz, ny, nx, kmax), A (nz, ny, nx, kmax) (|u| of each arrival),
    overflow flag."""
    nz, ny, nx = S.nz, S.ny, S.nx
    flag = _flags(S, lab)
    X = (np.arange(nx) * S.hx + S.p.origin[0] - S.xs[0])[None, None, :]
    Y = (np.arange(ny) * S.hy + S.p.origin[1] - S.xs[1])[None, :, None]
    Z = (np.arange(nz) * S.hz + S.p.origin[2] - S.xs[2])[:, None, None]
    D = np.stack(np.broadcast_arrays(X, Y, Z), -1)
    r = np.linalg.norm(D, axis=-1)
    node_ok = r > S.r0
    rhat = D / np.where(r > 0, r, 1.0)[..., None]
    e1, e2 = frame(np.where(node_ok[..., None], rhat, np.array([0.0, 0.0, 1.0])))
    b = np.stack([lab['bx'], lab['by'], lab['bz']], -1)          # (nph, nth, nz, ny, nx, 3)
    beta = np.stack([np.einsum('...i,...i->...', b, e1[None, None]),
                     np.einsum('...i,...i->...', b, e2[None, None])], -1)
    brad = np.einsum('...i,...i->...', b, rhat[None, None])
    found = []
    for t in sphere_triangles(S.nth, S.nph):
        P = [beta[kk, jj] for kk, jj in t]
        inside, w = origin_in_triangle(*P)
        ok = inside & node_ok & flag[t[0][0], t[0][1]] & flag[t[1][0], t[1][1]] & flag[t[2][0], t[2][1]]
        if not ok.any():
            continue
        iz, iy, ix = np.nonzero(ok)
        ww = [wi[iz, iy, ix] for wi in w]
        bdot = sum(ww[v] * brad[t[v][0], t[v][1], iz, iy, ix] for v in range(3))
        keep = np.abs(bdot) <= 0.25 * r[iz, iy, ix]
        if not keep.any():
            continue
        found.append((t, iz[keep], iy[keep], ix[keep], [wi[keep] for wi in ww]))
    count = np.zeros((nz, ny, nx), np.uint8)
    T = np.zeros((nz, ny, nx, kmax))
    A = np.zeros((nz, ny, nx, kmax))
    if not found:
        return count, T, A, False
    rows = []
    for t, iz, iy, ix, ww in found:
        cells = [(np.full_like(iz, t[v][0]), np.full_like(iz, t[v][1]), iz, iy, ix) for v in range(3)]
        g = _gather(S, lab, cells, ww)
        n0, vs, Vs, Vsn, f_e1, f_e2, f1, f2 = _source_frames(S, g['n0'])
        nc = g['n'] / np.linalg.norm(g['n'], axis=-1, keepdims=True)
        t1, t2 = frame(nc)
        R = _rows(g['gb'], g['gn'], f_e1, f_e2, f1, f2, g['V'], g['ndot'], t1, t2)
        rhs = np.zeros(R.shape[:-2] + (5, 2))
        rhs[..., 2, 0] = 1.0
        rhs[..., 3, 1] = 1.0
        d = np.linalg.solve(R, rhs)
        Xm = np.stack([d[..., :3, 0], d[..., :3, 1], g['V']], -1)
        Jps = np.linalg.det(Xm)
        Aval = S.c_ref ** 2 * np.sqrt(S.rho_s / g['rho']) / (4 * np.pi * vs ** 1.5 * np.sqrt(np.abs(Jps)))
        ang = t[0][0] * S.nth + t[0][1]
        rows.append((iz, iy, ix, g['tau'], Aval, np.full_like(iz, ang)))
    iz, iy, ix, Tv, Av, ang = (np.concatenate(c) for c in zip(*rows))
    order = np.lexsort((ang, Tv, ix, iy, iz))
    overflow = False
    per = {}
    for q in order:
        per.setdefault((iz[q], iy[q], ix[q]), []).append(q)
    for key, qs in per.items():
        if len(qs) > kmax:
            overflow = True
        qs = qs[:kmax]
        count[key] = len(qs)
        T[key][:len(qs)] = Tv[qs]
        A[key][:len(qs)] = Av[qs]
    return count, T, A, overflow


# axis normal to the plane -> (state axis of the plane index, the two in-plane Cartesian components)
_PLANES = {'z': (2, (0, 1)), 'y': (3, (0, 2)), 'x': (4, (1, 2))}


def _plane_triangles(n1, n2):
    """Triangles of an n1 x n2 node grid (indices (i1, i2), i2 fastest), each quad split along its
    (i1, i2)-(i1+1, i2+1) diagonal, consistently oriented."""
    tri = []
    for i1 in range(n1 - 1):
        for i2 in range(n2 - 1):
            tri.append(((i1, i2), (i1, i2 + 1), (i1 + 1, i2 + 1)))
            tri.append(((i1, i2), (i1 + 1, i2 + 1), (i1 + 1, i2)))
    return np.array(tri, np.int64)


def beam_centres3d(S, lab, axis_name):
    """Points of Gamma on the grid planes normal to one axis, for every direction cell: list of dicts
    (direction k, j; plane index; centre position relative to x_s; vertex cells; weights)."""
    saxis, _ = _PLANES[axis_name]
    flag = _flags(S, lab)
    shape = {2: S.nz, 3: S.ny, 4: S.nx}
    inplane = [a for a in (2, 3, 4) if a != saxis]
    tri = _plane_triangles(shape[inplane[0]], shape[inplane[1]])
    pos = [(np.arange(n) * h + o - s) for n, h, o, s in
           ((S.nx, S.hx, S.p.origin[0], S.xs[0]), (S.ny, S.hy, S.p.origin[1], S.xs[1]),
            (S.nz, S.hz, S.p.origin[2], S.xs[2]))]
    out = []
    for k in range(S.nph):
        for j in range(S.nth):
            g = S.gs[k, j]
            e1, e2 = frame(g[None])
            b = np.stack([lab['bx'][k, j], lab['by'][k, j], lab['bz'][k, j]], -1)   # (nz, ny, nx, 3)
            bb = np.moveaxis(b, saxis - 2, 0)
            fl = np.moveaxis(flag[k, j], saxis - 2, 0)
            beta = np.stack([bb @ e1[0], bb @ e2[0]], -1)
            bg = bb @ g
            P = [beta[:, tri[:, v, 0], tri[:, v, 1]] for v in range(3)]
            inside, w = origin_in_triangle(*P)
            ok = (inside & fl[:, tri[:, 0, 0], tri[:, 0, 1]] & fl[:, tri[:, 1, 0], tri[:, 1, 1]]
                  & fl[:, tri[:, 2, 0], tri[:, 2, 1]])
            if not ok.any():
                continue
            ip, it = np.nonzero(ok)
            ww = [wi[ip, it] for wi in w]
            xc = 0.0
            cells = []
            for v in range(3):
                idx = {saxis: ip, inplane[0]: tri[it, v, 0], inplane[1]: tri[it, v, 1]}
                pv = np.stack([pos[0][idx[4]], pos[1][idx[3]], pos[2][idx[2]]], -1)
                xc = xc + ww[v][:, None] * pv
                cells.append((np.full_like(ip, k), np.full_like(ip, j), idx[2], idx[3], idx[4]))
            bgc = sum(ww[v] * bg[ip, tri[it, v, 0], tri[it, v, 1]] for v in range(3))
            keep = np.abs(bgc) <= 0.25 * np.linalg.norm(xc, axis=-1)
            if not keep.any():
                continue
            out.append(dict(k=np.full(keep.sum(), k), j=np.full(keep.sum(), j), plane=ip[keep],
                            xc=xc[keep], cells=[tuple(a[keep] for a in c) for c in cells],
                            w=[wi[keep] for wi in ww]))
    return out


def green3d(S, lab, omegas, beam_width):
    """u(omega, z, y, x) complex128: Gaussian beams centred on Gamma summed over the direction cells
    (Eq. 34) in the three plane families."""
    nz, ny, nx = S.nz, S.ny, S.nx
    u = np.zeros((len(omegas), nz, ny, nx), np.complex128)
    pos = [np.arange(nx) * S.hx + S.p.origin[0] - S.xs[0], np.arange(ny) * S.hy + S.p.origin[1] - S.xs[1],
           np.arange(nz) * S.hz + S.p.origin[2] - S.xs[2]]
    for name in ('z', 'y', 'x'):
        _, (c1, c2) = _PLANES[name]
        drop = {'z': 2, 'y': 1, 'x': 0}[name]
        for blk in beam_centres3d(S, lab, name):
            g = _gather(S, lab, blk['cells'], blk['w'])
            th = S.theta[blk['j']]
            n = _ch.direction_3d(th, S.phi[blk['k']])
            V, v, pdot = g['V'], g['v'], g['pdot']
            p = n / v[:, None]
            t1, t2 = frame(n)
            # dp/dn along the tangent directions: dp = dn / v - n (V . dn) / v^2
            dp_da = [t / v[:, None] - n * (np.einsum('ni,ni->n', V, t) / v ** 2)[:, None] for t in (t1, t2)]
            n0, vs, Vs, Vsn, e1, e2, f1, f2 = _source_frames(S, g['n0'])
            R = _rows(g['gb'], g['gn'], e1, e2, f1, f2, V, g['ndot'], t1, t2)
            # pairing of offsets with take-off rotations (source Hessian M0 = i c Pi^T Pi)
            Amat = np.stack([np.stack([np.einsum('ni,ni->n', e, f) / vs
                                       - np.einsum('ni,ni->n', e, n0) * np.einsum('ni,ni->n', Vs, f) / vs ** 2
                                       for f in (f1, f2)], -1) for e in (e1, e2)], -2)
            Pi_e = [e - Vs * (np.einsum('ni,ni->n', n0, e) / vs)[:, None] for e in (e1, e2)]
            Q = np.stack([np.stack([np.einsum('ni,ni->n', a, b) for b in Pi_e], -1) for a in Pi_e], -2)
            AQ = np.linalg.solve(Amat, Q)
            # blend of the plane families times the take-off measure
            Eb, Fn = R[:, 0:2, :], R[:, 2:4, :]
            dets = {a: np.linalg.det(Eb[:, :, [c for c in (0, 1, 2) if c != a]]) for a in (0, 1, 2)}
            Ssum = dets[0] ** 2 + dets[1] ** 2 + dets[2] ** 2
            Ja = np.concatenate([Eb, Fn], -2)[:, :, [c1, c2, 3, 4]]
            wj = np.abs(dets[drop]) * np.abs(np.linalg.det(Ja)) / Ssum
            for io, om in enumerate(omegas):
                kappa = 2j / (om * beam_width ** 2)
                rhs = np.zeros(R.shape[:-2] + (5, 2), np.complex128)
                rhs[:, 0, 0] = 1.0
                rhs[:, 1, 1] = 1.0
                rhs[:, 2:4, :] = kappa * AQ
                d = np.linalg.solve(R.astype(np.complex128), rhs)
                dx = d[:, :3, :]
                dp = (p[:, :, None] * np.einsum('ni,nij->nj', pdot, dx)[:, None, :]
                      + dp_da[0][:, :, None] * d[:, 3, None, :] + dp_da[1][:, :, None] * d[:, 4, None, :])
                Xm = np.concatenate([dx, V[:, :, None]], -1)
                Pm = np.concatenate([dp, pdot[:, :, None]], -1)
                M = np.swapaxes(np.linalg.solve(np.swapaxes(Xm, -1, -2), np.swapaxes(Pm, -1, -2)), -1, -2)
                J = np.linalg.det(Xm)
                sigma = np.where(np.angle(J) < -KMAH_ARG, -1.0, 1.0)
                amp = sigma * np.sqrt(S.rho_s * Vsn / (g['rho'] * J))
                W = 1j * om * S.c_ref ** 2 / (8 * np.pi ** 2 * vs ** 3)
                coef = W * S.dth * S.dph * np.sin(th) * wj * amp
                ok = np.isfinite(coef) & np.all(np.isfinite(M), axis=(-1, -2))
                coef = np.where(ok, coef, 0.0)
                M = np.where(ok[:, None, None], M, 0.0)
                d1 = pos[c1][None, :, None] - blk['xc'][:, c1, None, None]
                d2 = pos[c2][None, None, :] - blk['xc'][:, c2, None, None]
                quad = (M[:, c1, c1, None, None] * d1 * d1
                        + (M[:, c1, c2, None, None] + M[:, c2, c1, None, None]) * d1 * d2
                        + M[:, c2, c2, None, None] * d2 * d2)
                lin = p[:, c1, None, None] * d1 + p[:, c2, None, None] * d2
                ph_ = om * (g['tau'][:, None, None] + lin + 0.5 * quad.real)
                gauss = np.exp(-0.5 * om * np.maximum(quad.imag, 0.0))
                contrib = coef[:, None, None] * gauss * np.exp(1j * ph_)
                # contrib[:, i1, i2] with i1 along component c1 and i2 along c2; the receiver planes
                # are stored with the later component first, hence the transpose
                for q_, plane in enumerate(blk['plane']):
                    if name == 'z':
                        u[io, plane] += contrib[q_].T
                    elif name == 'y':
                        u[io, :, plane, :] += contrib[q_].T
                    else:
                        u[io, :, :, plane] += contrib[q_].T
    return u


def ambiguous_nodes3d(S, lab, tol=1e-4, q_band=0.05, spur_band=1e-3):
    """Nodes whose arrival count hinges on a decision below the rounding of an FP32 evaluation, for
    triangles of the direction sphere that (nearly) contain the projected origin (barycentric
    weights all >= -tol) and (nearly) pass the |b . r_hat| <= |x - x_s|/4 test: the origin within
    a relative distance tol of the triangle's boundary with every vertex flagged; a vertex source
    indicator within q_band of 1/2 (no vertex frozen); or |b . r_hat| within a relative spur_band of
    the bound with every vertex flagged."""
    nz, ny, nx = S.nz, S.ny, S.nx
    X = (np.arange(nx) * S.hx + S.p.origin[0] - S.xs[0])[None, None, :]
    Y = (np.arange(ny) * S.hy + S.p.origin[1] - S.xs[1])[None, :, None]
    Z = (np.arange(nz) * S.hz + S.p.origin[2] - S.xs[2])[:, None, None]
    D = np.stack(np.broadcast_arrays(X, Y, Z), -1)
    r = np.linalg.norm(D, axis=-1)
    rhat = D / np.where(r > 0, r, 1.0)[..., None]
    e1, e2 = frame(np.where((r > S.r0)[..., None], rhat, np.array([0.0, 0.0, 1.0])))
    b = np.stack([lab['bx'], lab['by'], lab['bz']], -1)
    beta = np.stack([np.einsum('...i,...i->...', b, e1[None, None]),
                     np.einsum('...i,...i->...', b, e2[None, None])], -1)
    brad = np.einsum('...i,...i->...', b, rhat[None, None])
    q = lab['q']
    flag = _flags(S, lab)
    out = np.zeros((nz, ny, nx), bool)
    lim = 0.25 * r
    for t in sphere_triangles(S.nth, S.nph):
        P = [beta[kk, jj] for kk, jj in t]
        area = _cross2(P[1] - P[0], P[2] - P[0])
        with np.errstate(divide='ignore', invalid='ignore', over='ignore'):
            w = [_cross2(P[1], P[2]) / area, _cross2(P[2], P[0]) / area, _cross2(P[0], P[1]) / area]
            wmin = np.minimum(np.minimum(w[0], w[1]), w[2])
            cand = np.isfinite(wmin) & (wmin >= -tol)
            bdot = np.where(cand, sum(np.where(cand, w[v], 0.0) * brad[t[v][0], t[v][1]] for v in range(3)), np.inf)
        fl = flag[t[0][0], t[0][1]] & flag[t[1][0], t[1][1]] & flag[t[2][0], t[2][1]]
        nofrozen = ~(S.frozen[t[0][0], t[0][1]] | S.frozen[t[1][0], t[1][1]] | S.frozen[t[2][0], t[2][1]])
        passes = cand & (np.abs(bdot) <= lim * (1 + spur_band))
        qn = np.zeros_like(cand)
        for kk, jj in t:
            qn |= np.abs(q[kk, jj] - 0.5) < q_band
        out |= passes & fl & (wmin <= tol)
        out |= passes & nofrozen & qn
        out |= cand & fl & (np.abs(np.abs(bdot) - lim) <= spur_band * lim)
    return out & (r > S.r0)
