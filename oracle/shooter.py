"""Lagrangian ray shooter (oracle pin for heterogeneous media).  Test infrastructure only.

Brute force, independent of the level-set machinery: a fan of take-off phase angles leaves the
source; every ray integrates the Hamiltonian system of the qP eigenvalue (the kinematics behind
Eqs. 8-12: dx/dt = V = a p g g, dp/dt = -1/2 g Gamma(grad a, p) g) with classical RK4 in
traveltime, in a medium interpolated bilinearly from the nodes (a and its node gradient).  Each
pair of neighbouring rays and consecutive time steps spans a ray-tube quadrilateral; every grid
node inside one (split into two triangles) is an arrival, with the traveltime interpolated
barycentrically.  The geometrical amplitude of an arrival uses the tube's spreading
J_t = |dx/dtheta_0 x V| (take-off angle, traveltime):
    A = c_ref^2 sqrt(rho_s / rho) / (v_s(theta_0) sqrt(8 pi J_t)),
the far field of the acoustic-scaled qP Green's function |u| sqrt(omega).
"""
from __future__ import annotations

import math

import numpy as np

from . import christoffel as _ch
from . import medium as _md


class Medium2D:
    """Bilinear interpolation of a, grad a, rho on the node grid of a 2-D problem."""

    def __init__(self, problem):
        self.p = problem
        self.a, self.dax, self.daz, self.rho = _md.medium_2d(problem)

    def _w(self, x, z):
        p = self.p
        fx = (x - p.origin[0]) / p.hx
        fz = (z - p.origin[1]) / p.hz
        ix = np.clip(np.floor(fx).astype(int), 0, p.nx - 2)
        iz = np.clip(np.floor(fz).astype(int), 0, p.nz - 2)
        tx = np.clip(fx - ix, 0.0, 1.0)[..., None]
        tz = np.clip(fz - iz, 0.0, 1.0)[..., None]
        return ix, iz, tx, tz

    def sample(self, field, x, z):
        ix, iz, tx, tz = self._w(x, z)
        shp = field.shape[2:]
        f00 = field[iz, ix].reshape(len(x), -1)
        f01 = field[iz, ix + 1].reshape(len(x), -1)
        f10 = field[iz + 1, ix].reshape(len(x), -1)
        f11 = field[iz + 1, ix + 1].reshape(len(x), -1)
        out = (1 - tz) * ((1 - tx) * f00 + tx * f01) + tz * ((1 - tx) * f10 + tx * f11)
        return out.reshape((len(x),) + shp)


def _rhs(M, x, z, px, pz):
    """Hamiltonian ray velocities at slowness (px, 0, pz) (the medium is interpolated)."""
    a = M.sample(M.a, x, z)
    dax = M.sample(M.dax, x, z)
    daz = M.sample(M.daz, x, z)
    p = np.stack([px, np.zeros_like(px), pz], -1)
    G = _ch.christoffel(a, p)
    lam, g = _ch.qp_eigen(G)
    ap = np.einsum('nijkl,nl->nijk', a, p)
    V = np.einsum('nijk,nj,nk->ni', ap, g, g)
    pdx = -0.5 * np.einsum('njl,nj,nl->n', _ch.christoffel(dax, p), g, g)
    pdz = -0.5 * np.einsum('njl,nj,nl->n', _ch.christoffel(daz, p), g, g)
    return V[:, 0], V[:, 2], pdx, pdz, lam


def shoot(problem, n_rays=2048, dt=None, t_max=None):
    """Trace the fan; returns dict with positions X, Z (steps, rays), times, take-off angles."""
    M = Medium2D(problem)
    xs, zs = problem.xs
    a_s = _md.bilinear_at(M.a, problem, xs, zs)
    th0 = 2 * np.pi * np.arange(n_rays) / n_rays
    vs, _, _, _ = _ch.source_quantities(a_s, th0)
    px, pz = np.sin(th0) / vs, np.cos(th0) / vs
    x = np.full(n_rays, float(xs))
    z = np.full(n_rays, float(zs))
    h = min(problem.hx, problem.hz)
    if dt is None:
        dt = 0.25 * h / float(np.max(vs) * 1.6)
    L = (problem.nx - 1) * problem.hx, (problem.nz - 1) * problem.hz
    if t_max is None:
        t_max = 3.0 * math.hypot(*L) / float(np.min(vs))
    X, Z, T = [x.copy()], [z.copy()], [0.0]
    alive = np.ones(n_rays, bool)
    exit_time = np.full(n_rays, np.nan)
    t = 0.0
    ox, oz = problem.origin
    while t < t_max and alive.any():
        def f(x_, z_, px_, pz_):
            Vx, Vz, pdx, pdz, _ = _rhs(M, x_, z_, px_, pz_)
            return Vx, Vz, pdx, pdz
        k1 = f(x, z, px, pz)
        k2 = f(x + 0.5 * dt * k1[0], z + 0.5 * dt * k1[1], px + 0.5 * dt * k1[2], pz + 0.5 * dt * k1[3])
        k3 = f(x + 0.5 * dt * k2[0], z + 0.5 * dt * k2[1], px + 0.5 * dt * k2[2], pz + 0.5 * dt * k2[3])
        k4 = f(x + dt * k3[0], z + dt * k3[1], px + dt * k3[2], pz + dt * k3[3])
        x = x + dt / 6 * (k1[0] + 2 * k2[0] + 2 * k3[0] + k4[0])
        z = z + dt / 6 * (k1[1] + 2 * k2[1] + 2 * k3[1] + k4[1])
        px = px + dt / 6 * (k1[2] + 2 * k2[2] + 2 * k3[2] + k4[2])
        pz = pz + dt / 6 * (k1[3] + 2 * k2[3] + 2 * k3[3] + k4[3])
        t += dt
        inside = (x >= ox) & (x <= ox + L[0]) & (z >= oz) & (z <= oz + L[1])
        newly = alive & ~inside
        exit_time[newly] = t
        alive &= inside
        X.append(x.copy())
        Z.append(z.copy())
        T.append(t)
    V = _rhs(M, x, z, px, pz)
    return dict(X=np.array(X), Z=np.array(Z), T=np.array(T), th0=th0, vs=vs, dt=dt,
                exit_time=exit_time, medium=M, a_s=a_s)


def arrivals(problem, fan, min_dist=0.0, node_mask=None):
    """Ray-tube arrivals at the grid nodes: count, sorted times and GO amplitudes per node.

    Each arrival is (T, A, J_t, m), m its KMAH index: the number of caustics the tube has passed,
    counted as sign changes of the signed spreading dx/dtheta_0 x V along the tube; the arrival's
    geometrical field is A exp(i (omega T + pi/4 - m pi/2)) / sqrt(omega).

    node_mask (nz, nx) bool, optional: collect arrivals only at these nodes (the others report 0),
    which bounds the work on large grids; the arrivals of a node do not depend on the others."""
    X, Z, T = fan['X'], fan['Z'], fan['T']
    M = fan['medium']
    nx, nz = problem.nx, problem.nz
    ox, oz = problem.origin
    ns, nr = X.shape
    i1 = np.roll(np.arange(nr), -1)
    dth = 2 * np.pi / nr
    # quad corners: (j, i), (j, i+1), (j+1, i+1), (j+1, i)
    ax, az = X[:-1, :], Z[:-1, :]
    bx, bz = X[:-1, i1], Z[:-1, i1]
    cx, cz = X[1:, i1], Z[1:, i1]
    dx_, dz_ = X[1:, :], Z[1:, :]
    t0 = T[:-1][:, None] * np.ones((1, nr))
    t1 = T[1:][:, None] * np.ones((1, nr))
    # spreading of each tube: |dx/dtheta0 x V| with V ~ (x(t+dt) - x(t)) / dt
    gx, gz = (bx - ax) / dth, (bz - az) / dth
    vx, vz = (dx_ - ax) / (T[1] - T[0]), (dz_ - az) / (T[1] - T[0])
    Js = gx * vz - gz * vx
    Jt = np.abs(Js)
    # KMAH index of each tube: the signed spreading changes sign once per caustic the tube passes
    sg = np.sign(Js)
    flips = np.zeros(Js.shape, np.int64)
    flips[1:] = (sg[1:] * sg[:-1]) < 0
    kmah = np.cumsum(flips, axis=0)
    out = {}
    s_rho = float(_md.bilinear_at(M.rho, problem, *problem.xs))
    vs = fan['vs']
    for tri in ((ax, az, bx, bz, cx, cz, t0, t0, t1), (ax, az, cx, cz, dx_, dz_, t0, t1, t1)):
        Ax, Az, Bx, Bz, Cx, Cz, ta, tb, tc = (np.asarray(q).ravel() for q in tri)
        ray = np.tile(np.arange(nr), ns - 1)
        jt = Jt.ravel()
        km = kmah.ravel()
        xmin = np.floor((np.minimum(np.minimum(Ax, Bx), Cx) - ox) / problem.hx).astype(int)
        xmax = np.floor((np.maximum(np.maximum(Ax, Bx), Cx) - ox) / problem.hx).astype(int)
        zmin = np.floor((np.minimum(np.minimum(Az, Bz), Cz) - oz) / problem.hz).astype(int)
        zmax = np.floor((np.maximum(np.maximum(Az, Bz), Cz) - oz) / problem.hz).astype(int)
        span = max(int(np.max(xmax - xmin)), int(np.max(zmax - zmin))) + 1 if len(xmin) else 0
        for di in range(span + 1):
            for dj in range(span + 1):
                ix = xmin + di
                iz = zmin + dj
                ok = (ix <= xmax) & (iz <= zmax) & (ix >= 0) & (ix < nx) & (iz >= 0) & (iz < nz)
                if not ok.any():
                    continue
                px = ox + ix * problem.hx
                pz = oz + iz * problem.hz
                den = (Bz - Cz) * (Ax - Cx) + (Cx - Bx) * (Az - Cz)
                with np.errstate(divide='ignore', invalid='ignore'):
                    l1 = ((Bz - Cz) * (px - Cx) + (Cx - Bx) * (pz - Cz)) / den
                    l2 = ((Cz - Az) * (px - Cx) + (Ax - Cx) * (pz - Cz)) / den
                    l3 = 1 - l1 - l2
                # half-open inclusion so a node on a shared edge is counted once
                inside = ok & (den != 0) & (l1 >= 0) & (l2 >= 0) & (l3 > 0)
                if node_mask is not None:
                    inside[inside] = node_mask[iz[inside], ix[inside]]
                for q in np.nonzero(inside)[0]:
                    key = (int(iz[q]), int(ix[q]))
                    tt = l1[q] * ta[q] + l2[q] * tb[q] + l3[q] * tc[q]
                    r = ray[q]
                    rho_r = float(M.sample(M.rho[..., None], np.array([px[q]]), np.array([pz[q]]))[0, 0])
                    c_ref = float(_ch.source_quantities(fan['a_s'], np.array([0.0]))[0][0])
                    A = c_ref ** 2 * math.sqrt(s_rho / rho_r) / (vs[r] * math.sqrt(8 * math.pi * max(jt[q], 1e-300)))
                    out.setdefault(key, []).append((tt, A, jt[q], int(km[q])))
    count = np.zeros((nz, nx), np.int32)
    first = np.full((nz, nx), np.nan)
    arr = {}
    for key, lst in out.items():
        lst.sort()
        # merge duplicates from coincident tube vertices (same time within a tiny tolerance)
        merged = []
        for item in lst:
            if merged and abs(item[0] - merged[-1][0]) < 1e-9:
                continue
            merged.append(item)
        count[key] = len(merged)
        first[key] = merged[0][0]
        arr[key] = merged
    return count, first, arr
