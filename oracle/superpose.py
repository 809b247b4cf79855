"""Gaussian-beam superposition and arrival extraction (oracle, float64).  Test infrastructure only.

The paper forms a Gaussian beam about each point of the source manifold Gamma = {X = x_s} (Eq. 35)
with complex traveltime tau + p.(x - X) + 1/2 (x - X)^T M (x - X) (Eq. 25, M = B C^-1 from the
dynamic ray tracing of Eq. 21 with the complex initial data of Eq. 24), amplitude from det C
(Eq. 26), and sums the beams over Gamma with the weight Psi_0 of Eq. 33 (Eq. 34).

Reading taken here (the paper's Eqs. 24 and 28-33 are garbled or isotropic-only):

* The ray through a phase cell (x, theta) carries the level-set labels (b, q, vartheta, tau): b
  its signed distance from x_s at closest approach (2-D cross product a x b = a_x b_z - a_z b_x),
  q = 1 when those labels come from the source manifold, so Gamma = {b = 0} (Eq. 35).
* Beam centres: for every theta and every grid row, each sign change of b between neighbouring
  ball-origin cells is one point of Gamma; everything there is interpolated linearly.  The beam is
  evaluated at the receivers of the same row with the horizontal offset (the paper's same-depth
  evaluation); flat rays are served the same way along grid columns, and the two are blended by
  the partition of unity b_x^2/|grad b|^2 + b_z^2/|grad b|^2 = 1 of the level line of b (in a
  homogeneous medium grad b is normal to the ray, so this is g_z^2 + g_x^2 of the group direction).
* Dynamic ray tracing from the level sets (in place of advecting Eq. 21): with k1 = grad b,
  k2 = grad vartheta (centred differences in x, z, theta) and e_t = (Vx, Vz, thetadot), the
  phase-space perturbation with (db, dvartheta) = (1, kappa) is
      d = (k2 x e_t + kappa e_t x k1) / (e_t . (k1 x k2));
  kappa = 2 i |V_s| / (omega w0^2) gives the beam a wavefront Hessian i 2/(omega w0^2) at the source
  (|beam| = 1/e at w0; the complex initial data of Eq. 24).  With dx = (d_x, d_z) and
  dp = p (pdot . dx) + dp/dtheta d_theta, M [dx, V] = [dp, pdot] gives the Cartesian Hessian
  (Eq. 25's M = B C^-1) and J = dx x V the complex spreading (det C of Eq. 26).
* Amplitude (Eq. 26 with the elastic transport div(rho U^2 V) = 0): rho_s |V_s| / (rho J) under a
  square root continued along the ray.  J never vanishes for the complex beam family (its real and
  imaginary parts, the offset and take-off families, never vanish together), and its argument grows
  by pi at every caustic (KMAH index), so the principal root is right only up to the first
  crossing of the negative real axis.  The continued argument is followed per phase cell through
  the pseudo-time evolution (`track_branch`): alpha, the argument of the reference spreading
  J_ref = J_b + i J_T / w0 (offset family plus the take-off family scaled by 1/w0), is re-lifted
  every BRANCH_SAMPLE steps to the value of the current principal argument nearest to it.  With the
  labels fixed, the homotopy from the initial straight-ray data (no caustic) to the steady state
  carries alpha continuously onto the argument continued along the ray.  At a beam centre
  k = rint((alpha_c - arg J_ref) / 2 pi) and sigma = (-1)^k multiplies the principal root: every
  frequency's J = J_b + kappa J_T has the sign of Im J_ref, so the same k continues all of them.
* Weight (the calibrated Psi_0 of Eqs. 30-33): i c_ref^2 / (4 pi v_s(vartheta)^2) times the
  take-off measure |d vartheta_c / d theta| dtheta, so that a homogeneous isotropic medium gives
  the 2-D Helmholtz Green's function (i/4) H0^(1)(kr) as kr -> inf; the output is rho_s c_ref^2
  times the scalar qP Green's function (c_ref: source phase velocity along +z), phase exp(+i omega T)
  (Eq. 2).
* Only rays that carry source labels and have left the frozen manifold count (q > 1/2, not frozen).

Arrivals (late arrivals included, Eq. 35): along theta at a node, every sign change of b between
cells k and k+1 (sign(0) = +1) where both cells are flagged; T is tau interpolated
linearly at b = 0 and A the geometrical amplitude |u| sqrt(omega) of that ray,
      A = c_ref^2 sqrt(rho_s / rho_r) / (v_r sqrt(8 pi |V_s| |d_theta b|)),
interpolated the same way.  Arrivals are sorted by T (then by angle index), at most kmax kept.
"""
from __future__ import annotations

import math

import numpy as np

from . import christoffel as _ch


# steps between two samples of the continued argument of the complex spreading (track_branch)
BRANCH_SAMPLE = 9


def _wrap(d):
    return (d + np.pi) % (2.0 * np.pi) - np.pi


def _grad_axis(f, h, axis, wrap):
    """Second-order centred difference along x or z, second-order one-sided at the two edges."""
    f = np.moveaxis(f, axis, -1)
    out = np.empty_like(f)
    d = (lambda a: _wrap(a)) if wrap else (lambda a: a)
    out[..., 1:-1] = d(f[..., 2:] - f[..., :-2]) / (2 * h)
    out[..., 0] = (4 * d(f[..., 1] - f[..., 0]) - d(f[..., 2] - f[..., 0])) / (2 * h)
    out[..., -1] = (4 * d(f[..., -1] - f[..., -2]) - d(f[..., -1] - f[..., -3])) / (2 * h)
    return np.moveaxis(out, -1, axis)


def _grad_theta(f, dth, wrap):
    d = np.roll(f, -1, axis=0) - np.roll(f, 1, axis=0)
    if wrap:
        d = _wrap(d)
    return d / (2 * dth)


def _label_gradients(S, b, Th):
    return dict(bx=_grad_axis(b, S.hx, 2, False), bz=_grad_axis(b, S.hz, 1, False),
                bt=_grad_theta(b, S.dth, False),
                Tx=_grad_axis(Th, S.hx, 2, True), Tz=_grad_axis(Th, S.hz, 1, True),
                Tt=_grad_theta(Th, S.dth, True))


def _families(et, k1, k2):
    """Phase-space perturbations (last axis 3) with (db, dvartheta) = (1, 0) and (0, 1) that keep the
    ray direction e_t: d_b = (k2 x e_t) / D, d_T = (e_t x k1) / D, D = e_t . (k1 x k2).

    D is the orientation of the label coordinates (b, vartheta, tau): e_t is parallel to
    k1 x k2, and D / |e_t|^2 = det[grad b, grad vartheta, grad tau].  The label map is one-to-one on
    the source tube and equals the straight-ray data there at the start, where D < 0, so D < 0
    throughout; a positive discrete D (centred differences of under-resolved labels) is taken as
    -|D|, which keeps J's orientation (a sign flip of D alone would multiply the amplitude by
    +-i) and makes the argument of J continuous where the discrete D passes through zero."""
    D = -np.abs(np.einsum('...i,...i->...', et, np.cross(k1, k2)))
    return np.cross(k2, et) / D[..., None], np.cross(et, k1) / D[..., None]


def reference_arg(S, b, Th):
    """Per cell: principal argument of J_ref = J_b + i J_T / w0, the complex spreading dx x V of the
    offset family (J_b) plus the take-off family scaled by the beam width (J_T), from the centred
    label gradients; NaN where the level-set Jacobian is singular."""
    G = _label_gradients(S, b, Th)
    et = np.stack([S.vel['Vx'], S.vel['Vz'], S.vel['thetadot']], -1)
    k1 = np.stack([G['bx'], G['bz'], G['bt']], -1)
    k2 = np.stack([G['Tx'], G['Tz'], G['Tt']], -1)
    with np.errstate(divide='ignore', invalid='ignore'):
        d_b, d_T = _families(et, k1, k2)
        Jb = d_b[..., 0] * S.vel['Vz'] - d_b[..., 1] * S.vel['Vx']
        JT = d_T[..., 0] * S.vel['Vz'] - d_T[..., 1] * S.vel['Vx']
        a = np.arctan2(JT / S.p.beam_width, Jb)
    return np.where(np.isfinite(Jb) & np.isfinite(JT), a, np.nan)


def lift_branch(alpha, a):
    """The value a + 2 pi k (k integer) nearest to alpha; alpha itself where a is undefined."""
    lifted = a + 2.0 * np.pi * np.rint((alpha - a) / (2.0 * np.pi))
    return np.where(np.isfinite(a), lifted, alpha)


def track_branch(S, lab, alpha=None):
    """One sample of the continued argument of the complex spreading on every cell (interior
    labels b, vartheta of shape (n_theta, nz, nx)): alpha lifted to the current principal argument,
    or that argument itself when alpha is None (the initial data, which has no caustic)."""
    a = reference_arg(S, lab['b'], lab['Th'])
    if alpha is None:
        return np.where(np.isfinite(a), a, 0.0)
    return lift_branch(alpha, a)


# The last beam_fields result with the objects it was computed from (held, so that their ids stay
# theirs): the label arrays are treated as immutable, so a later call on the same setup and the same
# label arrays returns it instead of recomputing (the per-cell eigen-solves dominate a beam sum).
_fields_memo = {'key': None, 'F': None}


def beam_fields(S, lab):
    """Frequency-independent per-cell quantities of the superposition (all float64)."""
    key = (S, lab) + tuple(lab.get(k) for k in ('b', 'q', 'Th', 'tau', 'alpha'))
    old = _fields_memo['key']
    if old is not None and len(old) == len(key) and all(a is c for a, c in zip(old, key)):
        return _fields_memo['F']
    F = _beam_fields(S, lab)
    _fields_memo['key'], _fields_memo['F'] = key, F
    return F


def _beam_fields(S, lab):
    b, q, Th, tau = lab['b'], lab['q'], lab['Th'], lab['tau']
    vs, Vs, Vsn, gs = _ch.source_quantities(S.a_s, Th)
    F = dict(b=b, tau=tau, vs=vs, Vs=Vs, Vsn=Vsn, gs=gs, Th=Th,
             # rays whose labels came from the source manifold and that have left it
             flag=(q > 0.5) & ~S.frozen)
    F.update(_label_gradients(S, b, Th))
    # the continued argument, sampled once more on the labels being superposed; labels given without
    # one (closed-form steady states of caustic-free media) take the principal argument
    F['alpha'] = track_branch(S, lab, lab.get('alpha'))
    return F


def _interp(a, i0, i1, t):
    return a[i0] + t * (a[i1] - a[i0])


def crossings(S, lab, F, axis):
    """Points of the source manifold Gamma = {b = 0} on grid rows (axis=2) or columns (axis=1).

    For each theta and each row (column), every sign change of b between neighbouring nodes
    (both flagged as ball-origin, sign(0) = +1) is one beam centre; its position and every per-cell
    quantity are interpolated linearly between the two nodes.  Returns a dict of 1-D arrays.
    """
    b, flag = F['b'], F['flag']
    sl0 = [slice(None)] * 3
    sl1 = [slice(None)] * 3
    sl0[axis] = slice(0, -1)
    sl1[axis] = slice(1, None)
    b0, b1 = b[tuple(sl0)], b[tuple(sl1)]
    cross = flag[tuple(sl0)] & flag[tuple(sl1)] & ((b0 >= 0) != (b1 >= 0))
    k, iz, ix = np.nonzero(cross)
    c1 = (k, iz + (axis == 1), ix + (axis == 2))
    c0 = (k, iz, ix)
    t = b[c0] / (b[c0] - b[c1])
    out = dict(k=k, iz=iz, ix=ix, t=t)
    names = ('tau', 'bx', 'bz', 'bt', 'Tx', 'Tz', 'Tt', 'alpha')
    for nm in names:
        out[nm] = _interp(F[nm], c0, c1, t)
    for nm in ('Vx', 'Vz', 'thetadot', 'pdx', 'pdz', 'v'):
        out[nm] = _interp(S.vel[nm], c0, c1, t)
    rho = np.broadcast_to(S.rho[None], b.shape)
    out['rho'] = _interp(rho, c0, c1, t)
    Th = lab['Th']
    out['Th'] = Th[c0] + t * _wrap(Th[c1] - Th[c0])
    return out


def beam_centres(S, lab, F, axis, omega, beam_width):
    """Complex Gaussian beam at each crossing of Gamma with a row (axis=2) or column (axis=1).

    Dynamic ray tracing from the level sets (Eqs. 21-24): with k1 = grad b, k2 = grad vartheta and
    e_t = (Vx, Vz, thetadot) (the null direction of both), the phase-space perturbation with
    (db, dvartheta) = (1, kappa) is d = (k2 x e_t + kappa e_t x k1) / (e_t . (k1 x k2)).
    kappa = 2 i |V_s| / (omega w0^2) makes the beam's wavefront Hessian at the source i 2/(omega w0^2)
    (the complex initial data of Eq. 24, w0 the beam width).  With dx = (d_x, d_z) and
    dp = p (pdot . dx) + dp/dtheta d_theta, the Cartesian Hessian solves M [dx, V] = [dp, pdot]
    (Eq. 25's M = B C^-1) and the complex spreading is J = dx x V (det C of Eq. 26).
    """
    c = crossings(S, lab, F, axis)
    if c['k'].size == 0:
        return c, None
    th = S.theta[c['k']]
    n = np.stack([np.sin(th), np.cos(th)], -1)
    nth_ = np.stack([np.cos(th), -np.sin(th)], -1)
    V = np.stack([c['Vx'], c['Vz']], -1)
    pdot = np.stack([c['pdx'], c['pdz']], -1)
    v = c['v']
    et = np.stack([c['Vx'], c['Vz'], c['thetadot']], -1)
    k1 = np.stack([c['bx'], c['bz'], c['bt']], -1)
    k2 = np.stack([c['Tx'], c['Tz'], c['Tt']], -1)
    d_b, d_T = _families(et, k1, k2)
    vs, _, Vsn, _ = _ch.source_quantities(S.a_s, c['Th'])
    kappa = 2j * Vsn / (omega * beam_width ** 2)
    d = d_b + kappa[:, None] * d_T
    dx = d[:, :2]
    dth = d[:, 2]
    p = n / v[:, None]
    v_th = np.einsum('ni,ni->n', nth_, V)
    dp_dth = (nth_ * v[:, None] - n * v_th[:, None]) / (v ** 2)[:, None]
    dp = p * np.einsum('ni,ni->n', pdot, dx)[:, None] + dp_dth * dth[:, None]
    J = dx[:, 0] * V[:, 1] - dx[:, 1] * V[:, 0]
    J_theta = d_T[:, 0] * V[:, 1] - d_T[:, 1] * V[:, 0]
    Mxx = (dp[:, 0] * V[:, 1] - pdot[:, 0] * dx[:, 1]) / J
    Mzz = (-dp[:, 1] * V[:, 0] + pdot[:, 1] * dx[:, 0]) / J
    # Square root continued along the ray: the continued argument alpha of J_ref at the centre
    # fixes the sheet, k = rint((alpha - arg J_ref) / 2 pi), sigma = (-1)^k on the principal root.
    Jb = d_b[:, 0] * V[:, 1] - d_b[:, 1] * V[:, 0]
    a_ref = np.arctan2(J_theta / S.p.beam_width, Jb)
    k = np.rint((c['alpha'] - a_ref) / (2.0 * np.pi))
    sigma = np.where(np.mod(k, 2.0) == 0.0, 1.0, -1.0)
    amp = sigma * np.sqrt(S.rho_s * Vsn / (c['rho'] * J))
    # Take-off measure along the line times the row/column blend.  Along a row the beam centre moves
    # with theta as dx_c/dtheta = -b_theta/b_x, so d vartheta_c/dtheta = vartheta_theta -
    # vartheta_x b_theta/b_x; the blend is b_x^2/|grad_x b|^2 for rows and b_z^2/|grad_x b|^2 for
    # columns (the two add up to 1; in a homogeneous medium grad_x b is normal to the ray and this is
    # g_z^2 and g_x^2).  Their product stays bounded where the level line of b runs along the grid
    # line: |vartheta_theta b_l - vartheta_l b_theta| |b_l| / |grad_x b|^2.
    g2 = c['bx'] ** 2 + c['bz'] ** 2
    if axis == 2:
        wj = np.abs(c['Tt'] * c['bx'] - c['Tx'] * c['bt']) * np.abs(c['bx']) / g2
        M, pl = Mxx, p[:, 0]
    else:
        wj = np.abs(c['Tt'] * c['bz'] - c['Tz'] * c['bt']) * np.abs(c['bz']) / g2
        M, pl = Mzz, p[:, 1]
    weight = 1j * S.c_ref ** 2 / (4 * np.pi * vs ** 2)
    coef = S.dth * wj * weight * amp
    # A centre where the level-set Jacobian is singular (no finite beam) carries no weight.
    ok = np.isfinite(coef) & np.isfinite(M)
    coef = np.where(ok, coef, 0.0)
    M = np.where(ok, M, 0.0)
    return c, dict(coef=coef, M=M, p=pl)


def _scatter_add(u, flat, vals):
    """u.flat[flat] += vals, summing repeated indices (np.add.at, written with bincount)."""
    n = u.size
    f, v = flat.ravel(), vals.ravel()
    u += (np.bincount(f, weights=v.real, minlength=n)
          + 1j * np.bincount(f, weights=v.imag, minlength=n)).reshape(u.shape)


def green(S, lab, omegas, beam_width):
    """u(omega, z, x) complex128: Gaussian beams centred on Gamma summed over theta (Eq. 34).

    Beams are centred where Gamma crosses the receiver's row (offset x0 - x_c along the row, the
    paper's same-depth evaluation) and where it crosses the receiver's column (offset along the
    column, for flat rays); the two are blended by b_x^2/|grad b|^2 and b_z^2/|grad b|^2.  Each adds
        dtheta |d vartheta_c / d theta| w c exp(i omega (tau_c + p_l delta + M_ll delta^2 / 2))
    with c = i c_ref^2 / (4 pi v_s(vartheta)^2) sigma sqrt(rho_s |V_s| / (rho J)).
    """
    F = beam_fields(S, lab)
    out = []
    xg = S.hx * np.arange(S.nx)
    zg = S.hz * np.arange(S.nz)
    for om in omegas:
        u = np.zeros((S.nz, S.nx), np.complex128)
        for axis in (2, 1):
            c, bc = beam_centres(S, lab, F, axis, om, beam_width)
            if bc is None:
                continue
            if axis == 2:
                xc = xg[c['ix']] + c['t'] * S.hx
                delta = xg[None, :] - xc[:, None]
            else:
                zc = zg[c['iz']] + c['t'] * S.hz
                delta = zg[None, :] - zc[:, None]
            # Im M annihilates V, so Im M_ll >= 0 along a grid line up to discretisation error; the
            # Gaussian factor uses max(Im M_ll, 0) so that no beam grows away from its centre
            M = bc['M'][:, None]
            Mc = M.real + 1j * np.maximum(M.imag, 0.0)
            ph = np.exp(1j * om * (c['tau'][:, None] + bc['p'][:, None] * delta
                                   + 0.5 * Mc * delta ** 2))
            contrib = bc['coef'][:, None] * ph
            if axis == 2:
                _scatter_add(u, c['iz'][:, None] * S.nx + np.arange(S.nx)[None, :], contrib)
            else:
                _scatter_add(u, np.arange(S.nz)[None, :] * S.nx + c['ix'][:, None], contrib)
        out.append(u)
    return np.stack(out)


def green_receiver(S, lab, omegas, beam_width):
    """u(omega, z, x) complex128 by the receiver-side (reciprocal) reduction of the same labels.

    Eq. 34 read from the receiver: by reciprocity the Green's function at x0 of the source x_s is
    that at x_s of a source at x0, and it is summed from Gaussian beams launched at x0 along every
    ray through x0 that carries source labels (q > 1/2, not frozen), evaluated at x_s.  The ray
    through the cell (x0, theta) passes closest to x_s at C, at signed offset b, with phase angle
    vartheta, tau after C.  A beam launched back along it with the perturbation
    (dx_perp, dtheta) = (1, kappa0), kappa0 = -2 i |V0| / (omega w0^2) (the source side's initial
    data mirrored for the reversed direction), reaches C with the offset and angle changes
        db = b_perp + kappa0 b_theta,   dvartheta = vartheta_perp + kappa0 vartheta_theta
    (the label Jacobian at x0 is the ray propagator to C; perp is along the unit normal
    (g_z, -g_x) of the group direction g, the direction in which b grows).  Its Hessian there is
    M = -(dp/dvartheta . (g_z, -g_x)) dvartheta / db (slowness of the source medium at vartheta; the
    minus for the reversed ray), and its phase at x_s is tau + M b^2 / 2: tau already holds the
    plane-wave part p_C . (x_C - x_s) of the offset.  Im M is taken from the beam's Wronskian
    instead of the label Jacobian: the ray propagator is symplectic, so Im(conj(Q) P) keeps its
    initial value and Im M = 2 |V0| (dp/dtheta . (g_z, -g_x))_x0 / (omega w0^2 |db|^2) exactly; the
    label Jacobian satisfies this only up to its discretisation error, which near the edge of the
    source-ray tube (labels bending onto boundary data) can leave Im M near zero at a small |db|, a
    large undamped term whose phase then hangs on the last digit of the labels.  With the elastic
    transport the amplitude there is sqrt(rho0 |V0| / (rho_s |V_s(vartheta)| db)) (principal root:
    rays with no caustic, KMAH index 0), the weight per dtheta is i c0^2 / (4 pi v0(theta)^2) (c0 the phase velocity along +z at x0;
    the same calibration as the source side, which gives (i/4) H0^(1)(kr) in a homogeneous isotropic
    medium), and the sum, rho0 c0^2 times the Green's function, is rescaled by
    rho_s c_s^2 / (rho0 c0^2) to the source side's normalisation.
    """
    # the label gradients, the source flag and the source medium at vartheta are those of the
    # source-side sum (beam_fields)
    G = beam_fields(S, lab)
    b, Th, tau, flag = G['b'], G['Th'], G['tau'], G['flag']
    Vx, Vz, v0 = S.vel['Vx'], S.vel['Vz'], S.vel['v']
    V0 = np.hypot(Vx, Vz)
    gx, gz = Vx / V0, Vz / V0
    b_perp = G['bx'] * gz - G['bz'] * gx
    t_perp = G['Tx'] * gz - G['Tz'] * gx
    # source medium at the closest approach: slowness derivative along vartheta, |V_s|
    vs, Vs, Vsn, gs = G['vs'], G['Vs'], G['Vsn'], G['gs']
    n = np.stack([np.sin(Th), np.cos(Th)], -1)
    n_t = np.stack([np.cos(Th), -np.sin(Th)], -1)
    vs_t = np.einsum('...i,...i->...', Vs, n_t)
    dp_dt = (n_t * vs[..., None] - n * vs_t[..., None]) / (vs ** 2)[..., None]
    dp_perp = dp_dt[..., 0] * gs[..., 1] - dp_dt[..., 1] * gs[..., 0]
    # receiver medium at the cell's own angle theta: dp/dtheta . (g_z, -g_x), which fixes Im M
    # (n = (sin, cos), n_t = dn/dtheta = (cos, -sin), dv/dtheta = V . n_t)
    sn, cn = np.sin(S.theta)[:, None, None], np.cos(S.theta)[:, None, None]
    v0_t = Vx * cn - Vz * sn
    dp0_x = (cn * v0 - sn * v0_t) / v0 ** 2
    dp0_z = (-sn * v0 - cn * v0_t) / v0 ** 2
    dp0_perp = dp0_x * gz - dp0_z * gx
    # receiver medium: density and the qP phase velocity along +z (c0) per node
    rho0 = S.rho[None, :, :]
    lam, _ = _ch.qp_eigen(_ch.christoffel(S.a, np.array([0.0, 0.0, 1.0])))
    c0 = np.sqrt(lam)[None, :, :]
    out = []
    for om in omegas:
        kap = -2j * V0 / (om * beam_width ** 2)
        db = b_perp + kap * G['bt']
        dth = t_perp + kap * G['Tt']
        M = (-dp_perp * dth / db).real + 1j * 2 * V0 * dp0_perp / (om * beam_width ** 2 * np.abs(db) ** 2)
        amp = np.sqrt(rho0 * V0 / (S.rho_s * Vsn * db))
        w = 1j * c0 ** 2 / (4 * np.pi * v0 ** 2) * S.dth
        term = w * amp * np.exp(1j * om * (tau + 0.5 * M * b ** 2))
        term = np.where(flag & np.isfinite(term), term, 0.0)
        u = term.sum(axis=0)
        out.append(u * (S.rho_s * S.c_ref ** 2) / (S.rho * c0[0] ** 2))
    return np.stack(out)


def arrivals(S, lab, kmax=8, kmah=False):
    """count (nz, nx) uint8, T (nz, nx, kmax) float64, A (nz, nx, kmax) float64, overflow flag;
    with kmah=True also M (nz, nx, kmax) int, each arrival's KMAH index: the number of caustics its
    ray has passed, floor(alpha / pi) of the continued argument alpha of the complex spreading,
    interpolated at the crossing like T (it grows by pi at every caustic; 0 < alpha < pi on the
    straight-ray initial data downstream of the source)."""
    F = beam_fields(S, lab)
    v_r = S.vel['v']
    rho_r = S.rho[None, :, :]
    # Cells with d b / d theta = 0 (b constant along theta: rays from the boundary, or a caustic of
    # the point-source family) have no finite geometrical amplitude; they are inf here and must not
    # reach a counted crossing (checked below).
    with np.errstate(divide='ignore'):
        Acell = S.c_ref ** 2 * np.sqrt(S.rho_s / rho_r) / (
            v_r * np.sqrt(8 * np.pi * F['Vsn'] * np.abs(F['bt'])))
    b, tau, flag, alpha = F['b'], F['tau'], F['flag'], F['alpha']
    bn, taun, flagn, An, alphan = (np.roll(a, -1, axis=0) for a in (b, tau, flag, Acell, alpha))
    cross = flag & flagn & ((b >= 0) != (bn >= 0))
    nth, nz, nx = b.shape
    count = np.zeros((nz, nx), np.uint8)
    T = np.zeros((nz, nx, kmax))
    A = np.zeros((nz, nx, kmax))
    overflow = False
    ks, izs, ixs = np.nonzero(cross)
    t = b[ks, izs, ixs] / (b[ks, izs, ixs] - bn[ks, izs, ixs])
    Tval = tau[ks, izs, ixs] + t * (taun[ks, izs, ixs] - tau[ks, izs, ixs])
    with np.errstate(invalid='ignore'):
        Aval = Acell[ks, izs, ixs] + t * (An[ks, izs, ixs] - Acell[ks, izs, ixs])
    if not np.all(np.isfinite(Aval)):
        bad = np.flatnonzero(~np.isfinite(Aval))[0]
        raise FloatingPointError(
            'arrival at node (%d, %d), angle cell %d lies on a cell with d b / d theta = 0: '
            'its geometrical amplitude is undefined' % (izs[bad], ixs[bad], ks[bad]))
    Mval = np.floor((alpha[ks, izs, ixs] + t * (alphan[ks, izs, ixs] - alpha[ks, izs, ixs])) / np.pi)
    M = np.zeros((nz, nx, kmax), np.int64)
    order = np.lexsort((ks, Tval, ixs, izs))
    per_node = {}
    for j in order:
        per_node.setdefault((izs[j], ixs[j]), []).append(j)
    for (iz, ix), js in per_node.items():
        if len(js) > kmax:
            overflow = True
        js = js[:kmax]
        count[iz, ix] = len(js)
        T[iz, ix, :len(js)] = Tval[js]
        A[iz, ix, :len(js)] = Aval[js]
        M[iz, ix, :len(js)] = Mval[js]
    if kmah:
        return count, T, A, overflow, M
    return count, T, A, overflow


def min_abs_b_at_crossings(S, lab):
    """Per node, the smallest |b| over the two cells of any counted crossing (inf if none)."""
    F = beam_fields(S, lab)
    b, flag = F['b'], F['flag']
    bn, flagn = np.roll(b, -1, axis=0), np.roll(flag, -1, axis=0)
    cross = flag & flagn & ((b >= 0) != (bn >= 0))
    m = np.where(cross, np.minimum(np.abs(b), np.abs(bn)), np.inf)
    return m.min(axis=0)


def ambiguous_nodes(S, lab, b_tol, q_band=0.05):
    """Nodes whose arrival count hinges on a decision below the rounding of an FP32 evaluation:
    a sign change of b (between any two theta-neighbours) with min |b| < b_tol, or with a source
    indicator q within q_band of the 1/2 threshold at either cell."""
    b, q = lab['b'], lab['q']
    bn, qn = np.roll(b, -1, axis=0), np.roll(q, -1, axis=0)
    cross = (b >= 0) != (bn >= 0)
    near_b = cross & (np.minimum(np.abs(b), np.abs(bn)) < b_tol)
    near_q = cross & ((np.abs(q - 0.5) < q_band) | (np.abs(qn - 0.5) < q_band))
    return (near_b | near_q).any(axis=0)
