"""Pins for the oracle's level-set advection (Eqs. 16, 19, 20 in pseudo-time; HJ-WENO3 + TVD-RK3).

Checked against: exactness of WENO3 on linear data, its third-order convergence on smooth data,
exact rotation of the angle label across the 2 pi wrap, frozen source ball and Dirichlet ghosts left
bit-for-bit untouched, agreement of the compiled loop with the array code, and the closed-form
steady state of a homogeneous VTI medium (straight rays: b = (x - x_s) x g(theta), vartheta = theta,
tau = p(theta) . (x - x_s)).
"""
import math
import types

import numpy as np
import pytest

import synthmedia
from oracle import christoffel as CH
from oracle import liouville as L
from oracle import superpose as SP


def test_weno3_exact_on_linear_data():
    rng = np.random.default_rng(0)
    slope = rng.normal(size=50)
    d = [slope] * 4
    um, up = L._weno3_pair(*d, eps=1e-6)
    assert np.allclose(um, slope, rtol=1e-14) and np.allclose(up, slope, rtol=1e-14)


def test_weno3_third_order_on_smooth_data():
    errs = []
    for n in (40, 80, 160):
        h = 1.0 / n
        x = np.arange(-2, 3) * h + 0.3
        u = np.sin(2 * np.pi * x)
        d = np.diff(u)
        um, up = L._weno3_pair(d[0], d[1], d[2], d[3], eps=1e-6 * h * h)
        exact = 2 * np.pi * np.cos(2 * np.pi * 0.3)
        errs.append(max(abs(um / h - exact), abs(up / h - exact)))
    rates = np.log2(np.array(errs[:-1]) / np.array(errs[1:]))
    assert np.all(rates > 2.6), rates


def _fake_setup(nth, nz, nx, vx=0.0, vz=0.0, vt=0.0, h=1.0):
    S = types.SimpleNamespace()
    S.nth, S.nz, S.nx = nth, nz, nx
    S.hx = S.hz = h
    S.dth = 2 * math.pi / nth
    shape = (nth, nz, nx)
    S.vel = {'Vx': np.full(shape, vx), 'Vz': np.full(shape, vz), 'thetadot': np.full(shape, vt)}
    S.frozen = np.zeros((nth, nz, nx), bool)
    S.eps = {'b': 1e-6, 'q': 1e-6, 'Th': 1e-6 * S.dth ** 2, 'tau': 1e-6}
    return S


def _padded(S, f):
    return np.pad(f, ((0, 0), (L.GHOST, L.GHOST), (L.GHOST, L.GHOST)), mode='edge')


def test_angle_label_rotates_exactly_across_wrap():
    """d_t Th + w d_theta Th = 0 with Th = theta: solution theta - w t, across the 2 pi seam."""
    S = _fake_setup(32, 3, 3, vt=1.3)
    th = S.dth * np.arange(32)
    st = {f: _padded(S, np.zeros((32, 3, 3))) for f in L.FIELDS}
    st['Th'] = _padded(S, np.broadcast_to(th[:, None, None], (32, 3, 3)).copy())
    dt = 0.4 * S.dth / 1.3
    for _ in range(10):
        st = L.rk3_step(st, S, dt)
    got = L._interior(st['Th'], S)[:, 1, 1]
    exp = th - 1.3 * 10 * dt
    assert np.max(np.abs(L._wrap(got - exp))) < 1e-12


def test_smooth_theta_advection_third_order():
    errs = []
    for nth in (64, 128, 256):
        S = _fake_setup(nth, 3, 3, vt=1.0)
        th = S.dth * np.arange(nth)
        u0 = np.exp(np.cos(th))
        st = {f: _padded(S, np.zeros((nth, 3, 3))) for f in L.FIELDS}
        st['b'] = _padded(S, np.broadcast_to(u0[:, None, None], (nth, 3, 3)).copy())
        T = 0.5
        steps = int(math.ceil(T / (0.3 * S.dth)))
        dt = T / steps
        for _ in range(steps):
            st = L.rk3_step(st, S, dt)
        got = L._interior(st['b'], S)[:, 1, 1]
        errs.append(np.max(np.abs(got - np.exp(np.cos(th - T)))))
    rates = np.log2(np.array(errs[:-1]) / np.array(errs[1:]))
    assert np.all(rates > 2.5), (errs, rates)


@pytest.fixture(scope='module')
def vti_small():
    p = synthmedia.vti_homogeneous(n=40, h=10.0, n_theta=48, steps=140)
    S = L.Setup(p)
    return p, S


def test_c_loop_equals_array_code(vti_small):
    p, S = vti_small
    st0 = S.initial_state()
    _, a, _ = L.evolve(p, steps=2, S=S, state=st0, backend='numpy')
    _, b, _ = L.evolve(p, steps=2, S=S, state=st0, backend='c')
    for f in L.FIELDS:
        assert np.max(np.abs(a[f] - b[f])) <= 1e-12 * max(1.0, np.max(np.abs(a[f])))


def test_frozen_cells_and_ghosts_untouched(vti_small):
    p, S = vti_small
    st0 = S.initial_state()
    _, st, _ = L.evolve(p, steps=5, S=S, state=st0)
    G = L.GHOST
    for f in L.FIELDS:
        a, b = st[f], st0[f]
        assert np.array_equal(a[:, :G], b[:, :G]) and np.array_equal(a[:, -G:], b[:, -G:])
        assert np.array_equal(a[:, :, :G], b[:, :, :G]) and np.array_equal(a[:, :, -G:], b[:, :, -G:])
        ia, ib = L._interior(a, S), L._interior(b, S)
        assert np.array_equal(ia[S.frozen], ib[S.frozen])


def test_homogeneous_vti_steady_state_closed_form(vti_small):
    """After the transients leave, every source-labelled cell carries the straight-ray invariants."""
    p, S = vti_small
    _, st, dt = L.evolve(p)
    lab = L.interior_state(st, S)
    F = SP.beam_fields(S, lab)
    x = np.arange(S.nx) * S.hx - S.xs[0]
    z = np.arange(S.nz) * S.hz - S.xs[1]
    Z, X = np.meshgrid(z, x, indexing='ij')
    v, V, Vn, g = CH.source_quantities(S.a_s, S.theta)
    b_ref = X[None] * g[:, 1, None, None] - Z[None] * g[:, 0, None, None]
    tau_ref = (np.sin(S.theta) / v)[:, None, None] * X[None] + (np.cos(S.theta) / v)[:, None, None] * Z[None]
    # cells whose ray passed closest to the source inside the disc, a few cells away from its edge
    sel = F['flag'] & (np.abs(b_ref) < 0.5 * S.R_sigma)
    assert sel.sum() > 1000
    assert np.max(np.abs(lab['b'][sel] - b_ref[sel])) < 1e-9
    assert np.max(np.abs(L._wrap(lab['Th'][sel] - np.broadcast_to(S.theta[:, None, None], sel.shape)[sel]))) < 1e-9
    assert np.max(np.abs(lab['tau'][sel] - tau_ref[sel])) < 1e-9
    # the source indicator is 1 up to the smeared edge of the tube (|b| ~ R_Sigma)
    assert np.mean(lab['q'][sel] > 0.99) > 0.99


def test_pooled_velocity_planes_equal_the_serial_ones():
    p = synthmedia.tti_heterogeneous(n=24, n_theta=12, length=2560.0, steps=5, freqs=(10.0,))
    from oracle import medium as OM
    a, dx, dz, _ = OM.medium_2d(p)
    serial = CH.velocity_field_2d(a, dx, dz, p.n_theta)
    pooled = L.velocity_field_pooled(p, processes=3)
    for key in serial:
        assert np.array_equal(serial[key], pooled[key]), key
