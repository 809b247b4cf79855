"""Pins for the oracle's Gaussian-beam superposition and arrival extraction (Eqs. 24-26, 33-35).

The labels fed in here are the closed-form steady state of a homogeneous medium, so these tests
check the superposition alone:
* isotropic: u -> (i/4) H0^(1)(kr) with a relative L2 error that falls as kr grows, and the result
  does not depend on the beam width to the same order (Gaussian-beam summation theory);
* isotropic arrivals: exactly one arrival per node, T = r/v, A = |(i/4) H0| sqrt(omega) = sqrt(v/(8 pi r));
* VTI: the far field of the exact plane-wave integral (stationary phase), traveltimes r/|V_g| along
  the Thomsen group direction.
"""
import math

import numpy as np
import pytest

import synthmedia
from oracle import christoffel as CH
from oracle import closed_forms as CF
from oracle import liouville as L
from oracle import superpose as SP


def _exact_setup(problem, vel=None):
    S = L.Setup(problem, vel=vel)
    x = np.arange(S.nx) * S.hx - S.xs[0]
    z = np.arange(S.nz) * S.hz - S.xs[1]
    Z, X = np.meshgrid(z, x, indexing='ij')
    v, V, Vn, g = CH.source_quantities(S.a_s, S.theta)
    p = np.stack([np.sin(S.theta) / v, np.cos(S.theta) / v], -1)
    lab = CF.homogeneous_labels(S.theta, X, Z, g, p, S.R_sigma)
    edge = np.minimum(np.minimum(X - X.min(), X.max() - X), np.minimum(Z - Z.min(), Z.max() - Z))
    return S, lab, X, Z, edge


@pytest.fixture(scope='module')
def iso():
    p = synthmedia.isotropic_homogeneous(n=128, h=10.0, n_theta=384, freqs=[60.0])
    return (p,) + _exact_setup(p)


def _band_errors(u, ref, kr, mask, bands):
    out = []
    for lo, hi in bands:
        m = mask & (kr >= lo) & (kr < hi)
        out.append(np.linalg.norm(u[m] - ref[m]) / np.linalg.norm(ref[m]))
    return np.array(out)


def test_isotropic_hankel_convergence(iso):
    p, S, lab, X, Z, edge = iso
    om = 2 * math.pi * 60.0
    k = om / p.meta['vp']
    r = np.hypot(X, Z)
    ref = CF.hankel_green_2d(k, np.where(r > 0, r, 1.0))
    u = SP.green(S, lab, [om], 100.0)[0]
    bands = [(5, 10), (10, 20), (20, 40)]
    err = _band_errors(u, ref, k * r, edge > 0.25 * 128 * 10.0, bands)
    assert err[-1] < 0.02, err
    assert np.all(np.diff(err) < 0), err


def test_isotropic_beam_width_independence(iso):
    p, S, lab, X, Z, edge = iso
    om = 2 * math.pi * 60.0
    k = om / p.meta['vp']
    r = np.hypot(X, Z)
    u1 = SP.green(S, lab, [om], 100.0)[0]
    u2 = SP.green(S, lab, [om], 200.0)[0]
    m = (edge > 0.25 * 128 * 10.0) & (k * r >= 20) & (k * r < 40)
    assert np.linalg.norm(u1[m] - u2[m]) / np.linalg.norm(u1[m]) < 0.02


def test_isotropic_arrivals(iso):
    p, S, lab, X, Z, edge = iso
    c = p.meta['vp']
    cnt, T, A, overflow = SP.arrivals(S, lab)
    r = np.hypot(X, Z)
    m = r > 3 * S.r0
    assert not overflow
    assert np.all(cnt[m] == 1)
    assert np.max(np.abs(T[..., 0][m] - r[m] / c) / (r[m] / c)) < 2e-4
    Aref = np.sqrt(c / (8 * math.pi * r[m]))
    assert np.max(np.abs(A[..., 0][m] - Aref) / Aref) < 2e-4


@pytest.fixture(scope='module')
def vti():
    p = synthmedia.vti_homogeneous(n=128, h=10.0, n_theta=384, freqs=[60.0])
    return (p,) + _exact_setup(p)


def test_vti_far_field_matches_plane_wave_integral(vti):
    p, S, lab, X, Z, edge = vti
    m = p.meta
    om = 2 * math.pi * 60.0
    v_of = lambda th: CF.thomsen_vti_phase_velocity(th, m['vp0'], m['vs0'], m['eps'], m['delta'])
    V_of = lambda th: CF.vti_group_velocity(th, m['vp0'], m['vs0'], m['eps'], m['delta'])[1:]
    r = np.hypot(X, Z)
    sel = (edge > 0.25 * 128 * 10.0) & (r > 350.0)
    ref, T, _ = CF.homogeneous_go_green(X[sel], Z[sel], 0.0, 0.0, om, v_of, V_of, m['vp0'])
    u = SP.green(S, lab, [om], 100.0)[0][sel]
    assert np.linalg.norm(u - ref) / np.linalg.norm(ref) < 0.03
    cnt, Ta, A, _ = SP.arrivals(S, lab)
    assert np.all(cnt[sel] == 1)
    assert np.max(np.abs(Ta[..., 0][sel] - T) / T) < 2e-4
    Aref = np.abs(ref) * math.sqrt(om)
    assert np.max(np.abs(A[..., 0][sel] - Aref) / Aref) < 2e-3


def test_heterogeneous_wavefield_is_bounded():
    """In a heterogeneous TTI medium every beam that enters the sum decays along its evaluation
    line, so the Green's function stays of the order of the homogeneous one (no runaway Gaussians)."""
    p = synthmedia.tti_heterogeneous(n=80, n_theta=48, length=2560.0, steps=220, freqs=(10.0, 20.0))
    S, st, dt = L.evolve(p)
    lab = L.interior_state(st, S)
    u = SP.green(S, lab, p.omegas, p.beam_width)
    assert np.all(np.isfinite(u))
    assert np.max(np.abs(u)) < 1.0


# ---- receiver-side (reciprocal) reduction of the same labels (Eq. 34 read through reciprocity) ----

def _wide_tube(p, R_sigma, vel=None):
    """The same medium with a source-ray tube of radius R_sigma (vel: its velocity fields, when
    already computed, which do not depend on the tube)."""
    import dataclasses
    return _exact_setup(dataclasses.replace(p, R_sigma=R_sigma), vel=vel)


@pytest.fixture(scope='module')
def iso_wide(iso):
    """The isotropic medium with a 400 m source-ray tube: the receiver-side beams reach x_s about
    w(r) = w0 sqrt(1 + (2 r / (k w0^2))^2) wide (143 m at 640 m, 60 Hz, w0 = 100 m) and need the
    labels of rays up to about 2 w(r) from the source."""
    p, S = iso[0], iso[1]
    return (p,) + _wide_tube(p, 400.0, vel=S.vel)


def test_receiver_side_hankel_convergence(iso_wide):
    p, S, lab, X, Z, edge = iso_wide
    om = 2 * math.pi * 60.0
    k = om / p.meta['vp']
    r = np.hypot(X, Z)
    ref = CF.hankel_green_2d(k, np.where(r > 0, r, 1.0))
    u = SP.green_receiver(S, lab, [om], 100.0)[0]
    err = _band_errors(u, ref, k * r, edge > 0.25 * 128 * 10.0, [(5, 10), (10, 20), (20, 40), (40, 80)])
    print('receiver-side vs (i/4) H0 by kr band', err)
    assert np.all(np.diff(err) < 0) and err[2] < 0.01 and err[3] < 0.01, err


def test_receiver_side_beam_width_independence(iso_wide):
    p, S, lab, X, Z, edge = iso_wide
    om = 2 * math.pi * 60.0
    k = om / p.meta['vp']
    r = np.hypot(X, Z)
    u1, u2 = (SP.green_receiver(S, lab, [om], w)[0] for w in (100.0, 150.0))
    m = (edge > 0.25 * 128 * 10.0) & (k * r >= 20) & (k * r < 80)
    assert np.linalg.norm(u1[m] - u2[m]) / np.linalg.norm(u1[m]) < 0.02


def test_receiver_side_vti_far_field(vti):
    """VTI: the receiver-side sum of the closed-form labels (tube widened to 400 m) against the
    stationary-phase evaluation of the exact plane-wave integral, and against the source-side sum."""
    p0 = vti[0]
    p, S, lab, X, Z, edge = (p0,) + _wide_tube(p0, 400.0, vel=vti[1].vel)
    m = p.meta
    om = 2 * math.pi * 60.0
    v_of = lambda th: CF.thomsen_vti_phase_velocity(th, m['vp0'], m['vs0'], m['eps'], m['delta'])
    V_of = lambda th: CF.vti_group_velocity(th, m['vp0'], m['vs0'], m['eps'], m['delta'])[1:]
    r = np.hypot(X, Z)
    sel = (edge > 0.25 * 128 * 10.0) & (r > 350.0)
    ref, T, _ = CF.homogeneous_go_green(X[sel], Z[sel], 0.0, 0.0, om, v_of, V_of, m['vp0'])
    ur = SP.green_receiver(S, lab, [om], 100.0)[0][sel]
    us = SP.green(S, lab, [om], 100.0)[0][sel]
    assert np.linalg.norm(ur - ref) / np.linalg.norm(ref) < 0.015
    assert np.linalg.norm(ur - us) / np.linalg.norm(us) < 0.03


@pytest.mark.slow
def test_receiver_side_agrees_with_source_side_in_a_heterogeneous_medium():
    """TTI (64^2 at 40 m, 96 angles) with a 900 m source-ray tube: at receivers 200-600 m from
    the source, well inside the tube, the two reductions of the same labels agree as the frequency
    grows.  (Beyond the frozen disc's radius they part: the disc's straight-ray closest-approach
    data are only accurate where the medium varies little across it.)"""
    import dataclasses
    p = synthmedia.tti_heterogeneous(n=64, n_theta=96, length=2560.0, steps=400, freqs=(20.0, 40.0, 80.0),
                                     beam_width=150.0)
    p = dataclasses.replace(p, R_sigma=900.0)
    S, st, dt = L.evolve(p)
    lab = L.interior_state(st, S)
    us = SP.green(S, lab, p.omegas, p.beam_width)
    ur = SP.green_receiver(S, lab, p.omegas, p.beam_width)
    x = np.arange(p.nx) * p.hx - p.xs[0]
    z = np.arange(p.nz) * p.hz - p.xs[1]
    Z, X = np.meshgrid(z, x, indexing='ij')
    r = np.hypot(X, Z)
    m = (r >= 200) & (r < 600)
    e = [np.linalg.norm(ur[w][m] - us[w][m]) / np.linalg.norm(us[w][m]) for w in range(3)]
    med = [np.median(np.abs(ur[w][m] / us[w][m] - 1)) for w in range(3)]
    print('receiver vs source side, L2', e, 'median', med)
    assert e[1] < 0.1 and e[2] < 0.1 and med[2] < med[0] and med[2] < 0.06
