"""Pins for the advected dynamic ray tracing of the depth march (Eq. 21, oracle/zmarch_drt.py).

* Homogeneous VTI: the point-source family is Q2 = ((z - z_s) dU/dtheta, 1) and the offset family
  Q1 = (1 / ghat_z, 0), with U = Vx/Vz and ghat from Thomsen's exact phase velocity (closed form);
* homogeneous isotropic: the wavefield equals the label-gradient one (the two routes coincide
  algebraically there) and (i/4) H0^(1)(kr) inside the cone;
* heterogeneous TTI: geometrical amplitudes of the point-source family against the Lagrangian ray
  shooter on both branches, and the downgoing wavefield against the label-gradient reading.
"""
import math

import numpy as np
import pytest

import synthmedia
from oracle import closed_forms as CF
from oracle import zmarch as ZM
from oracle import zmarch_drt as DR

THETA_MAX = math.radians(60.0)


def test_homogeneous_vti_perturbation_families():
    p = synthmedia.vti_homogeneous(n=48, n_theta=32, steps=1)
    m = p.meta
    U = lambda th: np.divide(*CF.vti_group_velocity(th, m['vp0'], m['vs0'], m['eps'], m['delta'])[1:])
    errs = []
    for nth in (32, 64):
        Z = ZM.ZSetup(p, nth, THETA_MAX, 1, 0.5)
        Q = DR.march_q(Z)
        e = 1e-6
        dU = (U(Z.theta + e) - U(Z.theta - e)) / (2 * e)
        zeta = (Z.rows * p.hz + p.origin[1] - p.xs[1])[None, :, None]
        ref = zeta * dU[:, None, None]
        rel = np.abs(Q['x2'] - ref) / np.max(np.abs(ref))
        inner = np.abs(Z.theta) < math.radians(45.0)
        errs.append(rel[inner].max())
        assert rel.max() < 2.5e-2
        assert np.abs(Q['t2'] - 1).max() < 1e-10 and np.abs(Q['t1']).max() < 1e-10
        v, Vx, Vz = CF.vti_group_velocity(Z.theta, m['vp0'], m['vs0'], m['eps'], m['delta'])
        gz = Vz / np.hypot(Vx, Vz)
        assert np.max(np.abs(Q['x1'] * gz[:, None, None] - 1)) < 1e-6
    # dU/dtheta of the tabulated U is a second-order difference: halving dtheta quarters the error
    assert errs[0] < 4e-3 and errs[0] / errs[1] > 3.0, errs


def test_homogeneous_isotropic_wavefield():
    p = synthmedia.isotropic_homogeneous(n=96, h=10.0, n_theta=64, freqs=[60.0])
    Z = ZM.ZSetup(p, 144, THETA_MAX, 1, 0.5)
    H = ZM.march(Z)
    Q = DR.march_q(Z)
    om = 2 * math.pi * 60.0
    ua = ZM.green_rows(Z, H, [om], 100.0)[0]
    ub = DR.green_rows_q(Z, H, Q, [om], 100.0)[0]
    assert np.linalg.norm(ua - ub) / np.linalg.norm(ua) < 1e-6
    x = Z.x - p.xs[0]
    z = Z.rows * p.hz - p.xs[1]
    Zg, Xg = np.meshgrid(z, x, indexing='ij')
    r = np.hypot(Xg, Zg)
    ang = np.degrees(np.arctan2(np.abs(Xg), np.abs(Zg)))
    k = om / p.meta['vp']
    ref = CF.hankel_green_2d(k, np.where(r > 0, r, 1.0))
    sel = (k * r >= 20) & (ang < 30)
    assert np.linalg.norm(ub[sel] - ref[sel]) / np.linalg.norm(ref[sel]) < 0.04


@pytest.fixture(scope='module')
def tti(tti64_shooter):
    p, fan, sc, first, arr = tti64_shooter
    return p, sc, arr, ZM.solve(p, 64, THETA_MAX, 0.5), DR.solve(p, 64, THETA_MAX, 0.5)


def _geometry(p):
    x = np.arange(p.nx) * p.hx - p.xs[0]
    z = np.arange(p.nz) * p.hz - p.xs[1]
    Zg, Xg = np.meshgrid(z, x, indexing='ij')
    return Zg, np.hypot(Xg, Zg), np.degrees(np.arctan2(np.abs(Xg), np.abs(Zg)))


def test_tti_amplitudes_of_the_point_source_family_match_the_shooter(tti):
    p, sc, arr, a, b = tti
    Zg, r, ang = _geometry(p)
    for side in (Zg > 0, Zg < 0):
        m = side & (b['count'] == 1) & (sc == 1) & (ang < 35) & (r > 160)
        As = np.array([arr[(i, j)][0][1] for i, j in zip(*np.nonzero(m))])
        rel = np.abs(b['A'][..., 0][m] - As) / As
        assert m.sum() > 500 and np.median(rel) < 5e-3 and np.quantile(rel, 0.95) < 2e-2


def test_tti_downgoing_wavefield_matches_the_label_gradient_reading(tti):
    p, sc, arr, a, b = tti
    Zg, r, ang = _geometry(p)
    m = (Zg > 0) & (ang < 30) & (r > 200)
    assert np.array_equal(a['count'], b['count'])
    assert np.linalg.norm(a['u'][0][m] - b['u'][0][m]) / np.linalg.norm(a['u'][0][m]) < 1e-2
