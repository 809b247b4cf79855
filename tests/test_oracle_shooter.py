"""Brute-force pin of the Eulerian oracle in a heterogeneous TTI medium: the Lagrangian ray shooter
(RK4 on the same Hamiltonian, ray-tube rasterisation) gives the arrival count, the first-arrival
traveltime and the geometrical amplitude at every node; the level-set oracle must agree away from
the source (discretisation errors of a 40 m grid).  The beam-sum wavefield is pinned against the
geometrical field built from the shooter's traveltimes and amplitudes, which it approaches as the
frequency grows."""
import numpy as np
import pytest

import synthmedia
from oracle import liouville as L
from oracle import superpose as SP


@pytest.fixture(scope='module')
def both(tti64_shooter):
    p, fan, cnt, first, arr = tti64_shooter
    S, st, dt = L.evolve(p)
    lab = L.interior_state(st, S)
    ec, eT, eA, _ = SP.arrivals(S, lab, 8)
    x = np.arange(p.nx) * p.hx - p.xs[0]
    z = np.arange(p.nz) * p.hz - p.xs[1]
    Z, X = np.meshgrid(z, x, indexing='ij')
    far = np.hypot(X, Z) > 4 * S.r0
    return p, fan, cnt, first, arr, S, ec, eT, eA, far


def test_every_ray_leaves_the_domain_before_the_evolution_ends(both):
    p, fan, *_ , S, ec, eT, eA, far = both
    t_exit = np.nanmax(fan['exit_time'])
    assert np.isfinite(t_exit) and p.steps * S.dt(p.cfl) > t_exit


def test_arrival_counts_agree(both):
    p, fan, cnt, first, arr, S, ec, eT, eA, far = both
    assert np.mean(ec[far] == cnt[far]) > 0.99


def test_first_arrival_traveltimes_agree(both):
    p, fan, cnt, first, arr, S, ec, eT, eA, far = both
    m = far & (ec >= 1) & (cnt >= 1)
    rel = np.abs(eT[..., 0][m] - first[m]) / first[m]
    assert np.median(rel) < 5e-3 and np.quantile(rel, 0.95) < 3e-2


def test_single_arrival_amplitudes_agree(both):
    p, fan, cnt, first, arr, S, ec, eT, eA, far = both
    m = far & (ec == 1) & (cnt == 1)
    As = np.array([arr[(i, j)][0][1] for i, j in zip(*np.nonzero(m))])
    rel = np.abs(eA[..., 0][m] - As) / As
    assert np.median(rel) < 2e-2 and np.quantile(rel, 0.9) < 1.5e-1


@pytest.fixture(scope='module')
def field128(tti64_shooter):
    """The same medium evolved with 128 angles (the beam sum needs finer take-off sampling than the
    arrivals at the frequencies where it is asymptotic)."""
    import dataclasses
    p, fan, cnt, first, arr = tti64_shooter
    S, st, dt = L.evolve(dataclasses.replace(p, n_theta=128))
    lab = L.interior_state(st, S)
    ec, eT, eA, _ = SP.arrivals(S, lab, 8)
    x = np.arange(p.nx) * p.hx - p.xs[0]
    z = np.arange(p.nz) * p.hz - p.xs[1]
    Z, X = np.meshgrid(z, x, indexing='ij')
    iz, ix = np.indices(Z.shape)
    edge = np.minimum(np.minimum(iz, ix), np.minimum(p.nz - 1 - iz, p.nx - 1 - ix)) * p.hx
    m = (np.hypot(X, Z) > 4 * S.r0) & (ec == 1) & (cnt == 1) & (edge > 6 * p.hx)
    T = np.zeros(Z.shape)
    A = np.ones(Z.shape)
    for i, j in zip(*np.nonzero(m)):
        T[i, j], A[i, j] = arr[(i, j)][0][:2]
    return S, lab, m, Z, T, A


def test_no_tube_passes_a_caustic_in_the_tti_medium(tti64_shooter):
    """The medium has no caustic (one arrival at every node reached): the shooter's KMAH counter
    (sign changes of the signed tube spreading) stays 0 on every arrival."""
    p, fan, cnt, first, arr = tti64_shooter
    assert cnt.max() == 1
    assert all(a[3] == 0 for lst in arr.values() for a in lst)


@pytest.mark.slow
def test_heterogeneous_wavefield_tends_to_the_shooters_geometrical_field(field128):
    """Away from caustics the beam sum (Eq. 34) tends, as omega grows at fixed beam width, to the
    geometrical field A exp(i (omega T + pi/4)) / sqrt(omega) of a single ray (the far field of the
    2-D point-source Green's function), with T and A from the Lagrangian shooter.  Single-arrival
    nodes beyond 4 r0 and 6 cells inside the grid; w0 = 150 m (k w0 = 25 at 80 Hz near the source).
    The signed amplitude medians above and below the source pin the density factor sqrt(rho_s/rho)
    (it changes them by -2.3 % and +1.4 % here)."""
    import math
    S, lab, m, Z, T, A = field128
    err = {}
    for f in (20.0, 40.0, 80.0):
        om = 2 * math.pi * f
        u = SP.green(S, lab, [om], 150.0)[0][m]
        go = A[m] / math.sqrt(om) * np.exp(1j * (om * T[m] + math.pi / 4))
        ratio = np.abs(u) / np.abs(go)
        err[f] = np.median(np.abs(ratio - 1))
        if f == 80.0:
            # the phase error (omega times the 40 m grid's traveltime error) grows with omega, so the
            # complex error is bounded here rather than required to fall (0.072 and 0.204 measured:
            # the spatially varying epsilon and delta add to the traveltime error of the 40 m grid)
            e = np.abs(u - go) / np.abs(go)
            assert np.median(e) < 0.09 and np.quantile(e, 0.9) < 0.25, (np.median(e), np.quantile(e, 0.9))
            up, down = np.median(ratio[Z[m] < 0]), np.median(ratio[Z[m] > 0])
            assert _density_medians_ok(up, down), (up, down)
    assert err[20.0] > 2 * err[40.0] and err[40.0] > 1.3 * err[80.0] and err[80.0] < 0.04, err


def _density_medians_ok(up, down):
    return abs(up - 1) < 0.03 and abs(down - 1) < 0.03 and abs(up - down) < 0.025


@pytest.mark.slow
def test_wavefield_pin_detects_a_dropped_density_factor(field128):
    """Planted mistake in the oracle: with the receiver density replaced by the source's, the beam
    sum loses its sqrt(rho_s / rho) factor and the amplitude medians above and below the source
    leave the bounds the pin above holds them to."""
    import copy
    import math
    S, lab, m, Z, T, A = field128
    bad = copy.copy(S)
    bad.rho = np.full_like(S.rho, S.rho_s)
    om = 2 * math.pi * 80.0
    u = SP.green(bad, lab, [om], 150.0)[0][m]
    ratio = np.abs(u) * math.sqrt(om) / A[m]
    up, down = np.median(ratio[Z[m] < 0]), np.median(ratio[Z[m] > 0])
    assert not _density_medians_ok(up, down), (up, down)
