"""Brute-force pin of the Eulerian oracle in a heterogeneous TTI medium: the Lagrangian ray shooter
(RK4 on the same Hamiltonian, ray-tube rasterisation) gives the arrival count, the first-arrival
traveltime and the geometrical amplitude at every node; the level-set oracle must agree away from
the source (discretisation errors of a 40 m grid)."""
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
