"""The amplitude's square root continued past two caustics and more (Eq. 26 with the phase of
Eq. 31), pinned against the Lagrangian ray shooter in a low-velocity channel.

In synthmedia.v_channel trapped rays oscillate about the channel axis and touch a caustic every half
period, so late in the channel a node sees arrivals that passed no, one and two caustics.  The
shooter counts the caustics of each arrival independently (sign changes of its ray-tube spreading).
The oracle follows the argument of the complex spreading J of the beam family through the
pseudo-time evolution (superpose.track_branch) and

* reads each arrival's KMAH index from it, floor(alpha / pi): it must equal the shooter's index for
  every arrival at the nodes where both see the same arrivals (index 2 included);
* sums the beams with the square root on the sheet alpha selects.  Against the stateless rule that
  holds only up to index 1 (sheet -1 wherever arg J < -1e-3), the sheet differs exactly for the
  beams of arrivals that passed two caustics, so the difference of the two beam sums is twice
  their contribution; at nodes with an index-2 arrival it must approach the matching difference
  of geometrical fields, 2 sum_{m_k = 2} A_k exp(i (omega T_k + pi/4 - pi)) / sqrt(omega) (the
  oracle's own T_k, A_k), and be far from its negative (what the stateless rule would need).
"""
import math

import numpy as np
import pytest

import synthmedia
from oracle import liouville as L
from oracle import shooter as SH
from oracle import superpose as SP


@pytest.fixture(scope='module')
def channel():
    from scipy import ndimage
    p = synthmedia.v_channel(n_theta=256)
    fan = SH.shoot(p, n_rays=2048, dt=1.0e-3)
    sc, first, arr = SH.arrivals(p, fan)
    S = L.Setup(p)
    steps = int(math.ceil(1.05 * np.nanmax(fan['exit_time']) / S.dt(p.cfl)))
    S, st, dt = L.evolve(p, steps=steps, S=S)
    lab = L.interior_state(st, S)
    cnt, T, A, _, M = SP.arrivals(S, lab, 8, kmah=True)
    calm = ndimage.maximum_filter(sc, 5) == ndimage.minimum_filter(sc, 5)
    X, Z = np.meshgrid(np.arange(p.nx) * p.hx - p.xs[0], np.arange(p.nz) * p.hz - p.xs[1])
    same = calm & (np.hypot(X, Z) > 100) & (cnt == sc) & (sc > 0)
    idx2 = np.zeros(sc.shape, bool)
    for key, lst in arr.items():
        idx2[key] = any(a[3] == 2 for a in lst)
    return p, S, lab, arr, T, A, M, same, idx2


@pytest.mark.slow
def test_arrival_kmah_indices_equal_the_shooters(channel):
    p, S, lab, arr, T, A, M, same, idx2 = channel
    total, equal, by_index = 0, 0, {}
    for key in zip(*np.nonzero(same)):
        for j, a in enumerate(arr[key]):
            total += 1
            equal += int(M[key][j] == a[3])
            by_index[a[3]] = by_index.get(a[3], 0) + 1
    print('arrivals compared', total, 'equal', equal, 'by shooter index', by_index)
    assert by_index.get(2, 0) >= 20 and by_index.get(1, 0) >= 100
    assert equal == total


@pytest.mark.slow
def test_beams_past_two_caustics_carry_their_kmah_phase(channel):
    p, S, lab, arr, T, A, M, same, idx2 = channel
    nodes = same & idx2
    assert nodes.sum() >= 20
    u = SP.green(S, lab, p.omegas, p.beam_width)
    a = SP.reference_arg(S, lab['b'], lab['Th'])
    stateless = dict(lab, alpha=np.where(a < -1e-3, a + 2 * np.pi, np.nan_to_num(a)))
    u0 = SP.green(S, stateless, p.omegas, p.beam_width)
    for w, om in enumerate(p.omegas):
        dgo = np.zeros(T.shape[:2], complex)
        for key in zip(*np.nonzero(nodes)):
            for j, x in enumerate(arr[key]):
                if x[3] == 2:
                    dgo[key] += 2 * A[key][j] / math.sqrt(om) * np.exp(1j * (om * T[key][j] + math.pi / 4 - math.pi))
        du = (u[w] - u0[w])[nodes]
        e = np.median(np.abs(du - dgo[nodes]) / np.abs(dgo[nodes]))
        e_neg = np.median(np.abs(du + dgo[nodes]) / np.abs(dgo[nodes]))
        print(f'{om / 2 / math.pi:.0f} Hz, {nodes.sum()} nodes: median {e:.3f}, against the negative {e_neg:.3f}')
        assert e < 0.6 and e_neg > 2.5 * e, (e, e_neg)
