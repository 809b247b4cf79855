"""The amplitude's square root continued past two caustics and more (Eq. 26; the phase shift of
Eq. 31) on the CUDA path, in a low-velocity channel whose trapped rays touch a caustic every half
period (synthmedia.v_channel: arrivals with KMAH index 0, 1 and 2 at the same node).

* Parity with the FP64 oracle, which follows the continued argument of the complex spreading the
  same way (every BRANCH_SAMPLE steps, per phase cell): wavefield, counts, traveltimes, amplitudes.
* Against the Lagrangian ray shooter (independent of both): at nodes with an index-2 arrival, the
  CUDA beam sum tends to sum_k A_k exp(i (omega T_k + pi/4 - m_k pi/2)) / sqrt(omega) with the
  solve's own T_k, A_k and the shooter's m_k; flipping the sign of the index-2 terms (what a
  principal-branch rule valid up to index 1 does) is far off.
"""
import dataclasses
import math

import numpy as np
import pytest

import synthmedia
from oracle import shooter as SH
from tests.gpu_common import compare_outputs, run_gpu, run_oracle

pytestmark = pytest.mark.gpu


def _steps(p, fan):
    from oracle import liouville as OL
    return int(math.ceil(1.05 * np.nanmax(fan['exit_time']) / OL.Setup(p).dt(p.cfl)))


@pytest.fixture(scope='module')
def channel():
    from scipy import ndimage
    p = synthmedia.v_channel(n_theta=256)
    fan = SH.shoot(p, n_rays=2048, dt=1.0e-3)
    sc, first, arr = SH.arrivals(p, fan)
    p = dataclasses.replace(p, steps=_steps(p, fan))
    calm = ndimage.maximum_filter(sc, 5) == ndimage.minimum_filter(sc, 5)
    X, Z = np.meshgrid(np.arange(p.nx) * p.hx - p.xs[0], np.arange(p.nz) * p.hz - p.xs[1])
    idx2 = np.zeros(sc.shape, bool)
    for key, lst in arr.items():
        idx2[key] = any(a[3] == 2 for a in lst)
    res, info, _, _ = run_gpu(p)
    return p, fan, sc, arr, calm & (np.hypot(X, Z) > 100), idx2, res


def test_channel_parity_with_the_oracle(channel):
    """128 angles (the oracle's share of the test time); the beams past two caustics are there too."""
    p, fan, sc, arr, calm, idx2, _ = channel
    q = dataclasses.replace(p, n_theta=128)
    q = dataclasses.replace(q, steps=_steps(q, fan))
    res, info, _, _ = run_gpu(q)
    ref = run_oracle(q)
    m = compare_outputs(res, ref)
    print('channel parity', m)
    # Wavefield tolerance of this caustic-rich medium: a few beam centres near its caustics have a
    # level-set Jacobian D about 1/70 of its typical size, so their FP32 families carry about 70
    # times the usual relative rounding; one such beam along a row near x = 1200 m gives most of the
    # FP32-vs-FP64 difference at 200 Hz (4.4e-3; 1.5e-3 and 2.0e-3 at 50 and 100 Hz).
    assert m['u_rel_l2'] < 5e-3, m
    assert m['count_mismatch'] == 0, m
    assert m['T_rel_max'] < 1e-5 and m['A_rel_max'] < 1e-3, m


def test_beam_sum_carries_the_kmah_phase_past_two_caustics(channel):
    p, fan, sc, arr, calm, idx2, res = channel
    nodes = calm & idx2 & (res.count == sc)
    print('index-2 nodes', int((calm & idx2).sum()), 'with equal counts', int(nodes.sum()))
    assert nodes.sum() >= 20
    for w, om in enumerate(p.omegas):
        go = np.zeros(sc.shape, complex)
        flipped = np.zeros(sc.shape, complex)
        for key in zip(*np.nonzero(nodes)):
            for j, a in enumerate(arr[key]):
                g = res.A[key][j] / math.sqrt(om) * np.exp(1j * (om * res.T[key][j] + math.pi / 4)) * (-1j) ** a[3]
                go[key] += g
                flipped[key] += -g if a[3] == 2 else g
        u = res.u[w].astype(np.complex128)
        e = np.abs(u[nodes] - go[nodes]) / np.abs(go[nodes])
        ef = np.abs(u[nodes] - flipped[nodes]) / np.abs(flipped[nodes])
        print(f'{om / 2 / math.pi:.0f} Hz: median {np.median(e):.3f} q90 {np.quantile(e, 0.9):.3f}; '
              f'index-2 terms flipped: median {np.median(ef):.3f}')
        # the beam sum's own error in this channel is large (beams wider than the channel's
        # structure); the pin is that the tracked sheet is far closer than the flipped one
        assert np.median(e) < 0.8 and np.median(ef) > 2 * np.median(e), (np.median(e), np.median(ef))
