"""The receiver-side (reciprocal) reduction of a solve's labels (egb_superpose_receiver, Eq. 34 read
through reciprocity) on the GPU, through the C ABI:

* parity with the FP64 oracle's green_receiver on the same problem (homogeneous VTI; heterogeneous
  TTI with a 900 m source-ray tube) at the wavefield bar;
* against the source-side sum of the same state at a finer grid: receivers well inside the tube
  agree as the frequency grows (the receiver-side beams reach x_s up to about 2 w(r) off their
  rays, and the frozen disc's straight-ray data hold only where the medium varies little across it);
* argument errors.
"""
import dataclasses

import numpy as np
import pytest

import synthmedia

pytestmark = pytest.mark.gpu


def _gpu(p):
    import paper_2006_11945_gb300 as egb
    with egb.Context(0) as ctx:
        m = ctx.medium_2d(p)
        s = ctx.source_2d(m, p)
        ctx.evolve(s, p.steps, p.cfl)
        ur = ctx.superpose_receiver(s, len(p.freqs), p.nz, p.nx)
        us = ctx.superpose(s, len(p.freqs), p.nz, p.nx, 8).u
        egb.egb_sync(ctx.h)
    return ur.astype(np.complex128), us.astype(np.complex128)


def _oracle(p):
    from oracle import liouville as OL
    from oracle import superpose as OS
    S, st, dt = OL.evolve(p)
    lab = OL.interior_state(st, S)
    return OS.green_receiver(S, lab, p.omegas, p.beam_width)


@pytest.mark.parametrize('case', ['vti', 'vti_ragged', 'vti_10_freqs', 'tti'])
def test_receiver_side_matches_the_oracle(case):
    if case == 'vti':
        p = dataclasses.replace(synthmedia.vti_homogeneous(n=64, n_theta=64, steps=150, freqs=(30.0, 60.0)),
                                R_sigma=200.0)
    elif case == 'vti_10_freqs':
        # more frequencies than one pass of the kernel accumulates (8)
        p = dataclasses.replace(synthmedia.vti_homogeneous(n=40, n_theta=32, steps=80,
                                                           freqs=tuple(10.0 + 5.0 * i for i in range(10))),
                                R_sigma=150.0)
    elif case == 'vti_ragged':
        # rows of 45 receivers (a block serves 32) and 44 angles (8 warps take 6 or 5 of them)
        p = dataclasses.replace(synthmedia.vti_homogeneous(n=45, n_theta=44, steps=100, freqs=(30.0,)),
                                R_sigma=150.0)
    else:
        p = synthmedia.tti_heterogeneous(n=64, n_theta=96, length=2560.0, steps=400, freqs=(20.0, 40.0, 80.0),
                                         beam_width=150.0)
        p = dataclasses.replace(p, R_sigma=900.0)
    ur, _ = _gpu(p)
    ref = _oracle(p)
    rel = np.linalg.norm(ur - ref) / np.linalg.norm(ref)
    print(case, 'receiver-side parity', rel)
    assert np.all(np.isfinite(ur)) and rel < 2e-3


def test_receiver_side_agrees_with_source_side_on_a_finer_grid():
    p = synthmedia.tti_heterogeneous(n=256, n_theta=256, length=2560.0, steps=1400, freqs=(20.0, 40.0, 80.0),
                                     beam_width=150.0)
    p = dataclasses.replace(p, R_sigma=900.0)
    ur, us = _gpu(p)
    x = np.arange(p.nx) * p.hx - p.xs[0]
    z = np.arange(p.nz) * p.hz - p.xs[1]
    Z, X = np.meshgrid(z, x, indexing='ij')
    r = np.hypot(X, Z)
    m = (r >= 200) & (r < 600)
    e = [np.linalg.norm(ur[w][m] - us[w][m]) / np.linalg.norm(us[w][m]) for w in range(3)]
    med = [np.median(np.abs(ur[w][m] / us[w][m] - 1)) for w in range(3)]
    print('receiver vs source side (256^2, 10 m): L2', e, 'median', med)
    assert e[2] < 0.1 and med[2] < 0.05 and med[2] < med[0]


def test_receiver_side_argument_errors():
    import paper_2006_11945_gb300 as egb
    p = synthmedia.vti_homogeneous(n=16, n_theta=16, steps=1)
    q = synthmedia.vti_homogeneous_3d(n=8, n_theta=4, n_phi=8, steps=1)
    with egb.Context(0) as ctx:
        m = ctx.medium_2d(p)
        s = ctx.source_2d(m, p)
        with pytest.raises(egb.EgbError) as e:
            egb.egb_superpose_receiver(ctx.h, s, None)
        assert e.value.status == egb.EGB_E_INVALID
        m3 = ctx.medium_3d(q)
        s3 = ctx.source_3d(m3, q)
        u3 = np.zeros((1, q.nz, q.ny, q.nx), np.complex64)
        with pytest.raises(egb.EgbError) as e:
            egb.egb_superpose_receiver(ctx.h, s3, u3)
        assert e.value.status == egb.EGB_E_INVALID
        with pytest.raises(egb.EgbError) as e:
            egb.egb_source(ctx.h, m, (p.xs[0], 0.0, p.xs[1]), p.omegas, 50.0, 16, r0=40.0, R_sigma=20.0)
        assert e.value.status == egb.EGB_E_INVALID


def test_receiver_side_of_an_fp64_solve_matches_the_oracle():
    """A solve of the plain FP64 form: egb_superpose_receiver converts its state before summing."""
    import paper_2006_11945_gb300 as egb
    p = dataclasses.replace(synthmedia.vti_homogeneous(n=48, n_theta=48, steps=100, freqs=(30.0, 45.0)),
                            R_sigma=150.0)
    with egb.Context(0, precision=egb.EGB_FP64) as ctx:
        m = ctx.medium_2d(p)
        s = ctx.source_2d(m, p)
        ctx.evolve(s, p.steps, p.cfl)
        ur = ctx.superpose_receiver(s, len(p.freqs), p.nz, p.nx).astype(np.complex128)
        egb.egb_sync(ctx.h)
    ref = _oracle(p)
    rel = np.linalg.norm(ur - ref) / np.linalg.norm(ref)
    print('FP64-form receiver-side parity', rel)
    assert np.all(np.isfinite(ur)) and rel < 2e-3
