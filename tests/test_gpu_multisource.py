"""Several sources on one medium share its characteristic velocities (they depend on the medium
and the phase angles only): every solve gives bit for bit what it gives on a medium of its own,
and the solves after the first hold 24 bytes per phase-space cell less device memory."""
import dataclasses

import numpy as np
import pytest

import synthmedia

pytestmark = pytest.mark.gpu


def _problems():
    p = synthmedia.tti_heterogeneous(n=64, n_theta=40, length=2560.0, steps=60, freqs=(10.0, 20.0))
    q = dataclasses.replace(p, xs=(20 * p.hx, 41 * p.hz))
    return p, q


def test_sources_sharing_a_medium_equal_separate_solves():
    import paper_2006_11945_gb300 as egb
    p, q = _problems()
    shared = []
    with egb.Context(0) as ctx:
        m = ctx.medium_2d(p)
        ids = [ctx.source_2d(m, x) for x in (p, q)]
        infos = [egb.egb_get_solve_info(ctx.h, s) for s in ids]
        for s, x in zip(ids, (p, q)):
            ctx.evolve(s, x.steps, x.cfl)
            shared.append((ctx.superpose(s, len(x.freqs), x.nz, x.nx, 8), ctx.read_state(s, x.n_theta, x.nz, x.nx)))
        egb.egb_sync(ctx.h)
    for x, (res, state), info in zip((p, q), shared, infos):
        with egb.Context(0) as ctx:
            m = ctx.medium_2d(x)
            s = ctx.source_2d(m, x)
            alone_info = egb.egb_get_solve_info(ctx.h, s)
            ctx.evolve(s, x.steps, x.cfl)
            alone = ctx.superpose(s, len(x.freqs), x.nz, x.nx, 8)
            alone_state = ctx.read_state(s, x.n_theta, x.nz, x.nx)
        assert np.array_equal(alone_state, state)
        for a, b in ((alone.u, res.u), (alone.count, res.count), (alone.T, res.T), (alone.A, res.A)):
            assert np.array_equal(a, b)
        assert info['dt'] == alone_info['dt']
    cells = infos[0]['cells']
    assert infos[0]['device_bytes'] - infos[1]['device_bytes'] == 24 * cells


def test_sources_sharing_a_medium_match_the_oracle():
    """Both solves on the shared medium (the second reusing the first's velocities) against the FP64
    oracle run for each source on its own, at the parity bar."""
    import paper_2006_11945_gb300 as egb
    from tests.gpu_common import compare_outputs, run_oracle
    p, q = _problems()
    with egb.Context(0) as ctx:
        m = ctx.medium_2d(p)
        ids = [ctx.source_2d(m, x) for x in (p, q)]
        res = []
        for s, x in zip(ids, (p, q)):
            ctx.evolve(s, x.steps, x.cfl)
            res.append(ctx.superpose(s, len(x.freqs), x.nz, x.nx, 8))
        egb.egb_sync(ctx.h)
    for x, r in zip((p, q), res):
        mt = compare_outputs(r, run_oracle(x))
        print(x.xs, mt)
        assert mt['u_rel_l2'] < 2e-3 and mt['count_mismatch'] == 0, mt
        assert mt['T_rel_max'] < 1e-5 and mt['A_rel_max'] < 1e-3, mt
