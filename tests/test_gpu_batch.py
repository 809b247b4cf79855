"""Batched evolution (one persistent launch per stage over several solves, CUDA-graph replay):
every solve's level sets are bit-identical to advancing it alone, and steps compose."""
import numpy as np
import pytest

import synthmedia

pytestmark = pytest.mark.gpu


def _problems():
    return [synthmedia.tti_heterogeneous(n=72, n_theta=40, length=2560.0, steps=11, seed=5),
            synthmedia.tti_heterogeneous(n=100, n_theta=64, length=2000.0, steps=7, seed=6),
            synthmedia.vti_homogeneous(n=45, n_theta=24, steps=16)]


def _state(ctx, s, p):
    return ctx.read_state(s, p.n_theta, p.nz, p.nx)


def test_batch_equals_individual():
    import paper_2006_11945_gb300 as egb
    ps = _problems()
    alone = []
    with egb.Context(0) as ctx:
        for p in ps:
            m = ctx.medium_2d(p)
            s = ctx.source_2d(m, p)
            ctx.evolve(s, p.steps, p.cfl)
            alone.append(_state(ctx, s, p))
    with egb.Context(0) as ctx:
        ids = []
        for p in ps:
            m = ctx.medium_2d(p)
            ids.append(ctx.source_2d(m, p))
        egb.egb_evolve_batch(ctx.h, ids, [p.steps for p in ps], ps[0].cfl)
        egb.egb_sync(ctx.h)
        for p, s, a in zip(ps, ids, alone):
            b = _state(ctx, s, p)
            assert np.array_equal(a, b), p.name
            info = egb.egb_get_solve_info(ctx.h, s)
            assert info['steps_done'] == p.steps and info['tile_chunk'] in (8, 16, 32, 64)


def test_steps_compose():
    import paper_2006_11945_gb300 as egb
    p = synthmedia.tti_heterogeneous(n=64, n_theta=32, length=2560.0, steps=10, seed=7)
    with egb.Context(0) as ctx:
        m = ctx.medium_2d(p)
        s1 = ctx.source_2d(m, p)
        s2 = ctx.source_2d(m, p)
        ctx.evolve(s1, 10, p.cfl)
        for k in (4, 1, 5):
            ctx.evolve(s2, k, p.cfl)
        assert np.array_equal(_state(ctx, s1, p), _state(ctx, s2, p))


def test_batch_of_twenty_samples_the_spreading_argument_like_solves_alone():
    """Twenty small uneven solves with different step counts: the branch tracking of the due solves
    runs in launches of up to 16 of them, and every solve's state and superposition (whose square
    root sheet comes from the tracked argument) equal the same solve advanced alone, bit for bit."""
    import paper_2006_11945_gb300 as egb
    ps = [synthmedia.tti_heterogeneous(n=24 + 4 * (i % 5), n_theta=16 + 8 * (i % 3), length=1600.0,
                                       steps=9 + 3 * i, freqs=(15.0, 30.0), seed=20 + i)
          for i in range(20)]
    alone = []
    with egb.Context(0) as ctx:
        for p in ps:
            m = ctx.medium_2d(p)
            s = ctx.source_2d(m, p)
            ctx.evolve(s, p.steps, p.cfl)
            r = ctx.superpose(s, len(p.freqs), p.nz, p.nx)
            alone.append((_state(ctx, s, p), r))
    with egb.Context(0) as ctx:
        ids = [ctx.source_2d(ctx.medium_2d(p), p) for p in ps]
        egb.egb_evolve_batch(ctx.h, ids, [p.steps for p in ps], ps[0].cfl)
        egb.egb_sync(ctx.h)
        for p, s, (st, r) in zip(ps, ids, alone):
            assert np.array_equal(_state(ctx, s, p), st), p.name
            b = ctx.superpose(s, len(p.freqs), p.nz, p.nx)
            assert np.array_equal(b.u, r.u) and np.array_equal(b.count, r.count)
            assert np.array_equal(b.T, r.T) and np.array_equal(b.A, r.A)
