"""Continuous batching on the GPU: requests that arrive while others run are admitted into the
running batch (requests on the same medium share it), and every result equals the result of the
same request solved alone."""
import dataclasses

import numpy as np
import pytest

import synthmedia
from paper_2006_11945_gb300.serve import Request, Backend, serve

pytestmark = pytest.mark.gpu


_VTI = synthmedia.vti_homogeneous(n=48, n_theta=32, steps=60, freqs=(15.0, 25.0))


def _problem(i):
    if i % 2 == 0:
        # the even requests share one medium (and its characteristic velocities) in the backend
        return dataclasses.replace(_VTI, steps=60 + 7 * i, xs=(_VTI.xs[0] + 10.0 * (i % 3), _VTI.xs[1]))
    return synthmedia.tti_heterogeneous(n=64, n_theta=40, length=2560.0, steps=90 + 5 * i,
                                        freqs=(10.0,), seed=20 + i)


def test_results_alone_equal_results_in_the_mix():
    import paper_2006_11945_gb300 as egb
    reqs = [Request(i, 0.0 if i < 3 else 0.002 * i, _problem(i)) for i in range(6)]
    be = Backend(0)
    try:
        st = serve(reqs, be, chunk_steps=17)
    finally:
        be.close()
    assert len(st.completed) == 6 and st.max_active >= 2
    with egb.Context(0) as ctx:
        for r in st.completed:
            alone, _ = ctx.solve_problem(r.problem, kmax=r.kmax)
            assert np.array_equal(alone.u, r.result.u), r.rid
            assert np.array_equal(alone.count, r.result.count)
            assert np.array_equal(alone.T, r.result.T)
            assert np.array_equal(alone.A, r.result.A)
    s = st.summary(len(reqs))
    assert s['p99_latency_s'] >= s['p50_latency_s'] > 0
