"""Failure paths on the GPU, all provoked from the host or by a bounded wait (nothing faults or hangs):

* the stencil's waits on its own TMA copies are bounded; with a bound of one poll they give up while
  the copies are still in flight, the kernel latches EGB_E_TIMEOUT after draining those copies, and
  egb_sync reports it with the CUDA context intact;
* a device allocation of a medium or a solve that fails (injected on the host with EGB_FAIL_ALLOC, at
  every allocation site in turn) returns EGB_E_NOMEM, leaks nothing, and the context goes on;
* a non-finite stiffness value is refused like a non-positive-definite one.
"""
import dataclasses

import numpy as np
import pytest

import synthmedia

pytestmark = pytest.mark.gpu


def _status(fn):
    import paper_2006_11945_gb300 as egb
    try:
        fn()
    except egb.EgbError as e:
        return e.status
    return egb.EGB_OK


def _solve(ctx, p, steps):
    m = ctx.medium_2d(p)
    s = ctx.source_2d(m, p)
    ctx.evolve(s, steps, p.cfl)
    return m, s, ctx.superpose(s, len(p.freqs), p.nz, p.nx, 8)


def test_stencil_wait_bound_latches_timeout_and_the_context_stays_usable():
    torch = pytest.importorskip('torch')
    import paper_2006_11945_gb300 as egb
    p = synthmedia.vti_homogeneous(n=48, n_theta=32, steps=12)
    with egb.Context(0) as ref_ctx:
        _, _, ref = _solve(ref_ctx, p, p.steps)
    with egb.Context(0, wait_polls=1) as ctx:
        m = ctx.medium_2d(p)
        s = ctx.source_2d(m, p)   # the stencil autotuner already runs stage launches here
        egb.egb_evolve(ctx.h, s, 6, p.cfl)
        assert _status(lambda: egb.egb_sync(ctx.h)) == egb.EGB_E_TIMEOUT
        torch.cuda.synchronize()                      # the CUDA context is intact
        assert _status(lambda: egb.egb_sync(ctx.h)) == egb.EGB_OK   # reported once, then cleared
        st = ctx.read_state(s, p.n_theta, p.nz, p.nx)   # the library still answers on this context
        assert st.shape == (4, p.n_theta, p.nz, p.nx)
        egb.egb_release(ctx.h, s)
        egb.egb_release(ctx.h, m)
    # a context with the default bound in the same process reproduces the reference solve
    with egb.Context(0) as ctx2:
        _, _, res = _solve(ctx2, p, p.steps)
    assert np.array_equal(res.count, ref.count)
    assert np.array_equal(res.u, ref.u)


def test_injected_allocation_failures_return_nomem_and_leak_nothing(monkeypatch):
    torch = pytest.importorskip('torch')
    import paper_2006_11945_gb300 as egb
    p = synthmedia.vti_homogeneous(n=40, n_theta=16, steps=6)
    with egb.Context(0) as ctx:
        _, _, ref = _solve(ctx, p, p.steps)
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    failed_at = []
    for n in range(16):
        monkeypatch.setenv('EGB_FAIL_ALLOC', str(n))
        with egb.Context(0) as ctx:
            holder = {}
            st_m = _status(lambda: holder.setdefault('m', ctx.medium_2d(p)))
            if st_m != egb.EGB_OK:
                assert st_m == egb.EGB_E_NOMEM
                failed_at.append(('medium', n))
                m = ctx.medium_2d(p)          # the one injected failure is spent: this succeeds
            else:
                m = holder['m']
            st_s = _status(lambda: holder.setdefault('s', ctx.source_2d(m, p)))
            if st_s != egb.EGB_OK:
                assert st_s == egb.EGB_E_NOMEM
                failed_at.append(('source', n))
                s = ctx.source_2d(m, p)
            else:
                s = holder['s']
            ctx.evolve(s, p.steps, p.cfl)
            res = ctx.superpose(s, len(p.freqs), p.nz, p.nx, 8)
            egb.egb_sync(ctx.h)
            assert np.array_equal(res.u, ref.u) and np.array_equal(res.count, ref.count), n
    monkeypatch.delenv('EGB_FAIL_ALLOC')
    torch.cuda.synchronize()
    leak = free0 - torch.cuda.mem_get_info()[0]
    kinds = {k for k, _ in failed_at}
    assert kinds == {'medium', 'source'}, failed_at
    assert len(failed_at) >= 12, failed_at          # every allocation site was hit once
    assert leak < (8 << 20), leak


def test_non_finite_stiffness_is_refused():
    import paper_2006_11945_gb300 as egb
    p = synthmedia.vti_homogeneous(n=16, n_theta=8, steps=1)
    for bad in (np.nan, np.inf):
        c21 = np.array(p.c21, copy=True)
        c21[77, 2] = bad
        q = dataclasses.replace(p, c21=c21)
        with egb.Context(0) as ctx:
            m = ctx.medium_2d(q)
            assert _status(lambda: ctx.source_2d(m, q)) == egb.EGB_E_NOT_PD
            # the context takes a valid medium afterwards
            _, _, res = _solve(ctx, p, 1)
            assert res.count.max() <= 1
