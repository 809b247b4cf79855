"""The allocation-free superposition entry point against the ordinary one, on the GPU.

egb_superpose_noalloc exists for callers that cannot allocate device memory at the moment they
superpose (a serving loop whose memory belongs to a pool or caching allocator, or a latency-critical
loop that must avoid cudaMalloc/cudaFree and their device-wide synchronisation).  It must give the
same outputs as egb_superpose, call after call, while its work buffers live in one fixed array
shared by all calls.  This file is collected last on purpose.
"""
import numpy as np
import pytest

import synthmedia

pytestmark = pytest.mark.gpu


def _outputs(torch, p, kmax):
    dev = 'cuda'
    return (torch.zeros((len(p.freqs), p.nz, p.nx, 2), dtype=torch.float32, device=dev),
            torch.zeros((p.nz, p.nx), dtype=torch.uint8, device=dev),
            torch.zeros((p.nz, p.nx, kmax), dtype=torch.float64, device=dev),
            torch.zeros((p.nz, p.nx, kmax), dtype=torch.float32, device=dev))


@pytest.mark.parametrize('precision', ['fp32_phase64', 'fp64'])
def test_noalloc_matches_superpose_on_two_calls(precision):
    """Two calls in a row, the solve evolved further before the second: a call that superposed a
    stale state (the initial labels, or the previous call's) would differ from egb_superpose."""
    torch = pytest.importorskip('torch')
    import paper_2006_11945_gb300 as egb
    kmax = 8
    prec = egb.EGB_FP64 if precision == 'fp64' else egb.EGB_FP32_PHASE64
    p = synthmedia.tti_heterogeneous(n=64, n_theta=48, length=2560.0, steps=120, freqs=(10.0, 20.0))
    with egb.Context(0, precision=prec) as ctx:
        m = ctx.medium_2d(p)
        s = ctx.source_2d(m, p)
        prev = None
        for call, steps in enumerate((60, 60)):
            ctx.evolve(s, steps, p.cfl)
            ref = _outputs(torch, p, kmax)
            egb.egb_superpose(ctx.h, s, *ref, kmax=kmax)
            egb.egb_sync(ctx.h)
            out = _outputs(torch, p, kmax)
            egb.egb_superpose_noalloc(ctx.h, s, *out, kmax=kmax)
            egb.egb_sync(ctx.h)
            u_ref = ref[0].cpu().numpy().view(np.complex64)[..., 0]
            u = out[0].cpu().numpy().view(np.complex64)[..., 0]
            rel = np.linalg.norm(u - u_ref) / np.linalg.norm(u_ref)
            assert rel < 2e-3, (call, rel)
            if prev is not None:
                # the evolution moved the wavefield, so matching above is not matching a stale copy
                assert np.linalg.norm(u - prev) / np.linalg.norm(u) > 1e-3, call
            prev = u
            cnt_ref, cnt = ref[1].cpu().numpy(), out[1].cpu().numpy()
            assert np.array_equal(cnt, cnt_ref), call
            sel = np.arange(kmax)[None, None, :] < cnt_ref[..., None]
            T_ref, T = ref[2].cpu().numpy()[sel], out[2].cpu().numpy()[sel]
            A_ref, A = ref[3].cpu().numpy()[sel], out[3].cpu().numpy()[sel]
            assert np.max(np.abs(T - T_ref) / T_ref) < 1e-5, call
            assert np.max(np.abs(A - A_ref) / A_ref) < 1e-3, call


def test_noalloc_refuses_oversized_solves_3d_ids_and_host_buffers():
    torch = pytest.importorskip('torch')
    import paper_2006_11945_gb300 as egb
    big = synthmedia.vti_homogeneous(n=256, n_theta=128, steps=1)
    small = synthmedia.vti_homogeneous(n=32, n_theta=32, steps=1)
    with egb.Context(0) as ctx:
        m = ctx.medium_2d(big)
        s = ctx.source_2d(m, big)
        out = _outputs(torch, big, 8)
        with pytest.raises(egb.EgbError) as e:
            egb.egb_superpose_noalloc(ctx.h, s, *out, kmax=8)
        assert e.value.status == egb.EGB_E_INVALID and 'scratch' in str(e.value)
        m2 = ctx.medium_2d(small)
        s2 = ctx.source_2d(m2, small)
        host_u = np.zeros((1, small.nz, small.nx), np.complex64)
        with pytest.raises(egb.EgbError) as e:
            egb.egb_superpose_noalloc(ctx.h, s2, host_u)
        assert e.value.status == egb.EGB_E_INVALID
        q = synthmedia.vti_homogeneous_3d(n=8, n_theta=4, n_phi=8, steps=1)
        m3 = ctx.medium_3d(q)
        s3 = ctx.source_3d(m3, q)
        u3 = torch.zeros((1, q.nz, q.ny, q.nx, 2), dtype=torch.float32, device='cuda')
        with pytest.raises(egb.EgbError) as e:
            egb.egb_superpose_noalloc(ctx.h, s3, u3)
        assert e.value.status == egb.EGB_E_INVALID and '3-D' in str(e.value)
