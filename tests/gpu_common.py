"""Helpers shared by the GPU parity tests (CUDA path through the C ABI vs the FP64 oracle)."""
import math

import numpy as np

import synthmedia


def run_gpu(problem, steps=None, kmax=8, read_state=False):
    import paper_2006_11945_gb300 as egb
    with egb.Context(0) as ctx:
        m = ctx.medium_2d(problem)
        s = ctx.source_2d(m, problem)
        ctx.evolve(s, problem.steps if steps is None else steps, problem.cfl)
        res = ctx.superpose(s, len(problem.freqs), problem.nz, problem.nx, kmax)
        egb.egb_sync(ctx.h)
        state = ctx.read_state(s, problem.n_theta, problem.nz, problem.nx) if read_state else None
        vel = ctx.read_velocity(s, problem.n_theta, problem.nz, problem.nx) if read_state else None
        info = egb.egb_get_solve_info(ctx.h, s)
    return res, info, state, vel


def run_oracle(problem, steps=None, kmax=8):
    from oracle import liouville as OL
    from oracle import superpose as OS
    S, st, dt = OL.evolve(problem, steps=steps)
    lab = OL.interior_state(st, S)
    u = OS.green(S, lab, problem.omegas, problem.beam_width)
    cnt, T, A, over = OS.arrivals(S, lab, kmax)
    amb = OS.ambiguous_nodes(S, lab, 1e-4 * max(problem.hx, problem.hz))
    return dict(S=S, lab=lab, u=u, count=cnt, T=T, A=A, overflow=over, ambiguous=amb, dt=dt)


def wrap(d):
    return (d + np.pi) % (2 * np.pi) - np.pi


def compare_outputs(res, ref):
    """Error metrics of the GPU outputs against the oracle."""
    out = {}
    u, ur = res.u.astype(np.complex128), ref['u']
    out['u_rel_l2'] = float(np.linalg.norm(u - ur) / np.linalg.norm(ur))
    ok = ~ref['ambiguous']
    out['count_mismatch'] = int(np.sum((res.count != ref['count']) & ok))
    same = (res.count == ref['count']) & ok
    kk = np.arange(res.T.shape[-1])[None, None, :] < ref['count'][..., None]
    sel = same[..., None] & kk
    Tr, Ar = ref['T'][sel], ref['A'][sel]
    out['T_rel_max'] = float(np.max(np.abs(res.T[sel] - Tr) / Tr)) if sel.any() else 0.0
    out['A_rel_max'] = float(np.max(np.abs(res.A[sel] - Ar) / Ar)) if sel.any() else 0.0
    out['A_rel_p99'] = float(np.quantile(np.abs(res.A[sel] - Ar) / Ar, 0.99)) if sel.any() else 0.0
    out['arrivals'] = int(sel.sum())
    out['ambiguous_nodes'] = int(ref['ambiguous'].sum())
    return out
