"""Benchmark: phase-space cell-updates/s of the anisotropic Eulerian Gaussian beam solver on GB300.

One step = one whole solve of the workload through the C ABI: medium upload and validation,
characteristic velocities and initial level sets (egb_medium, egb_source), the pseudo-time evolution
(egb_evolve: HJ-WENO3 / TVD-RK3 on every phase-space cell for the workload's step count) and the
Gaussian-beam superposition with arrival extraction at every frequency (egb_superpose).

Default workload: the heterogeneous 2-D TTI medium on a 512 x 512 grid at 5 m with 256 phase
angles, frequencies 10, 20 and 40 Hz, single source at the centre.  `value` is cell-updates per
second with the medium already resident in HBM; `e2e` is the same metric through the C ABI with
host buffers (medium uploaded from pinned host memory, every output copied back, inside the timed
region).  The state (1.3 GB per copy) is far larger than L2, so no flush is needed between steps.

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl egb|reference]
Under torchrun every rank runs its own replica (independent solves, no collective): weak scaling.
Other workloads (--workload): tti256 / tti128 / vti64 (smaller 2-D cases), tri96 / tri48 (3-D),
batch (uneven batched solves), serve (continuous batching on a Poisson request stream) and zmarch
(the paper's paraxial depth march, --zm-drt 1 for the dynamic ray tracing advected as Eq. 21).
"""
from __future__ import annotations

import argparse
import json
import math
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import synthmedia  # noqa: E402

HBM_FALLBACK_GBS = 6800.0
# Algorithmic bytes of the stencil per cell-update: the 2-D state (3 FP32 labels + 8-byte tau) read
# and written once per TVD-RK3 step (40 B) plus the stored characteristic velocities read once
# (Vx, Vz, dtheta/dt: 12 B).
ALGO_BYTES_PER_CELL_UPDATE = 52.0
# DRAM traffic of k_rk3_tma measured by ncu (dram__bytes_read.sum + dram__bytes_write.sum) on the
# 256 x 256 x 256 TTI case, per cell and launch, averaged over the three stage launches
# (stage 1: 917 MB, stages 2 and 3: 1285 and 1284 MB per 16.8 M cells), with the SHA-256 of the
# kernel's device source it was taken on; traffic grows with the cells a launch processes, so the
# figure is scaled to the timed workload.  Reported as null once the device source differs.
STENCIL_TRAFFIC = {'bytes_per_cell_launch': (55.04 + 77.42 + 77.34) / 3.0,
                   'device_source_sha256': '327db6ccac3f8c6d4fba2645ac44b331cd09c4c937f6076f8595bc09c97e0faa'}


def stencil_traffic_per_launch(cells):
    import hashlib
    src = open(os.path.join(ROOT, 'paper_2006_11945_gb300', 'csrc', 'liouville_tma.cu')).read()
    a, b = src.index('// ---- packed two-cell arithmetic'), src.index('// ---- host side')
    if hashlib.sha256(src[a:b].encode()).hexdigest() != STENCIL_TRAFFIC['device_source_sha256']:
        return None
    return STENCIL_TRAFFIC['bytes_per_cell_launch'] * cells


# Instruction issue of k_rk3_tma per cell and stage launch (ncu, thread-level instructions of the
# stage-2 launch on the 256^2 x 256 TTI case: 317.3, of which FP32 182.1 and integer 60.4), and
# GB300's issue ceiling: 4 schedulers per SM issue one warp instruction (32 thread instructions)
# per cycle.
STENCIL_THREAD_INST_PER_CELL_STAGE = 317.3


def issue_ceiling_thread_inst_per_s(sm_mhz):
    return 152 * 4 * 32 * sm_mhz * 1e6


# 3-D: the state (six FP32 labels b, n0, the indicator q and the double-float tau: 36 B) read and
# written once per step, plus the five stored characteristic velocities (20 B) read once.
ALGO_BYTES_PER_CELL_UPDATE_3D = 92.0


def workload(name):
    if name in ('tti512', 'zmarch'):
        return synthmedia.tti_heterogeneous(n=512, h=5.0, n_theta=256, freqs=(10.0, 20.0, 40.0))
    if name == 'vti64':
        return synthmedia.vti_homogeneous()
    if name == 'tti256':
        return synthmedia.tti_heterogeneous(n=256, n_theta=256, length=2560.0, steps=1400,
                                            freqs=(10.0, 20.0, 40.0))
    if name == 'tri96':
        return synthmedia.triclinic_3d(n=96, h=10.0, n_theta=24, n_phi=48, freqs=(15.0,))
    if name == 'tri48':
        return synthmedia.triclinic_3d(n=48, n_theta=12, n_phi=24, length=960.0, freqs=(15.0,))
    if name == 'tti128':
        return synthmedia.tti_heterogeneous(n=128, n_theta=128, length=2560.0, steps=400,
                                            freqs=(10.0, 20.0, 40.0))
    raise ValueError(name)


def measured_peaks():
    p = os.path.join(ROOT, 'MEASURED_PEAKS.json')
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return float(d['hbm_gbs']), 'measured'
    return HBM_FALLBACK_GBS, 'fallback'


class ClockSampler:
    """nvidia-smi clock / throttle sampling while the timed region runs."""

    def __init__(self, index):
        self.index = index
        self.samples = []
        self.proc = None

    def __enter__(self):
        q = ('clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,'
             'clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,'
             'clocks_event_reasons.sw_power_cap')
        try:
            self.proc = subprocess.Popen(
                ['nvidia-smi', '-i', str(self.index), f'--query-gpu={q}', '--format=csv,noheader,nounits',
                 '-lms', '200'], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except OSError:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            parts = [x.strip() for x in line.split(',')]
            if len(parts) >= 7:
                self.samples.append(parts)

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        if not self.samples:
            return {'sm_mhz': None, 'sm_max_mhz': None, 'reasons': ['no samples']}
        sm = [float(s[0]) for s in self.samples if s[0].replace('.', '', 1).isdigit()]
        mx = [float(s[1]) for s in self.samples if s[1].replace('.', '', 1).isdigit()]
        names = ['hw_slowdown', 'hw_thermal_slowdown', 'sw_thermal_slowdown', 'sw_power_cap']
        reasons = sorted({names[i] for s in self.samples for i in range(4) if s[3 + i] == 'Active'})
        return {'sm_mhz': float(np.median(sm)) if sm else None,
                'sm_max_mhz': max(mx) if mx else None, 'reasons': reasons, 'samples': len(self.samples)}


def dist_env():
    ws = int(os.environ.get('WORLD_SIZE', '1'))
    rank = int(os.environ.get('RANK', '0'))
    local = int(os.environ.get('LOCAL_RANK', '0'))
    return ws, rank, local


def max_over_ranks(ms, dist, device):
    """The largest per-rank time of a timed region (every rank receives it); ms on one rank."""
    if dist is None:
        return ms
    import torch
    t = torch.tensor([ms], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_rate(units_per_rank, ranks, ms):
    """Whole-job throughput: the units all ranks processed over the slowest rank's time (weak
    scaling: every rank runs its own replica of the workload)."""
    return ranks * units_per_rank / (ms / 1e3)


def run_egb(args):
    import torch
    import paper_2006_11945_gb300 as egb

    ws, rank, local = dist_env()
    torch.cuda.set_device(local)
    dist = None
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group('nccl', device_id=torch.device('cuda', local))
    p = workload(args.workload)
    steps_evolve = p.steps if args.evolve_steps is None else args.evolve_steps
    stream = torch.cuda.Stream()
    ctx = egb.Context(local, stream.cuda_stream)
    nodes = p.nx * p.nz
    c21_d = torch.from_numpy(np.ascontiguousarray(p.c21)).cuda()
    rho_d = torch.from_numpy(np.ascontiguousarray(p.rho)).cuda()
    c21_h = torch.from_numpy(np.ascontiguousarray(p.c21)).pin_memory()
    rho_h = torch.from_numpy(np.ascontiguousarray(p.rho)).pin_memory()
    no, kmax = len(p.freqs), 8
    u_d = torch.empty((no, p.nz, p.nx, 2), dtype=torch.float32, device='cuda')
    cnt_d = torch.empty((p.nz, p.nx), dtype=torch.uint8, device='cuda')
    T_d = torch.empty((p.nz, p.nx, kmax), dtype=torch.float64, device='cuda')
    A_d = torch.empty((p.nz, p.nx, kmax), dtype=torch.float32, device='cuda')
    u_h = torch.empty((no, p.nz, p.nx, 2), dtype=torch.float32).pin_memory()
    cnt_h = torch.empty((p.nz, p.nx), dtype=torch.uint8).pin_memory()
    T_h = torch.empty((p.nz, p.nx, kmax), dtype=torch.float64).pin_memory()
    A_h = torch.empty((p.nz, p.nx, kmax), dtype=torch.float32).pin_memory()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    evolve_ms = []

    def solve(host):
        n = (p.nx, 1, p.nz)
        hs = (p.hx, 1.0, p.hz)
        org = (p.origin[0], 0.0, p.origin[1])
        c21, rho = (c21_h, rho_h) if host else (c21_d, rho_d)
        m = egb.egb_medium(ctx.h, n, hs, org, c21, rho)
        s = egb.egb_source(ctx.h, m, (p.xs[0], 0.0, p.xs[1]), p.omegas, p.beam_width, p.n_theta, 0.0)
        with torch.cuda.stream(stream):
            ev0.record(stream)
        egb.egb_evolve(ctx.h, s, steps_evolve, p.cfl)
        with torch.cuda.stream(stream):
            ev1.record(stream)
        if host:
            egb.egb_superpose(ctx.h, s, u_h, cnt_h, T_h, A_h, kmax)
        else:
            egb.egb_superpose(ctx.h, s, u_d, cnt_d, T_d, A_d, kmax)
        egb.egb_sync(ctx.h)
        evolve_ms.append(ev0.elapsed_time(ev1))
        info = egb.egb_get_solve_info(ctx.h, s)
        egb.egb_release(ctx.h, s)
        egb.egb_release(ctx.h, m)
        return info

    def timed(host, K, W):
        for _ in range(W):
            solve(host)
        evolve_ms.clear()
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()
        t0 = torch.cuda.Event(enable_timing=True)
        t1 = torch.cuda.Event(enable_timing=True)
        with torch.cuda.stream(stream):
            t0.record(stream)
        for _ in range(K):
            info = solve(host)
        with torch.cuda.stream(stream):
            t1.record(stream)
        torch.cuda.synchronize()
        ms = max_over_ranks(t0.elapsed_time(t1), dist, 'cuda')
        return ms, info

    with ClockSampler(local) as clk:
        ms, info = timed(False, args.steps, args.warmup)
    evolve_avg_ms = float(np.mean(evolve_ms))
    k_e2e = max(1, min(3, args.steps))
    e2e_ms, _ = timed(True, k_e2e, 1)
    cells = info['cells']
    cu_per_solve = cells * steps_evolve
    per_step_ms = ms / args.steps
    value = job_rate(cu_per_solve * args.steps, ws, ms)
    e2e_value = job_rate(cu_per_solve * k_e2e, ws, e2e_ms)
    peak, peak_kind = measured_peaks()
    launch_ms = evolve_avg_ms / (3 * steps_evolve)
    achieved = ALGO_BYTES_PER_CELL_UPDATE * cells / 3.0 / (launch_ms / 1e3) / 1e9
    # per timed solve: k_medium_a, k_medium_grad; k_source, k_velocity, k_frozen, k_init,
    # k_zero_frozen, the first k_track_branch; 3 stage launches per step and a k_track_branch every
    # 9 steps; k_beam_fields, 2 x k_centres, k_sum, k_arrivals (the theta-chunk autotuner ran in
    # the warm-up solve and is cached per grid shape)
    launches = 2 + 6 + 3 * steps_evolve + steps_evolve // 9 + 5
    h2d = p.c21.nbytes + p.rho.nbytes
    d2h = u_h.numel() * 4 + cnt_h.numel() + T_h.numel() * 8 + A_h.numel() * 4
    line = {
        'metric': 'phase-space cell-updates/s',
        'value': value,
        'unit': 'cell-updates/s',
        'n_gpus': ws,
        'steps': args.steps,
        'warmup': args.warmup,
        'ms_per_step': per_step_ms,
        'higher_is_better': True,
        'scaling': 'weak',
        'vs_baseline': None,
        'dtype': 'f32 (double-float tau and phase)',
        'data': 'synthetic (seeded TTI medium)',
        'config': {'workload': f'{p.name} {p.nx}x{p.nz} at {p.hx:g} m x {p.n_theta} angles, '
                               f'{steps_evolve} TVD-RK3 steps, {len(p.freqs)} frequencies',
                   'cells': cells, 'evolve_steps': steps_evolve, 'freqs_hz': p.freqs,
                   'tile_chunk': info.get('tile_chunk'),
                   'parallelism': f'replicas x{ws}', 'l2': 'state (1.3 GB) larger than L2, no flush'},
        'solves_per_s': ws * args.steps / (ms / 1e3),
        'beam_point_sums_per_s': ws * args.steps * p.nx * p.nz * p.n_theta * len(p.freqs) / (ms / 1e3),
        'e2e': {'value': e2e_value, 'unit': 'cell-updates/s', 'h2d_bytes_per_step': int(h2d),
                'd2h_bytes_per_step': int(d2h), 'timed_steps': k_e2e},
        'roofline': {'bound': 'hbm', 'kernel': 'k_rk3_tma', 'achieved': achieved, 'peak': peak,
                     'unit': 'GB/s', 'frac': achieved / peak, 'traffic': stencil_traffic_per_launch(cells),
                     'peak_kind': peak_kind, 'launch_ms': launch_ms},
        'gpu_launches': launches * args.steps,
        'clocks': clk.summary(),
    }
    # the stencil against its instruction-issue ceiling (at the median SM clock of the timed region)
    mhz = line['clocks'].get('sm_mhz') or 2070.0
    inst_rate = STENCIL_THREAD_INST_PER_CELL_STAGE * cells / (launch_ms / 1e3)
    line['issue_ceiling'] = {'kernel': 'k_rk3_tma', 'thread_inst_per_cell_stage': STENCIL_THREAD_INST_PER_CELL_STAGE,
                             'achieved': inst_rate, 'peak': issue_ceiling_thread_inst_per_s(mhz),
                             'unit': 'thread instructions/s', 'frac': inst_rate / issue_ceiling_thread_inst_per_s(mhz),
                             'hbm_frac_at_ceiling': ALGO_BYTES_PER_CELL_UPDATE * issue_ceiling_thread_inst_per_s(mhz)
                             / (3 * STENCIL_THREAD_INST_PER_CELL_STAGE) / (peak * 1e9)}
    if not args.no_fp64_form:
        line['fp64_form'] = fp64_form(p, args.fp64_steps, local)
        line['fp64_form']['speedup'] = line['value'] / ws / line['fp64_form']['value']
    if rank == 0 and not args.no_cpu_baseline and ws == 1:
        line['cpu_baseline'] = cpu_baseline(p, budget_s=args.cpu_seconds)
    ctx.close()
    if ws == 1 and args.workload == 'tti512' and not args.no_sub:
        # the other configurations of the metric, each measured on its own with its own clocks
        p3 = workload('tri96')
        line['sub'] = {
            'tri96': measure_3d(p3, p3.steps, 1, 1, warmup_steps=3),
            'batch': measure_batch_waves(synthmedia.batched_instances(count=args.batch_count),
                                         args.evolve_steps or 10, 1, 1),
            'batch_small': measure_batch_small(),
            'reductions': measure_receiver(p),
            'serve': measure_serve(args.serve_seconds, 1.0, args.serve_chunk,
                                   args.serve_wall if args.serve_wall is not None else 60.0,
                                   args.serve_chunk_work, args.serve_max_chunk_work),
        }
    if rank == 0:
        print(json.dumps(line))
    if dist is not None:
        dist.destroy_process_group()


def run_egb3d(args):
    """The 3-D (5-D phase space) workload: whole solves (medium, source, evolve, superpose) through
    the C ABI with --evolve-steps TVD-RK3 steps each (default 20 of the workload's full count)."""
    import torch
    torch.cuda.set_device(0)
    p = workload(args.workload)
    print(json.dumps(measure_3d(p, args.evolve_steps or 20, args.steps, args.warmup)))


def measure_receiver(p, K=5, W=2):
    """The two reductions of one evolved state, each timed on its own (CUDA events on the context's
    stream, W untimed calls first): the source-side superposition with arrivals (egb_superpose) and
    the receiver-side reciprocal sum (egb_superpose_receiver), both into device buffers.  Their unit
    is a beam-point sum: one phase cell at one frequency."""
    import torch
    import paper_2006_11945_gb300 as egb
    stream = torch.cuda.Stream()
    no, kmax = len(p.freqs), 8
    u_d = torch.empty((no, p.nz, p.nx, 2), dtype=torch.float32, device='cuda')
    cnt_d = torch.empty((p.nz, p.nx), dtype=torch.uint8, device='cuda')
    T_d = torch.empty((p.nz, p.nx, kmax), dtype=torch.float64, device='cuda')
    A_d = torch.empty((p.nz, p.nx, kmax), dtype=torch.float32, device='cuda')
    out = {}
    with egb.Context(0, stream.cuda_stream) as ctx:
        m = ctx.medium_2d(p)
        s = ctx.source_2d(m, p)
        ctx.evolve(s, p.steps, p.cfl)
        calls = {'source_side': lambda: egb.egb_superpose(ctx.h, s, u_d, cnt_d, T_d, A_d, kmax),
                 'receiver_side': lambda: egb.egb_superpose_receiver(ctx.h, s, u_d)}
        cells = p.nx * p.nz * p.n_theta
        for name, fn in calls.items():
            for _ in range(W):
                fn()
            egb.egb_sync(ctx.h)
            t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            with torch.cuda.stream(stream):
                t0.record(stream)
            for _ in range(K):
                fn()
            with torch.cuda.stream(stream):
                t1.record(stream)
            egb.egb_sync(ctx.h)
            ms = t0.elapsed_time(t1) / K
            out[name] = {'ms': ms, 'beam_point_sums_per_s': cells * no / (ms / 1e3)}
    out['workload'] = (f'{p.name} {p.nx}x{p.nz} x {p.n_theta} angles after {p.steps} steps, '
                       f'{no} frequencies; state resident, no flush (the reductions read it once)')
    out['calls'] = K
    return out


def measure_3d(p, steps_evolve, K, W, warmup_steps=None):
    """K timed whole 3-D solves of problem p with steps_evolve TVD-RK3 steps each, after W untimed
    ones (of warmup_steps steps each, default steps_evolve); returns the bench record."""
    import torch
    import paper_2006_11945_gb300 as egb
    stream = torch.cuda.Stream()
    ctx = egb.Context(0, stream.cuda_stream)
    c21_d = torch.from_numpy(np.ascontiguousarray(p.c21)).cuda()
    rho_d = torch.from_numpy(np.ascontiguousarray(p.rho)).cuda()
    no, kmax = len(p.freqs), 8
    nodes = p.nx * p.ny * p.nz
    u_d = torch.empty((no, nodes, 2), dtype=torch.float32, device='cuda')
    cnt_d = torch.empty((nodes,), dtype=torch.uint8, device='cuda')
    T_d = torch.empty((nodes, kmax), dtype=torch.float64, device='cuda')
    A_d = torch.empty((nodes, kmax), dtype=torch.float32, device='cuda')
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    evolve_ms = []

    def solve(steps=steps_evolve):
        m = egb.egb_medium(ctx.h, (p.nx, p.ny, p.nz), (p.hx, p.hy, p.hz), tuple(p.origin), c21_d, rho_d, dim=3)
        s = egb.egb_source(ctx.h, m, tuple(p.xs), p.omegas, p.beam_width, p.n_theta, 0.0, n_phi=p.n_phi)
        with torch.cuda.stream(stream):
            ev0.record(stream)
        egb.egb_evolve(ctx.h, s, steps, p.cfl)
        with torch.cuda.stream(stream):
            ev1.record(stream)
        egb.egb_superpose(ctx.h, s, u_d, cnt_d, T_d, A_d, kmax)
        egb.egb_sync(ctx.h)
        evolve_ms.append(ev0.elapsed_time(ev1))
        info = egb.egb_get_solve_info(ctx.h, s)
        egb.egb_release(ctx.h, s)
        egb.egb_release(ctx.h, m)
        return info

    for _ in range(W):
        solve(warmup_steps or steps_evolve)
    evolve_ms.clear()
    with ClockSampler(0) as clk:
        torch.cuda.synchronize()
        t0 = torch.cuda.Event(enable_timing=True)
        t1 = torch.cuda.Event(enable_timing=True)
        with torch.cuda.stream(stream):
            t0.record(stream)
        for _ in range(K):
            info = solve()
        with torch.cuda.stream(stream):
            t1.record(stream)
        torch.cuda.synchronize()
    ms = t0.elapsed_time(t1)
    cells = info['cells']
    launch_ms = float(np.mean(evolve_ms)) / (3 * steps_evolve)
    achieved = ALGO_BYTES_PER_CELL_UPDATE_3D * cells / 3.0 / (launch_ms / 1e3) / 1e9
    peak, peak_kind = measured_peaks()
    ctx.close()
    return {
        'metric': 'phase-space cell-updates/s', 'value': cells * steps_evolve * K / (ms / 1e3),
        'unit': 'cell-updates/s', 'n_gpus': 1, 'steps': K, 'warmup': W,
        'ms_per_step': ms / K, 'higher_is_better': True, 'scaling': 'weak', 'vs_baseline': None,
        'dtype': 'f32 (double-float tau and phase)', 'data': 'synthetic (seeded triclinic medium)',
        'config': {'workload': f'{p.name} {p.nx}^3 at {p.hx:g} m x {p.n_theta} polar x {p.n_phi} azimuth, '
                               f'{steps_evolve} of {p.steps} TVD-RK3 steps per solve, {len(p.freqs)} frequency',
                   'cells': cells, 'evolve_steps': steps_evolve, 'device_GB': info['device_bytes'] / 1e9,
                   'l2': 'state larger than L2, no flush'},
        'evolve_cell_updates_per_s': cells * steps_evolve / (float(np.mean(evolve_ms)) / 1e3),
        'solves_per_s': K / (ms / 1e3),
        'roofline': {'bound': 'hbm', 'kernel': 'k_rk3_3d', 'achieved': achieved, 'peak': peak, 'unit': 'GB/s',
                     'frac': achieved / peak, 'traffic': None, 'peak_kind': peak_kind, 'launch_ms': launch_ms},
        'gpu_launches': (2 + 4 + 3 * steps_evolve + 5) * K,
        'clocks': clk.summary(),
    }


def run_batch(args):
    """The uneven batch: the first --batch-count instances of the batched recipe at full size (grids
    256^2-1024^2 at 5 m, 128-512 angles, 1-4 frequencies, one TTI medium each), resident together.
    One bench step = every instance advanced --evolve-steps TVD-RK3 steps by egb_evolve_batch (one
    persistent launch per stage over the work items of all instances, 3-step rotations replayed
    from a CUDA graph) and superposed.  The same steps taken one instance at a time with egb_evolve
    are timed for comparison."""
    import torch
    import paper_2006_11945_gb300 as egb
    torch.cuda.set_device(0)
    ps = synthmedia.batched_instances(count=args.batch_count)
    S = args.evolve_steps or 10
    stream = torch.cuda.Stream()
    ctx = egb.Context(0, stream.cuda_stream)
    ids, outs = [], []
    for p in ps:
        m = ctx.medium_2d(p)
        ids.append(ctx.source_2d(m, p))
        outs.append((torch.empty((len(p.freqs), p.nz, p.nx, 2), dtype=torch.float32, device='cuda'),
                     torch.empty((p.nz, p.nx), dtype=torch.uint8, device='cuda'),
                     torch.empty((p.nz, p.nx, 8), dtype=torch.float64, device='cuda'),
                     torch.empty((p.nz, p.nx, 8), dtype=torch.float32, device='cuda')))
    egb.egb_sync(ctx.h)
    cells = sum(egb.egb_get_solve_info(ctx.h, s)['cells'] for s in ids)

    def step():
        egb.egb_evolve_batch(ctx.h, ids, [S] * len(ids), ps[0].cfl)
        for s, (u, c, T, A) in zip(ids, outs):
            egb.egb_superpose(ctx.h, s, u, c, T, A, 8)

    def timed(fn, K):
        torch.cuda.synchronize()
        t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        with torch.cuda.stream(stream):
            t0.record(stream)
        for _ in range(K):
            fn()
        with torch.cuda.stream(stream):
            t1.record(stream)
        torch.cuda.synchronize()
        return t0.elapsed_time(t1)

    for _ in range(args.warmup):
        step()
    with ClockSampler(0) as clk:
        ms = timed(step, args.steps)
    egb.egb_sync(ctx.h)

    def evolve_batch_only():
        egb.egb_evolve_batch(ctx.h, ids, [S] * len(ids), ps[0].cfl)

    def evolve_one_by_one():
        for s in ids:
            egb.egb_evolve(ctx.h, s, S, ps[0].cfl)
    ms_b = timed(evolve_batch_only, 1)
    ms_1 = timed(evolve_one_by_one, 1)
    egb.egb_sync(ctx.h)
    value = cells * S * args.steps / (ms / 1e3)
    print(json.dumps({
        'metric': 'phase-space cell-updates/s', 'value': value, 'unit': 'cell-updates/s', 'n_gpus': 1,
        'steps': args.steps, 'warmup': args.warmup, 'ms_per_step': ms / args.steps, 'higher_is_better': True,
        'scaling': 'weak', 'vs_baseline': None, 'dtype': 'f32 (double-float tau and phase)',
        'data': 'synthetic (seeded TTI media)',
        'config': {'workload': f'uneven batch: first {len(ps)} instances of the 64 (grids '
                               f'{min(p.nx for p in ps)}^2-{max(p.nx for p in ps)}^2 at 5 m, '
                               f'{min(p.n_theta for p in ps)}-{max(p.n_theta for p in ps)} angles), '
                               f'{S} TVD-RK3 steps per instance per step, all superposed',
                   'cells': cells, 'instances': [[p.nx, p.n_theta, len(p.freqs)] for p in ps],
                   'l2': 'state larger than L2, no flush'},
        'evolve_batched_cell_updates_per_s': cells * S / (ms_b / 1e3),
        'evolve_one_by_one_cell_updates_per_s': cells * S / (ms_1 / 1e3),
        'gpu_launches': (3 * S + 5 * len(ps)) * args.steps,
        'clocks': clk.summary(),
    }))
    ctx.close()


def measure_batch_small(steps=60, K=3):
    """Batching where it pays: small instances advanced by one egb_evolve_batch call against one
    egb_evolve per instance, both timed with CUDA events on the context stream (K calls after one
    untimed).  Two sets: 32 copies of the 64^2 x 64 VTI instance (the small class of the serving
    stream) and 64 instances of the uneven recipe scaled by 1/8 (72^2-120^2 grids, 20-62 angles)."""
    import torch
    import paper_2006_11945_gb300 as egb
    sets = {'vti64x32': [synthmedia.vti_homogeneous(n=64, n_theta=64, steps=steps) for _ in range(32)],
            'uneven_1_8x64': synthmedia.batched_instances(count=64, size_scale=0.125)}
    out = {}
    for name, ps in sets.items():
        stream = torch.cuda.Stream()
        with egb.Context(0, stream.cuda_stream) as ctx:
            ids = [ctx.source_2d(ctx.medium_2d(p), p) for p in ps]
            egb.egb_sync(ctx.h)
            cells = sum(p.nx * p.nz * p.n_theta for p in ps)

            def timed(fn):
                fn()
                egb.egb_sync(ctx.h)
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                with torch.cuda.stream(stream):
                    e0.record(stream)
                for _ in range(K):
                    fn()
                with torch.cuda.stream(stream):
                    e1.record(stream)
                egb.egb_sync(ctx.h)
                return e0.elapsed_time(e1) / K
            cfl = ps[0].cfl
            b = timed(lambda: egb.egb_evolve_batch(ctx.h, ids, [steps] * len(ids), cfl))
            o = timed(lambda: [egb.egb_evolve(ctx.h, i, steps, cfl) for i in ids])
        out[name] = {'instances': len(ps), 'cells': cells, 'steps': steps, 'batched_ms': b, 'one_by_one_ms': o,
                     'speedup': o / b, 'batched_cell_updates_per_s': cells * steps / (b / 1e3)}
    return out


def measure_batch_waves(ps, S, K, W):
    """Uneven batched solves admitted in waves by free HBM (the library refuses a solve that does not
    fit with EGB_E_NOMEM): each wave is every instance that fits beside the ones already admitted,
    advanced S TVD-RK3 steps together by egb_evolve_batch (one persistent launch per stage over all
    their work items), superposed and released before the next wave.  One bench step is one pass
    over all instances; K timed after W untimed."""
    import torch
    import paper_2006_11945_gb300 as egb
    stream = torch.cuda.Stream()
    ctx = egb.Context(0, stream.cuda_stream)
    outs = [(torch.empty((len(p.freqs), p.nz, p.nx, 2), dtype=torch.float32, device='cuda'),
             torch.empty((p.nz, p.nx), dtype=torch.uint8, device='cuda'),
             torch.empty((p.nz, p.nx, 8), dtype=torch.float64, device='cuda'),
             torch.empty((p.nz, p.nx, 8), dtype=torch.float32, device='cuda')) for p in ps]
    c21 = [torch.from_numpy(np.ascontiguousarray(p.c21)).cuda() for p in ps]
    rho = [torch.from_numpy(np.ascontiguousarray(p.rho)).cuda() for p in ps]
    waves = []

    def one_pass():
        i, sizes = 0, []
        while i < len(ps):
            wave = []
            while i < len(ps):
                p = ps[i]
                try:
                    m = egb.egb_medium(ctx.h, (p.nx, 1, p.nz), (p.hx, 1.0, p.hz), (p.origin[0], 0.0, p.origin[1]),
                                       c21[i], rho[i])
                except egb.EgbError as e:
                    if e.status != egb.EGB_E_NOMEM or not wave:
                        raise
                    break
                try:
                    s = egb.egb_source(ctx.h, m, (p.xs[0], 0.0, p.xs[1]), p.omegas, p.beam_width, p.n_theta, 0.0)
                except egb.EgbError as e:
                    egb.egb_release(ctx.h, m)
                    if e.status != egb.EGB_E_NOMEM or not wave:
                        raise
                    break
                wave.append((i, m, s))
                i += 1
            egb.egb_evolve_batch(ctx.h, [s for _, _, s in wave], [S] * len(wave), ps[0].cfl)
            for j, m, s in wave:
                egb.egb_superpose(ctx.h, s, *outs[j], 8)
                egb.egb_release(ctx.h, s)
                egb.egb_release(ctx.h, m)
            sizes.append(len(wave))
        egb.egb_sync(ctx.h)
        waves.append(sizes)

    for _ in range(W):
        one_pass()
    with ClockSampler(0) as clk:
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(K):
            one_pass()
        torch.cuda.synchronize()
        ms = (time.perf_counter() - t0) * 1e3
    ctx.close()
    cells = sum(p.cells for p in ps)
    return {
        'metric': 'phase-space cell-updates/s', 'value': cells * S * K / (ms / 1e3), 'unit': 'cell-updates/s',
        'n_gpus': 1, 'steps': K, 'warmup': W, 'ms_per_step': ms / K, 'higher_is_better': True,
        'scaling': 'weak', 'dtype': 'f32 (double-float tau and phase)', 'data': 'synthetic (seeded TTI media)',
        'config': {'workload': f'uneven batch: {len(ps)} instances of the 64-instance recipe (grids '
                               f'{min(p.nx for p in ps)}^2-{max(p.nx for p in ps)}^2 at 5 m, '
                               f'{min(p.n_theta for p in ps)}-{max(p.n_theta for p in ps)} angles, 1-4 '
                               f'frequencies), admitted in waves by free HBM, {S} TVD-RK3 steps each, '
                               f'every instance set up, superposed and released per step',
                   'cells': cells, 'waves': waves[-1],
                   'l2': 'state larger than L2, no flush'},
        'solves_per_s': len(ps) * K / (ms / 1e3),
        'timing': 'host wall clock around whole passes (setup, evolve, superpose, release)',
        'gpu_launches': K * (len(ps) * (2 + 5 + 5) + 3 * S * len(waves[-1])),
        'clocks': clk.summary(),
    }


def fp64_form(p, steps, device):
    """The plain all-FP64 GPU form on the same workload, evolution timed over `steps` steps.

    Returns its cell-update rate and the solves/s it implies for the workload's full step count
    (setup and superposition excluded, which favours the FP64 form)."""
    import torch
    import paper_2006_11945_gb300 as egb
    stream = torch.cuda.Stream()
    ctx = egb.Context(device, stream.cuda_stream, precision=egb.EGB_FP64)
    m = ctx.medium_2d(p)
    s = ctx.source_2d(m, p)
    egb.egb_evolve(ctx.h, s, 1, p.cfl)
    egb.egb_sync(ctx.h)
    t0 = torch.cuda.Event(enable_timing=True)
    t1 = torch.cuda.Event(enable_timing=True)
    with torch.cuda.stream(stream):
        t0.record(stream)
    egb.egb_evolve(ctx.h, s, steps, p.cfl)
    with torch.cuda.stream(stream):
        t1.record(stream)
    egb.egb_sync(ctx.h)
    ms = t0.elapsed_time(t1)
    egb.egb_release(ctx.h, s)
    egb.egb_release(ctx.h, m)
    ctx.close()
    rate = p.cells * steps / (ms / 1e3)
    return {'value': rate, 'unit': 'cell-updates/s', 'timed_steps': steps,
            'solves_per_s': rate / (p.cells * p.steps),
            'note': 'plain FP64 stencil, one thread per cell, evolution only'}


# Depth march (--workload zmarch): per (theta, x) cell and stage launch the nf state fields are
# read and written (4 nf B each), u^n is read in stages 2 and 3 (4 nf B) and the coefficients U, W, S
# of the two bounding rows are read (24 B); with the advected dynamic ray tracing (nf = 9 instead of
# 5) also the Jacobian of (U, W) of the two rows (32 B).  Averaged over the three stage launches.
def algo_bytes_per_cell_stage_zm(drt):
    nf = 9 if drt else 5
    rows = 24 + (32 if drt else 0)
    s1 = 8 * nf + rows
    return (s1 + 2 * (s1 + 4 * nf)) / 3.0


def run_zmarch(args):
    """The paper's paraxial depth march (egb_zmarch) on the 512 x 512 TTI medium: whole solves
    (medium upload, both branches, 3-frequency superposition and arrivals) through the C ABI."""
    import torch
    import paper_2006_11945_gb300 as egb
    torch.cuda.set_device(0)
    p = workload('zmarch')
    if args.zm_n != 512:  # a smaller grid of the same physical extent (profiling captures)
        p = synthmedia.tti_heterogeneous(n=args.zm_n, h=2560.0 / args.zm_n, n_theta=256,
                                         freqs=(10.0, 20.0, 40.0))
    nth, tmax = args.zm_theta, math.radians(args.zm_theta_max)
    stream = torch.cuda.Stream()
    ctx = egb.Context(0, stream.cuda_stream)
    c21_d = torch.from_numpy(np.ascontiguousarray(p.c21)).cuda()
    rho_d = torch.from_numpy(np.ascontiguousarray(p.rho)).cuda()
    c21_h = torch.from_numpy(np.ascontiguousarray(p.c21)).pin_memory()
    rho_h = torch.from_numpy(np.ascontiguousarray(p.rho)).pin_memory()
    no, kmax = len(p.freqs), 8
    outs_d = (torch.empty((no, p.nz, p.nx, 2), dtype=torch.float32, device='cuda'),
              torch.empty((p.nz, p.nx), dtype=torch.uint8, device='cuda'),
              torch.empty((p.nz, p.nx, kmax), dtype=torch.float64, device='cuda'),
              torch.empty((p.nz, p.nx, kmax), dtype=torch.float32, device='cuda'))
    outs_h = tuple(torch.empty(o.shape, dtype=o.dtype).pin_memory() for o in outs_d)
    infos = []

    def solve(host):
        c21, rho = (c21_h, rho_h) if host else (c21_d, rho_d)
        m = egb.egb_medium(ctx.h, (p.nx, 1, p.nz), (p.hx, 1.0, p.hz), (p.origin[0], 0.0, p.origin[1]), c21, rho)
        u, cnt, T, A = outs_h if host else outs_d
        info = egb.egb_zmarch(ctx.h, m, p.xs, p.omegas, p.beam_width, nth, tmax, p.cfl, u, cnt, T, A, kmax,
                              drt=args.zm_drt)
        egb.egb_release(ctx.h, m)
        infos.append(info)
        return info

    def timed(host, K, W):
        for _ in range(W):
            solve(host)
        infos.clear()
        torch.cuda.synchronize()
        t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        with torch.cuda.stream(stream):
            t0.record(stream)
        for _ in range(K):
            info = solve(host)
        with torch.cuda.stream(stream):
            t1.record(stream)
        torch.cuda.synchronize()
        return t0.elapsed_time(t1), info

    with ClockSampler(0) as clk:
        ms, info = timed(False, args.steps, args.warmup)
    march_ms = float(np.mean([i['march_ms'] for i in infos]))
    setup_ms = float(np.mean([i['setup_ms'] for i in infos]))
    sup_ms = float(np.mean([i['superpose_ms'] for i in infos]))
    e2e_ms, _ = timed(True, max(1, args.steps), 1)
    cu = info['cell_updates']
    # a stage launch advances one or both branches; per pass over one branch's plane the algorithmic
    # bytes and the device time are in the same ratio as per launch
    pass_ms = march_ms / info['stage_passes']
    achieved = algo_bytes_per_cell_stage_zm(args.zm_drt) * nth * p.nx / (pass_ms / 1e3) / 1e9
    peak, peak_kind = measured_peaks()
    h2d = p.c21.nbytes + p.rho.nbytes
    d2h = sum(o.numel() * o.element_size() for o in outs_h)
    line = {
        'metric': 'phase-space cell-updates/s', 'value': cu * args.steps / (ms / 1e3),
        'unit': 'cell-updates/s', 'n_gpus': 1, 'steps': args.steps, 'warmup': args.warmup,
        'ms_per_step': ms / args.steps, 'higher_is_better': True, 'scaling': 'weak', 'vs_baseline': None,
        'dtype': 'f32 (double-float tau and phase)', 'data': 'synthetic (seeded TTI medium)',
        'config': {'workload': f'paraxial depth march (Eqs. 13-20), {p.name} {p.nx}x{p.nz} at {p.hx:g} m, '
                               f'{nth} angles per branch within +-{args.zm_theta_max:g} deg, both branches, '
                               f'{len(p.freqs)} frequencies, dynamic ray tracing '
                               f'{"advected (Eq. 21)" if args.zm_drt else "from label gradients"}',
                   'cells_per_row': nth * p.nx, 'drt': args.zm_drt,
                   'n_sub': info['n_sub'], 'rows': info['rows'], 'freqs_hz': p.freqs,
                   'l2': 'per-row state (2 MB) L2-resident; coefficient and history volumes (1.9 GB) larger than L2, no flush'},
        'solves_per_s': args.steps / (ms / 1e3),
        'phase_ms': {'setup': setup_ms, 'march': march_ms, 'superpose': sup_ms},
        'e2e': {'value': cu * max(1, args.steps) / (e2e_ms / 1e3), 'unit': 'cell-updates/s',
                'h2d_bytes_per_step': int(h2d), 'd2h_bytes_per_step': int(d2h)},
        'roofline': {'bound': 'hbm', 'kernel': 'k_zm_stage', 'achieved': achieved, 'peak': peak, 'unit': 'GB/s',
                     'frac': achieved / peak, 'traffic': None, 'peak_kind': peak_kind, 'pass_ms': pass_ms},
        'gpu_launches': (2 + info['kernel_launches']) * args.steps,
        'clocks': clk.summary(),
    }
    if not args.no_cpu_baseline:
        line['cpu_baseline'] = cpu_baseline_zmarch(p, args.cpu_seconds)
    print(json.dumps(line))
    ctx.close()


def _zmarch_sample(p):
    """128 x 128 sub-block of the workload medium with 64 angles per branch (downgoing branch)."""
    from oracle import zmarch as ZM
    q = _oracle_sample(p, 128)
    return q, ZM.ZSetup(q, 64, math.radians(60.0), 1, q.cfl)


def cpu_baseline_zmarch(p, budget_s=20.0):
    """Time the FP64 oracle's depth march (downgoing branch, setup excluded) on a bounded sample."""
    from oracle import zmarch as ZM
    q, Z = _zmarch_sample(p)
    t = time.perf_counter()
    ZM.march(Z)
    el = time.perf_counter() - t
    cu = (len(Z.rows) - 1) * Z.n_sub * Z.nth * Z.nx
    cores = int(os.environ.get('OMP_NUM_THREADS', os.cpu_count() or 1))
    return {'value': cu / el, 'unit': 'cell-updates/s', 'cores': cores, 'kind': 'oracle',
            'sample': f'{q.nx}x{q.nz} sub-block of the workload medium, 64 angles within +-60 deg, the '
                      f'downgoing branch ({len(Z.rows)} rows x {Z.n_sub} substeps) of the float64 '
                      f'oracle march, setup excluded ({el:.1f} s)'}


def _oracle_sample(p, sub=128):
    """A sub-block of the workload's medium (same spacing and angle count) for the CPU oracle."""
    n = min(sub, p.nx)
    c21 = p.c21.reshape(p.nz, p.nx, 21)[:n, :n].reshape(-1, 21).copy()
    rho = p.rho.reshape(p.nz, p.nx)[:n, :n].reshape(-1).copy()
    q = synthmedia.Problem2D(p.name + '_sample', n, n, p.hx, p.hz, c21, rho,
                             ((n // 2) * p.hx, (n // 2) * p.hz), p.n_theta, p.freqs, p.beam_width,
                             p.steps, p.cfl)
    return q


def cpu_baseline(p, budget_s=20.0):
    """Time the FP64 oracle's evolution on a bounded sample of the workload (host cores)."""
    from oracle import liouville as OL
    q = _oracle_sample(p)
    S = OL.Setup(q)
    st = S.initial_state()
    t = time.perf_counter()
    S2, st, dt = OL.evolve(q, steps=1, S=S, state=st)
    one = time.perf_counter() - t
    steps = max(1, min(200, int(budget_s / max(one, 1e-3))))
    t = time.perf_counter()
    OL.evolve(q, steps=steps, S=S, state=st)
    el = time.perf_counter() - t
    cores = int(os.environ.get('OMP_NUM_THREADS', os.cpu_count() or 1))
    return {'value': q.cells * steps / el, 'unit': 'cell-updates/s', 'cores': cores, 'kind': 'oracle',
            'sample': f'{q.nx}x{q.nz}x{q.n_theta} sub-block of the workload medium, {steps} TVD-RK3 '
                      f'steps of the float64 oracle (compiled loop), evolution only'}


def run_reference(args):
    ws, rank, local = dist_env()
    if rank != 0:
        return
    p = workload(args.workload)
    if args.workload == 'zmarch':
        return run_reference_zmarch(args, p, ws)
    q = _oracle_sample(p)
    from oracle import liouville as OL
    S = OL.Setup(q)
    st = S.initial_state()
    per = 2
    for _ in range(args.warmup):
        _, st, _ = OL.evolve(q, steps=per, S=S, state=st)
    t = time.perf_counter()
    for _ in range(args.steps):
        _, st, _ = OL.evolve(q, steps=per, S=S, state=st)
    el = time.perf_counter() - t
    value = q.cells * per * args.steps / el
    cores = int(os.environ.get('OMP_NUM_THREADS', os.cpu_count() or 1))
    sample = f'{q.nx}x{q.nz}x{q.n_theta} sub-block of the workload medium, {per} TVD-RK3 steps per step'
    print(json.dumps({
        'impl': 'reference', 'metric': 'phase-space cell-updates/s', 'value': value,
        'unit': 'cell-updates/s', 'n_gpus': ws, 'steps': args.steps, 'warmup': args.warmup,
        'ms_per_step': el / args.steps * 1e3, 'higher_is_better': True, 'scaling': 'weak',
        'vs_baseline': None, 'dtype': 'f64', 'data': 'synthetic (seeded TTI medium)',
        'config': {'workload': f'{p.name} {p.nx}x{p.nz} at {p.hx:g} m x {p.n_theta} angles (oracle sample)'},
        'cpu_baseline': {'value': value, 'unit': 'cell-updates/s', 'cores': cores, 'kind': 'oracle',
                         'sample': sample},
        'e2e': {'value': value, 'unit': 'cell-updates/s', 'h2d_bytes_per_step': 0, 'd2h_bytes_per_step': 0},
    }))


def run_reference_zmarch(args, p, ws):
    """Reference arm of the depth-march workload: the FP64 oracle march on its bounded sample."""
    from oracle import zmarch as ZM
    q, Z = _zmarch_sample(p)
    cu = (len(Z.rows) - 1) * Z.n_sub * Z.nth * Z.nx
    for _ in range(args.warmup):
        ZM.march(Z)
    t = time.perf_counter()
    for _ in range(args.steps):
        ZM.march(Z)
    el = time.perf_counter() - t
    value = cu * args.steps / el
    cores = int(os.environ.get('OMP_NUM_THREADS', os.cpu_count() or 1))
    sample = f'{q.nx}x{q.nz} sub-block, 64 angles, downgoing branch of the float64 oracle march per step'
    print(json.dumps({
        'impl': 'reference', 'metric': 'phase-space cell-updates/s', 'value': value,
        'unit': 'cell-updates/s', 'n_gpus': ws, 'steps': args.steps, 'warmup': args.warmup,
        'ms_per_step': el / args.steps * 1e3, 'higher_is_better': True, 'scaling': 'weak',
        'vs_baseline': None, 'dtype': 'f64', 'data': 'synthetic (seeded TTI medium)',
        'config': {'workload': f'paraxial depth march, {p.name} {p.nx}x{p.nz} (oracle sample)'},
        'cpu_baseline': {'value': value, 'unit': 'cell-updates/s', 'cores': cores, 'kind': 'oracle',
                         'sample': sample},
        'e2e': {'value': value, 'unit': 'cell-updates/s', 'h2d_bytes_per_step': 0, 'd2h_bytes_per_step': 0},
    }))


def serve_requests(duration, seed=4, rate=200.0, large_scale=1.0):
    """The Poisson request stream (50/50 small/large, 1-8 frequencies in 8-40 Hz) as Requests."""
    import dataclasses
    from paper_2006_11945_gb300.serve import Request
    out = []
    media = {}
    small = synthmedia.vti_homogeneous()
    for i, (t, kind, nf, freqs) in enumerate(synthmedia.request_stream(rate=rate, duration=duration,
                                                                       seed=seed)):
        if kind == 'small':
            p = dataclasses.replace(small, freqs=list(freqs))
        else:
            # eight seeded large media, reused across requests (building one takes seconds on the host)
            key = i % 8
            if key not in media:
                n = int(512 * large_scale) // 4 * 4
                media[key] = synthmedia.tti_heterogeneous(n=n, h=2560.0 / n,
                                                          n_theta=max(16, int(256 * large_scale)),
                                                          seed=100 + key)
            p = dataclasses.replace(media[key], freqs=list(freqs))
        out.append(Request(i, t, p))
    return out


def measure_serve_curve(rates=(5.0, 10.0, 20.0, 40.0, 80.0, 160.0), seconds=4.0, large_scale=0.25,
                        chunk=60, chunk_work=4e9, max_chunk_work=2e10):
    """Offered against sustained load: the serving loop on Poisson streams of increasing rate (the
    same 50/50 mix, large requests scaled by large_scale), arrivals admitted for `seconds`, then
    everything admitted drained.  Per rate: offered requests/s, completed and never-admitted
    requests, completed/s over the whole run, p50/p99 latency of the completed ones."""
    from paper_2006_11945_gb300.serve import Backend, serve
    points = []
    be = Backend(0)
    # warm-up: the first solve of each grid shape runs the stencil autotuner, the first of each
    # medium its characteristic velocities
    serve(serve_requests(2.0, seed=9, rate=8.0, large_scale=large_scale), be, chunk_steps=chunk,
          chunk_work=chunk_work, max_chunk_work=max_chunk_work)
    for rate in rates:
        reqs = serve_requests(seconds, rate=rate, large_scale=large_scale)
        st = serve(reqs, be, chunk_steps=chunk, time_limit=seconds, chunk_work=chunk_work,
                   max_chunk_work=max_chunk_work)
        s = st.summary(len(reqs))
        points.append({'offered_per_s': len(reqs) / seconds, 'offered': len(reqs), 'completed': s['completed'],
                       'not_admitted': s['not_admitted'], 'completed_per_s': s['solves_per_s'],
                       'p50_s': s['p50_latency_s'], 'p99_s': s['p99_latency_s'], 'wall_s': s['wall_s'],
                       'device_cell_updates_per_s': s['device_cell_updates_per_s']})
    be.close()
    n = int(512 * large_scale) // 4 * 4
    return {'metric': 'serving: completed solves/s against offered requests/s', 'unit': 'solves/s',
            'config': {'workload': f'Poisson streams, {seconds:g} s of arrivals each, 50/50 64x64x64 VTI / '
                                   f'{n}^2 x {max(16, int(256 * large_scale))} TTI, 1-8 frequencies, '
                                   'admitted ones drained', 'chunk_steps': chunk, 'chunk_work': chunk_work,
                       'max_chunk_work': max_chunk_work},
            'points': points}


def run_serve(args):
    """Serving measurement: arrivals for --serve-seconds, then drain what was admitted."""
    import torch
    torch.cuda.set_device(0)
    print(json.dumps(measure_serve(args.serve_seconds, args.serve_large_scale, args.serve_chunk,
                                   args.serve_wall, args.serve_chunk_work, args.serve_max_chunk_work)))


def measure_serve(seconds, large_scale, chunk, wall=None, chunk_work=4e9, max_chunk_work=2e10):
    """Continuous batching on the Poisson request stream: arrivals for `seconds`, admitted by free
    HBM; the loop then drains what was admitted, stopping at `wall` seconds (requests still on the
    device are released and counted unfinished).  Returns the serving record."""
    from paper_2006_11945_gb300.serve import Backend, serve
    reqs = serve_requests(seconds, large_scale=large_scale)
    be = Backend(0)
    with ClockSampler(0) as clk:
        st = serve(reqs, be, chunk_steps=chunk, time_limit=seconds, wall_limit=wall, chunk_work=chunk_work,
                   max_chunk_work=max_chunk_work)
    be.close()
    s = st.summary(len(reqs))
    small = [r.finished - r.arrival for r in st.completed if r.problem.name == 'vti_homogeneous']
    large = [r.finished - r.arrival for r in st.completed if r.problem.name != 'vti_homogeneous']
    for name, lat in (('small', small), ('large', large)):
        if lat:
            s[f'{name}_p50_s'] = float(np.percentile(lat, 50))
            s[f'{name}_p99_s'] = float(np.percentile(lat, 99))
            s[f'{name}_completed'] = len(lat)
    small_p = synthmedia.vti_homogeneous()
    n_large = int(512 * large_scale) // 4 * 4
    large_cu = n_large * n_large * max(16, int(256 * large_scale)) * synthmedia.tti_default_steps(
        n_large, 2560.0 / n_large)
    s['offered_per_s'] = len(reqs) / seconds
    s['offered_cell_updates_per_s'] = s['offered_per_s'] * 0.5 * (small_p.cells * small_p.steps + large_cu)
    return {'metric': 'serving: solves/s and p50/p99 latency', 'value': s['solves_per_s'],
            'unit': 'solves/s', 'higher_is_better': True,
            'config': {'workload': f'Poisson 200 req/s for {seconds:g} s, 50/50 64x64x64 VTI (150 steps) / '
                                   f'{n_large}^2 TTI ({large_cu / n_large ** 2:.0f} cell-updates per node), '
                                   f'1-8 frequencies, admission by free HBM, drain stopped at '
                                   f'{wall if wall is not None else "completion"} s',
                       'chunk_steps': chunk, 'chunk_work': chunk_work, 'max_chunk_work': max_chunk_work},
            'serving': s, 'clocks': clk.summary()}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument('--gpus', type=int, default=1)
    ap.add_argument('--steps', type=int, default=3)
    ap.add_argument('--warmup', type=int, default=3)
    ap.add_argument('--impl', default='egb', choices=['egb', 'reference'])
    ap.add_argument('--workload', default='tti512',
                    choices=['tti512', 'tti256', 'tti128', 'vti64', 'tri96', 'tri48', 'batch', 'serve',
                             'serve_curve', 'zmarch'])
    ap.add_argument('--zm-theta', type=int, default=256)
    ap.add_argument('--zm-n', type=int, default=512)
    ap.add_argument('--zm-drt', type=int, default=0, choices=[0, 1])
    ap.add_argument('--zm-theta-max', type=float, default=60.0)
    ap.add_argument('--batch-count', type=int, default=6)
    ap.add_argument('--serve-seconds', type=float, default=2.0)
    ap.add_argument('--serve-large-scale', type=float, default=1.0)
    ap.add_argument('--serve-chunk', type=int, default=60)
    ap.add_argument('--serve-wall', type=float, default=None)
    ap.add_argument('--serve-chunk-work', type=float, default=4e9,
                    help='cell-updates a request advances per chunk (a small solve finishes in one)')
    ap.add_argument('--serve-max-chunk-work', type=float, default=2e10,
                    help='bound on the work of one chunk: admission shortest-work-first under it')
    ap.add_argument('--no-sub', action='store_true', help='skip the 3-D, batch and serving sub-records')
    ap.add_argument('--reductions', action='store_true',
                    help='time only the source-side and receiver-side reductions of one evolved state')
    ap.add_argument('--evolve-steps', type=int, default=None)
    ap.add_argument('--no-cpu-baseline', action='store_true')
    ap.add_argument('--cpu-seconds', type=float, default=20.0)
    ap.add_argument('--no-fp64-form', action='store_true')
    ap.add_argument('--fp64-steps', type=int, default=20)
    args = ap.parse_args()
    if args.impl == 'reference':
        run_reference(args)
    elif args.workload == 'serve_curve':
        import torch
        torch.cuda.set_device(0)
        print(json.dumps(measure_serve_curve()))
    elif args.workload == 'serve':
        run_serve(args)
    elif args.reductions:
        import dataclasses
        import torch
        torch.cuda.set_device(0)
        p = workload(args.workload)
        if args.evolve_steps is not None:
            p = dataclasses.replace(p, steps=args.evolve_steps)
        print(json.dumps(measure_receiver(p, K=args.steps, W=args.warmup)))
    elif args.workload in ('tri96', 'tri48'):
        run_egb3d(args)
    elif args.workload == 'batch':
        run_batch(args)
    elif args.workload == 'zmarch':
        run_zmarch(args)
    else:
        run_egb(args)


if __name__ == '__main__':
    main()
