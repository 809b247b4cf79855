"""Python binding of libegb, the GB300 anisotropic Eulerian Gaussian beam library.

Argument marshalling only: every step of the method runs in the CUDA kernels behind
``include/egb.h``.  The functions keep the C names (``egb_create``, ``egb_medium``, ``egb_source``,
``egb_evolve``, ``egb_superpose``, ``egb_sync``, ``egb_release``, ``egb_destroy``, ...) and accept
numpy arrays (host memory) or torch CUDA tensors (device memory); ``Context`` wraps them.

The library is loaded from ``_lib/libegb.so`` next to this file (build it with
``python -m paper_2006_11945_gb300.build``).  There is no fallback: if the library or a CUDA device
is missing, the calls raise.
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass
from typing import Optional, Sequence

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, '_lib', 'libegb.so')

EGB_OK, EGB_E_INVALID, EGB_E_NOT_PD, EGB_E_NOMEM, EGB_E_CUDA = 0, 1, 2, 3, 4
EGB_E_TIMEOUT, EGB_E_NUMERIC, EGB_E_ARRIVAL_OVERFLOW, EGB_E_BUSY = 5, 6, 7, 8
STATUS_NAMES = {0: 'EGB_OK', 1: 'EGB_E_INVALID', 2: 'EGB_E_NOT_PD', 3: 'EGB_E_NOMEM', 4: 'EGB_E_CUDA',
                5: 'EGB_E_TIMEOUT', 6: 'EGB_E_NUMERIC', 7: 'EGB_E_ARRIVAL_OVERFLOW', 8: 'EGB_E_BUSY'}
EGB_FP32_PHASE64, EGB_FP64 = 0, 1

EXPORTED = ('egb_create', 'egb_destroy', 'egb_medium', 'egb_source', 'egb_evolve', 'egb_superpose',
            'egb_sync', 'egb_release', 'egb_last_error', 'egb_get_solve_info', 'egb_read_state',
            'egb_read_velocity', 'egb_superpose_noalloc', 'egb_evolve_batch', 'egb_zmarch',
            'egb_superpose_receiver')


class EgbError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f'{STATUS_NAMES.get(status, status)}: {msg}')
        self.status = status


class egb_opts(ctypes.Structure):
    _fields_ = [('precision', ctypes.c_int), ('store_velocity', ctypes.c_int), ('wait_polls', ctypes.c_int)]


class egb_zmarch_info(ctypes.Structure):
    _fields_ = [('n_sub', ctypes.c_int * 2), ('rows', ctypes.c_int * 2), ('cell_updates', ctypes.c_uint64),
                ('stage_passes', ctypes.c_uint64), ('kernel_launches', ctypes.c_uint64),
                ('setup_ms', ctypes.c_double), ('march_ms', ctypes.c_double), ('superpose_ms', ctypes.c_double)]


class egb_solve_info(ctypes.Structure):
    _fields_ = [('nx', ctypes.c_int), ('nz', ctypes.c_int), ('n_theta', ctypes.c_int),
                ('n_omega', ctypes.c_int), ('steps_done', ctypes.c_int), ('dt', ctypes.c_double),
                ('max_rate', ctypes.c_double), ('c_ref', ctypes.c_double),
                ('cells', ctypes.c_uint64), ('device_bytes', ctypes.c_uint64),
                ('tile_chunk', ctypes.c_int), ('dim', ctypes.c_int), ('ny', ctypes.c_int),
                ('n_phi', ctypes.c_int)]


_lib = None


def load(path: Optional[str] = None):
    """Load libegb.so (raises if it is missing: there is no CPU fallback)."""
    global _lib
    if _lib is not None and path is None:
        return _lib
    p = path or LIB_PATH
    if not os.path.exists(p):
        raise RuntimeError(f'libegb.so not found at {p}; build it with '
                           f'`python -m paper_2006_11945_gb300.build` (needs nvcc)')
    lib = ctypes.CDLL(p)
    vp, i, d, u64 = ctypes.c_void_p, ctypes.c_int, ctypes.c_double, ctypes.c_uint64
    P = ctypes.POINTER
    lib.egb_create.argtypes = [P(vp), i, vp, P(egb_opts)]
    lib.egb_destroy.argtypes = [vp]
    lib.egb_medium.argtypes = [vp, i, P(i), P(d), P(d), vp, vp, P(u64)]
    lib.egb_source.argtypes = [vp, u64, P(d), i, P(d), d, P(i), d, d, P(u64)]
    lib.egb_evolve.argtypes = [vp, u64, i, d]
    lib.egb_evolve_batch.argtypes = [vp, i, P(u64), P(i), d]
    lib.egb_superpose.argtypes = [vp, u64, vp, vp, vp, vp, i]
    lib.egb_superpose_noalloc.argtypes = [vp, u64, vp, vp, vp, vp, i]
    lib.egb_superpose_receiver.argtypes = [vp, u64, vp]
    lib.egb_sync.argtypes = [vp]
    lib.egb_release.argtypes = [vp, u64]
    lib.egb_last_error.argtypes = [vp]
    lib.egb_last_error.restype = ctypes.c_char_p
    lib.egb_get_solve_info.argtypes = [vp, u64, P(egb_solve_info)]
    lib.egb_read_state.argtypes = [vp, u64, vp]
    lib.egb_read_velocity.argtypes = [vp, u64, vp]
    lib.egb_zmarch.argtypes = [vp, u64, P(d), i, P(d), d, i, d, d, i, vp, vp, vp, vp, i, P(egb_zmarch_info)]
    for name in EXPORTED:
        if name != 'egb_last_error':
            getattr(lib, name).restype = i
    if path is None:
        _lib = lib
    return lib


def _ptr(a):
    """Address of a numpy array or a torch tensor (device or host)."""
    if a is None:
        return None
    if hasattr(a, 'data_ptr'):
        if not a.is_contiguous():
            raise ValueError('tensors must be contiguous')
        return ctypes.c_void_p(a.data_ptr())
    if isinstance(a, np.ndarray):
        if not a.flags['C_CONTIGUOUS']:
            raise ValueError('arrays must be C-contiguous')
        return ctypes.c_void_p(a.ctypes.data)
    raise TypeError(f'unsupported buffer type {type(a)}')


def _check(ctx_handle, status):
    if status != EGB_OK:
        msg = load().egb_last_error(ctx_handle)
        raise EgbError(status, msg.decode() if msg else '')


# ---- thin functions with the C names ------------------------------------------------------------

def egb_create(device: int = 0, stream: int = 0, precision: int = EGB_FP32_PHASE64, wait_polls: int = 0):
    lib = load()
    h = ctypes.c_void_p()
    opts = egb_opts(precision, 1, wait_polls)
    st = lib.egb_create(ctypes.byref(h), device, ctypes.c_void_p(stream or None), ctypes.byref(opts))
    if st != EGB_OK:
        raise EgbError(st, 'egb_create failed (no CUDA device?)')
    return h


def egb_destroy(h):
    _check(h, load().egb_destroy(h))


def egb_medium(h, n, hsp, origin, c21, rho, dim=2):
    n_ = (ctypes.c_int * 3)(*n)
    h_ = (ctypes.c_double * 3)(*hsp)
    o_ = (ctypes.c_double * 3)(*origin)
    out = ctypes.c_uint64()
    _check(h, load().egb_medium(h, dim, n_, h_, o_, _ptr(c21), _ptr(rho), ctypes.byref(out)))
    return out.value


def egb_source(h, medium, xs, omegas: Sequence[float], beam_width, n_theta, r0=0.0, n_phi=0, R_sigma=0.0):
    xs_ = (ctypes.c_double * 3)(*xs)
    om = (ctypes.c_double * len(omegas))(*omegas)
    na = (ctypes.c_int * 2)(n_theta, n_phi)
    out = ctypes.c_uint64()
    _check(h, load().egb_source(h, medium, xs_, len(omegas), om, beam_width, na, r0, R_sigma or 0.0,
                                ctypes.byref(out)))
    return out.value


def egb_superpose_receiver(h, solve, u_out):
    _check(h, load().egb_superpose_receiver(h, solve, _ptr(u_out)))


def egb_evolve(h, solve, steps, cfl):
    _check(h, load().egb_evolve(h, solve, int(steps), float(cfl)))


def egb_evolve_batch(h, solves: Sequence[int], steps: Sequence[int], cfl):
    n = len(solves)
    ids = (ctypes.c_uint64 * max(n, 1))(*solves)
    st = (ctypes.c_int * max(n, 1))(*[int(x) for x in steps])
    _check(h, load().egb_evolve_batch(h, n, ids, st, float(cfl)))


def egb_superpose(h, solve, u_out=None, count=None, T=None, A=None, kmax=8):
    _check(h, load().egb_superpose(h, solve, _ptr(u_out), _ptr(count), _ptr(T), _ptr(A), kmax))


def egb_superpose_noalloc(h, solve, u_out=None, count=None, T=None, A=None, kmax=8):
    """egb_superpose into caller-owned DEVICE buffers without any device allocation (the work
    buffers are a fixed 32 MiB array inside the library); see include/egb.h."""
    _check(h, load().egb_superpose_noalloc(h, solve, _ptr(u_out), _ptr(count), _ptr(T), _ptr(A), kmax))


def egb_zmarch(h, medium, xs, omegas, beam_width, n_theta, theta_max, cfl=0.5, u_out=None, count=None,
               T=None, A=None, kmax=8, drt=0):
    """The paper's paraxial depth march from the source row, both branches, with its same-row
    superposition (see include/egb.h).  Returns the run's egb_zmarch_info as a dict."""
    om = (ctypes.c_double * max(len(omegas), 1))(*[float(w) for w in omegas])
    xs = tuple(xs)
    x = (ctypes.c_double * 3)(*((xs[0], 0.0, xs[1]) if len(xs) == 2 else xs))
    info = egb_zmarch_info()
    _check(h, load().egb_zmarch(h, medium, x, len(omegas), om, float(beam_width), int(n_theta),
                                 float(theta_max), float(cfl), int(drt), _ptr(u_out), _ptr(count), _ptr(T),
                                 _ptr(A), kmax, ctypes.byref(info)))
    out = {k: getattr(info, k) for k, _ in egb_zmarch_info._fields_}
    out['n_sub'], out['rows'] = list(info.n_sub), list(info.rows)
    return out


def egb_sync(h):
    _check(h, load().egb_sync(h))


def egb_release(h, ident):
    _check(h, load().egb_release(h, ident))


def egb_get_solve_info(h, solve):
    info = egb_solve_info()
    _check(h, load().egb_get_solve_info(h, solve, ctypes.byref(info)))
    return {f: getattr(info, f) for f, _ in egb_solve_info._fields_}


def egb_read_state(h, solve, out):
    _check(h, load().egb_read_state(h, solve, _ptr(out)))


def egb_read_velocity(h, solve, out):
    _check(h, load().egb_read_velocity(h, solve, _ptr(out)))


# ---- convenience wrapper ------------------------------------------------------------------------

@dataclass
class SolveResult:
    u: np.ndarray          # complex64 [n_omega][nz][nx]
    count: np.ndarray      # uint8 [nz][nx]
    T: np.ndarray          # float64 [nz][nx][kmax]
    A: np.ndarray          # float32 [nz][nx][kmax]


class Context:
    """Owns one egb context on a CUDA stream (an int cudaStream_t handle; 0 = legacy default)."""

    def __init__(self, device=0, stream=0, precision=EGB_FP32_PHASE64, wait_polls=0):
        self.h = egb_create(device, stream, precision, wait_polls)

    def close(self):
        if self.h is not None:
            egb_destroy(self.h)
            self.h = None

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def medium_2d(self, problem):
        return egb_medium(self.h, (problem.nx, 1, problem.nz), (problem.hx, 1.0, problem.hz),
                          (problem.origin[0], 0.0, problem.origin[1]),
                          np.ascontiguousarray(problem.c21, np.float32),
                          np.ascontiguousarray(problem.rho, np.float32))

    def source_2d(self, medium, problem):
        return egb_source(self.h, medium, (problem.xs[0], 0.0, problem.xs[1]), problem.omegas,
                          problem.beam_width, problem.n_theta, problem.r0 or 0.0,
                          R_sigma=getattr(problem, 'R_sigma', None) or 0.0)

    def superpose_receiver(self, solve, n_omega, nz, nx):
        """egb_superpose_receiver into a host array (n_omega, nz, nx) complex64."""
        u = np.zeros((n_omega, nz, nx), np.complex64)
        egb_superpose_receiver(self.h, solve, u)
        return u

    def evolve(self, solve, steps, cfl):
        egb_evolve(self.h, solve, steps, cfl)

    def superpose(self, solve, n_omega, nz, nx, kmax=8):
        u = np.zeros((n_omega, nz, nx), np.complex64)
        cnt = np.zeros((nz, nx), np.uint8)
        T = np.zeros((nz, nx, kmax), np.float64)
        A = np.zeros((nz, nx, kmax), np.float32)
        egb_superpose(self.h, solve, u, cnt, T, A, kmax)
        return SolveResult(u, cnt, T, A)

    def read_state(self, solve, nth, nz, nx):
        out = np.zeros((4, nth, nz, nx), np.float64)
        egb_read_state(self.h, solve, out)
        return out

    def read_velocity(self, solve, nth, nz, nx):
        out = np.zeros((6, nth, nz, nx), np.float32)
        egb_read_velocity(self.h, solve, out)
        return out

    # ---- 3-D ----
    def medium_3d(self, problem):
        return egb_medium(self.h, (problem.nx, problem.ny, problem.nz), (problem.hx, problem.hy, problem.hz),
                          tuple(problem.origin), np.ascontiguousarray(problem.c21, np.float32),
                          np.ascontiguousarray(problem.rho, np.float32), dim=3)

    def source_3d(self, medium, problem):
        return egb_source(self.h, medium, tuple(problem.xs), problem.omegas, problem.beam_width,
                          problem.n_theta, problem.r0 or 0.0, n_phi=problem.n_phi,
                          R_sigma=getattr(problem, "R_sigma", None) or 0.0)

    def superpose_3d(self, solve, n_omega, nz, ny, nx, kmax=8):
        u = np.zeros((n_omega, nz, ny, nx), np.complex64)
        cnt = np.zeros((nz, ny, nx), np.uint8)
        T = np.zeros((nz, ny, nx, kmax), np.float64)
        A = np.zeros((nz, ny, nx, kmax), np.float32)
        egb_superpose(self.h, solve, u, cnt, T, A, kmax)
        return SolveResult(u, cnt, T, A)

    def read_state_3d(self, solve, nph, nth, nz, ny, nx):
        out = np.zeros((8, nph, nth, nz, ny, nx), np.float64)
        egb_read_state(self.h, solve, out)
        return out

    def read_velocity_3d(self, solve, nph, nth, nz, ny, nx):
        out = np.zeros((9, nph, nth, nz, ny, nx), np.float32)
        egb_read_velocity(self.h, solve, out)
        return out

    def solve_problem_3d(self, problem, steps=None, kmax=8):
        """medium -> source -> evolve -> superpose for one 3-D problem; returns (result, info)."""
        m = self.medium_3d(problem)
        s = self.source_3d(m, problem)
        self.evolve(s, problem.steps if steps is None else steps, problem.cfl)
        res = self.superpose_3d(s, len(problem.freqs), problem.nz, problem.ny, problem.nx, kmax)
        egb_sync(self.h)
        info = egb_get_solve_info(self.h, s)
        egb_release(self.h, s)
        egb_release(self.h, m)
        return res, info

    def zmarch(self, medium, problem, n_theta, theta_max, cfl=0.5, kmax=8, drt=0):
        """Depth march of a 2-D problem's source on `medium` (both branches); returns the outputs
        (u (n_omega, nz, nx), count, T, A) like superpose."""
        nz, nx = problem.nz, problem.nx
        u = np.zeros((len(problem.freqs), nz, nx), np.complex64)
        cnt = np.zeros((nz, nx), np.uint8)
        T = np.zeros((nz, nx, kmax), np.float64)
        A = np.zeros((nz, nx, kmax), np.float32)
        egb_zmarch(self.h, medium, problem.xs, problem.omegas, problem.beam_width, n_theta, theta_max,
                   cfl, u, cnt, T, A, kmax, drt)
        return SolveResult(u, cnt, T, A)

    def solve_problem(self, problem, steps=None, kmax=8):
        """medium -> source -> evolve -> superpose for one 2-D problem; returns (result, info)."""
        m = self.medium_2d(problem)
        s = self.source_2d(m, problem)
        self.evolve(s, problem.steps if steps is None else steps, problem.cfl)
        res = self.superpose(s, len(problem.freqs), problem.nz, problem.nx, kmax)
        egb_sync(self.h)
        info = egb_get_solve_info(self.h, s)
        egb_release(self.h, s)
        egb_release(self.h, m)
        return res, info
