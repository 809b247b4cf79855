"""Compile the oracle's C stepping loop (test infrastructure only).

``python -m oracle.build`` or ``oracle.build.library()`` builds ``oracle/_build/liboracle.so`` from
the 2-D and 3-D loops with gcc (-O3, OpenMP, no floating-point contraction, so IEEE arithmetic in
the order written) on the machine it runs on.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRCS = [os.path.join(_HERE, 'liouville_c.c'), os.path.join(_HERE, 'liouville3d_c.c')]
_OUT = os.path.join(_HERE, '_build', 'liboracle.so')
_lib = None


def build(force=False):
    os.makedirs(os.path.dirname(_OUT), exist_ok=True)
    if force or not os.path.exists(_OUT) or os.path.getmtime(_OUT) < max(map(os.path.getmtime, _SRCS)):
        tmp = _OUT + f'.{os.getpid()}.tmp'
        subprocess.check_call(['gcc', '-O3', '-fopenmp', '-ffp-contract=off', '-fPIC', '-shared',
                               '-o', tmp] + _SRCS + ['-lm'])
        os.replace(tmp, _OUT)
    return _OUT


def library():
    global _lib
    if _lib is None:
        _lib = ctypes.CDLL(build())
        d, i, p = ctypes.c_double, ctypes.c_int, ctypes.c_void_p
        _lib.oracle_rk3_steps.argtypes = [i, i, i, d, d, d, p, p, p, p, p, d, i, p, p, p, p]
        _lib.oracle_rk3_steps.restype = i
        _lib.oracle3d_rk3_steps.argtypes = [i, i, i, i, i, d, d, d, d, d, p, p, p, p, p, p, p, d, i, p]
        _lib.oracle3d_rk3_steps.restype = i
    return _lib


if __name__ == '__main__':
    print(build(force=True))
