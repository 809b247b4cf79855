"""Build libegb.so (the CUDA library behind include/egb.h) in-tree for sm_103a.

``python -m paper_2006_11945_gb300.build`` compiles every ``csrc/*.cu`` translation unit with nvcc
(in parallel, one -gencode for compute_103a/sm_103a) and links ``_lib/libegb.so``.
"""
from __future__ import annotations

import concurrent.futures as cf
import glob
import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, 'csrc')
OUT_DIR = os.path.join(HERE, '_lib')
LIB = os.path.join(OUT_DIR, 'libegb.so')
ARCH = ['-gencode', 'arch=compute_103a,code=sm_103a']
FLAGS = ['-O3', '-lineinfo', '-std=c++17', '-Xcompiler', '-fPIC', '-Xcompiler', '-O2',
         '--expt-relaxed-constexpr']


def _nvcc():
    for cand in (os.environ.get('NVCC'), shutil.which('nvcc'), '/usr/local/cuda/bin/nvcc'):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError('nvcc not found: the CUDA library cannot be built')


def _stale(sources, headers):
    if not os.path.exists(LIB):
        return True
    t = os.path.getmtime(LIB)
    return any(os.path.getmtime(f) > t for f in sources + headers + [__file__])


def build(force=False, verbose=False, extra_flags=()):
    sources = sorted(glob.glob(os.path.join(CSRC, '*.cu')))
    headers = sorted(glob.glob(os.path.join(CSRC, '*.cuh'))) + [
        os.path.join(HERE, '..', 'include', 'egb.h')]
    if not force and not _stale(sources, headers):
        return LIB
    os.makedirs(OUT_DIR, exist_ok=True)
    nvcc = _nvcc()
    objs = [os.path.join(OUT_DIR, os.path.basename(s)[:-3] + '.o') for s in sources]

    def compile_one(src_obj):
        src, obj = src_obj
        cmd = [nvcc, *ARCH, *FLAGS, *extra_flags, '-c', src, '-o', obj]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f'nvcc failed for {os.path.basename(src)}:\n{r.stderr}')
        if verbose and r.stderr:
            sys.stderr.write(r.stderr)
        return obj

    with cf.ThreadPoolExecutor(max_workers=min(8, len(sources))) as ex:
        list(ex.map(compile_one, zip(sources, objs)))
    tmp = LIB + f'.{os.getpid()}.tmp'
    r = subprocess.run([nvcc, *ARCH, '-shared', '-o', tmp, *objs], capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f'link failed:\n{r.stderr}')
    os.replace(tmp, LIB)
    return LIB


if __name__ == '__main__':
    print(build(force=True, verbose=True))
