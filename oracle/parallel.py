"""The paper's multicore method on the host CPU (OpenMP, plain C) -- the timed
CPU baseline.  TEST AND BENCHMARK INFRASTRUCTURE ONLY, like the serial oracle:
only ``tests/`` and the CPU legs of ``bench.py`` may import it.  It shares no
code with the CUDA library.

  bfs       Sec. 2.3.2, Algorithm "Parallel BFS" (level-synchronous, the
            level's edges split among the threads; a compare-and-swap on the
            level array claims each vertex once; parent = the claiming
            frontier vertex)
  kron_csr  the Kronecker graph of Sec. 2.1 built as the CSR of Sec. 2.2 in
            parallel (radix sort of the symmetric keys, Sec. 4.2), with the
            per-vertex counts of tuples starting there (the TEPS numerator of
            Sec. 4.3 sums them over the reached vertices)

Both are pinned to the serial oracle in tests/test_oracle_parallel.py.
"""
import ctypes

import numpy as np

from . import build as _build

_lib = None
_i64p = ctypes.POINTER(ctypes.c_int64)
_i32p = ctypes.POINTER(ctypes.c_int32)


def lib():
    global _lib
    if _lib is None:
        L = ctypes.CDLL(_build.build_parallel())
        L.gbp_max_threads.restype = ctypes.c_int
        L.gbp_max_threads.argtypes = []
        L.gbp_kron_csr.restype = ctypes.c_int
        L.gbp_kron_csr.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_double, ctypes.c_double,
                                   ctypes.c_double, ctypes.c_uint64, ctypes.c_uint64, ctypes.c_int,
                                   _i64p, _i32p, _i64p, _i64p]
        L.gbp_bfs.restype = ctypes.c_int64
        L.gbp_bfs.argtypes = [_i64p, _i32p, ctypes.c_int64, ctypes.c_int64, ctypes.c_int, _i32p, _i32p]
        L.gbp_teps_edges.restype = ctypes.c_int64
        L.gbp_teps_edges.argtypes = [_i64p, _i32p, ctypes.c_int64, ctypes.c_int]
        _lib = L
    return _lib


def _p(a, t):
    return a.ctypes.data_as(t)


def max_threads():
    """Threads the OpenMP runtime offers (the host's cores unless limited)."""
    return int(lib().gbp_max_threads())


def kron_csr(scale, edgefactor, a, b, c, seed_gen, seed_perm, seed_shuf=None, threads=0):
    """(off int64 [n+1], col int32 [nnz], starts int64 [n]) of the Kronecker
    graph; seed_shuf (the tuple order) is accepted and not needed."""
    n = 1 << scale
    m = n * edgefactor
    off = np.empty(n + 1, dtype=np.int64)
    col = np.empty(max(2 * m, 1), dtype=np.int32)
    starts = np.empty(n, dtype=np.int64)
    nnz = ctypes.c_int64(0)
    rc = lib().gbp_kron_csr(scale, edgefactor, a, b, c, seed_gen & (2**64 - 1),
                            seed_perm & (2**64 - 1), int(threads), _p(off, _i64p), _p(col, _i32p),
                            _p(starts, _i64p), ctypes.byref(nnz))
    if rc != 0:
        raise RuntimeError("gbp_kron_csr failed with status %d" % rc)
    return off, col[: nnz.value], starts


def bfs(off, col, root, threads=0):
    """(parent, level, nlevels) of the paper's parallel BFS from `root`."""
    off = np.ascontiguousarray(off, dtype=np.int64)
    col = np.ascontiguousarray(col, dtype=np.int32)
    n = off.size - 1
    parent = np.empty(n, dtype=np.int32)
    level = np.empty(n, dtype=np.int32)
    colp = col if col.size else np.zeros(1, dtype=np.int32)
    nl = lib().gbp_bfs(_p(off, _i64p), _p(colp, _i32p), n, int(root), int(threads),
                       _p(parent, _i32p), _p(level, _i32p))
    if nl < 0:
        raise RuntimeError("gbp_bfs failed with status %d" % nl)
    return parent, level, int(nl)


def teps_edges(starts, level, threads=0):
    """Tuples whose start vertex is reached (Sec. 4.3), from per-vertex counts."""
    starts = np.ascontiguousarray(starts, dtype=np.int64)
    level = np.ascontiguousarray(level, dtype=np.int32)
    return int(lib().gbp_teps_edges(_p(starts, _i64p), _p(level, _i32p), level.size, int(threads)))
