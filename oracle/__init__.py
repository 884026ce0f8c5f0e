"""Graph500 oracle (serial CPU, plain C) -- TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU legs of ``bench.py``
(``cpu_baseline`` and ``--impl reference``) may import this package.  It shares
no code with the CUDA library and imports nothing from it.

Every function follows the paper "Graph500 from OCaml-Multicore Perspective"
(arXiv 2012.13548); the C source names the section each one restates:
  kron_generate / kron_raw / vertex_perm / hash_order   Sec. 2.1 (Kronecker)
  csr_build                                             Sec. 2.2 (kernel 1, CSR)
  bfs                                                   Sec. 2.3.1 (kernel 2)
  validate, teps_edges                                  Sec. 2 outline step 5, Sec. 4.3
  kron_weights, csr_build_weighted                      Sec. 2.1 weight row, Sec. 2.2
  sssp, sssp_tree, sssp_validate                        Sec. 2.4 (kernel 3, Dijkstra)
"""
import ctypes
import numpy as np

from . import build as _build

_lib = None
_i64p = ctypes.POINTER(ctypes.c_int64)
_i32p = ctypes.POINTER(ctypes.c_int32)
_u64p = ctypes.POINTER(ctypes.c_uint64)
_f64p = ctypes.POINTER(ctypes.c_double)


def lib():
    global _lib
    if _lib is None:
        path = _build.build()
        L = ctypes.CDLL(path)
        L.gbo_sm64.restype = ctypes.c_uint64
        L.gbo_sm64.argtypes = [ctypes.c_uint64, ctypes.c_uint64]
        L.gbo_kron_thresholds.restype = None
        L.gbo_kron_thresholds.argtypes = [ctypes.c_double] * 3 + [_u64p]
        L.gbo_kron_raw.restype = ctypes.c_int
        L.gbo_kron_raw.argtypes = [ctypes.c_int, ctypes.c_int64, ctypes.c_double,
                                   ctypes.c_double, ctypes.c_double, ctypes.c_uint64,
                                   _i64p, _i64p]
        L.gbo_hash_order.restype = ctypes.c_int
        L.gbo_hash_order.argtypes = [ctypes.c_int64, ctypes.c_uint64, _i64p]
        L.gbo_vertex_perm.restype = ctypes.c_int
        L.gbo_vertex_perm.argtypes = [ctypes.c_int, ctypes.c_uint64, _i64p]
        L.gbo_kron_generate.restype = ctypes.c_int
        L.gbo_kron_generate.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_double,
                                        ctypes.c_double, ctypes.c_double, ctypes.c_uint64,
                                        ctypes.c_uint64, ctypes.c_uint64, _i64p]
        L.gbo_csr_build.restype = ctypes.c_int
        L.gbo_csr_build.argtypes = [_i64p, ctypes.c_int64, ctypes.c_int, _i64p, _i32p, _i64p]
        L.gbo_bfs.restype = ctypes.c_int64
        L.gbo_bfs.argtypes = [_i64p, _i32p, ctypes.c_int64, ctypes.c_int64, _i32p, _i32p]
        L.gbo_validate.restype = ctypes.c_int
        L.gbo_validate.argtypes = [_i64p, _i32p, ctypes.c_int64, ctypes.c_int64, _i32p, _i32p]
        L.gbo_teps_edges.restype = ctypes.c_int64
        L.gbo_teps_edges.argtypes = [_i64p, ctypes.c_int64, _i32p]
        L.gbo_component_edges.restype = ctypes.c_int64
        L.gbo_component_edges.argtypes = [_i64p, ctypes.c_int64, _i32p]
        L.gbo_kron_weights.restype = ctypes.c_int
        L.gbo_kron_weights.argtypes = [ctypes.c_int64, ctypes.c_uint64, _f64p]
        L.gbo_csr_build_weighted.restype = ctypes.c_int
        L.gbo_csr_build_weighted.argtypes = [_i64p, _f64p, ctypes.c_int64, ctypes.c_int, _i64p,
                                             _i32p, _f64p, _i64p]
        L.gbo_sssp.restype = ctypes.c_int64
        L.gbo_sssp.argtypes = [_i64p, _i32p, _f64p, ctypes.c_int64, ctypes.c_int64, _f64p, _i32p]
        L.gbo_sssp_tree.restype = ctypes.c_int
        L.gbo_sssp_tree.argtypes = [_i64p, _i32p, _f64p, ctypes.c_int64, ctypes.c_int64, _f64p,
                                    _i32p]
        L.gbo_sssp_validate.restype = ctypes.c_int
        L.gbo_sssp_validate.argtypes = [_i64p, _i32p, _f64p, ctypes.c_int64, ctypes.c_int64,
                                        _i32p, _f64p]
        _lib = L
    return _lib


def _p(a, t):
    return a.ctypes.data_as(t)


def _check(rc, what):
    if rc < 0:
        raise RuntimeError("oracle %s failed with status %d" % (what, rc))
    return rc


def sm64(seed: int, i: int) -> int:
    """SplitMix64 output for counter i of a generator seeded with `seed`."""
    return int(lib().gbo_sm64(seed & (2**64 - 1), i & (2**64 - 1)))


def kron_thresholds(a, b, c):
    t = np.zeros(3, dtype=np.uint64)
    lib().gbo_kron_thresholds(a, b, c, _p(t, _u64p))
    return t


def kron_raw(scale, m, a, b, c, seed_gen):
    u = np.empty(m, dtype=np.int64)
    v = np.empty(m, dtype=np.int64)
    _check(lib().gbo_kron_raw(scale, m, a, b, c, seed_gen, _p(u, _i64p), _p(v, _i64p)), "kron_raw")
    return u, v


def hash_order(count, seed):
    o = np.empty(count, dtype=np.int64)
    _check(lib().gbo_hash_order(count, seed, _p(o, _i64p)), "hash_order")
    return o


def vertex_perm(scale, seed_perm):
    pi = np.empty(1 << scale, dtype=np.int64)
    _check(lib().gbo_vertex_perm(scale, seed_perm, _p(pi, _i64p)), "vertex_perm")
    return pi


def kron_generate(scale, edgefactor, a, b, c, seed_gen, seed_perm, seed_shuf):
    """Edge list [2, m] int64 (row 0 start, row 1 end), m = edgefactor * 2^scale."""
    m = (1 << scale) * edgefactor
    e = np.empty((2, m), dtype=np.int64)
    _check(lib().gbo_kron_generate(scale, edgefactor, a, b, c, seed_gen, seed_perm,
                                   seed_shuf, _p(e, _i64p)), "kron_generate")
    return e


def csr_build(edges, scale):
    """(off int64 [n+1], col int32 [nnz]) of the undirected simple graph."""
    edges = np.ascontiguousarray(edges, dtype=np.int64)
    m = edges.shape[1]
    n = 1 << scale
    off = np.empty(n + 1, dtype=np.int64)
    col = np.empty(max(2 * m, 1), dtype=np.int32)
    nnz = ctypes.c_int64(0)
    _check(lib().gbo_csr_build(_p(edges, _i64p), m, scale, _p(off, _i64p), _p(col, _i32p),
                               ctypes.byref(nnz)), "csr_build")
    return off, col[: nnz.value].copy()


def bfs(off, col, root):
    """(parent int32 [n], level int32 [n]); parent is the canonical (min-id) tree."""
    off = np.ascontiguousarray(off, dtype=np.int64)
    col = np.ascontiguousarray(col, dtype=np.int32)
    if col.size == 0:
        col = np.zeros(1, dtype=np.int32)
    n = off.size - 1
    parent = np.empty(n, dtype=np.int32)
    level = np.empty(n, dtype=np.int32)
    _check(lib().gbo_bfs(_p(off, _i64p), _p(col, _i32p), n, root, _p(parent, _i32p),
                         _p(level, _i32p)), "bfs")
    return parent, level


def validate(off, col, root, parent, level):
    """0 if (parent, level) pass the Graph500 rules, else the failed rule's number."""
    off = np.ascontiguousarray(off, dtype=np.int64)
    col = np.ascontiguousarray(col, dtype=np.int32)
    if col.size == 0:
        col = np.zeros(1, dtype=np.int32)
    parent = np.ascontiguousarray(parent, dtype=np.int32)
    level = np.ascontiguousarray(level, dtype=np.int32)
    n = off.size - 1
    return int(lib().gbo_validate(_p(off, _i64p), _p(col, _i32p), n, root,
                                  _p(parent, _i32p), _p(level, _i32p)))


def teps_edges(edges, level):
    edges = np.ascontiguousarray(edges, dtype=np.int64)
    level = np.ascontiguousarray(level, dtype=np.int32)
    return int(lib().gbo_teps_edges(_p(edges, _i64p), edges.shape[1], _p(level, _i32p)))


def component_edges(off, level):
    off = np.ascontiguousarray(off, dtype=np.int64)
    level = np.ascontiguousarray(level, dtype=np.int32)
    return int(lib().gbo_component_edges(_p(off, _i64p), off.size - 1, _p(level, _i32p)))


def kron_weights(m, seed_w):
    """The weight row: float64 [m], each a multiple of 2^-24 in (0, 1]."""
    w = np.empty(max(m, 1), dtype=np.float64)
    _check(lib().gbo_kron_weights(m, seed_w & (2**64 - 1), _p(w, _f64p)), "kron_weights")
    return w[:m].copy()


def csr_build_weighted(edges, w, scale):
    """(off, col, wgt float64 [nnz]): csr_build's graph, each entry with the least
    weight among the tuples joining its pair."""
    edges = np.ascontiguousarray(edges, dtype=np.int64)
    w = np.ascontiguousarray(w, dtype=np.float64)
    m = edges.shape[1]
    if w.shape != (m,):
        raise ValueError("one weight per tuple")
    n = 1 << scale
    off = np.empty(n + 1, dtype=np.int64)
    col = np.empty(max(2 * m, 1), dtype=np.int32)
    wgt = np.empty(max(2 * m, 1), dtype=np.float64)
    nnz = ctypes.c_int64(0)
    _check(lib().gbo_csr_build_weighted(_p(edges, _i64p), _p(w if m else np.zeros(1), _f64p), m,
                                        scale, _p(off, _i64p), _p(col, _i32p), _p(wgt, _f64p),
                                        ctypes.byref(nnz)), "csr_build_weighted")
    return off, col[: nnz.value].copy(), wgt[: nnz.value].copy()


def _csr_args(off, col, wgt):
    off = np.ascontiguousarray(off, dtype=np.int64)
    col = np.ascontiguousarray(col, dtype=np.int32)
    wgt = np.ascontiguousarray(wgt, dtype=np.float64)
    if col.size == 0:
        col = np.zeros(1, dtype=np.int32)
        wgt = np.zeros(1, dtype=np.float64)
    return off, col, wgt


def sssp(off, col, wgt, root):
    """(dist float64 [n], prev int32 [n]) of Algorithm "Sequential SSSP"."""
    off, col, wgt = _csr_args(off, col, wgt)
    n = off.size - 1
    dist = np.empty(n, dtype=np.float64)
    prev = np.empty(n, dtype=np.int32)
    _check(lib().gbo_sssp(_p(off, _i64p), _p(col, _i32p), _p(wgt, _f64p), n, root,
                          _p(dist, _f64p), _p(prev, _i32p)), "sssp")
    return dist, prev


def sssp_tree(off, col, wgt, root, dist):
    """The canonical tree of `dist`: the smallest-id tight neighbour per vertex."""
    off, col, wgt = _csr_args(off, col, wgt)
    n = off.size - 1
    dist = np.ascontiguousarray(dist, dtype=np.float64)
    parent = np.empty(n, dtype=np.int32)
    _check(lib().gbo_sssp_tree(_p(off, _i64p), _p(col, _i32p), _p(wgt, _f64p), n, root,
                               _p(dist, _f64p), _p(parent, _i32p)), "sssp_tree")
    return parent


def sssp_validate(off, col, wgt, root, parent, dist):
    """0 if (parent, dist) pass the SSSP rules, else the failed rule's number."""
    off, col, wgt = _csr_args(off, col, wgt)
    n = off.size - 1
    parent = np.ascontiguousarray(parent, dtype=np.int32)
    dist = np.ascontiguousarray(dist, dtype=np.float64)
    return int(lib().gbo_sssp_validate(_p(off, _i64p), _p(col, _i32p), _p(wgt, _f64p), n, root,
                                       _p(parent, _i32p), _p(dist, _f64p)))
