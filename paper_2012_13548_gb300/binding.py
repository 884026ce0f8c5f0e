"""Python binding of the C ABI in ``include/gb300bfs.h``.

Argument marshalling only: every function checks its tensors, passes their
device pointers and the current CUDA stream to the library and raises
``GbError`` on a non-zero status.  There is no fallback: if the CUDA library
has not been built, importing a function raises.
"""
import ctypes
import os

import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
# GB_CHECKED=1 selects the index-checking debug build (build_ext --checked).
LIB_PATH = os.path.join(_HERE, "_build_checked" if os.environ.get("GB_CHECKED") == "1" else "_build",
                        "libgb300bfs.so")

GB_OK, GB_ERR_INVALID, GB_ERR_NOMEM, GB_ERR_CUDA = 0, -1, -2, -3
GB_ERR_TIMEOUT, GB_ERR_RANGE, GB_ERR_BUSY, GB_ERR_UNIMPLEMENTED = -4, -5, -6, -7
_NAMES = {0: "GB_OK", -1: "GB_ERR_INVALID", -2: "GB_ERR_NOMEM", -3: "GB_ERR_CUDA",
          -4: "GB_ERR_TIMEOUT", -5: "GB_ERR_RANGE", -6: "GB_ERR_BUSY", -7: "GB_ERR_UNIMPLEMENTED"}


class GbError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__("%s: %s" % (_NAMES.get(status, status), msg))
        self.status = status


class gb_bfs_options(ctypes.Structure):
    _fields_ = [("canonical_parents", ctypes.c_int), ("alpha", ctypes.c_double),
                ("beta", ctypes.c_double), ("big_degree", ctypes.c_int),
                ("ms_alpha", ctypes.c_double), ("ms_beta", ctypes.c_double),
                ("timeout_ms", ctypes.c_double), ("blocks_per_sm", ctypes.c_int)]


GB_STAT_LEVELS = 32


class gb_bfs_stats(ctypes.Structure):
    _fields_ = [(f, ctypes.c_int64) for f in
                ("nlevels", "edges_examined", "vertices_touched", "reached", "td_levels",
                 "bu_levels")] + [("level_ns", ctypes.c_int64 * GB_STAT_LEVELS),
                                  ("level_frontier", ctypes.c_int64 * GB_STAT_LEVELS),
                                  ("level_dir", ctypes.c_int32 * GB_STAT_LEVELS)]


class gb_validation(ctypes.Structure):
    _fields_ = [("code", ctypes.c_int32), ("max_level", ctypes.c_int32), ("where", ctypes.c_int64),
                ("reached", ctypes.c_int64), ("component_edges", ctypes.c_int64),
                ("teps_edges", ctypes.c_int64)]


class gb_sssp_stats(ctypes.Structure):
    _fields_ = [(f, ctypes.c_int64) for f in
                ("rounds", "buckets", "processed", "scanned", "won", "reached")] + \
        [("delta", ctypes.c_double), ("phase_ns", ctypes.c_int64 * 4)]


class gb_server_options(ctypes.Structure):
    _fields_ = [("single_source_min_vertices", ctypes.c_int64), ("slots_per_graph", ctypes.c_int),
                ("full_grid", ctypes.c_int), ("verbose", ctypes.c_int)]


class gb_server_stats(ctypes.Structure):
    _fields_ = [(f, ctypes.c_int64) for f in ("budget_bytes", "fixed_bytes", "used_bytes", "queued",
                                              "running", "done", "released", "cancelled")]


class gb_sssp_validation(ctypes.Structure):
    _fields_ = [("code", ctypes.c_int32), ("pad", ctypes.c_int32), ("where", ctypes.c_int64),
                ("reached", ctypes.c_int64), ("component_edges", ctypes.c_int64),
                ("teps_edges", ctypes.c_int64), ("max_dist", ctypes.c_double)]


_lib = None
_vp = ctypes.c_void_p
_i64 = ctypes.c_int64


def lib():
    """The loaded CUDA library (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(
                "CUDA library %s is missing: run __graft_entry__.build() (nvcc, sm_103a) first"
                % LIB_PATH)
        L = ctypes.CDLL(LIB_PATH)
        sigs = {
            "gb_last_error": (ctypes.c_char_p, []),
            "gb_abi_version": (ctypes.c_int, []),
            "gb_kernel_launches": (ctypes.c_uint64, []),
            "gb_set_sort_portion": (ctypes.c_int, [_i64]),
            "gb_debug_fail_allocations": (ctypes.c_int, [_i64, _i64]),
            "gb_debug_live_allocations": (_i64, []),
            "gb_sort_portion": (_i64, []),
            "gb_device_status": (ctypes.c_int, [_vp]),
            "kron_generate": (ctypes.c_int, [ctypes.c_int, ctypes.c_int, ctypes.c_double,
                                             ctypes.c_double, ctypes.c_double, ctypes.c_uint64,
                                             ctypes.c_uint64, ctypes.c_uint64, _vp, _vp]),
            "graph_build_csr": (ctypes.c_int, [_vp, _i64, ctypes.c_int, ctypes.POINTER(_vp), _vp]),
            "graph_from_csr": (ctypes.c_int, [_vp, _vp, _i64, _i64, ctypes.POINTER(_vp), _vp]),
            "graph_build_csr_counting": (ctypes.c_int, [_vp, _i64, ctypes.c_int, ctypes.POINTER(_vp),
                                                        _vp]),
            "graph_generate_csr": (ctypes.c_int, [ctypes.c_int, ctypes.c_int, ctypes.c_double,
                                                  ctypes.c_double, ctypes.c_double, ctypes.c_uint64,
                                                  ctypes.c_uint64, ctypes.POINTER(_vp), _vp]),
            "graph_free": (ctypes.c_int, [_vp]),
            "graph_info": (ctypes.c_int, [_vp, ctypes.POINTER(_i64), ctypes.POINTER(_i64)]),
            "graph_csr_view": (ctypes.c_int, [_vp, ctypes.POINTER(_vp), ctypes.POINTER(_vp)]),
            "graph_prepare_batched": (ctypes.c_int, [_vp, _vp]),
            "bfs_get_options": (ctypes.c_int, [ctypes.POINTER(gb_bfs_options)]),
            "bfs_set_options": (ctypes.c_int, [ctypes.POINTER(gb_bfs_options)]),
            "bfs": (ctypes.c_int, [_vp, _i64, _vp, _vp, _vp]),
            "bfs_batch": (ctypes.c_int, [_vp, ctypes.POINTER(_i64), ctypes.c_int, _vp, _vp, _vp]),
            "bfs_multi_graph": (ctypes.c_int, [ctypes.POINTER(_vp), ctypes.c_int,
                                               ctypes.POINTER(_i64), ctypes.c_int,
                                               ctypes.POINTER(_vp), ctypes.POINTER(_vp), _vp]),
            "bfs_last_stats": (ctypes.c_int, [ctypes.POINTER(gb_bfs_stats)]),
            "bfs_noalloc": (ctypes.c_int, [_vp, _vp, _i64, _i64, _i64, _vp, _vp, _vp]),
            "bfs_validate": (ctypes.c_int, [_vp, _i64, _vp, _vp, _vp, _i64,
                                            ctypes.POINTER(gb_validation), _vp]),
            "kron_weights": (ctypes.c_int, [_i64, ctypes.c_uint64, _vp, _vp]),
            "graph_build_csr_weighted": (ctypes.c_int, [_vp, _vp, _i64, ctypes.c_int,
                                                        ctypes.POINTER(_vp), _vp]),
            "graph_weights_view": (ctypes.c_int, [_vp, ctypes.POINTER(_vp)]),
            "sssp": (ctypes.c_int, [_vp, _i64, ctypes.c_double, _vp, _vp, _vp]),
            "sssp_last_stats": (ctypes.c_int, [ctypes.POINTER(gb_sssp_stats)]),
            "sssp_validate": (ctypes.c_int, [_vp, _i64, _vp, _vp, _vp, _i64,
                                             ctypes.POINTER(gb_sssp_validation), _vp]),
            "server_create": (ctypes.c_int, [ctypes.POINTER(_vp), ctypes.c_int, ctypes.c_size_t,
                                             ctypes.POINTER(_vp)]),
            "server_default_options": (ctypes.c_int, [ctypes.POINTER(gb_server_options)]),
            "server_create_with_options": (ctypes.c_int, [ctypes.POINTER(_vp), ctypes.c_int,
                                                          ctypes.c_size_t,
                                                          ctypes.POINTER(gb_server_options),
                                                          ctypes.POINTER(_vp)]),
            "server_cancel": (ctypes.c_int, [_vp, _i64]),
            "server_stats": (ctypes.c_int, [_vp, ctypes.POINTER(gb_server_stats)]),
            "server_submit": (ctypes.c_int, [_vp, ctypes.c_int, _i64, ctypes.POINTER(_i64)]),
            "server_poll": (ctypes.c_int, [_vp, _i64, ctypes.POINTER(_vp), ctypes.POINTER(_vp)]),
            "server_release": (ctypes.c_int, [_vp, _i64]),
            "server_run_trace": (ctypes.c_int, [_vp, _i64, _vp, _vp, _vp, ctypes.c_int, _vp]),
            "server_destroy": (ctypes.c_int, [_vp]),
        }
        for name, (res, args) in sigs.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


def exported_symbols():
    """Names of the C-ABI functions this binding wraps."""
    return ["gb_last_error", "gb_abi_version", "gb_kernel_launches", "gb_set_sort_portion",
            "gb_sort_portion", "gb_debug_fail_allocations", "gb_debug_live_allocations",
            "gb_device_status", "kron_generate",
            "graph_build_csr", "graph_build_csr_counting", "graph_from_csr", "graph_generate_csr",
            "graph_free", "graph_info", "graph_csr_view", "graph_prepare_batched",
            "bfs_get_options", "bfs_set_options", "bfs", "bfs_batch", "bfs_multi_graph",
            "bfs_last_stats", "bfs_noalloc", "bfs_validate", "kron_weights", "graph_build_csr_weighted",
            "graph_weights_view", "sssp", "sssp_last_stats", "sssp_validate", "server_create",
            "server_default_options", "server_create_with_options", "server_cancel", "server_stats",
            "server_submit", "server_poll", "server_release", "server_run_trace", "server_destroy"]


def _check(rc):
    if rc != GB_OK:
        raise GbError(rc, lib().gb_last_error().decode(errors="replace"))


def _stream(stream=None):
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


def _dev(t, dtype, name):
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError("%s must be a CUDA tensor" % name)
    if t.dtype != dtype:
        raise TypeError("%s must be %s, got %s" % (name, dtype, t.dtype))
    if not t.is_contiguous():
        raise ValueError("%s must be contiguous" % name)
    return ctypes.c_void_p(t.data_ptr())


class _DevArray:
    """A borrowed device array exposed through __cuda_array_interface__."""

    def __init__(self, ptr, shape, typestr, owner):
        self.__cuda_array_interface__ = {"shape": shape, "typestr": typestr,
                                         "data": (ptr, False), "version": 3, "strides": None}
        self._owner = owner


class Graph:
    """A library-owned device CSR graph (Sec. 2.2)."""

    def __init__(self, handle):
        self._h = ctypes.c_void_p(handle)
        n, nnz = _i64(), _i64()
        _check(lib().graph_info(self._h, ctypes.byref(n), ctypes.byref(nnz)))
        self.n, self.nnz = n.value, nnz.value

    @property
    def handle(self):
        if not self._h:
            raise ValueError("graph has been freed")
        return self._h

    def csr(self):
        """Borrowed (off int64 [n+1], col int32 [nnz]) CUDA tensors; valid until free()."""
        off, col = _vp(), _vp()
        _check(lib().graph_csr_view(self.handle, ctypes.byref(off), ctypes.byref(col)))
        dev = torch.cuda.current_device()
        o = torch.as_tensor(_DevArray(off.value, (self.n + 1,), "<i8", self), device="cuda:%d" % dev)
        c = torch.as_tensor(_DevArray(col.value, (self.nnz,), "<i4", self), device="cuda:%d" % dev)
        return o, c

    def weights(self):
        """Borrowed uint32 [nnz] weights of a weighted graph, in units of 2^-24
        (torch has no uint32 arithmetic on every version: returned as int32
        bits, all values below 2^31)."""
        w = _vp()
        _check(lib().graph_weights_view(self.handle, ctypes.byref(w)))
        dev = torch.cuda.current_device()
        return torch.as_tensor(_DevArray(w.value, (self.nnz,), "<i4", self), device="cuda:%d" % dev)

    def prepare_batched(self, stream=None):
        """Build the degree-ordered copy bfs_batch searches (graph_prepare_batched)."""
        _check(lib().graph_prepare_batched(self.handle, _stream(stream)))
        return self

    def free(self):
        if self._h:
            _check(lib().graph_free(self._h))
            self._h = ctypes.c_void_p(None)

    def __del__(self):
        try:
            if self._h and _lib is not None:
                _lib.graph_free(self._h)
        except Exception:
            pass


def gb_kernel_launches():
    """Kernels this library has launched so far in this process."""
    return int(lib().gb_kernel_launches())


def sort_portion(keys=None):
    """Keys per portion of the library's radix sort: returns the current value,
    after setting it to `keys` if given (0 restores the default 2^28)."""
    if keys is not None:
        _check(lib().gb_set_sort_portion(int(keys)))
    return int(lib().gb_sort_portion())


def debug_fail_allocations(skip=0, count=0):
    """Make the library's next `count` device allocations, after `skip` more,
    fail as if the device were out of memory (count 0 disarms)."""
    _check(lib().gb_debug_fail_allocations(int(skip), int(count)))


def debug_live_allocations():
    """Device blocks the library holds now (allocated and not yet freed)."""
    return int(lib().gb_debug_live_allocations())


def gb_device_status(stream=None):
    """Synchronise the stream and raise if a kernel recorded an error."""
    _check(lib().gb_device_status(_stream(stream)))


def kron_generate(scale, edgefactor, a, b, c, seed_gen, seed_perm, seed_shuf, edges=None,
                  stream=None):
    """Kronecker edge list (Sec. 2.1) as an int64 [2, m] CUDA tensor."""
    m = (1 << scale) * edgefactor
    if edges is None:
        edges = torch.empty((2, m), dtype=torch.int64, device="cuda")
    if tuple(edges.shape) != (2, m):
        raise ValueError("edges must have shape (2, %d)" % m)
    _check(lib().kron_generate(scale, edgefactor, a, b, c, seed_gen & (2**64 - 1),
                               seed_perm & (2**64 - 1), seed_shuf & (2**64 - 1),
                               _dev(edges, torch.int64, "edges"), _stream(stream)))
    return edges


def graph_build_csr(edges, scale, stream=None):
    """Kernel 1 (Sec. 2.2): the undirected CSR of an int64 [2, m] edge list."""
    if edges.dim() != 2 or edges.shape[0] != 2:
        raise ValueError("edges must have shape (2, m)")
    h = _vp()
    _check(lib().graph_build_csr(_dev(edges, torch.int64, "edges"), edges.shape[1], scale,
                                 ctypes.byref(h), _stream(stream)))
    return Graph(h.value)


def graph_build_csr_counting(edges, scale, stream=None):
    """Kernel 1 by counting sort (rows scattered, then each sorted): the same
    Graph as graph_build_csr(edges, scale), for comparison."""
    if edges.dim() != 2 or edges.shape[0] != 2:
        raise ValueError("edges must have shape (2, m)")
    h = _vp()
    _check(lib().graph_build_csr_counting(_dev(edges, torch.int64, "edges"), edges.shape[1], scale,
                                          ctypes.byref(h), _stream(stream)))
    return Graph(h.value)


def graph_generate_csr(scale, edgefactor, a, b, c, seed_gen, seed_perm, seed_shuf=None,
                       stream=None):
    """Generator and kernel 1 fused: the Graph that graph_build_csr(kron_generate(...))
    gives for the same parameters, built without the edge list (seed_shuf, which
    only orders the tuples, is accepted and ignored)."""
    h = ctypes.c_void_p()
    _check(lib().graph_generate_csr(int(scale), int(edgefactor), float(a), float(b), float(c),
                                    int(seed_gen), int(seed_perm), ctypes.byref(h), _stream(stream)))
    return Graph(h.value)


def graph_from_csr(off, col, stream=None):
    """Wrap a caller CSR (copied into library memory)."""
    h = _vp()
    _check(lib().graph_from_csr(_dev(off, torch.int64, "off"),
                                _dev(col, torch.int32, "col") if col.numel() else ctypes.c_void_p(None),
                                off.numel() - 1, col.numel(), ctypes.byref(h), _stream(stream)))
    return Graph(h.value)


def bfs_get_options():
    o = gb_bfs_options()
    _check(lib().bfs_get_options(ctypes.byref(o)))
    return {f: getattr(o, f) for f, _ in gb_bfs_options._fields_}


def bfs_set_options(**kw):
    """Update any of canonical_parents, alpha, beta, big_degree, ms_alpha, ms_beta,
    timeout_ms, blocks_per_sm."""
    cur = bfs_get_options()
    unknown = set(kw) - set(cur)
    if unknown:
        raise KeyError("unknown options %s" % sorted(unknown))
    cur.update(kw)
    o = gb_bfs_options(**cur)
    _check(lib().bfs_set_options(ctypes.byref(o)))


def bfs(graph, root, parent=None, level=None, stream=None):
    """Kernel 2 (Sec. 2.3): (parent, level) int32 [n] CUDA tensors from `root`."""
    if parent is None:
        parent = torch.empty(graph.n, dtype=torch.int32, device="cuda")
    if level is None:
        level = torch.empty(graph.n, dtype=torch.int32, device="cuda")
    if parent.numel() != graph.n or level.numel() != graph.n:
        raise ValueError("outputs must have n = %d entries" % graph.n)
    _check(lib().bfs(graph.handle, int(root), _dev(parent, torch.int32, "parent"),
                     _dev(level, torch.int32, "level"), _stream(stream)))
    return parent, level


def bfs_batch(graph, roots, parents=None, levels=None, stream=None):
    """Multi-source BFS: (parents, levels) int32 [k, n], row i for roots[i]."""
    roots = [int(r) for r in roots]
    k = len(roots)
    if parents is None:
        parents = torch.empty((k, graph.n), dtype=torch.int32, device="cuda")
    if levels is None:
        levels = torch.empty((k, graph.n), dtype=torch.int32, device="cuda")
    if parents.numel() != k * graph.n or levels.numel() != k * graph.n:
        raise ValueError("outputs must have k*n entries")
    arr = (_i64 * max(k, 1))(*roots)
    _check(lib().bfs_batch(graph.handle, arr, k, _dev(parents, torch.int32, "parents"),
                           _dev(levels, torch.int32, "levels"), _stream(stream)))
    return parents, levels


def bfs_multi_graph(graphs, roots, parents=None, levels=None, stream=None):
    """BFS of r roots on each of ng graphs in one launch.  roots: [ng][r] ints.
    Returns lists of (parents [r, n_i], levels [r, n_i])."""
    ng = len(graphs)
    r = len(roots[0]) if ng else 0
    if any(len(x) != r for x in roots):
        raise ValueError("every graph needs the same number of roots")
    if parents is None:
        parents = [torch.empty((r, g.n), dtype=torch.int32, device="cuda") for g in graphs]
    if levels is None:
        levels = [torch.empty((r, g.n), dtype=torch.int32, device="cuda") for g in graphs]
    gh = (_vp * ng)(*[g.handle.value for g in graphs])
    rr = (_i64 * (ng * r))(*[int(x) for row in roots for x in row])
    pp = (_vp * ng)(*[_dev(p, torch.int32, "parents").value for p in parents])
    ll = (_vp * ng)(*[_dev(x, torch.int32, "levels").value for x in levels])
    _check(lib().bfs_multi_graph(gh, ng, rr, r, pp, ll, _stream(stream)))
    return parents, levels


def bfs_noalloc(off, col, root, parent, level, stream=None):
    """Allocation-free single-source BFS into caller tensors parent/level (int32 [n]).

    For callers that must not allocate device memory: the library keeps this
    call's temporaries in a fixed built-in device array, so graphs are limited
    to 2^20 vertices.  off/col are a CSR in CUDA tensors (int64 [n+1], int32
    [nnz]); the call synchronises the stream.  Nothing here allocates."""
    n = off.numel() - 1
    if parent.numel() != n or level.numel() != n:
        raise ValueError("outputs must have n = %d entries" % n)
    _check(lib().bfs_noalloc(_dev(off, torch.int64, "off"),
                             _dev(col, torch.int32, "col") if col.numel() else ctypes.c_void_p(None),
                             n, col.numel(), int(root), _dev(parent, torch.int32, "parent"),
                             _dev(level, torch.int32, "level"), _stream(stream)))
    return parent, level


def bfs_validate(graph, root, parent, level, edges=None, stream=None):
    """Graph500 validation of one search on the device (synchronises the
    stream).  parent/level: int32 [n] CUDA tensors; edges: the int64 [2, m]
    input tuples for the TEPS numerator, or None.  Returns a dict with code
    (0 = valid, else the first failing rule 1..7), where, reached,
    component_edges, teps_edges (-1 without edges) and max_level."""
    if parent.numel() != graph.n or level.numel() != graph.n:
        raise ValueError("parent/level must have n = %d entries" % graph.n)
    if edges is not None:
        if edges.dim() != 2 or edges.shape[0] != 2:
            raise ValueError("edges must be a [2, m] tensor")
        ep, m = _dev(edges, torch.int64, "edges"), int(edges.shape[1])
    else:
        ep, m = ctypes.c_void_p(None), 0
    out = gb_validation()
    _check(lib().bfs_validate(graph.handle, int(root), _dev(parent, torch.int32, "parent"),
                              _dev(level, torch.int32, "level"), ep, m, ctypes.byref(out),
                              _stream(stream)))
    return {f: getattr(out, f) for f, _ in gb_validation._fields_}


def bfs_last_stats():
    """Counters of this thread's last BFS call (synchronises its stream)."""
    s = gb_bfs_stats()
    _check(lib().bfs_last_stats(ctypes.byref(s)))
    out = {f: getattr(s, f) for f, _ in gb_bfs_stats._fields_[:6]}
    k = min(out["nlevels"], GB_STAT_LEVELS)
    out["level_ns"] = list(s.level_ns)[:k]
    out["level_frontier"] = list(s.level_frontier)[:k]
    out["level_dir"] = ["td" if d == 1 else "bu" if d == 2 else "-" for d in list(s.level_dir)[:k]]
    return out


class Server:
    """Continuous-batching BFS server over resident graphs (C ABI server_*).

    Queries are admitted as slots free up while their output buffers fit in
    `mem_budget` bytes (which also holds the server's own search state):
    concurrent single-source searches on large graphs, bit-slots of one
    multi-source search (admitted at level boundaries) on small ones."""

    def __init__(self, graphs, mem_budget, **options):
        """options: any of single_source_min_vertices, slots_per_graph,
        full_grid, verbose (gb_server_options); the rest keep their defaults."""
        self.graphs = list(graphs)
        arr = (_vp * len(self.graphs))(*[g.handle.value for g in self.graphs])
        o = gb_server_options()
        _check(lib().server_default_options(ctypes.byref(o)))
        names = {f for f, _ in gb_server_options._fields_}
        if set(options) - names:
            raise KeyError("unknown server options %s" % sorted(set(options) - names))
        for k, v in options.items():
            setattr(o, k, int(v))
        h = _vp()
        _check(lib().server_create_with_options(arr, len(self.graphs), int(mem_budget), ctypes.byref(o),
                                                ctypes.byref(h)))
        self._h = h

    def cancel(self, ticket):
        _check(lib().server_cancel(self._h, int(ticket)))

    def stats(self):
        """Budget, fixed and used bytes and the query counts (server_stats)."""
        st = gb_server_stats()
        _check(lib().server_stats(self._h, ctypes.byref(st)))
        return {f: getattr(st, f) for f, _ in gb_server_stats._fields_}

    def submit(self, graph_id, root):
        t = _i64()
        _check(lib().server_submit(self._h, int(graph_id), int(root), ctypes.byref(t)))
        return t.value

    def poll(self, ticket):
        """(parent, level) borrowed int32 CUDA tensors once done, else None."""
        p, l = _vp(), _vp()
        rc = lib().server_poll(self._h, int(ticket), ctypes.byref(p), ctypes.byref(l))
        if rc == GB_ERR_BUSY:
            return None
        _check(rc)
        return p.value, l.value

    def result(self, ticket, graph_id, timeout_s=60.0):
        """Wait for a query and return copies of its (parent, level) tensors."""
        import time
        t0 = time.time()
        while True:
            r = self.poll(ticket)
            if r is not None:
                break
            if time.time() - t0 > timeout_s:
                raise TimeoutError("query %d not finished" % ticket)
            time.sleep(1e-4)
        n = self.graphs[graph_id].n
        dev = "cuda:%d" % torch.cuda.current_device()
        par = torch.as_tensor(_DevArray(r[0], (n,), "<i4", self), device=dev).clone()
        lev = torch.as_tensor(_DevArray(r[1], (n,), "<i4", self), device=dev).clone()
        return par, lev

    def release(self, ticket):
        _check(lib().server_release(self._h, int(ticket)))

    def run_trace(self, t_arrival_s, graph_id, roots, keep_results=False):
        """Replay an open-loop trace; returns arrival-to-done latencies in ms."""
        import numpy as np
        t = np.ascontiguousarray(t_arrival_s, dtype=np.float64)
        gid = np.ascontiguousarray(graph_id, dtype=np.int32)
        rr = np.ascontiguousarray(roots, dtype=np.int64)
        lat = np.zeros(t.size, dtype=np.float64)
        _check(lib().server_run_trace(self._h, t.size, ctypes.c_void_p(t.ctypes.data),
                                      ctypes.c_void_p(gid.ctypes.data), ctypes.c_void_p(rr.ctypes.data),
                                      1 if keep_results else 0, ctypes.c_void_p(lat.ctypes.data)))
        return lat

    def close(self):
        if self._h:
            _check(lib().server_destroy(self._h))
            self._h = _vp()

    def __del__(self):
        try:
            if self._h and _lib is not None:
                _lib.server_destroy(self._h)
        except Exception:
            pass



def kron_weights(m, seed_weight, w=None, stream=None):
    """The weight row of the tuple matrix (Sec. 2.1): float32 [m] CUDA tensor,
    multiples of 2^-24 in (0, 1]."""
    if w is None:
        w = torch.empty(max(int(m), 1), dtype=torch.float32, device="cuda")[: int(m)]
    if w.numel() != m:
        raise ValueError("w must have m = %d entries" % m)
    _check(lib().kron_weights(int(m), int(seed_weight) & (2**64 - 1),
                              _dev(w, torch.float32, "w") if m else ctypes.c_void_p(None),
                              _stream(stream)))
    return w


def graph_build_csr_weighted(edges, w, scale, stream=None):
    """Kernel 1 with weights: graph_build_csr's graph, each entry with the least
    weight (float32 [m], each in (0, 1]) among the tuples joining its pair."""
    if edges.dim() != 2 or edges.shape[0] != 2:
        raise ValueError("edges must have shape (2, m)")
    m = int(edges.shape[1])
    if w.numel() != m:
        raise ValueError("w must have one weight per tuple")
    h = _vp()
    _check(lib().graph_build_csr_weighted(
        _dev(edges, torch.int64, "edges") if m else ctypes.c_void_p(None),
        _dev(w, torch.float32, "w") if m else ctypes.c_void_p(None), m, int(scale),
        ctypes.byref(h), _stream(stream)))
    return Graph(h.value)


def sssp(graph, root, delta=0.0, dist=None, parent=None, stream=None):
    """Kernel 3 (Sec. 2.4): (dist float64 [n], parent int32 [n]) CUDA tensors of
    the shortest paths from `root`; delta = bucket width (<= 0: the default)."""
    if dist is None:
        dist = torch.empty(graph.n, dtype=torch.float64, device="cuda")
    if parent is None:
        parent = torch.empty(graph.n, dtype=torch.int32, device="cuda")
    if dist.numel() != graph.n or parent.numel() != graph.n:
        raise ValueError("outputs must have n = %d entries" % graph.n)
    _check(lib().sssp(graph.handle, int(root), float(delta), _dev(dist, torch.float64, "dist"),
                      _dev(parent, torch.int32, "parent"), _stream(stream)))
    return dist, parent


def sssp_last_stats():
    """Counters of this thread's last sssp call (synchronises its stream)."""
    s = gb_sssp_stats()
    _check(lib().sssp_last_stats(ctypes.byref(s)))
    out = {f: getattr(s, f) for f, _ in gb_sssp_stats._fields_[:7]}
    out["phase_ns"] = list(s.phase_ns)
    return out


def sssp_validate(graph, root, parent, dist, edges=None, stream=None):
    """SSSP result validation on the device (synchronises the stream): a dict with
    code (0 = valid, else the first failing rule 1..7), where, reached,
    component_edges, teps_edges (-1 without edges) and max_dist."""
    if parent.numel() != graph.n or dist.numel() != graph.n:
        raise ValueError("parent/dist must have n = %d entries" % graph.n)
    if edges is not None:
        if edges.dim() != 2 or edges.shape[0] != 2:
            raise ValueError("edges must be a [2, m] tensor")
        ep, m = _dev(edges, torch.int64, "edges"), int(edges.shape[1])
    else:
        ep, m = ctypes.c_void_p(None), 0
    out = gb_sssp_validation()
    _check(lib().sssp_validate(graph.handle, int(root), _dev(parent, torch.int32, "parent"),
                               _dev(dist, torch.float64, "dist"), ep, m, ctypes.byref(out),
                               _stream(stream)))
    return {f: getattr(out, f) for f, _ in gb_sssp_validation._fields_ if f != "pad"}
