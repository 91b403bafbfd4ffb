"""GB300 k-clique listing (SDegree / BitCol with Pre-Core and Pre-List).

Thin Python binding of the C ABI in ``include/kcl.h``: every function here has
the name of the C entry point it calls and only marshals arguments (numpy
arrays or torch tensors in, plain pointers and sizes out).  All work runs in
the CUDA library ``libkcl.so``; there is no CPU fallback, and importing this
package fails loudly if the library has not been built
(``python -c "import __graft_entry__ as g; g.build()"``).
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libkcl.so")

if not os.path.exists(LIB_PATH):
    raise ImportError(
        "libkcl.so is missing: build the CUDA library first "
        "(python -c 'import __graft_entry__ as g; g.build()')")

_lib = ctypes.CDLL(LIB_PATH)

KCL_OK, KCL_EINVAL, KCL_ENOMEM, KCL_EOVERFLOW, KCL_ETRUNC = 0, 1, 2, 3, 4
KCL_ETIMEOUT, KCL_ECUDA, KCL_EABORT, KCL_ELIMIT = 5, 6, 7, 8
KCL_ORDER_DEGREE, KCL_ORDER_COLOR = 0, 1
KCL_MAX_K = 32
KCL_NUM_STAGES = 5
KCL_MAX_CLASSES = 16
STAGES = ("pre_core", "pre_list", "orientation", "listing", "total")
ORDERINGS = {"degree": KCL_ORDER_DEGREE, "color": KCL_ORDER_COLOR,
             "sdegree": KCL_ORDER_DEGREE, "bitcol": KCL_ORDER_COLOR}


class KclError(RuntimeError):
    def __init__(self, status, what):
        msg = _lib.kcl_strerror(status).decode()
        super().__init__("%s: %s (status %d)" % (what, msg, status))
        self.status = status


class _Ring(ctypes.Structure):
    _fields_ = [("ids", ctypes.c_void_p), ("capacity", ctypes.c_uint64), ("wrap", ctypes.c_int)]


class _Timing(ctypes.Structure):
    _fields_ = [("ms", ctypes.c_float * KCL_NUM_STAGES),
                ("launches", ctypes.c_uint32 * KCL_NUM_STAGES),
                ("n_classes", ctypes.c_uint32),
                ("class_lo", ctypes.c_uint32 * KCL_MAX_CLASSES),
                ("class_hi", ctypes.c_uint32 * KCL_MAX_CLASSES),
                ("class_roots", ctypes.c_uint32 * KCL_MAX_CLASSES),
                ("class_ms", ctypes.c_float * KCL_MAX_CLASSES)]

    def classes(self):
        return [{"lo": int(self.class_lo[c]), "hi": int(self.class_hi[c]),
                 "roots": int(self.class_roots[c]), "ms": float(self.class_ms[c])}
                for c in range(min(int(self.n_classes), KCL_MAX_CLASSES))]


class _Tuning(ctypes.Structure):
    _fields_ = [("sdegree_gallop", ctypes.c_uint32 * KCL_MAX_CLASSES),
                ("sdegree_gallop_list", ctypes.c_uint32 * KCL_MAX_CLASSES),
                ("sdegree_bitmap", ctypes.c_uint32 * KCL_MAX_CLASSES),
                ("sdegree_cta_warps", ctypes.c_uint32 * KCL_MAX_CLASSES),
                ("bitcol_cta_warps", ctypes.c_uint32 * KCL_MAX_CLASSES),
                ("sdegree_split", ctypes.c_uint32 * KCL_MAX_CLASSES),
                ("bitcol_split", ctypes.c_uint32 * KCL_MAX_CLASSES)]

    def as_dict(self):
        return {f: [int(x) for x in getattr(self, f)] for f, _ in self._fields_}


_P, _U32, _U64, _I = ctypes.c_void_p, ctypes.c_uint32, ctypes.c_uint64, ctypes.c_int
_sig = {
    "kcl_load_csr": ([_U32, _P, _P, _I, _P, ctypes.POINTER(_P)], _I),
    "kcl_free_graph": ([_P], None),
    "kcl_set_stream": ([_P, _P], _I),
    "kcl_num_vertices": ([_P], _U32),
    "kcl_num_edges": ([_P], _U64),
    "kcl_count": ([_P, _U32, _I, ctypes.POINTER(_U64)], _I),
    "kcl_list": ([_P, _U32, _I, ctypes.POINTER(_Ring), ctypes.POINTER(_U64),
                  ctypes.POINTER(_U64), ctypes.POINTER(_U64)], _I),
    "kcl_count_per_root": ([_P, _U32, _I, _P, ctypes.POINTER(_U64), ctypes.POINTER(_U64)], _I),
    "kcl_stage_info": ([_P, _U32, _I, _P, _P, _P, _P, ctypes.POINTER(_U64),
                        ctypes.POINTER(_U32)], _I),
    "kcl_enable_timing": ([_P, _I], _I),
    "kcl_last_timing": ([_P, ctypes.POINTER(_Timing)], _I),
    "kcl_set_options": ([_P, _U32], _I),
    "kcl_get_options": ([_P, ctypes.POINTER(_U32)], _I),
    "kcl_scratch_bytes": ([_P, ctypes.POINTER(_U64), ctypes.POINTER(_U64)], _I),
    "kcl_get_tuning": ([_P, ctypes.POINTER(_Tuning)], _I),
    "kcl_set_tuning": ([_P, ctypes.POINTER(_Tuning)], _I),
    "kcl_autotune": ([_P, _U32, _I, _I, ctypes.POINTER(_Tuning)], _I),
    "kcl_strerror": ([_I], ctypes.c_char_p),
    "kcl_root_colouring": ([_P, _U32, _U32, _U32, _P, _P, ctypes.POINTER(_U32)], _I),
}
for _name, (_args, _res) in _sig.items():
    _f = getattr(_lib, _name)
    _f.argtypes = _args
    _f.restype = _res


def _ord(ordering):
    if isinstance(ordering, str):
        return ORDERINGS[ordering.lower()]
    return int(ordering)


def _check(st, what, ok=(KCL_OK,)):
    if st not in ok:
        raise KclError(st, what)
    return st


def _current_stream():
    try:
        import torch
        if torch.cuda.is_available():
            return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    except ImportError:
        pass
    return ctypes.c_void_p(0)


def _dev_ptr(t, dtype_name, numel=None):
    import torch
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError("expected a CUDA tensor")
    if str(t.dtype) != "torch." + dtype_name:
        raise TypeError("expected dtype %s, got %s" % (dtype_name, t.dtype))
    if not t.is_contiguous():
        raise TypeError("expected a contiguous tensor")
    if numel is not None and t.numel() < numel:
        raise ValueError("tensor too small: %d < %d" % (t.numel(), numel))
    return ctypes.c_void_p(t.data_ptr())


class Graph:
    """Owning handle of a device-resident graph (``kcl_graph*``)."""

    def __init__(self, handle, n, m):
        self._h = handle
        self.n = n
        self.m = m

    @property
    def handle(self):
        if self._h is None:
            raise ValueError("graph already freed")
        return self._h

    def free(self):
        if self._h is not None:
            _lib.kcl_free_graph(self._h)
            self._h = None

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass


def kcl_load_csr(row_ptr, col, stream=None):
    """Copy a symmetric CSR graph into the library (validated on the device).

    ``row_ptr``/``col`` are numpy arrays (host) or CUDA tensors (device),
    dtypes uint64/uint32 (torch: int64/int32 reinterpreted)."""
    try:
        import torch
        on_dev = isinstance(row_ptr, torch.Tensor) and row_ptr.is_cuda
    except ImportError:
        on_dev = False
    if on_dev:
        # device CSR: int64 row offsets and int32 ids, bit-identical to the
        # uint64 / uint32 layout of the C ABI
        n = row_ptr.numel() - 1
        rp_p = _dev_ptr(row_ptr, "int64")
        c_p = _dev_ptr(col, "int32") if col.numel() else None
        keep = (row_ptr, col)
    else:
        rp = np.ascontiguousarray(row_ptr, dtype=np.uint64)
        c = np.ascontiguousarray(col, dtype=np.uint32)
        n = len(rp) - 1
        rp_p = ctypes.c_void_p(rp.ctypes.data)
        c_p = ctypes.c_void_p(c.ctypes.data) if c.size else None
        keep = (rp, c)
    h = ctypes.c_void_p()
    s = stream if stream is not None else _current_stream()
    st = _lib.kcl_load_csr(n, rp_p, c_p, 1 if on_dev else 0, s, ctypes.byref(h))
    del keep
    _check(st, "kcl_load_csr")
    return Graph(h, n, int(_lib.kcl_num_edges(h)))


def kcl_free_graph(g):
    g.free()


def kcl_set_stream(g, stream=None):
    _check(_lib.kcl_set_stream(g.handle, stream if stream is not None else _current_stream()),
           "kcl_set_stream")


def kcl_count(g, k, ordering="color"):
    """Exact number of k-cliques (Algorithms 5 / 6)."""
    c = ctypes.c_uint64()
    _check(_lib.kcl_count(g.handle, k, _ord(ordering), ctypes.byref(c)), "kcl_count")
    return int(c.value)


def kcl_list(g, k, ordering="color", ring=None, wrap=False):
    """List the k-cliques into ``ring`` (CUDA int32/uint32 tensor of
    capacity*k entries, or None for checksum only).  Returns
    (count, checksum, written, truncated)."""
    r = _Ring()
    if ring is not None:
        if ring.numel() % k:
            raise ValueError("ring size must be a multiple of k")
        r.ids = ctypes.c_void_p(ring.data_ptr())
        r.capacity = ring.numel() // k
        r.wrap = 1 if wrap else 0
    c, s, w = ctypes.c_uint64(), ctypes.c_uint64(), ctypes.c_uint64()
    st = _lib.kcl_list(g.handle, k, _ord(ordering), ctypes.byref(r), ctypes.byref(c),
                       ctypes.byref(s), ctypes.byref(w))
    _check(st, "kcl_list", ok=(KCL_OK, KCL_ETRUNC))
    return int(c.value), int(s.value), int(w.value), st == KCL_ETRUNC


def kcl_count_per_root(g, k, ordering, per_root):
    """Fill ``per_root`` (CUDA int64 tensor, n entries) with per-root counts;
    returns (total, prelist_count)."""
    c, p = ctypes.c_uint64(), ctypes.c_uint64()
    ptr = ctypes.c_void_p(per_root.data_ptr())
    if per_root.numel() < g.n:
        raise ValueError("per_root too small")
    _check(_lib.kcl_count_per_root(g.handle, k, _ord(ordering), ptr, ctypes.byref(c),
                                   ctypes.byref(p)), "kcl_count_per_root")
    return int(c.value), int(p.value)


_lib.kcl_count_roots.argtypes = [_P, _U32, _I, _P, _U32, _P, ctypes.POINTER(_U64)]
_lib.kcl_count_roots.restype = _I


def kcl_count_roots(g, k, ordering, roots, per_root):
    """Per-root counts of the given roots only (numpy uint32 ids) into
    ``per_root`` (CUDA int64 tensor, n entries); returns their sum."""
    r = np.ascontiguousarray(roots, dtype=np.uint32)
    if per_root.numel() < g.n:
        raise ValueError("per_root too small")
    c = ctypes.c_uint64()
    _check(_lib.kcl_count_roots(g.handle, k, _ord(ordering), r.ctypes.data if r.size else None,
                                r.size, ctypes.c_void_p(per_root.data_ptr()), ctypes.byref(c)),
           "kcl_count_roots")
    return int(c.value)


def kcl_stage_info(g, k, ordering):
    """Front-end intermediates as numpy arrays: alive_core, alive_final,
    outdeg, key, prelist_count, max_outdeg."""
    n = g.n
    ac = np.zeros(max(n, 1), np.uint8)
    af = np.zeros(max(n, 1), np.uint8)
    od = np.zeros(max(n, 1), np.uint32)
    ky = np.zeros(max(n, 1), np.uint32)
    pc, mo = ctypes.c_uint64(), ctypes.c_uint32()
    _check(_lib.kcl_stage_info(g.handle, k, _ord(ordering), ac.ctypes.data, af.ctypes.data,
                               od.ctypes.data, ky.ctypes.data, ctypes.byref(pc), ctypes.byref(mo)),
           "kcl_stage_info")
    return {"alive_core": ac[:n], "alive_final": af[:n], "outdeg": od[:n], "key": ky[:n],
            "prelist_count": int(pc.value), "max_outdeg": int(mo.value)}


def kcl_root_colouring(g, k, root):
    """The colouring BitCol's subproblem builder gives G_root (the subgraph
    induced by root's out-neighbours in the degeneracy DAG after the front
    end for k): (out-neighbours in ascending id, their colours), numpy
    uint32 arrays; empty when root has no out-neighbours."""
    d = ctypes.c_uint32()
    st = _lib.kcl_root_colouring(g.handle, k, root, 0, None, None, ctypes.byref(d))
    if st not in (KCL_OK, KCL_EINVAL) or (st == KCL_EINVAL and d.value == 0):
        _check(st, "kcl_root_colouring")
    nb = np.zeros(max(d.value, 1), np.uint32)
    co = np.zeros(max(d.value, 1), np.uint32)
    if d.value:
        _check(_lib.kcl_root_colouring(g.handle, k, root, d.value, nb.ctypes.data, co.ctypes.data,
                                       ctypes.byref(d)), "kcl_root_colouring")
    return nb[: d.value], co[: d.value]


def kcl_enable_timing(g, enable=True):
    _check(_lib.kcl_enable_timing(g.handle, 1 if enable else 0), "kcl_enable_timing")


KCL_OPT_NO_PRECORE = 1
KCL_OPT_NO_PRELIST = 2
KCL_OPT_NO_COLOR_PRUNE = 4


_lib.kcl_set_time_limit.argtypes = [_P, _U64]
_lib.kcl_set_time_limit.restype = _I


def kcl_set_time_limit(g, ms):
    """Time limit of the listing stage of later calls on g, in ms (0: none);
    a call that exceeds it raises KclError with status KCL_ETIMEOUT."""
    _check(_lib.kcl_set_time_limit(g.handle, int(ms)), "kcl_set_time_limit")


def kcl_set_options(g, flags):
    """Ablation switches (KCL_OPT_* bits); results do not change."""
    _check(_lib.kcl_set_options(g.handle, int(flags)), "kcl_set_options")


def kcl_get_options(g):
    f = ctypes.c_uint32()
    _check(_lib.kcl_get_options(g.handle, ctypes.byref(f)), "kcl_get_options")
    return int(f.value)


def kcl_scratch_bytes(g):
    """(workspace, arena) device bytes the handle holds now."""
    a, b = ctypes.c_uint64(), ctypes.c_uint64()
    _check(_lib.kcl_scratch_bytes(g.handle, ctypes.byref(a), ctypes.byref(b)), "kcl_scratch_bytes")
    return int(a.value), int(b.value)


def kcl_get_tuning(g):
    """The graph's listing-kernel tuning as a dict of per-class lists."""
    t = _Tuning()
    _check(_lib.kcl_get_tuning(g.handle, ctypes.byref(t)), "kcl_get_tuning")
    return t.as_dict()


def kcl_set_tuning(g, tuning):
    """Set the tuning from a dict like kcl_get_tuning's (missing classes: 0)."""
    t = _Tuning()
    for f, _ in _Tuning._fields_:
        arr = getattr(t, f)
        for c, v in enumerate(tuning.get(f, [])[:KCL_MAX_CLASSES]):
            arr[c] = int(v)
    _check(_lib.kcl_set_tuning(g.handle, ctypes.byref(t)), "kcl_set_tuning")


def kcl_autotune(g, k, ordering, listing=False):
    """Run the autotuner for (k, ordering) in counting or listing mode on g;
    returns the chosen tuning."""
    t = _Tuning()
    _check(_lib.kcl_autotune(g.handle, k, _ord(ordering), 1 if listing else 0, ctypes.byref(t)),
           "kcl_autotune")
    return t.as_dict()


def kcl_last_timing(g):
    t = _Timing()
    _check(_lib.kcl_last_timing(g.handle, ctypes.byref(t)), "kcl_last_timing")
    return ({STAGES[i]: float(t.ms[i]) for i in range(KCL_NUM_STAGES)},
            {STAGES[i]: int(t.launches[i]) for i in range(KCL_NUM_STAGES)}, t.classes())


class _IntPeaks(ctypes.Structure):
    _fields_ = [("num_sms", ctypes.c_uint32), ("sm_clock_mhz", ctypes.c_double),
                ("popc_per_sm_clk", ctypes.c_double), ("lop3_per_sm_clk", ctypes.c_double),
                ("iadd_per_sm_clk", ctypes.c_double), ("bitjoin_words_per_sm_clk", ctypes.c_double),
                ("lds128_bytes_per_sm_clk", ctypes.c_double), ("mix64_per_sm_clk", ctypes.c_double)]


_lib.kcl_measure_int_peaks.argtypes = [_P, ctypes.POINTER(_IntPeaks)]
_lib.kcl_measure_int_peaks.restype = _I


def kcl_measure_int_peaks(stream=None):
    """Measured per-SM-clock rates of POPC, LOP3, IADD, the BitJoin word,
    128-bit shared loads and the SplitMix64 round (see include/kcl.h)."""
    p = _IntPeaks()
    _check(_lib.kcl_measure_int_peaks(stream if stream is not None else _current_stream(),
                                      ctypes.byref(p)), "kcl_measure_int_peaks")
    return {f: (int(getattr(p, f)) if f == "num_sms" else float(getattr(p, f)))
            for f, _ in _IntPeaks._fields_}


def kcl_strerror(status):
    return _lib.kcl_strerror(status).decode()


def kcl_num_vertices(g):
    return int(_lib.kcl_num_vertices(g.handle))


def kcl_num_edges(g):
    return int(_lib.kcl_num_edges(g.handle))


KCL_ESIZE = 9
KCL_NOALLOC_MAX_VERTICES = 1 << 20
_lib.kcl_degeneracy_order_noalloc.argtypes = [_U32, _P, _P, _P, _P, _P, _P]
_lib.kcl_degeneracy_order_noalloc.restype = _I


def kcl_degeneracy_order_noalloc(row_ptr, col, alive, degree, round_out, stream=None):
    """Degeneracy peel rounds without any device allocation.

    For callers that must not allocate device memory from inside their own
    loops (a serving loop that cannot absorb the synchronisation an
    allocation may cause, or a program whose device memory belongs to
    another allocator): all scratch lives in a fixed array inside the
    library, sized for at most KCL_NOALLOC_MAX_VERTICES vertices.  Every
    argument is a CUDA tensor: row_ptr int64[n+1], col int32[nnz], alive
    uint8[n], degree int32[n] (alive-neighbour counts), round_out int32[n]
    (written).  Calls on one device share the scratch, so they must not
    overlap on the GPU."""
    n = row_ptr.numel() - 1
    st = _lib.kcl_degeneracy_order_noalloc(
        n, _dev_ptr(row_ptr, "int64"), _dev_ptr(col, "int32"), _dev_ptr(alive, "uint8", n),
        _dev_ptr(degree, "int32", n), _dev_ptr(round_out, "int32", n),
        stream if stream is not None else _current_stream())
    _check(st, "kcl_degeneracy_order_noalloc")


_lib.kcl_batch_create.argtypes = [_P, ctypes.POINTER(_P)]
_lib.kcl_batch_create.restype = _I
_lib.kcl_batch_free.argtypes = [_P]
_lib.kcl_batch_free.restype = None
_lib.kcl_count_batch.argtypes = [_P, _P, _P, _P, _U32, _P, _P]
_lib.kcl_count_batch.restype = _I


class Batch:
    """Owning handle of a kcl_batch (device scratch reused across calls)."""

    def __init__(self, handle):
        self._h = handle

    @property
    def handle(self):
        if self._h is None:
            raise ValueError("batch already freed")
        return self._h

    def free(self):
        if self._h is not None:
            _lib.kcl_batch_free(self._h)
            self._h = None

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass


def kcl_batch_create(stream=None):
    h = ctypes.c_void_p()
    _check(_lib.kcl_batch_create(stream if stream is not None else _current_stream(),
                                 ctypes.byref(h)), "kcl_batch_create")
    return Batch(h)


def kcl_batch_free(b):
    b.free()


def kcl_count_batch(b, graphs, ks, orderings, checksums=False):
    """Counts (and optionally listing checksums) of many loaded graphs at
    once: returns (counts, checksums-or-None) as lists."""
    G = len(graphs)
    handles = (ctypes.c_void_p * max(G, 1))(*[g.handle for g in graphs])
    karr = np.ascontiguousarray(ks, dtype=np.uint32)
    oarr = np.ascontiguousarray([_ord(o) for o in orderings], dtype=np.int32)
    counts = np.zeros(max(G, 1), dtype=np.uint64)
    cks = np.zeros(max(G, 1), dtype=np.uint64) if checksums else None
    _check(_lib.kcl_count_batch(b.handle, ctypes.cast(handles, ctypes.c_void_p),
                                karr.ctypes.data if G else None, oarr.ctypes.data if G else None,
                                G, counts.ctypes.data, cks.ctypes.data if checksums else None),
           "kcl_count_batch")
    return ([int(x) for x in counts[:G]],
            [int(x) for x in cks[:G]] if checksums else None)


# ------------------------------------------------------------ views, server
_lib.kcl_graph_view.argtypes = [_P, _P, ctypes.POINTER(_P)]
_lib.kcl_graph_view.restype = _I


def kcl_graph_view(g, stream=None):
    """Second handle on a loaded graph (shared CSR, own scratch and stream)."""
    h = ctypes.c_void_p()
    _check(_lib.kcl_graph_view(g.handle, stream if stream is not None else _current_stream(),
                               ctypes.byref(h)), "kcl_graph_view")
    v = Graph(h, g.n, g.m)
    v._parent = g  # the CSR belongs to g: keep it alive
    return v


class _ServerResult(ctypes.Structure):
    _fields_ = [("count", ctypes.c_uint64), ("checksum", ctypes.c_uint64),
                ("submit_s", ctypes.c_double), ("start_s", ctypes.c_double),
                ("done_s", ctypes.c_double), ("batch", ctypes.c_uint32), ("status", ctypes.c_int)]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_}


_lib.kcl_server_create.argtypes = [_U32, _U64, _U64, ctypes.POINTER(_P)]
_lib.kcl_server_create.restype = _I
_lib.kcl_server_add_graph.argtypes = [_P, _P, ctypes.POINTER(_U32)]
_lib.kcl_server_add_graph.restype = _I
_lib.kcl_server_submit.argtypes = [_P, _U32, _U32, _I, _I, ctypes.POINTER(_U64)]
_lib.kcl_server_submit.restype = _I
_lib.kcl_server_poll.argtypes = [_P, _U64, ctypes.POINTER(_I), ctypes.POINTER(_ServerResult)]
_lib.kcl_server_poll.restype = _I
_lib.kcl_server_wait.argtypes = [_P, _U64, ctypes.POINTER(_ServerResult)]
_lib.kcl_server_wait.restype = _I
_lib.kcl_server_clock.argtypes = [_P]
_lib.kcl_server_clock.restype = ctypes.c_double
_lib.kcl_server_destroy.argtypes = [_P]
_lib.kcl_server_destroy.restype = None


class Server:
    """Handle of a kcl_server (see kcl_server_create)."""

    def __init__(self, handle):
        self._h = handle
        self._graphs = []

    @property
    def handle(self):
        if self._h is None:
            raise ValueError("server already destroyed")
        return self._h

    def destroy(self):
        if self._h is not None:
            _lib.kcl_server_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.destroy()
        except Exception:
            pass


def kcl_server_create(slots=4, scratch_budget_bytes=100 << 30, small_nnz=1 << 20):
    h = ctypes.c_void_p()
    _check(_lib.kcl_server_create(slots, scratch_budget_bytes, small_nnz, ctypes.byref(h)),
           "kcl_server_create")
    return Server(h)


def kcl_server_add_graph(s, g):
    i = ctypes.c_uint32()
    _check(_lib.kcl_server_add_graph(s.handle, g.handle, ctypes.byref(i)), "kcl_server_add_graph")
    s._graphs.append(g)
    return int(i.value)


def kcl_server_submit(s, graph_id, k, ordering="color", listing=False):
    t = ctypes.c_uint64()
    _check(_lib.kcl_server_submit(s.handle, graph_id, k, _ord(ordering), 1 if listing else 0,
                                  ctypes.byref(t)), "kcl_server_submit")
    return int(t.value)


def kcl_server_poll(s, ticket):
    d, r = ctypes.c_int(), _ServerResult()
    _check(_lib.kcl_server_poll(s.handle, ticket, ctypes.byref(d), ctypes.byref(r)), "kcl_server_poll")
    return r.as_dict() if d.value else None


def kcl_server_wait(s, ticket):
    r = _ServerResult()
    _check(_lib.kcl_server_wait(s.handle, ticket, ctypes.byref(r)), "kcl_server_wait")
    return r.as_dict()


def kcl_server_clock(s):
    return float(_lib.kcl_server_clock(s.handle))


_lib.kcl_server_set_time_limit.argtypes = [_P, _U64]
_lib.kcl_server_set_time_limit.restype = _I
_lib.kcl_batch_set_time_limit.argtypes = [_P, _U64]
_lib.kcl_batch_set_time_limit.restype = _I


def kcl_server_set_time_limit(s, ms):
    """Time limit of each worker pass from now on (ms; 0 = none)."""
    _check(_lib.kcl_server_set_time_limit(s.handle, int(ms)), "kcl_server_set_time_limit")


def kcl_batch_set_time_limit(b, ms):
    """Time limit of each pipeline pass of later batched calls (ms; 0 = none)."""
    _check(_lib.kcl_batch_set_time_limit(b.handle, int(ms)), "kcl_batch_set_time_limit")


def kcl_server_destroy(s):
    s.destroy()


_lib.kcl_batch_enable_timing.argtypes = [_P, _I]
_lib.kcl_batch_enable_timing.restype = _I
_lib.kcl_batch_last_timing.argtypes = [_P, ctypes.POINTER(_Timing), ctypes.POINTER(_U32)]
_lib.kcl_batch_last_timing.restype = _I


def kcl_batch_enable_timing(b, enable=True):
    _check(_lib.kcl_batch_enable_timing(b.handle, 1 if enable else 0), "kcl_batch_enable_timing")


def kcl_batch_last_timing(b):
    t, gr = _Timing(), ctypes.c_uint32()
    _check(_lib.kcl_batch_last_timing(b.handle, ctypes.byref(t), ctypes.byref(gr)),
           "kcl_batch_last_timing")
    return ({STAGES[i]: float(t.ms[i]) for i in range(KCL_NUM_STAGES)},
            {STAGES[i]: int(t.launches[i]) for i in range(KCL_NUM_STAGES)}, int(gr.value))
