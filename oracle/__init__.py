"""Python binding of the plain CPU oracle (``kcl_oracle.c``).

TEST INFRASTRUCTURE ONLY: imported by ``tests/``, ``__graft_entry__.smoke()``
and the CPU-baseline leg of ``bench.py``.  The product library never imports,
links or executes anything under ``oracle/``.

Every call takes a symmetric CSR graph (``row_ptr`` uint64[n+1], ``col``
uint32[nnz], rows strictly ascending) and returns exact integers.  See the
header comment of ``kcl_oracle.c`` for what each mode computes and which
reading of the paper it takes.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "kcl_oracle.c")
_LIB = os.path.join(_HERE, "libkcl_oracle.so")
_lock = threading.Lock()
_lib = None

OK, EINVAL, ENOMEM, EOVERFLOW, ETRUNC = 0, 1, 2, 3, 4


class OracleError(RuntimeError):
    def __init__(self, code, what):
        super().__init__("%s failed with oracle status %d" % (what, code))
        self.code = code


class Counters(ctypes.Structure):
    _fields_ = [
        ("intersections", ctypes.c_uint64),
        ("merge_elems", ctypes.c_uint64),
        ("bitjoin_words", ctypes.c_uint64),
        ("build_reads", ctypes.c_uint64),
        ("roots", ctypes.c_uint64),
        ("max_outdeg", ctypes.c_uint64),
        ("bitrow_words", ctypes.c_uint64),
    ]

    def as_dict(self):
        return {f: int(getattr(self, f)) for f, _ in self._fields_}


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (plain -O2, no vectorisation tricks)."""
    with _lock:
        if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
            tmp = _LIB + ".%d.tmp" % os.getpid()
            subprocess.check_call(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-o", tmp, _SRC])
            os.replace(tmp, _LIB)
    return _LIB


_P = ctypes.c_void_p
_U32 = ctypes.c_uint32
_U64 = ctypes.c_uint64


def _load():
    global _lib
    if _lib is None:
        build()
        lib = ctypes.CDLL(_LIB)
        sig = {
            "oracle_mix64": ([_U64], _U64),
            "oracle_clique_hash": ([_U32, _P], _U64),
            "oracle_validate": ([_U32, _P, _P], ctypes.c_int),
            "oracle_plain": ([_U32, _P, _P, _U32, _P, _P, _P, _U64, _P], ctypes.c_int),
            "oracle_precore": ([_U32, _P, _P, _U32, _P], ctypes.c_int),
            "oracle_prelist": ([_U32, _P, _P, _U32, _P, _P, _P, _P, _P, _U64, _P], ctypes.c_int),
            "oracle_degeneracy_rounds": ([_U32, _P, _P, _P, _P, _P], ctypes.c_int),
            "oracle_outdegrees": ([_U32, _P, _P, _P, ctypes.c_int, _P], ctypes.c_int),
            "oracle_sdegree": ([_U32, _P, _P, _U32, ctypes.c_int, _P, _U32, _P, _P, _P, _P,
                                _P, _U64, _P, _P, _U64, _P, ctypes.c_int], ctypes.c_int),
            "oracle_bitcol": ([_U32, _P, _P, _U32, ctypes.c_int, _U32, _P, _U32, _P, _P, _P,
                               _P, _P, _U64, _P, ctypes.c_int], ctypes.c_int),
            "oracle_colour_graph": ([_U32, _P, _P, _P, _P], ctypes.c_int),
            "oracle_bitencode_graph": ([_U32, _P, _P, _U32, _P, _P], ctypes.c_int),
        }
        for name, (args, res) in sig.items():
            f = getattr(lib, name)
            f.argtypes = args
            f.restype = res
        _lib = lib
    return _lib


def _csr(row_ptr, col):
    rp = np.ascontiguousarray(row_ptr, dtype=np.uint64)
    c = np.ascontiguousarray(col, dtype=np.uint32)
    if c.size == 0:
        c = np.zeros(1, dtype=np.uint32)
    return len(rp) - 1, rp, c


def _ptr(a):
    return None if a is None else a.ctypes.data


def _check(rc, what, allow_trunc=False):
    if rc == OK or (allow_trunc and rc == ETRUNC):
        return
    raise OracleError(rc, what)


def mix64(x):
    return int(_load().oracle_mix64(x))


def clique_hash(ids):
    a = np.ascontiguousarray(sorted(int(i) for i in ids), dtype=np.uint32)
    return int(_load().oracle_clique_hash(len(a), _ptr(a)))


def validate(row_ptr, col):
    n, rp, c = _csr(row_ptr, col)
    return _load().oracle_validate(n, _ptr(rp), _ptr(c)) == OK


def plain(row_ptr, col, k, list_cap=0):
    """Reference answer (Algorithm 2 recursion over the degree DAG of the
    original graph).  Returns (count, checksum) or, with ``list_cap`` > 0,
    (count, checksum, cliques[written, k])."""
    n, rp, c = _csr(row_ptr, col)
    cnt, cks, wr = _U64(), _U64(), _U64()
    out = np.zeros(max(list_cap, 1) * k, dtype=np.uint32) if list_cap else None
    rc = _load().oracle_plain(n, _ptr(rp), _ptr(c), k, ctypes.byref(cnt), ctypes.byref(cks),
                              _ptr(out), list_cap, ctypes.byref(wr))
    _check(rc, "oracle_plain", allow_trunc=True)
    if list_cap:
        return int(cnt.value), int(cks.value), out[: wr.value * k].reshape(-1, k)
    return int(cnt.value), int(cks.value)


def precore(row_ptr, col, k):
    """Algorithm 3: survivors of the (k-1)-core peel, as uint8[n]."""
    n, rp, c = _csr(row_ptr, col)
    alive = np.zeros(max(n, 1), dtype=np.uint8)
    _check(_load().oracle_precore(n, _ptr(rp), _ptr(c), k, _ptr(alive)), "oracle_precore")
    return alive[:n]


def prelist(row_ptr, col, k, alive, list_cap=0):
    """Algorithm 4 on the alive subgraph.  Returns dict with the updated
    alive mask, count, checksum, removed component count (and cliques)."""
    n, rp, c = _csr(row_ptr, col)
    a = np.ascontiguousarray(alive, dtype=np.uint8).copy()
    if a.size == 0:
        a = np.zeros(1, dtype=np.uint8)
    cnt, cks, nrem, wr = _U64(), _U64(), _U32(), _U64()
    out = np.zeros(max(list_cap, 1) * k, dtype=np.uint32) if list_cap else None
    rc = _load().oracle_prelist(n, _ptr(rp), _ptr(c), k, _ptr(a), ctypes.byref(cnt),
                                ctypes.byref(cks), ctypes.byref(nrem), _ptr(out), list_cap,
                                ctypes.byref(wr))
    _check(rc, "oracle_prelist", allow_trunc=True)
    res = {"alive": a[:n], "count": int(cnt.value), "checksum": int(cks.value),
           "removed": int(nrem.value)}
    if list_cap:
        res["cliques"] = out[: wr.value * k].reshape(-1, k)
    return res


def degeneracy_rounds(row_ptr, col, alive=None):
    """Bulk peel rounds (degeneracy ordering key) and the final threshold."""
    n, rp, c = _csr(row_ptr, col)
    a = np.ones(max(n, 1), dtype=np.uint8) if alive is None else np.ascontiguousarray(alive, dtype=np.uint8)
    rd = np.zeros(max(n, 1), dtype=np.uint32)
    deg = _U32()
    _check(_load().oracle_degeneracy_rounds(n, _ptr(rp), _ptr(c), _ptr(a), _ptr(rd),
                                            ctypes.byref(deg)), "oracle_degeneracy_rounds")
    return rd[:n], int(deg.value)


def outdegrees(row_ptr, col, alive, mode):
    """Out-degrees of the DAG over ``alive``: mode 0 = degree ordering,
    mode 1 = degeneracy ordering."""
    n, rp, c = _csr(row_ptr, col)
    a = np.ascontiguousarray(alive, dtype=np.uint8)
    if a.size == 0:
        a = np.zeros(1, dtype=np.uint8)
    od = np.zeros(max(n, 1), dtype=np.uint32)
    _check(_load().oracle_outdegrees(n, _ptr(rp), _ptr(c), _ptr(a), mode, _ptr(od)),
           "oracle_outdegrees")
    return od[:n]


def _roots_arg(roots):
    if roots is None:
        return None, 0
    r = np.ascontiguousarray(roots, dtype=np.uint32)
    if r.size == 0:
        r = np.zeros(1, dtype=np.uint32)
        return r, 0
    return r, len(roots)


def sdegree(row_ptr, col, k, preprocess=True, roots=None, per_root=False, list_cap=0,
            trace_cap=0, count_only=False):
    """Algorithm 5.  Returns dict(count, checksum, counters[, per_root,
    cliques, trace]).  With ``roots`` only those roots are expanded and the
    Pre-List cliques are not included."""
    n, rp, c = _csr(row_ptr, col)
    r, nr = _roots_arg(roots)
    cnt, cks, wr, tl = _U64(), _U64(), _U64(), _U64()
    ctr = Counters()
    pr = np.zeros(max(n, 1), dtype=np.uint64) if per_root else None
    out = np.zeros(max(list_cap, 1) * k, dtype=np.uint32) if list_cap else None
    tr = np.zeros(max(trace_cap, 1), dtype=np.uint32) if trace_cap else None
    rc = _load().oracle_sdegree(n, _ptr(rp), _ptr(c), k, 1 if preprocess else 0, _ptr(r), nr,
                                ctypes.byref(cnt), ctypes.byref(cks), _ptr(pr), ctypes.byref(ctr),
                                _ptr(out), list_cap, ctypes.byref(wr), _ptr(tr), trace_cap,
                                ctypes.byref(tl), 1 if count_only else 0)
    _check(rc, "oracle_sdegree", allow_trunc=True)
    res = {"count": int(cnt.value), "checksum": int(cks.value), "counters": ctr.as_dict()}
    if per_root:
        res["per_root"] = pr[:n]
    if list_cap:
        res["cliques"] = out[: wr.value * k].reshape(-1, k)
    if trace_cap:
        res["trace"] = _parse_trace(tr[: tl.value])
    return res


def _parse_trace(t):
    calls, i = [], 0
    while i < len(t):
        l = int(t[i]); nr = int(t[i + 1])
        R = [int(x) for x in t[i + 2: i + 2 + nr]]
        nc = int(t[i + 2 + nr])
        C = [int(x) for x in t[i + 3 + nr: i + 3 + nr + nc]]
        calls.append((l, R, C))
        i += 3 + nr + nc
    return calls


def bitcol(row_ptr, col, k, preprocess=True, L=24, roots=None, per_root=False, list_cap=0,
           count_only=False):
    """Algorithm 6 with an L-bit bitmap word (the paper fixes L = 24)."""
    n, rp, c = _csr(row_ptr, col)
    r, nr = _roots_arg(roots)
    cnt, cks, wr = _U64(), _U64(), _U64()
    ctr = Counters()
    pr = np.zeros(max(n, 1), dtype=np.uint64) if per_root else None
    out = np.zeros(max(list_cap, 1) * k, dtype=np.uint32) if list_cap else None
    rc = _load().oracle_bitcol(n, _ptr(rp), _ptr(c), k, 1 if preprocess else 0, L, _ptr(r), nr,
                               ctypes.byref(cnt), ctypes.byref(cks), _ptr(pr), ctypes.byref(ctr),
                               _ptr(out), list_cap, ctypes.byref(wr), 1 if count_only else 0)
    _check(rc, "oracle_bitcol", allow_trunc=True)
    res = {"count": int(cnt.value), "checksum": int(cks.value), "counters": ctr.as_dict()}
    if per_root:
        res["per_root"] = pr[:n]
    if list_cap:
        res["cliques"] = out[: wr.value * k].reshape(-1, k)
    return res


def colour_graph(row_ptr, col):
    """Greedy colouring of an explicit graph (Section VII-A): (order, colour)."""
    n, rp, c = _csr(row_ptr, col)
    order = np.zeros(max(n, 1), dtype=np.uint32)
    colour = np.zeros(max(n, 1), dtype=np.uint32)
    _check(_load().oracle_colour_graph(n, _ptr(rp), _ptr(c), _ptr(order), _ptr(colour)),
           "oracle_colour_graph")
    return order[:n], colour[:n]


def bitencode_graph(row_ptr, col, L):
    """Colour an explicit graph and BitEncode it: (colour, B[n, ceil(n/L)])."""
    n, rp, c = _csr(row_ptr, col)
    nw = (n + L - 1) // L
    colour = np.zeros(max(n, 1), dtype=np.uint32)
    B = np.zeros(max(n * nw, 1), dtype=np.uint32)
    _check(_load().oracle_bitencode_graph(n, _ptr(rp), _ptr(c), L, _ptr(colour), _ptr(B)),
           "oracle_bitencode_graph")
    return colour[:n], B[: n * nw].reshape(n, nw)
