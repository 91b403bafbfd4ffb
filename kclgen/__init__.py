"""Seeded synthetic graph generators (inputs only; none of the method's arithmetic).

Shared by the tests, the benchmark and both sides of every parity check: the
oracle and the GPU path each receive the same CSR arrays built here.  The C
library is compiled with gcc on first use (``build()``) next to this file.

Every graph is an undirected simple graph returned as symmetric CSR:
``row_ptr`` uint64[n+1] and ``col`` uint32[row_ptr[n]], rows strictly ascending.

Workloads (all synthetic; the paper's NetworkRepository datasets are not used):

* ``chung_lu_planted_small``  n=10,000, 50,000 drawn pairs, exponent 2.5, plus
  20 planted 12-cliques on random vertices (seed 1).
* ``rmat``                    R-MAT scale 20, 16*2^20 unique undirected edges,
  a=0.57 b=0.19 c=0.19 d=0.05 (seed 1).
* ``chung_lu_communities``    n=4,000,000, 120M drawn pairs, exponent 2.1,
  expected degree capped at 40,000, plus 2,000 communities of 60-300 vertices
  at edge density 0.8.
* ``batch_graph(i)``          graph i of the 8,192-graph batch (n log-uniform in
  [50, 20000], mean degree uniform in [4, 40], exponent 2.3, 0-5 planted
  cliques of size 8-16, k uniform in 3..9).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "graphgen.c")
_LIB = os.path.join(_HERE, "libkclgen.so")
_lock = threading.Lock()
_lib = None


class _Params(ctypes.Structure):
    _fields_ = [
        ("kind", ctypes.c_int),
        ("n", ctypes.c_uint32),
        ("scale", ctypes.c_uint32),
        ("m", ctypes.c_uint64),
        ("gamma", ctypes.c_double),
        ("cap", ctypes.c_double),
        ("a", ctypes.c_double),
        ("b", ctypes.c_double),
        ("c", ctypes.c_double),
        ("n_groups", ctypes.c_uint32),
        ("group_lo", ctypes.c_uint32),
        ("group_hi", ctypes.c_uint32),
        ("group_p", ctypes.c_double),
        ("relabel", ctypes.c_int),
        ("seed", ctypes.c_uint64),
    ]


class _Csr(ctypes.Structure):
    _fields_ = [
        ("n", ctypes.c_uint32),
        ("nnz", ctypes.c_uint64),
        ("row_ptr", ctypes.POINTER(ctypes.c_uint64)),
        ("col", ctypes.POINTER(ctypes.c_uint32)),
    ]


def build(force: bool = False) -> str:
    """Compile libkclgen.so with gcc (portable flags, FP contraction off)."""
    with _lock:
        if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
            tmp = _LIB + ".%d.tmp" % os.getpid()
            subprocess.check_call([
                "gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-ffp-contract=off",
                "-fno-fast-math", "-o", tmp, _SRC,
            ])
            os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    if _lib is None:
        build()
        lib = ctypes.CDLL(_LIB)
        lib.kg_generate.argtypes = [ctypes.POINTER(_Params), ctypes.POINTER(_Csr)]
        lib.kg_generate.restype = ctypes.c_int
        lib.kg_from_edges.argtypes = [ctypes.c_uint32, ctypes.c_void_p, ctypes.c_void_p,
                                      ctypes.c_uint64, ctypes.POINTER(_Csr)]
        lib.kg_from_edges.restype = ctypes.c_int
        lib.kg_free.argtypes = [ctypes.POINTER(_Csr)]
        lib.kg_free.restype = None
        lib.kg_splitmix64.argtypes = [ctypes.c_uint64, ctypes.c_uint64]
        lib.kg_splitmix64.restype = ctypes.c_uint64
        lib.kg_batch_params.argtypes = [ctypes.c_uint64, ctypes.c_uint64,
                                        ctypes.POINTER(_Params), ctypes.POINTER(ctypes.c_uint32)]
        lib.kg_batch_params.restype = None
        _lib = lib
    return _lib


def _take(csr: _Csr):
    n = csr.n
    nnz = csr.nnz
    row_ptr = np.ctypeslib.as_array(csr.row_ptr, shape=(n + 1,)).copy()
    col = (np.ctypeslib.as_array(csr.col, shape=(nnz,)).copy() if nnz
           else np.zeros(0, dtype=np.uint32))
    _load().kg_free(ctypes.byref(csr))
    return row_ptr.astype(np.uint64, copy=False), col.astype(np.uint32, copy=False)


def _generate(p: _Params):
    csr = _Csr()
    rc = _load().kg_generate(ctypes.byref(p), ctypes.byref(csr))
    if rc != 0:
        raise RuntimeError("graph generator failed with code %d" % rc)
    return _take(csr)


def chung_lu(n, m, gamma, cap=0.0, groups=0, group_size=(0, 0), group_p=1.0,
             seed=1, relabel=True):
    """Chung-Lu graph: m endpoint pairs drawn i.i.d. proportional to
    w_i = c (i+1)^(-1/(gamma-1)) (scaled to sum 2m, clipped at ``cap``),
    self-loops and duplicates dropped, plus ``groups`` planted groups of a
    size drawn uniformly in ``group_size`` with edge probability ``group_p``."""
    p = _Params(kind=0, n=n, scale=0, m=m, gamma=gamma, cap=cap, a=0, b=0, c=0,
                n_groups=groups, group_lo=group_size[0], group_hi=group_size[1],
                group_p=group_p, relabel=1 if relabel else 0, seed=seed)
    return _generate(p)


def rmat(scale, m, a=0.57, b=0.19, c=0.19, seed=1, relabel=True):
    """R-MAT (quadrant recursion) sampled until ``m`` unique undirected
    non-loop edges exist on 2^scale vertices."""
    p = _Params(kind=1, n=0, scale=scale, m=m, gamma=0, cap=0, a=a, b=b, c=c,
                n_groups=0, group_lo=0, group_hi=0, group_p=1.0,
                relabel=1 if relabel else 0, seed=seed)
    return _generate(p)


def planted_only(n, groups, group_size, group_p=1.0, seed=1):
    """Empty base graph on n vertices plus planted groups."""
    p = _Params(kind=2, n=n, scale=0, m=0, gamma=0, cap=0, a=0, b=0, c=0,
                n_groups=groups, group_lo=group_size[0], group_hi=group_size[1],
                group_p=group_p, relabel=0, seed=seed)
    return _generate(p)


def from_edges(n, edges):
    """Symmetric sorted CSR from an iterable of (u, v) pairs (0-based)."""
    e = np.asarray(list(edges) if not isinstance(edges, np.ndarray) else edges,
                   dtype=np.uint32).reshape(-1, 2)
    eu = np.ascontiguousarray(e[:, 0])
    ev = np.ascontiguousarray(e[:, 1])
    csr = _Csr()
    rc = _load().kg_from_edges(n, eu.ctypes.data, ev.ctypes.data, len(eu), ctypes.byref(csr))
    if rc != 0:
        raise ValueError("bad edge list (code %d)" % rc)
    return _take(csr)


def splitmix64(seed, i):
    return int(_load().kg_splitmix64(seed, i))


# ---------------------------------------------------------------- workloads
def chung_lu_planted_small(seed=1):
    """n=10,000, 50,000 drawn pairs, exponent 2.5, 20 planted 12-cliques."""
    return chung_lu(10_000, 50_000, 2.5, 0.0, groups=20, group_size=(12, 12),
                    group_p=1.0, seed=seed)


def rmat20(seed=1, scale=20):
    """R-MAT at ``scale`` with 16 * 2^scale unique edges, a=.57 b=.19 c=.19."""
    return rmat(scale, 16 << scale, 0.57, 0.19, 0.19, seed=seed)


def chung_lu_communities(seed=1, n=4_000_000, m=120_000_000, groups=2000,
                         group_size=(60, 300)):
    """n=4M, 120M drawn pairs, exponent 2.1, expected degree capped at 40,000,
    plus ``groups`` communities of ``group_size`` vertices at density 0.8."""
    return chung_lu(n, m, 2.1, 40_000.0, groups=groups, group_size=group_size,
                    group_p=0.8, seed=seed)


def batch_params(i, base_seed=1):
    p = _Params()
    k = ctypes.c_uint32()
    _load().kg_batch_params(base_seed, i, ctypes.byref(p), ctypes.byref(k))
    return p, int(k.value)


def batch_graph(i, base_seed=1):
    """Graph i of the batched workload and its k."""
    p, k = batch_params(i, base_seed)
    rp, col = _generate(p)
    return rp, col, k
