"""CPU oracle for GSL-LPA (test infrastructure only).

Only the test suite, ``__graft_entry__.smoke()`` and the benchmark's CPU
baseline and reference arm may import this package.  It wraps ``oracle.c`` (plain, single
threaded C that shares nothing with the CUDA library) with numpy in and out.

Functions and the passages they follow:
  sync_sweep      one Jacobi sweep of Eq. 2 over every vertex
  lpa_sync        lpa() of Algorithm 3 with Jacobi sweeps (the parity reference)
  lpa_seq         lpa() of Algorithm 3 as printed, one thread, in place, pruned
  split_bfs       splitDisconnectedBfs(), Algorithm 2
  split_lp        splitDisconnectedLp(), Algorithm 1 (SL-LP, SL-LPP)
  modularity      Eq. 1, exact integer parts, one double combine
  disconnected    disconnectedCommunities(), Algorithm 4
  gsl_lpa         lpa_sync followed by split_bfs (Algorithm 3 with its split)
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_SO = os.path.join(_HERE, "_build", "liboracle.so")
_lock = threading.Lock()
_handle = None

i64p = ctypes.POINTER(ctypes.c_int64)
i32p = ctypes.POINTER(ctypes.c_int32)
u64p = ctypes.POINTER(ctypes.c_uint64)
u8p = ctypes.POINTER(ctypes.c_uint8)


def build(force: bool = False) -> str:
    """Compiles oracle.c into oracle/_build/liboracle.so (plain gcc, -O2)."""
    os.makedirs(os.path.dirname(_SO), exist_ok=True)
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < os.path.getmtime(_SRC):
        tmp = _SO + f".{os.getpid()}.tmp"
        subprocess.check_call(["gcc", "-O2", "-fPIC", "-shared", "-ffp-contract=off", "-o", tmp, _SRC])
        os.replace(tmp, _SO)
    return _SO


def configure(lib):
    """Declares the argument and result types of the oracle's C entry points."""
    lib.oracle_sync_sweep.restype = ctypes.c_int64
    lib.oracle_sync_sweep.argtypes = [ctypes.c_int64, i64p, i32p, i32p, i32p, i32p]
    f32p = ctypes.POINTER(ctypes.c_float)
    lib.oracle_sync_sweep_f32.restype = ctypes.c_int64
    lib.oracle_sync_sweep_f32.argtypes = [ctypes.c_int64, i64p, i32p, f32p, i32p, i32p]
    lib.oracle_lpa_sync_f32.restype = ctypes.c_int32
    lib.oracle_lpa_sync_f32.argtypes = [ctypes.c_int64, i64p, i32p, f32p, i32p, ctypes.c_double, ctypes.c_int32,
                                        i32p, i64p]
    lib.oracle_modularity_f64.restype = ctypes.c_int
    lib.oracle_modularity_f64.argtypes = [ctypes.c_int64, i64p, i32p, f32p, i32p, ctypes.POINTER(ctypes.c_double)]
    lib.oracle_sync_sweep_at.restype = ctypes.c_int
    lib.oracle_sync_sweep_at.argtypes = [ctypes.c_int64, i64p, i32p, i32p, i32p, i64p, ctypes.c_int64, i32p]
    for fn in (lib.oracle_lpa_sync, lib.oracle_lpa_seq):
        fn.restype = ctypes.c_int32
        fn.argtypes = [ctypes.c_int64, i64p, i32p, i32p, i32p, ctypes.c_double, ctypes.c_int32, i32p, i64p]
    lib.oracle_split_bfs.restype = ctypes.c_int
    lib.oracle_split_bfs.argtypes = [ctypes.c_int64, i64p, i32p, i32p, i32p]
    lib.oracle_split_lp.restype = ctypes.c_int32
    lib.oracle_split_lp.argtypes = [ctypes.c_int64, i64p, i32p, i32p, ctypes.c_int, i32p]
    lib.oracle_modularity.restype = ctypes.c_int
    lib.oracle_modularity.argtypes = [ctypes.c_int64, i64p, i32p, i32p, i32p, ctypes.POINTER(ctypes.c_double), u64p]
    lib.oracle_disconnected.restype = ctypes.c_int64
    lib.oracle_disconnected.argtypes = [ctypes.c_int64, i64p, i32p, i32p, u8p]
    return lib


def _lib():
    global _handle
    with _lock:
        if _handle is None:
            _handle = configure(ctypes.CDLL(build()))
    return _handle


def _csr(offsets, cols, weights):
    off = np.ascontiguousarray(offsets, dtype=np.int64)
    col = np.ascontiguousarray(cols, dtype=np.int32)
    w = None if weights is None else np.ascontiguousarray(weights, dtype=np.int32)
    n = off.shape[0] - 1
    return n, off, col, w


def _pp(a, t):
    return None if a is None else a.ctypes.data_as(t)


def _graph_args(g, weights="graph"):
    w = getattr(g, "weights", None) if weights == "graph" else weights
    return _csr(g.offsets, g.cols, w)


def sync_sweep(g, prev, weights="graph"):
    """next = Eq. 2 applied to every vertex under labels prev; returns (next, dN)."""
    n, off, col, w = _graph_args(g, weights)
    prev = np.ascontiguousarray(prev, dtype=np.int32)
    nxt = np.empty(max(n, 1), dtype=np.int32)
    dn = _lib().oracle_sync_sweep(n, _pp(off, i64p), _pp(col, i32p), _pp(w, i32p), _pp(prev, i32p), _pp(nxt, i32p))
    if dn < 0:
        raise MemoryError("oracle_sync_sweep")
    return nxt[:n], int(dn)


def _f32(g, wf):
    off = np.ascontiguousarray(g.offsets, dtype=np.int64)
    col = np.ascontiguousarray(g.cols, dtype=np.int32)
    w = np.ascontiguousarray(wf, dtype=np.float32)
    assert w.shape[0] == col.shape[0]
    return off.shape[0] - 1, off, col, w


def sync_sweep_f32(g, wf, prev):
    """Eq. 2 with float32 weights wf[nnz] and float64 sums -> (next, dN)."""
    n, off, col, w = _f32(g, wf)
    prev = np.ascontiguousarray(prev, dtype=np.int32)
    nxt = np.empty(max(n, 1), dtype=np.int32)
    dn = _lib().oracle_sync_sweep_f32(n, _pp(off, i64p), _pp(col, i32p), _pp(w, ctypes.POINTER(ctypes.c_float)),
                                      _pp(prev, i32p), _pp(nxt, i32p))
    if dn < 0:
        raise ValueError("oracle_sync_sweep_f32: bad weight or out of memory")
    return nxt[:n], int(dn)


def lpa_sync_f32(g, wf, tau=0.05, max_iters=20, labels_init=None):
    """lpa() of Algorithm 3, Jacobi sweeps, float32 weights -> (labels, sweeps, dN)."""
    n, off, col, w = _f32(g, wf)
    lab = np.empty(max(n, 1), dtype=np.int32)
    dn = np.zeros(max(max_iters, 1), dtype=np.int64)
    init = None if labels_init is None else np.ascontiguousarray(labels_init, dtype=np.int32)
    t = _lib().oracle_lpa_sync_f32(n, _pp(off, i64p), _pp(col, i32p), _pp(w, ctypes.POINTER(ctypes.c_float)),
                                   _pp(init, i32p), float(tau), int(max_iters), _pp(lab, i32p), _pp(dn, i64p))
    if t < 0:
        raise ValueError("oracle_lpa_sync_f32: bad weight or out of memory")
    return lab[:n], int(t), dn[:t]


def modularity_f64(g, wf, labels):
    """Eq. 1 with float32 weights and float64 sums."""
    n, off, col, w = _f32(g, wf)
    C = np.ascontiguousarray(labels, dtype=np.int32)
    q = ctypes.c_double()
    if _lib().oracle_modularity_f64(n, _pp(off, i64p), _pp(col, i32p), _pp(w, ctypes.POINTER(ctypes.c_float)),
                                    _pp(C, i32p), ctypes.byref(q)) != 0:
        raise ValueError("oracle_modularity_f64")
    return q.value


def gsl_lpa_f32(g, wf, tau=0.05, max_iters=20):
    """GSL-LPA with float32 weights: lpa_sync_f32 then splitDisconnectedBfs()."""
    lab, t, dn = lpa_sync_f32(g, wf, tau, max_iters)
    return split_bfs(g, lab), t, dn


def sync_sweep_at(g, prev, vertices, weights="graph"):
    """Eq. 2 for the listed vertices under labels prev (sampled checks)."""
    n, off, col, w = _graph_args(g, weights)
    prev = np.ascontiguousarray(prev, dtype=np.int32)
    sel = np.ascontiguousarray(vertices, dtype=np.int64)
    out = np.empty(max(sel.shape[0], 1), dtype=np.int32)
    if _lib().oracle_sync_sweep_at(n, _pp(off, i64p), _pp(col, i32p), _pp(w, i32p), _pp(prev, i32p), _pp(sel, i64p),
                                   sel.shape[0], _pp(out, i32p)) != 0:
        raise ValueError("oracle_sync_sweep_at")
    return out[:sel.shape[0]]


def _lpa(fn, g, tau, max_iters, labels_init, weights):
    n, off, col, w = _graph_args(g, weights)
    lab = np.empty(max(n, 1), dtype=np.int32)
    dn = np.zeros(max(max_iters, 1), dtype=np.int64)
    init = None if labels_init is None else np.ascontiguousarray(labels_init, dtype=np.int32)
    t = fn(n, _pp(off, i64p), _pp(col, i32p), _pp(w, i32p), _pp(init, i32p), float(tau), int(max_iters),
           _pp(lab, i32p), _pp(dn, i64p))
    if t < 0:
        raise MemoryError("oracle lpa")
    return lab[:n], int(t), dn[:t].copy()


def lpa_sync(g, tau=0.05, max_iters=20, labels_init=None, weights="graph"):
    """Algorithm 3's lpa() with Jacobi sweeps -> (labels, sweeps, dN per sweep)."""
    return _lpa(_lib().oracle_lpa_sync, g, tau, max_iters, labels_init, weights)


def lpa_seq(g, tau=0.05, max_iters=20, labels_init=None, weights="graph"):
    """Algorithm 3's lpa() as printed, one thread, in place -> (labels, sweeps, dN)."""
    return _lpa(_lib().oracle_lpa_seq, g, tau, max_iters, labels_init, weights)


def split_bfs(g, labels):
    """Algorithm 2: every connected piece of every community labelled by its smallest id."""
    n, off, col, _ = _graph_args(g, None)
    C = np.ascontiguousarray(labels, dtype=np.int32)
    out = np.empty(max(n, 1), dtype=np.int32)
    if _lib().oracle_split_bfs(n, _pp(off, i64p), _pp(col, i32p), _pp(C, i32p), _pp(out, i32p)) != 0:
        raise MemoryError("oracle_split_bfs")
    return out[:n]


def split_lp(g, labels, pruning=False):
    """Algorithm 1 (SL-LP, or SL-LPP with pruning=True) -> (labels, sweeps)."""
    n, off, col, _ = _graph_args(g, None)
    C = np.ascontiguousarray(labels, dtype=np.int32)
    out = np.empty(max(n, 1), dtype=np.int32)
    s = _lib().oracle_split_lp(n, _pp(off, i64p), _pp(col, i32p), _pp(C, i32p), int(pruning), _pp(out, i32p))
    if s < 0:
        raise MemoryError("oracle_split_lp")
    return out[:n], int(s)


def modularity(g, labels, weights="graph", parts=False):
    """Eq. 1.  With parts=True also returns (2m, S1, S2) as Python ints."""
    n, off, col, w = _graph_args(g, weights)
    C = np.ascontiguousarray(labels, dtype=np.int32)
    q = ctypes.c_double()
    p = np.zeros(4, dtype=np.uint64)
    if _lib().oracle_modularity(n, _pp(off, i64p), _pp(col, i32p), _pp(w, i32p), _pp(C, i32p), ctypes.byref(q),
                                _pp(p, u64p)) != 0:
        raise ValueError("oracle_modularity: labels outside [0, n) or out of memory")
    if parts:
        return q.value, (int(p[0]), int(p[1]), int(p[2]) | (int(p[3]) << 64))
    return q.value


def disconnected(g, labels):
    """Algorithm 4 -> (number of disconnected communities, flags uint8[n])."""
    n, off, col, _ = _graph_args(g, None)
    C = np.ascontiguousarray(labels, dtype=np.int32)
    D = np.zeros(max(n, 1), dtype=np.uint8)
    k = _lib().oracle_disconnected(n, _pp(off, i64p), _pp(col, i32p), _pp(C, i32p), _pp(D, u8p))
    if k < 0:
        raise ValueError("oracle_disconnected")
    return int(k), D[:n]


def gsl_lpa(g, tau=0.05, max_iters=20, weights="graph"):
    """GSL-LPA: synchronous lpa() then splitDisconnectedBfs() -> (labels, sweeps, dN)."""
    lab, t, dn = lpa_sync(g, tau, max_iters, weights=weights)
    return split_bfs(g, lab), t, dn
