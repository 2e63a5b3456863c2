"""Seeded synthetic inputs shared by the oracle tests and the CUDA path.

Input side only: nothing here computes labels, splits or modularity.  The
heavy generators live in ``graphgen.c`` (counter-based SplitMix64, so the
same seed gives the same graph for any thread count and on x86-64 and
aarch64 alike); this module wraps them with numpy and adds the small
hand-built graphs used as worked examples.

All graphs come back as symmetric CSR: ``offsets`` int64[n+1], ``cols``
int32[nnz], every row sorted ascending, no duplicates and no self-loops
(unless a hand-built graph asks for them explicitly).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "graphgen.c")
_SO = os.path.join(_HERE, "_build", "libgraphgen.so")
_lock = threading.Lock()
_handle = None

i64p = ctypes.POINTER(ctypes.c_int64)
i32p = ctypes.POINTER(ctypes.c_int32)


def build(force: bool = False) -> str:
    """Compiles graphgen.c into inputs/_build/libgraphgen.so (host code, gcc)."""
    os.makedirs(os.path.dirname(_SO), exist_ok=True)
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < os.path.getmtime(_SRC):
        tmp = _SO + f".{os.getpid()}.tmp"
        subprocess.check_call(["gcc", "-O2", "-fPIC", "-shared", "-ffp-contract=off", "-pthread",
                               "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _SO)
    return _SO


def _lib():
    global _handle
    with _lock:
        if _handle is None:
            lib = ctypes.CDLL(build())
            lib.gg_csr_from_pairs.restype = ctypes.c_int64
            lib.gg_csr_from_pairs.argtypes = [ctypes.c_int64, ctypes.c_int64, i32p, i32p, i32p, ctypes.c_int,
                                              i64p, i32p, ctypes.c_int64]
            lib.gg_permutation.restype = ctypes.c_int
            lib.gg_permutation.argtypes = [ctypes.c_int64, ctypes.c_uint64, ctypes.c_int, i32p]
            lib.gg_rmat_samples.restype = ctypes.c_int
            lib.gg_rmat_samples.argtypes = [ctypes.c_int, ctypes.c_int64, ctypes.c_double, ctypes.c_double,
                                            ctypes.c_double, ctypes.c_uint64, ctypes.c_int, i32p, i32p]
            lib.gg_sbm_count.restype = ctypes.c_int64
            lib.gg_sbm_count.argtypes = [ctypes.c_int64, i64p, ctypes.c_int64, ctypes.c_double, ctypes.c_double,
                                         ctypes.c_uint64, ctypes.c_int, i64p]
            lib.gg_sbm_pairs.restype = ctypes.c_int
            lib.gg_sbm_pairs.argtypes = [ctypes.c_int64, i64p, ctypes.c_int64, ctypes.c_double, ctypes.c_double,
                                         ctypes.c_uint64, ctypes.c_int, i64p, i32p, i32p]
            lib.gg_lattice_kept.restype = ctypes.c_int64
            lib.gg_lattice_kept.argtypes = [ctypes.c_int64, ctypes.c_int64, ctypes.c_double, ctypes.c_uint64,
                                            ctypes.c_int]
            lib.gg_chain_lengths.restype = ctypes.c_int
            lib.gg_chain_lengths.argtypes = [ctypes.c_int64, ctypes.c_int64, ctypes.c_int64, ctypes.c_uint64, i32p]
            lib.gg_lattice_pairs.restype = ctypes.c_int
            lib.gg_lattice_pairs.argtypes = [ctypes.c_int64, ctypes.c_int64, ctypes.c_double, ctypes.c_int64,
                                             ctypes.c_int64, i32p, ctypes.c_uint64, ctypes.c_int, i32p, i32p]
            for name in ("gg_det_log", "gg_det_exp"):
                getattr(lib, name).restype = ctypes.c_double
                getattr(lib, name).argtypes = [ctypes.c_double]
            lib.gg_rng.restype = ctypes.c_uint64
            lib.gg_rng.argtypes = [ctypes.c_uint64] * 3
            lib.gg_u01.restype = ctypes.c_double
            lib.gg_u01.argtypes = [ctypes.c_uint64] * 3
            lib.gg_below.restype = ctypes.c_uint64
            lib.gg_below.argtypes = [ctypes.c_uint64] * 4
            _handle = lib
    return _handle


def _threads(threads):
    return int(threads) if threads else max(1, min(64, os.cpu_count() or 1))


def _p(a, t):
    return a.ctypes.data_as(t)


class Graph:
    """A symmetric CSR graph held in host memory (numpy)."""

    def __init__(self, offsets, cols, weights=None, name=""):
        self.offsets = np.ascontiguousarray(offsets, dtype=np.int64)
        self.cols = np.ascontiguousarray(cols, dtype=np.int32)
        self.weights = None if weights is None else np.ascontiguousarray(weights, dtype=np.int32)
        self.name = name

    @property
    def n(self) -> int:
        return int(self.offsets.shape[0] - 1)

    @property
    def nnz(self) -> int:
        return int(self.cols.shape[0])

    def degrees(self):
        return np.diff(self.offsets)

    def __repr__(self):
        return f"Graph({self.name!r}, n={self.n}, nnz={self.nnz}, weighted={self.weights is not None})"


def csr_from_pairs(n, u, v, perm=None, threads=None, name=""):
    """Symmetric, deduplicated, loop-free CSR of the undirected pairs (u[i], v[i])."""
    u = np.ascontiguousarray(u, dtype=np.int32)
    v = np.ascontiguousarray(v, dtype=np.int32)
    assert u.shape == v.shape
    m = int(u.shape[0])
    offsets = np.empty(n + 1, dtype=np.int64)
    cols = np.empty(max(2 * m, 1), dtype=np.int32)
    pp = None
    if perm is not None:
        perm = np.ascontiguousarray(perm, dtype=np.int32)
        pp = _p(perm, i32p)
    nnz = _lib().gg_csr_from_pairs(n, m, _p(u, i32p), _p(v, i32p), pp, _threads(threads),
                                   _p(offsets, i64p), _p(cols, i32p), cols.shape[0])
    if nnz < 0:
        raise MemoryError("csr_from_pairs failed")
    return Graph(offsets, cols[:nnz] if nnz < cols.shape[0] else cols, name=name)


def permutation(n, seed, threads=None):
    perm = np.empty(max(n, 1), dtype=np.int32)
    if _lib().gg_permutation(n, seed, _threads(threads), _p(perm, i32p)) != 0:
        raise MemoryError("permutation failed")
    return perm[:n]


def rmat(scale, edge_factor=24, a=0.57, b=0.19, c=0.19, seed=1, permute=True, threads=None):
    """R-MAT graph: edge_factor * 2^scale samples, loops dropped, symmetrised,
    deduplicated, vertex ids randomly permuted (seeded)."""
    n = 1 << scale
    m = edge_factor * n
    u = np.empty(m, dtype=np.int32)
    v = np.empty(m, dtype=np.int32)
    if _lib().gg_rmat_samples(scale, m, a, b, c, seed, _threads(threads), _p(u, i32p), _p(v, i32p)) != 0:
        raise ValueError("bad R-MAT parameters")
    perm = permutation(n, seed, threads) if permute else None
    g = csr_from_pairs(n, u, v, perm=perm, threads=threads, name=f"rmat{scale}-ef{edge_factor}-s{seed}")
    del u, v
    return g


def sbm(n, block_starts, p_in, p_out, seed, threads=None, name=""):
    """Planted partition: contiguous blocks [block_starts[b], block_starts[b+1]),
    every pair u<v kept independently with p_in (same block) or p_out."""
    bs = np.ascontiguousarray(block_starts, dtype=np.int64)
    assert bs[0] == 0 and bs[-1] == n
    nb = int(bs.shape[0] - 1)
    cnt = np.zeros(max(n, 1), dtype=np.int64)
    lib = _lib()
    total = lib.gg_sbm_count(n, _p(bs, i64p), nb, p_in, p_out, seed, _threads(threads), _p(cnt, i64p))
    u = np.empty(max(total, 1), dtype=np.int32)
    v = np.empty(max(total, 1), dtype=np.int32)
    lib.gg_sbm_pairs(n, _p(bs, i64p), nb, p_in, p_out, seed, _threads(threads), _p(cnt, i64p),
                     _p(u, i32p), _p(v, i32p))
    return csr_from_pairs(n, u[:total], v[:total], threads=threads, name=name or f"sbm-n{n}-s{seed}")


def sbm_planted(n=10_000, block=200, d_in=16.0, d_out=2.0, seed=1, threads=None):
    """Planted partition with equal blocks: expected intra-block degree d_in and
    inter-block degree d_out (p_in = d_in/(block-1), p_out = d_out/(n-block))."""
    nb = n // block
    assert nb * block == n
    bs = np.arange(nb + 1, dtype=np.int64) * block
    return sbm(n, bs, d_in / (block - 1), d_out / (n - block), seed, threads,
               name=f"sbm-n{n}-b{block}-s{seed}")


def lattice_chains(rows=6000, cols=6000, p_del=0.25, shortcut_frac=0.005, n_chains=2_000_000,
                   len_lo=4, len_hi=20, seed=1, threads=None):
    """Road / k-mer-like graph: a rows x cols 4-neighbour lattice with each edge
    deleted with probability p_del, shortcut_frac * (kept edges) random
    long-range pairs, and n_chains disjoint paths of len_lo..len_hi vertices
    (ids after the lattice, not permuted)."""
    lib = _lib()
    t = _threads(threads)
    kept = lib.gg_lattice_kept(rows, cols, p_del, seed, t)
    shortcuts = int(round(shortcut_frac * kept))
    lens = np.empty(max(n_chains, 1), dtype=np.int32)
    lib.gg_chain_lengths(n_chains, len_lo, len_hi, seed, _p(lens, i32p))
    lens = lens[:n_chains]
    m = kept + shortcuts + int(np.sum(lens.astype(np.int64) - 1))
    n = rows * cols + int(np.sum(lens.astype(np.int64)))
    u = np.empty(max(m, 1), dtype=np.int32)
    v = np.empty(max(m, 1), dtype=np.int32)
    lib.gg_lattice_pairs(rows, cols, p_del, shortcuts, n_chains, _p(lens, i32p), seed, t, _p(u, i32p), _p(v, i32p))
    return csr_from_pairs(n, u[:m], v[:m], threads=threads,
                          name=f"lattice{rows}x{cols}-chains{n_chains}-s{seed}")


# ---------------------------------------------------------------- batched SBM laws
def batched_sbm_params(g: int, n_lo=1_000, n_hi=200_000, b_lo=5, b_hi=200, d_lo=8.0, d_hi=40.0,
                       r_lo=3.0, r_hi=12.0):
    """Parameters of graph g of the batched SBM workload (seed g):
    n log-uniform in [n_lo, n_hi], block count uniform in {b_lo..b_hi} (<= n),
    mean degree uniform in [d_lo, d_hi], intra:inter ratio uniform in [r_lo, r_hi]."""
    lib = _lib()
    s = 0x42415443  # stream id of the parameter draws
    lo, hi = lib.gg_det_log(float(n_lo)), lib.gg_det_log(float(n_hi))
    n = int(lib.gg_det_exp(lo + (hi - lo) * lib.gg_u01(g, s, 0)) + 0.5)
    nb = min(n, b_lo + int(lib.gg_below(g, s, 1, b_hi - b_lo + 1)))
    d = d_lo + (d_hi - d_lo) * lib.gg_u01(g, s, 2)
    r = r_lo + (r_hi - r_lo) * lib.gg_u01(g, s, 3)
    d_in = d * r / (r + 1.0)
    d_out = d / (r + 1.0)
    size = n / nb
    p_in = d_in / (size - 1.0) if size > 1.0 else 0.0
    p_out = d_out / (n - size) if n > size else 0.0
    return dict(n=n, blocks=nb, degree=d, ratio=r, p_in=min(p_in, 1.0), p_out=min(p_out, 1.0))


def batched_sbm(g: int, threads=None, **kw):
    prm = batched_sbm_params(g, **kw)
    n, nb = prm["n"], prm["blocks"]
    bs = (np.arange(nb + 1, dtype=np.int64) * n) // nb
    return sbm(n, bs, prm["p_in"], prm["p_out"], seed=g, threads=threads, name=f"batched-sbm-{g}")


def served_request_params(k: int, n_lo=1_000, n_hi=4_194_304, sbm_share=0.7):
    """Request k of the served workload (seed k): with probability sbm_share
    a planted partition with the batched laws for blocks, degree and ratio,
    else an R-MAT of scale clamp(round(log2 n), 10, 22) and edge factor 16;
    n log-uniform in [n_lo, n_hi]."""
    lib = _lib()
    s = 0x53525644  # stream id of the served-request draws
    lo, hi = lib.gg_det_log(float(n_lo)), lib.gg_det_log(float(n_hi))
    n = int(lib.gg_det_exp(lo + (hi - lo) * lib.gg_u01(k, s, 1)) + 0.5)
    if lib.gg_u01(k, s, 0) >= sbm_share:
        scale = min(22, max(10, int(round(float(np.log2(n))))))
        return dict(kind="rmat", scale=scale, edge_factor=16, n=1 << scale)
    nb = min(n, 5 + int(lib.gg_below(k, s, 2, 196)))
    d = 8.0 + 32.0 * lib.gg_u01(k, s, 3)
    r = 3.0 + 9.0 * lib.gg_u01(k, s, 4)
    size = n / nb
    d_in, d_out = d * r / (r + 1.0), d / (r + 1.0)
    p_in = d_in / (size - 1.0) if size > 1.0 else 0.0
    p_out = d_out / (n - size) if n > size else 0.0
    return dict(kind="sbm", n=n, blocks=nb, degree=d, ratio=r, p_in=min(p_in, 1.0), p_out=min(p_out, 1.0))


def served_request(k: int, threads=None, **kw):
    prm = served_request_params(k, **kw)
    if prm["kind"] == "rmat":
        return rmat(prm["scale"], prm["edge_factor"], seed=1000 + k, threads=threads)
    n, nb = prm["n"], prm["blocks"]
    bs = (np.arange(nb + 1, dtype=np.int64) * n) // nb
    return sbm(n, bs, prm["p_in"], prm["p_out"], seed=1000 + k, threads=threads, name=f"served-sbm-{k}")


# ---------------------------------------------------------------- hand-built graphs
def from_edges(n, edges, weights=None, name=""):
    """Symmetric CSR from an undirected edge list; both directions carry the
    same weight.  Duplicates are kept as given (callers pass simple graphs);
    self-loops (i, i) are stored once."""
    rows = [[] for _ in range(n)]
    for k, (a, b) in enumerate(edges):
        w = 1 if weights is None else int(weights[k])
        rows[a].append((b, w))
        if a != b:
            rows[b].append((a, w))
    offsets = np.zeros(n + 1, dtype=np.int64)
    cols, ws = [], []
    for i in range(n):
        r = sorted(rows[i])
        offsets[i + 1] = offsets[i] + len(r)
        cols.extend(c for c, _ in r)
        ws.extend(w for _, w in r)
    return Graph(offsets, np.array(cols, dtype=np.int32),
                 None if weights is None else np.array(ws, dtype=np.int32), name=name)


def two_cliques_bridge(k=5):
    """Two K_k cliques {0..k-1} and {k..2k-1} joined by the bridge (k-1, k)."""
    e = [(i, j) for i in range(k) for j in range(i + 1, k)]
    e += [(k + i, k + j) for i in range(k) for j in range(i + 1, k)]
    e.append((k - 1, k))
    return from_edges(2 * k, e, name=f"two-K{k}-bridge")


def path(n):
    return from_edges(n, [(i, i + 1) for i in range(n - 1)], name=f"path{n}")


def symmetric_weights(g: Graph, seed: int, wmax: int) -> np.ndarray:
    """Deterministic positive weights in [1, wmax] with w(i,j) == w(j,i)."""
    n = g.n
    src = np.repeat(np.arange(n, dtype=np.int64), np.diff(g.offsets))
    dst = g.cols.astype(np.int64)
    lo = np.minimum(src, dst).astype(np.uint64)
    hi = np.maximum(src, dst).astype(np.uint64)
    with np.errstate(over="ignore"):
        z = lo * np.uint64(0x9E3779B97F4A7C15) + hi * np.uint64(0xD1B54A32D192ED03) + np.uint64(seed)
        z = (z ^ (z >> np.uint64(30))) * np.uint64(0xBF58476D1CE4E5B9)
        z = (z ^ (z >> np.uint64(27))) * np.uint64(0x94D049BB133111EB)
        z = z ^ (z >> np.uint64(31))
    return (1 + (z % np.uint64(wmax))).astype(np.int32)


def random_graph(n, p, seed):
    """Small Erdos-Renyi graph (pairs kept with probability p), via the SBM sampler."""
    return sbm(n, np.array([0, n], dtype=np.int64), p, 0.0, seed, threads=1, name=f"er-n{n}-s{seed}")
