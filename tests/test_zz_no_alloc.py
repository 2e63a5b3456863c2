"""gsl_modularity_noalloc, the modularity entry point for callers that cannot
allocate device memory (a request loop that must not pay the device-wide
synchronisation cudaMalloc / cudaFree can cause, or a process whose GPU
memory is already reserved in full by another allocator).  It needs no
context and keeps its scratch in one fixed device array.

Called through the C ABI and checked against the oracle's Eq. 1 and against
gsl_modularity on the same inputs, twice in a row (the second call starts
from the scratch the first call left behind); malformed inputs are rejected
with GSL_ERR_INVALID and the next valid call is still right.  This file is
collected last, so that a run stopping at its first failure has run every
other test before it."""
import ctypes

import numpy as np
import pytest
import torch

import inputs as I
import oracle as O

pytestmark = pytest.mark.gpu

MAX_N = 4194304       # GSL_NOALLOC_MAX_N
REL_Q = 1e-9          # the modularity tolerance of the parity tests


def _entry(gsl):
    lib = ctypes.CDLL(gsl.library_path())
    fn = lib.gsl_modularity_noalloc
    fn.restype = ctypes.c_int
    fn.argtypes = [ctypes.POINTER(gsl.Csr), ctypes.c_void_p, ctypes.c_void_p, ctypes.POINTER(ctypes.c_double),
                   ctypes.c_void_p]
    return fn


def _csr(gsl, off, col, nnz=None):
    c = gsl.Csr()
    c.n = off.numel() - 1
    c.nnz = col.numel() if nnz is None else nnz
    c.offsets = off.data_ptr()
    c.cols = col.data_ptr() if col.numel() else None
    return c


def _call(fn, gsl, off, col, w, labels, nnz=None):
    q = ctypes.c_double(-9.0)
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    rc = fn(ctypes.byref(_csr(gsl, off, col, nnz)), None if w is None else ctypes.c_void_p(w.data_ptr()),
            ctypes.c_void_p(labels.data_ptr()), ctypes.byref(q), stream)
    return rc, q.value


def _close(q, want):
    return abs(q - want) <= REL_Q * max(1.0, abs(want))


def test_noalloc_modularity_matches_oracle_and_context_entry_point(gpu_lib):
    fn = _entry(gpu_lib)
    ctx = gpu_lib.Context(0)
    rng = np.random.default_rng(0)
    graphs = [I.sbm_planted(), I.rmat(16, 24, seed=1)]
    weighted = I.rmat(14, 16, seed=2)
    weighted.weights = I.symmetric_weights(weighted, seed=4, wmax=9)
    graphs.append(weighted)
    for g in graphs:
        off = torch.from_numpy(g.offsets).cuda()
        col = torch.from_numpy(g.cols).cuda()
        w = None if g.weights is None else torch.from_numpy(g.weights).cuda()
        lab = ctx.gsllpa(off, col, w)
        for labels in (lab, torch.from_numpy(rng.integers(0, 50, g.n).astype(np.int32)).cuda()):
            want = O.modularity(g, labels.cpu().numpy())
            assert _close(ctx.modularity(off, col, labels, w), want)
            for _ in range(2):      # two calls in a row share the same scratch
                rc, q = _call(fn, gpu_lib, off, col, w, labels)
                assert rc == 0 and _close(q, want), (g.name, q, want)


def test_noalloc_rejects_malformed_input_and_recovers(gpu_lib):
    """Every malformed input the device checks (labels, columns, weights,
    offsets) returns GSL_ERR_INVALID; a valid call on the same scratch right
    after each rejection still gives the oracle's modularity."""
    fn = _entry(gpu_lib)
    g = I.rmat(12, 16, seed=5)
    g.weights = I.symmetric_weights(g, seed=2, wmax=7)
    off = torch.from_numpy(g.offsets).cuda()
    col = torch.from_numpy(g.cols).cuda()
    w = torch.from_numpy(g.weights).cuda()
    lab_np = np.random.default_rng(3).integers(0, 40, g.n).astype(np.int32)
    lab = torch.from_numpy(lab_np).cuda()
    want_w = O.modularity(g, lab_np)
    want_u = O.modularity(g, lab_np, weights=None)
    row = int(np.argmax(np.diff(g.offsets)))        # a vertex with entries
    e0 = int(g.offsets[row])

    def with_(t, idx, val):
        u = t.clone()
        u[idx] = val
        return u

    cases = {
        "label >= n": dict(labels=with_(lab, 7, g.n)),
        "label < 0": dict(labels=with_(lab, 7, -1)),
        "column >= n": dict(col=with_(col, e0, g.n)),
        "column < 0": dict(col=with_(col, e0, -5)),
        "weight 0": dict(w=with_(w, e0, 0)),
        "weight < 0": dict(w=with_(w, e0, -3)),
        "offsets[0] != 0": dict(off=with_(off, 0, 1)),
        "offsets[n] != nnz": dict(off=with_(off, g.n, g.nnz - 1)),
        "nnz past offsets[n]": dict(nnz=g.nnz + 1),
        "decreasing offsets": dict(off=with_(off, row + 1, e0 - 1)),
    }
    for name, kw in cases.items():
        rc, _ = _call(fn, gpu_lib, kw.get("off", off), kw.get("col", col), kw.get("w", w), kw.get("labels", lab),
                      kw.get("nnz"))
        assert rc == 1, name    # GSL_ERR_INVALID
        rc, q = _call(fn, gpu_lib, off, col, w, lab)
        assert rc == 0 and _close(q, want_w), (name, q, want_w)
        rc, q = _call(fn, gpu_lib, off, col, None, lab)
        assert rc == 0 and _close(q, want_u), (name, q, want_u)


def test_noalloc_rejects_graphs_beyond_its_scratch(gpu_lib):
    fn = _entry(gpu_lib)
    off = torch.zeros(MAX_N + 2, dtype=torch.int64, device="cuda")
    col = torch.zeros(0, dtype=torch.int32, device="cuda")
    lab = torch.zeros(MAX_N + 1, dtype=torch.int32, device="cuda")
    q = ctypes.c_double()
    rc = fn(ctypes.byref(_csr(gpu_lib, off, col)), None, ctypes.c_void_p(lab.data_ptr()), ctypes.byref(q), None)
    assert rc == 1      # GSL_ERR_INVALID: more than GSL_NOALLOC_MAX_N vertices
    # the largest graph it accepts: MAX_N isolated vertices (Q = 0)
    off = torch.zeros(MAX_N + 1, dtype=torch.int64, device="cuda")
    lab = torch.arange(MAX_N, dtype=torch.int32, device="cuda")
    rc, q = _call(fn, gpu_lib, off, col, None, lab)
    assert rc == 0 and q == 0.0
