"""gsl_modularity_noalloc, the entry point for callers that cannot allocate
device memory (no context, fixed scratch), called through the C ABI and
checked against gsl_modularity on the same inputs, twice in a row (the
second call starts from the scratch the first call left behind)."""
import ctypes

import numpy as np
import pytest
import torch

import inputs as I

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


def _csr(gsl, off, col):
    c = gsl.Csr()
    c.n = off.numel() - 1
    c.nnz = col.numel()
    c.offsets = off.data_ptr()
    c.cols = col.data_ptr() if col.numel() else None
    return c


def test_noalloc_modularity_matches_context_entry_point(gpu_lib):
    fn = _entry(gpu_lib)
    ctx = gpu_lib.Context(0)
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
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
            want = ctx.modularity(off, col, labels, w)
            csr = _csr(gpu_lib, off, col)
            for _ in range(2):      # two calls in a row share the same scratch
                q = ctypes.c_double(-9.0)
                rc = fn(ctypes.byref(csr), None if w is None else ctypes.c_void_p(w.data_ptr()),
                        ctypes.c_void_p(labels.data_ptr()), ctypes.byref(q), stream)
                assert rc == 0
                assert abs(q.value - want) <= REL_Q * max(1.0, abs(want)), (g.name, q.value, want)


def test_noalloc_rejects_graphs_beyond_its_scratch(gpu_lib):
    fn = _entry(gpu_lib)
    off = torch.zeros(MAX_N + 2, dtype=torch.int64, device="cuda")
    col = torch.zeros(0, dtype=torch.int32, device="cuda")
    lab = torch.zeros(MAX_N + 1, dtype=torch.int32, device="cuda")
    q = ctypes.c_double()
    rc = fn(ctypes.byref(_csr(gpu_lib, off, col)), None, ctypes.c_void_p(lab.data_ptr()), ctypes.byref(q), None)
    assert rc == 1      # GSL_ERR_INVALID: more than GSL_NOALLOC_MAX_N vertices
