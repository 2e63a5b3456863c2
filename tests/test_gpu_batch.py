"""Batched GSL-LPA: every graph of a packed batch gets exactly its solo result."""
import numpy as np
import pytest
import torch

import inputs as I
import oracle as O

pytestmark = pytest.mark.gpu


def pack(graphs):
    """Disjoint union of graphs as one CSR (columns shifted by each graph's base)."""
    vptr = np.zeros(len(graphs) + 1, dtype=np.int64)
    for k, g in enumerate(graphs):
        vptr[k + 1] = vptr[k] + g.n
    offs, cols, ws = [np.zeros(1, dtype=np.int64)], [], []
    base_e = 0
    for k, g in enumerate(graphs):
        offs.append(g.offsets[1:] + base_e)
        cols.append(g.cols.astype(np.int64) + vptr[k])
        if g.weights is not None:
            ws.append(g.weights)
        base_e += g.nnz
    off = np.concatenate(offs)
    col = np.concatenate(cols).astype(np.int32) if cols else np.zeros(0, dtype=np.int32)
    w = np.concatenate(ws).astype(np.int32) if ws else None
    return off, col, w, vptr


def mixed_graphs(count, seed=0):
    rng = np.random.default_rng(seed)
    gs = []
    for k in range(count):
        kind = k % 4
        if kind == 0:
            gs.append(I.batched_sbm(k, n_lo=200, n_hi=5000))
        elif kind == 1:
            gs.append(I.rmat(int(rng.integers(6, 12)), 8, seed=k))
        elif kind == 2:
            gs.append(I.lattice_chains(int(rng.integers(3, 20)), int(rng.integers(3, 20)), n_chains=int(rng.integers(0, 5)), seed=k))
        else:
            gs.append(I.random_graph(int(rng.integers(1, 60)), 0.1, seed=k))
    return gs


def run_batch(ctx, graphs, **kw):
    off, col, w, vptr = pack(graphs)
    t = lambda a: torch.from_numpy(a).cuda()
    labels, iters = ctx.gsllpa_batch(t(off), t(col), vptr, None if w is None else t(w), **kw)
    return labels.cpu().numpy(), iters, vptr


@pytest.fixture(scope="module")
def ctx(gpu_lib):
    return gpu_lib.Context(0)


@pytest.mark.parametrize("max_iters", [20, 3, 1])
def test_batch_equals_solo_oracle(ctx, max_iters):
    graphs = mixed_graphs(24)
    labels, iters, vptr = run_batch(ctx, graphs, tolerance=0.05, max_iters=max_iters)
    for k, g in enumerate(graphs):
        want, t, _ = O.gsl_lpa(g, 0.05, max_iters)
        assert iters[k] == t, (k, g.name)
        assert np.array_equal(labels[vptr[k]:vptr[k + 1]], want), (k, g.name)


def test_batch_weighted_and_small_thresholds(gpu_lib):
    c = gpu_lib.Context(0)
    c.set_tuning(32, 48)
    graphs = mixed_graphs(12, seed=3)
    for g in graphs:
        if g.nnz:
            g.weights = I.symmetric_weights(g, seed=7, wmax=5)
        else:
            g.weights = np.zeros(0, dtype=np.int32)
    labels, iters, vptr = run_batch(c, graphs, tolerance=0.05, max_iters=20)
    for k, g in enumerate(graphs):
        want, t, _ = O.gsl_lpa(g, 0.05, 20)
        assert iters[k] == t and np.array_equal(labels[vptr[k]:vptr[k + 1]], want), (k, g.name)


def test_batch_replays_and_handles_empty_graphs(ctx):
    empty = I.Graph(np.zeros(1, dtype=np.int64), np.zeros(0, dtype=np.int32), name="empty")
    graphs = [empty] + mixed_graphs(6, seed=5) + [empty, I.path(1)]
    for _ in range(3):   # the captured sweep loop is replayed on repeat calls
        labels, iters, vptr = run_batch(ctx, graphs, tolerance=0.05, max_iters=20)
        for k, g in enumerate(graphs):
            want, t, _ = O.gsl_lpa(g, 0.05, 20) if g.n else (np.zeros(0, np.int32), 0, None)
            assert iters[k] == t and np.array_equal(labels[vptr[k]:vptr[k + 1]], want), (k, g.name)


def test_batch_async_invariants(ctx):
    graphs = mixed_graphs(8, seed=9)
    labels, iters, vptr = run_batch(ctx, graphs, tolerance=0.05, max_iters=20, mode=1)
    for k, g in enumerate(graphs):
        lab = labels[vptr[k]:vptr[k + 1]]
        v = np.arange(g.n)
        assert (lab <= v).all() and np.array_equal(lab[lab], lab)
        assert O.disconnected(g, lab)[0] == 0


def test_batch_rejects_edges_between_graphs(ctx, gpu_lib):
    a, b = I.path(4), I.path(3)
    off, col, _, vptr = pack([a, b])
    col = col.copy()
    col[0] = 5          # row 0 (graph 0) points into graph 1
    with pytest.raises(gpu_lib.GslError):
        ctx.gsllpa_batch(torch.from_numpy(off).cuda(), torch.from_numpy(col).cuda(), vptr)
    with pytest.raises(gpu_lib.GslError):
        ctx.gsllpa_batch(torch.from_numpy(off).cuda(), torch.from_numpy(col).cuda(), np.array([0, 3, 2], np.int64))


def test_batch_thresholds_changed_between_calls(gpu_lib):
    """A new threshold pair on the same buffers re-captures the sweep loop."""
    c = gpu_lib.Context(0)
    graphs = mixed_graphs(10, seed=11)
    off, col, w, vptr = pack(graphs)
    t = lambda a: torch.from_numpy(a).cuda()
    d_off, d_col = t(off), t(col)
    wants = [O.gsl_lpa(g, 0.05, 20) for g in graphs]
    for wm, bm in ((1024, 32768), (32, 40), (64, 4096), (1024, 32768)):
        c.set_tuning(wm, bm)
        labels, iters = c.gsllpa_batch(d_off, d_col, vptr)
        labels = labels.cpu().numpy()
        for k, (want, tt, _) in enumerate(wants):
            assert iters[k] == tt and np.array_equal(labels[vptr[k]:vptr[k + 1]], want), (wm, bm, k)
