"""Parity at full size, in the launch configuration the benchmark times.

Batched (4096 planted-partition graphs, 3.7 G entries): sampled graphs
against the oracle and against solo calls.

R-MAT scale 25 (33.5 M vertices, 1.56 G entries): the oracle cannot run
all sweeps here in reasonable time, so every GPU sweep is checked on
sampled vertices (random ones, the highest-degree hubs, degree-1 vertices)
against the oracle's Eq. 2 applied to the GPU's previous labels; the chain
of single sweeps must equal the benchmark's pruned run; the split, Eq. 1
and Algorithm 4 of the final labels are compared in full.

Lattice + chains (60 M vertices, the road / k-mer stand-in; synchronous LPA
oscillates on it for all 20 sweeps): compared with the full oracle run.
"""
import os
import sys
import tempfile

import numpy as np
import pytest
import torch

import inputs as I
import oracle as O

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
DEV = "cuda:0"
REL_Q = 1e-9


def _bench_graph(scale, edge_factor):
    sys.path.insert(0, ROOT)
    import bench
    cache = os.environ.get("GSL_BENCH_CACHE", os.path.join(tempfile.gettempdir(), "gsl_bench_cache"))
    off, col = bench.workload_graph(scale, edge_factor, cache, 0, 1)
    return I.Graph(np.asarray(off), np.asarray(col), name=f"rmat{scale}-ef{edge_factor}")


def _sample(g, rng, k=3000):
    d = np.diff(g.offsets)
    hubs = np.argsort(d)[-200:]
    ones = np.flatnonzero(d == 1)[:200]
    return np.unique(np.concatenate([rng.choice(g.n, k, replace=False), hubs, ones]).astype(np.int64))


@pytest.fixture(scope="module")
def ctx(gpu_lib):
    return gpu_lib.Context(0)


def test_rmat25_sampled_sweeps_and_full_split(ctx):
    g = _bench_graph(25, 24)
    assert g.n == 1 << 25
    off = torch.from_numpy(g.offsets).to(DEV)
    col = torch.from_numpy(g.cols).to(DEV)
    rng = np.random.default_rng(25)
    sel = _sample(g, rng)
    # the benchmark's call: all sweeps (pruned, streamed first sweep) + split
    final_lpa, st = ctx.lpa(off, col, tolerance=0.05, max_iters=20, stats=True)
    T = st["iterations"]
    # the same sweeps one at a time, each checked on the sample
    prev = np.arange(g.n, dtype=np.int32)
    cur_d = torch.from_numpy(prev).to(DEV)
    for t in range(1, T + 1):
        nxt_d = ctx.lpa(off, col, labels_init=cur_d, tolerance=0.0, max_iters=1)
        nxt = nxt_d.cpu().numpy()
        assert np.array_equal(nxt[sel], O.sync_sweep_at(g, prev, sel)), t
        assert int((nxt != prev).sum()) == st["changed"][t - 1], t
        prev, cur_d = nxt, nxt_d
    assert np.array_equal(final_lpa.cpu().numpy(), prev)
    assert st["changed"][T - 1] / g.n <= 0.05 and all(c / g.n > 0.05 for c in st["changed"][:T - 1])
    # split, modularity and Algorithm 4 of the final labels, in full
    got_split = ctx.gsllpa(off, col).cpu().numpy()
    want_split = O.split_bfs(g, prev)
    assert np.array_equal(got_split, want_split)
    q_gpu = ctx.modularity(off, col, torch.from_numpy(want_split).to(DEV))
    q_ref = O.modularity(g, want_split)
    assert abs(q_gpu - q_ref) <= REL_Q * max(1.0, abs(q_ref))
    k_gpu = ctx.disconnected(off, col, final_lpa)
    assert k_gpu == O.disconnected(g, prev)[0]


def test_lattice_chains_full_oracle(ctx):
    g = I.lattice_chains()
    off = torch.from_numpy(g.offsets).to(DEV)
    col = torch.from_numpy(g.cols).to(DEV)
    want, T, dn = O.lpa_sync(g, 0.05, 20)
    got, st = ctx.lpa(off, col, tolerance=0.05, max_iters=20, stats=True)
    assert st["iterations"] == T and st["changed"] == dn[:T].tolist()
    assert np.array_equal(got.cpu().numpy(), want)
    want_split = O.split_bfs(g, want)
    assert np.array_equal(ctx.gsllpa(off, col).cpu().numpy(), want_split)
    q_ref = O.modularity(g, want_split)
    assert abs(ctx.modularity(off, col, torch.from_numpy(want_split).to(DEV)) - q_ref) <= REL_Q * max(1.0, abs(q_ref))
    assert ctx.disconnected(off, col, got) == O.disconnected(g, want)[0]


def test_batched_4096_graphs_sampled(gpu_lib):
    """The benchmark's batched workload (4096 planted-partition graphs, one
    CUDA-graph sweep loop): 24 sampled graphs against the oracle, every 64th
    graph against its own solo call."""
    sys.path.insert(0, ROOT)
    import bench
    graphs = bench.batched_graphs(4096, 0)
    G = len(graphs)
    vptr = np.zeros(G + 1, dtype=np.int64)
    eptr = np.zeros(G + 1, dtype=np.int64)
    for k, (o, c) in enumerate(graphs):
        vptr[k + 1] = vptr[k] + (o.shape[0] - 1)
        eptr[k + 1] = eptr[k] + c.shape[0]
    off_u = np.empty(vptr[-1] + 1, dtype=np.int64)
    col_u = np.empty(eptr[-1], dtype=np.int32)
    off_u[0] = 0
    for k, (o, c) in enumerate(graphs):
        off_u[vptr[k] + 1:vptr[k + 1] + 1] = o[1:] + eptr[k]
        col_u[eptr[k]:eptr[k + 1]] = c + vptr[k]
    ctx = gpu_lib.Context(0)
    labels, iters = ctx.gsllpa_batch(torch.from_numpy(off_u).to(DEV), torch.from_numpy(col_u).to(DEV), vptr)
    labels = labels.cpu().numpy()
    rng = np.random.default_rng(4096)
    for k in sorted(rng.choice(G, 24, replace=False)):
        o, c = graphs[k]
        g = I.Graph(o, c)
        want, t, _ = O.gsl_lpa(g, 0.05, 20)
        assert iters[k] == t and np.array_equal(labels[vptr[k]:vptr[k + 1]], want), k
    solo = gpu_lib.Context(0)
    for k in range(0, G, 64):   # every 64th graph through the plain entry point as well
        o, c = graphs[k]
        got = solo.gsllpa(torch.from_numpy(o).to(DEV), torch.from_numpy(c).to(DEV)).cpu().numpy()
        assert np.array_equal(got, labels[vptr[k]:vptr[k + 1]]), k
