"""Float32 weights with float64 sums (the paper's precision) on the GPU.

With weights that are multiples of 1/8 every partial sum is exact in
float64, so labels, sweep counts and change counts must equal the oracle's
bit for bit; with arbitrary float weights one sweep is compared on every
vertex whose best label wins by more than rounding, and the full pipeline
is held to the split invariants and to modularity computed in float64.
"""
import numpy as np
import pytest
import torch

import inputs as I
import oracle as O
from fixtures import float_weights

pytestmark = pytest.mark.gpu

DEV = "cuda:0"


def dev(g, wf):
    return (torch.from_numpy(g.offsets).to(DEV), torch.from_numpy(g.cols).to(DEV), torch.from_numpy(wf).to(DEV))


def giant_hubs(seed=4):
    rng = np.random.default_rng(seed)
    base = I.sbm_planted(40_000, 400, 14.0, 3.0, seed=seed)
    src = np.repeat(np.arange(base.n), np.diff(base.offsets))
    keep = src < base.cols
    u, v = [src[keep]], [base.cols[keep]]
    for h, deg in enumerate((30_000, 9_000, 5_000)):
        nb = rng.choice(base.n, deg, replace=False)
        u.append(np.full(deg, base.n + h))
        v.append(nb)
    return I.csr_from_pairs(base.n + 3, np.concatenate(u), np.concatenate(v), name="sbm40k-hubs")


GRAPHS = {
    "two_k5": lambda: I.two_cliques_bridge(5),
    "sbm10k": lambda: I.sbm_planted(),
    "rmat14": lambda: I.rmat(14, 16, seed=2),
    "hubs": giant_hubs,
}


@pytest.fixture(scope="module", params=sorted(GRAPHS))
def graph(request):
    return GRAPHS[request.param]()


@pytest.fixture(scope="module")
def ctxs(gpu_lib):
    """Default context, small class bounds, and both again with the float64
    path forced (no fixed-point form of exact weights)."""
    out = []
    for fixed in (1, 0):
        a = gpu_lib.Context(0)
        b = gpu_lib.Context(0)
        b.set_tuning(32, 48)
        for c in (a, b):
            c.set_f32_fixed(fixed)
        out += [a, b]
    return out


def _took_integer_path(c, fn):
    """Runs fn() with profiling on; the integer sweep loop profiles its label
    initialisation, the float loop does not."""
    c.set_profiling(True)
    fn()
    prof = {p["name"]: p for p in c.profile()}
    c.set_profiling(False)
    return prof["init_labels"]["launches"] > 0


def test_dyadic_weights_bit_exact(graph, ctxs):
    wf = float_weights(graph, 3, dyadic=True)
    off, col, w = dev(graph, wf)
    want, t, dn = O.lpa_sync_f32(graph, wf, 0.05, 20)
    want_split, _, _ = O.gsl_lpa_f32(graph, wf, 0.05, 20)
    for c in ctxs:
        got, st = c.lpa_f32(off, col, w, stats=True)
        assert st["iterations"] == t and st["changed"] == dn.tolist()
        assert np.array_equal(got.cpu().numpy(), want)
        lab = c.gsllpa_f32(off, col, w)
        assert np.array_equal(lab.cpu().numpy(), want_split)
        q = c.modularity_f32(off, col, lab, w)
        assert abs(q - O.modularity_f64(graph, wf, want_split)) <= 1e-9 * max(1.0, abs(q))


def test_fine_dyadic_weights_fixed_point(gpu_lib, ctxs):
    """Weights 1 + k / 2^20: multiples of 2^-20 whose row totals stay far
    below 2^11, so every float64 sum is exact and the weights run on the
    integer sweeps as w * 2^20; the labels equal the oracle's and the
    float64 path's."""
    rng = np.random.default_rng(21)
    for g in (I.sbm_planted(), I.rmat(12, 8, seed=5)):
        src = np.repeat(np.arange(g.n), np.diff(g.offsets))
        key = np.minimum(src, g.cols).astype(np.int64) * g.n + np.maximum(src, g.cols)
        uniq, inv = np.unique(key, return_inverse=True)
        wf = (1.0 + rng.integers(0, 1 << 20, uniq.shape[0]) / float(1 << 20))[inv].astype(np.float32)
        off, col, w = dev(g, wf)
        want, t, dn = O.lpa_sync_f32(g, wf, 0.05, 20)
        for c in ctxs:
            got, st = c.lpa_f32(off, col, w, stats=True)
            assert np.array_equal(got.cpu().numpy(), want) and st["changed"] == dn.tolist(), g.name
        assert _took_integer_path(ctxs[0], lambda: ctxs[0].lpa_f32(off, col, w))
        assert not _took_integer_path(ctxs[2], lambda: ctxs[2].lpa_f32(off, col, w))
    # arbitrary floats (lowest bits down to 2^-30, values up to 3): float64 path
    g = I.sbm_planted(2000, 100, 12.0, 3.0, seed=2)
    off, col, w = dev(g, float_weights(g, 11, dyadic=False))
    assert not _took_integer_path(ctxs[0], lambda: ctxs[0].lpa_f32(off, col, w))
    with pytest.raises(gpu_lib.GslError):
        ctxs[0].set_f32_fixed(2)


def test_integer_valued_float_weights_equal_int32_path(graph, ctxs):
    wi = I.symmetric_weights(graph, 5, 7) if graph.nnz else np.zeros(0, np.int32)
    off, col, w = dev(graph, wi.astype(np.float32))
    wi_d = torch.from_numpy(wi).to(DEV)
    c = ctxs[0]
    assert np.array_equal(c.lpa_f32(off, col, w).cpu().numpy(), c.lpa(off, col, wi_d).cpu().numpy())
    lab = c.gsllpa(off, col, wi_d)
    assert abs(c.modularity_f32(off, col, lab, w) - c.modularity(off, col, lab, wi_d)) < 1e-12


def test_arbitrary_float_weights_one_sweep(ctxs):
    rng = np.random.default_rng(9)
    for g in (I.sbm_planted(2000, 100, 12.0, 3.0, seed=2), I.rmat(11, 16, seed=3)):
        wf = float_weights(g, 11, dyadic=False)
        off, col, w = dev(g, wf)
        prev = rng.integers(0, 40, g.n).astype(np.int32)
        want, _ = O.sync_sweep_f32(g, wf, prev)
        # margin between the best and second-best label sum, per vertex
        src = np.repeat(np.arange(g.n), np.diff(g.offsets))
        keep = src != g.cols
        S = np.zeros((g.n, 40))
        np.add.at(S, (src[keep], prev[g.cols[keep]]), wf[keep].astype(np.float64))
        top2 = -np.sort(-S, axis=1)[:, :2]
        clear = (top2[:, 0] - top2[:, 1]) > 1e-9 * np.maximum(1.0, top2[:, 0])
        for c in ctxs:
            got = c.lpa_f32(off, col, w, labels_init=torch.from_numpy(prev).to(DEV), tolerance=0.0, max_iters=1)
            assert np.array_equal(got.cpu().numpy()[clear], want[clear])


def test_float_pipeline_invariants_sync_and_async(graph, ctxs):
    wf = float_weights(graph, 7, dyadic=False)
    off, col, w = dev(graph, wf)
    for mode in (0, 1):
        lab = ctxs[mode * 2].gsllpa_f32(off, col, w, mode=mode).cpu().numpy()
        v = np.arange(graph.n)
        assert (lab <= v).all() and np.array_equal(lab[lab], lab)
        assert O.disconnected(graph, lab)[0] == 0
        q = ctxs[0].modularity_f32(off, col, torch.from_numpy(lab).to(DEV), w)
        assert abs(q - O.modularity_f64(graph, wf, lab)) <= 1e-9 * max(1.0, abs(q))


def test_bad_float_weights_are_rejected(gpu_lib, ctxs):
    g = I.path(6)
    for bad in (0.0, -2.0, np.nan, np.inf):
        wf = np.ones(g.nnz, dtype=np.float32)
        wf[2] = bad
        off, col, w = dev(g, wf)
        for c in (ctxs[0], ctxs[2]):
            with pytest.raises(gpu_lib.GslError):
                c.lpa_f32(off, col, w)
        with pytest.raises(gpu_lib.GslError):
            ctxs[0].modularity_f32(off, col, torch.zeros(6, dtype=torch.int32, device=DEV), w)
    off, col, w = dev(g, np.ones(g.nnz, dtype=np.float32))
    assert np.array_equal(ctxs[0].lpa_f32(off, col, w).cpu().numpy(), O.lpa_sync(g, 0.05, 20)[0])
