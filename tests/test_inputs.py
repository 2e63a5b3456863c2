"""Seeded input generators: determinism and CSR well-formedness."""
import numpy as np

import inputs as I


def _check_csr(g, loops_ok=False):
    o, c = g.offsets, g.cols
    assert o[0] == 0 and o[-1] == c.shape[0] and (np.diff(o) >= 0).all()
    assert ((c >= 0) & (c < g.n)).all()
    src = np.repeat(np.arange(g.n), np.diff(o))
    if not loops_ok:
        assert (src != c).all()
    key = src.astype(np.int64) * g.n + c
    rkey = c.astype(np.int64) * g.n + src
    assert np.array_equal(np.sort(key), np.sort(rkey))          # symmetric
    assert (np.diff(key) > 0).all()                              # sorted rows, no duplicates


def test_sbm_planted_shape_and_determinism():
    g = I.sbm_planted()
    _check_csr(g)
    assert g.n == 10_000
    # E[nnz] = 2 * (50 * C(200,2) * 16/199 + C(10000,2)... ) ~= 180,000
    assert abs(g.nnz - 180_000) < 3_000
    h = I.sbm_planted(threads=3)
    assert np.array_equal(g.offsets, h.offsets) and np.array_equal(g.cols, h.cols)
    src = np.repeat(np.arange(g.n), np.diff(g.offsets))
    intra = (src // 200 == g.cols // 200).mean() * g.nnz / g.n
    assert 15.5 < intra < 16.5


def test_rmat_small_and_thread_independent():
    a = I.rmat(12, 8, seed=5, threads=1)
    b = I.rmat(12, 8, seed=5, threads=7)
    _check_csr(a)
    assert np.array_equal(a.offsets, b.offsets) and np.array_equal(a.cols, b.cols)
    assert a.nnz <= 2 * 8 * (1 << 12)
    c = I.rmat(12, 8, seed=6)
    assert not np.array_equal(a.cols[:100], c.cols[:100])


def test_lattice_chains_structure():
    g = I.lattice_chains(30, 40, n_chains=25, seed=2)
    _check_csr(g)
    lens = g.n - 30 * 40
    assert 25 * 4 <= lens <= 25 * 20
    deg = np.diff(g.offsets)
    assert deg[:1200].max() <= 4 + 10    # lattice degree plus a few shortcuts


def test_batched_params_ranges():
    for gi in range(50):
        p = I.batched_sbm_params(gi)
        assert 1000 <= p["n"] <= 200_000 and 5 <= p["blocks"] <= 200
        assert 8 <= p["degree"] <= 40 and 3 <= p["ratio"] <= 12
    g = I.batched_sbm(3)
    _check_csr(g)
    assert g.n == I.batched_sbm_params(3)["n"]


def test_symmetric_weights():
    g = I.rmat(10, 8, seed=1)
    w = I.symmetric_weights(g, seed=3, wmax=9)
    src = np.repeat(np.arange(g.n), np.diff(g.offsets))
    d = dict(zip(zip(src.tolist(), g.cols.tolist()), w.tolist()))
    assert all(d[(b, a)] == x for (a, b), x in d.items())
    assert w.min() >= 1 and w.max() <= 9


def test_served_request_laws():
    ps = [I.served_request_params(k) for k in range(4000)]
    share = sum(p["kind"] == "sbm" for p in ps) / len(ps)
    assert 0.67 < share < 0.73
    ns = np.array([p["n"] for p in ps if p["kind"] == "sbm"])
    assert ns.min() >= 1000 and ns.max() <= 4_194_304
    # log-uniform: the median is near the geometric mean of the range
    assert abs(np.log(np.median(ns)) - 0.5 * (np.log(1e3) + np.log(4194304))) < 0.3
    scales = [p["scale"] for p in ps if p["kind"] == "rmat"]
    assert min(scales) == 10 and max(scales) == 22
    assert all(5 <= p["blocks"] <= 200 and 8 <= p["degree"] <= 40 for p in ps if p["kind"] == "sbm")
    assert I.served_request_params(17) == I.served_request_params(17)
    g = I.served_request(3)
    assert g.n == 1 << ps[3]["scale"] if ps[3]["kind"] == "rmat" else g.n == ps[3]["n"]
