"""Pins of the CPU oracle against facts fixed by the paper and by mathematics.

Each test checks the oracle against something other than itself: hand
derivations of Eq. 2 / Algorithm 3 on tiny graphs, closed forms, a dense
matrix formulation evaluated by numpy (argmax of A @ onehot(C)), textbook
connected components (scipy) and a library modularity (networkx).
"""
import itertools

import numpy as np
import pytest
import scipy.sparse as sp
from scipy.sparse.csgraph import connected_components

import inputs as I
import oracle as O
from fixtures import float_weights


# ------------------------------------------------------------------ helpers
def graph_from_adj(A):
    """Symmetric CSR (with weights) from a dense symmetric integer matrix."""
    A = np.asarray(A)
    n = A.shape[0]
    offsets = np.zeros(n + 1, dtype=np.int64)
    cols, ws = [], []
    for i in range(n):
        nz = np.nonzero(A[i])[0]
        cols.extend(nz.tolist())
        ws.extend(A[i, nz].tolist())
        offsets[i + 1] = len(cols)
    return I.Graph(offsets, np.array(cols, dtype=np.int32), np.array(ws, dtype=np.int32))


def dense(g):
    n = g.n
    A = np.zeros((n, n), dtype=np.int64)
    src = np.repeat(np.arange(n), np.diff(g.offsets))
    w = np.ones(g.nnz, dtype=np.int64) if g.weights is None else g.weights.astype(np.int64)
    np.add.at(A, (src, g.cols), w)
    return A


def dense_sweep(A, prev):
    """Eq. 2 as a matrix product: S = A' Y with A' = A without its diagonal
    (j != i) and Y the one-hot label matrix; np.argmax returns the first
    (smallest) label among equal maxima."""
    n = A.shape[0]
    Ad = A.copy()
    np.fill_diagonal(Ad, 0)
    Y = np.zeros((n, n), dtype=np.int64)
    Y[np.arange(n), prev] = 1
    S = Ad @ Y
    has = Ad.sum(axis=1) > 0
    return np.where(has, np.argmax(S, axis=1), prev).astype(np.int32)


def components_split(g, labels):
    """Connected components (scipy) of the subgraph of edges inside a
    community, each labelled by its smallest vertex."""
    n = g.n
    src = np.repeat(np.arange(n), np.diff(g.offsets))
    keep = labels[src] == labels[g.cols]
    M = sp.csr_matrix((np.ones(keep.sum()), (src[keep], g.cols[keep])), shape=(n, n))
    k, comp = connected_components(M, directed=False)
    rep = np.full(k, n, dtype=np.int64)
    np.minimum.at(rep, comp, np.arange(n))
    return rep[comp].astype(np.int32)


# ------------------------------------------------- Eq. 2 / Algorithm 3: worked
def test_two_k5_bridge_sweeps_by_hand():
    # Two K5 {0..4}, {5..9}, bridge 4-5, unit weights.
    # Sweep 1 (labels = ids): every vertex sees each neighbour label once, so
    # the smallest neighbour id wins: 0->1, 1..4->0, 5->4 (neighbours 4,6..9),
    # 6..9->5.  All 10 change.
    # Sweep 2: 0 sees {0,0,0,0} -> 0; 5 sees {0,5,5,5,5} -> 5; the rest keep.
    # dN = 2, 2/10 > 0.05.  Sweep 3: nothing changes, dN = 0 -> stop, T = 3.
    g = I.two_cliques_bridge(5)
    s1, dn1 = O.sync_sweep(g, np.arange(10, dtype=np.int32))
    assert s1.tolist() == [1, 0, 0, 0, 0, 4, 5, 5, 5, 5] and dn1 == 10
    s2, dn2 = O.sync_sweep(g, s1)
    assert s2.tolist() == [0, 0, 0, 0, 0, 5, 5, 5, 5, 5] and dn2 == 2
    lab, t, dn = O.lpa_sync(g, 0.05, 20)
    assert lab.tolist() == s2.tolist() and t == 3 and dn.tolist() == [10, 2, 0]


def test_stop_rule_boundaries():
    g = I.two_cliques_bridge(5)
    # dN/N after sweep 2 is exactly 0.2: "<= tau" stops there for tau = 0.2
    _, t, _ = O.lpa_sync(g, 0.2, 20)
    assert t == 2
    _, t, _ = O.lpa_sync(g, 0.19, 20)
    assert t == 3
    # sweep 1 changes every vertex: tau = 1.0 stops after one sweep
    lab, t, _ = O.lpa_sync(g, 1.0, 20)
    assert t == 1 and lab.tolist() == [1, 0, 0, 0, 0, 4, 5, 5, 5, 5]
    # max_iters = 0 performs no sweep
    lab, t, dn = O.lpa_sync(g, 0.05, 0)
    assert t == 0 and lab.tolist() == list(range(10)) and dn.size == 0


def test_single_edge_oscillates():
    # Jacobi: 0 takes 1's label and 1 takes 0's, every sweep (dN = 2 = N).
    g = I.path(2)
    for iters in range(1, 8):
        lab, t, dn = O.lpa_sync(g, 0.05, iters)
        assert t == iters and (dn == 2).all()
        assert lab.tolist() == ([1, 0] if iters % 2 else [0, 1])


def test_path4_two_sweeps_by_hand():
    # 0-1-2-3.  Sweep 1: 0->1, 1->min(0,2)=0, 2->min(1,3)=1, 3->2.
    # Sweep 2: 0 sees {0}; 1 sees {1,1} -> 1; 2 sees {0,2} tie -> 0; 3 sees {1}.
    g = I.path(4)
    lab, t, _ = O.lpa_sync(g, 0.0, 1)
    assert lab.tolist() == [1, 0, 1, 2]
    lab, t, _ = O.lpa_sync(g, 0.0, 2)
    assert lab.tolist() == [0, 1, 0, 1]


def test_weights_override_counts_and_ties():
    # vertex 0 with neighbours 1 (weight a), 2 and 3 (weight 1 each);
    # labels 1 -> 1, 2 -> 2, 3 -> 2.  Label 1 weighs a, label 2 weighs 2.
    for a, want in [(3, 1), (2, 1), (1, 2)]:
        A = np.zeros((4, 4), dtype=np.int64)
        for j, w in [(1, a), (2, 1), (3, 1)]:
            A[0, j] = A[j, 0] = w
        g = graph_from_adj(A)
        nxt, _ = O.sync_sweep(g, np.array([0, 1, 2, 2], dtype=np.int32))
        assert nxt[0] == want, (a, nxt)


def test_self_loop_is_ignored_and_isolated_vertex_keeps_label():
    # vertex 0: self-loop of weight 10 plus edge to 1; vertex 2 isolated.
    A = np.zeros((3, 3), dtype=np.int64)
    A[0, 0] = 10
    A[0, 1] = A[1, 0] = 1
    g = graph_from_adj(A)
    nxt, dn = O.sync_sweep(g, np.array([0, 1, 2], dtype=np.int32))
    assert nxt.tolist() == [1, 0, 2] and dn == 2


# ---------------------------------------------------------- closed forms
@pytest.mark.parametrize("n", [3, 4, 7, 12])
def test_complete_graph(n):
    # K_n, sweep 1: 0 -> 1, others -> 0.  Sweep 2: everybody sees label 0 at
    # least as often as any other (n-2 >= 1 copies vs one copy of 1) -> 0.
    A = np.ones((n, n), dtype=np.int64) - np.eye(n, dtype=np.int64)
    g = graph_from_adj(A)
    lab, t, dn = O.lpa_sync(g, 0.0, 20)
    assert lab.tolist() == [0] * n and t == 3 and dn.tolist() == [n, 1, 0]


@pytest.mark.parametrize("n", [3, 5, 8])
def test_cycle_first_sweep(n):
    # C_n: i sees {i-1, i+1} (mod n), one each -> the smaller id.
    g = I.from_edges(n, [(i, (i + 1) % n) for i in range(n)])
    nxt, _ = O.sync_sweep(g, np.arange(n, dtype=np.int32))
    want = [min((i - 1) % n, (i + 1) % n) for i in range(n)]
    assert nxt.tolist() == want


@pytest.mark.parametrize("k", [1, 3, 6])
def test_star_oscillates(k):
    # star, centre 0, leaves 1..k: sweep 1 gives [1, 0, ..., 0]; sweep 2
    # gives [0, 1, ..., 1]; it alternates from then on.
    g = I.from_edges(k + 1, [(0, i) for i in range(1, k + 1)])
    a, _, _ = O.lpa_sync(g, 0.0, 1)
    b, _, _ = O.lpa_sync(g, 0.0, 2)
    c, _, _ = O.lpa_sync(g, 0.0, 3)
    assert a.tolist() == [1] + [0] * k
    assert b.tolist() == [0] + [1] * k
    assert c.tolist() == a.tolist()


# ------------------------------------------------ brute force against numpy
def test_all_graphs_on_5_vertices_one_sweep():
    n = 5
    pairs = list(itertools.combinations(range(n), 2))
    rng = np.random.default_rng(0)
    for mask in range(1 << len(pairs)):
        A = np.zeros((n, n), dtype=np.int64)
        for b, (i, j) in enumerate(pairs):
            if mask >> b & 1:
                A[i, j] = A[j, i] = 1
        g = graph_from_adj(A)
        for prev in (np.arange(n, dtype=np.int32), rng.integers(0, n, n).astype(np.int32)):
            nxt, dn = O.sync_sweep(g, prev)
            want = dense_sweep(A, prev)
            assert np.array_equal(nxt, want), (mask, prev, nxt, want)
            assert dn == int((want != prev).sum())


def test_random_weighted_multigraphs_one_sweep():
    rng = np.random.default_rng(1)
    for trial in range(300):
        n = int(rng.integers(1, 14))
        A = np.zeros((n, n), dtype=np.int64)
        for _ in range(int(rng.integers(0, 3 * n + 1))):
            i, j = rng.integers(0, n, 2)
            w = int(rng.integers(1, 5))
            A[i, j] += w
            if i != j:
                A[j, i] += w
        g = graph_from_adj(A)
        prev = rng.integers(0, max(n, 1), n).astype(np.int32)
        nxt, _ = O.sync_sweep(g, prev)
        assert np.array_equal(nxt, dense_sweep(A, prev)), trial


def test_duplicate_entries_count_separately():
    # a CSR row may repeat a neighbour; each entry adds its weight (Eq. 2 sums
    # over entries).  Row 0 holds 1, 1, 2 under labels 1, 1, 2: label 1 weighs
    # 2 and beats label 2 (weight 1).
    g = I.Graph(np.array([0, 3, 5, 6], dtype=np.int64), np.array([1, 1, 2, 0, 0, 0], dtype=np.int32))
    nxt, _ = O.sync_sweep(g, np.array([0, 1, 2], dtype=np.int32))
    assert nxt[0] == 1


def test_lpa_loop_matches_iterated_dense_sweeps():
    rng = np.random.default_rng(2)
    for trial in range(60):
        n = int(rng.integers(2, 16))
        g = I.random_graph(n, float(rng.uniform(0.1, 0.6)), seed=trial)
        A = dense(g)
        lab, t, dn = O.lpa_sync(g, 0.0, 12)
        cur = np.arange(n, dtype=np.int32)
        for s in range(t):
            nxt = dense_sweep(A, cur)
            assert int((nxt != cur).sum()) == dn[s]
            cur = nxt
        assert np.array_equal(cur, lab)


# ------------------------------------------ Algorithm 3 as printed (in place)
def test_sequential_in_place_path4_by_hand():
    # 0-1-2-3, ascending, in place: 0 -> 1 ([1,1,2,3]); 1 sees {1,2} tie -> 1,
    # no change; 2 sees {1,3} -> 1 ([1,1,1,3]); 3 sees {1} -> 1.  dN = 3.
    # Sweep 2 processes 1 (re-marked by 2) and 2 (re-marked by 3): no change.
    lab, t, dn = O.lpa_seq(I.path(4), 0.05, 20)
    assert lab.tolist() == [1, 1, 1, 1] and t == 2 and dn.tolist() == [3, 0]


def test_sequential_reactivation_by_hand():
    # path 2-0-3-1 (edges 0-2, 0-3, 1-3), tau = 0, in place, ascending.
    # Sweep 1: 0 sees {2,3} tie -> 2; 1 sees {3} -> 3; 2 sees {2} keeps;
    # 3 sees {2,3} tie -> 2 and re-marks 0 and 1.  dN = 3, C = [2,3,2,2].
    # Sweep 2: 0 keeps 2; 1 sees {2} -> 2 and re-marks 3; 3 keeps.  dN = 1.
    # Sweep 3: nothing is unprocessed, dN = 0.  Without the re-marking of
    # Algorithm 3 sweep 2 would process nothing and stop at [2,3,2,2].
    g = I.from_edges(4, [(0, 2), (0, 3), (1, 3)])
    lab, t, dn = O.lpa_seq(g, 0.0, 20)
    assert lab.tolist() == [2, 2, 2, 2] and dn.tolist() == [3, 1, 0] and t == 3


def test_sequential_converged_state_is_a_fixed_point():
    for seed in range(20):
        g = I.random_graph(30, 0.15, seed=seed)
        lab, t, dn = O.lpa_seq(g, 0.0, 100)
        if dn[-1] == 0:
            assert np.array_equal(dense_sweep(dense(g), lab), lab)


# --------------------------------------------------------- Algorithm 2 split
def test_split_path_by_hand():
    g = I.path(5)
    out = O.split_bfs(g, np.array([0, 0, 9, 0, 0], dtype=np.int32))
    assert out.tolist() == [0, 0, 2, 3, 3]


def test_split_equals_scipy_components():
    rng = np.random.default_rng(3)
    for trial in range(200):
        n = int(rng.integers(1, 40))
        g = I.random_graph(n, float(rng.uniform(0.02, 0.3)), seed=100 + trial)
        labels = rng.integers(0, max(1, n // 3 + 1), n).astype(np.int32)
        assert np.array_equal(O.split_bfs(g, labels), components_split(g, labels)), trial


def test_all_labelings_of_small_graphs_split():
    for n in range(1, 6):
        for seed in range(3):
            g = I.random_graph(n, 0.5, seed=seed)
            for labels in itertools.product(range(n), repeat=n):
                lab = np.array(labels, dtype=np.int32)
                assert np.array_equal(O.split_bfs(g, lab), components_split(g, lab))


def test_split_lp_and_lpp_reach_the_bfs_labels():
    # Algorithm 1's fixed point is the minimum id of each piece, the same
    # labelling Algorithm 2 produces with ascending start vertices.
    rng = np.random.default_rng(4)
    for trial in range(60):
        g = I.random_graph(int(rng.integers(2, 60)), 0.08, seed=200 + trial)
        labels = rng.integers(0, 4, g.n).astype(np.int32)
        want = components_split(g, labels)
        assert np.array_equal(O.split_lp(g, labels, pruning=False)[0], want)
        assert np.array_equal(O.split_lp(g, labels, pruning=True)[0], want)


# ----------------------------------------------------------- Eq. 1 modularity
def test_modularity_two_k5_closed_form():
    # 2m = 42, sigma_c = 20 for both cliques, Sigma_c = 21 for both:
    # Q = 40/42 - 2 (21/42)^2 = 19/42.
    g = I.two_cliques_bridge(5)
    lab, _, _ = O.lpa_sync(g, 0.05, 20)
    q, (two_m, s1, s2) = O.modularity(g, lab, parts=True)
    assert (two_m, s1, s2) == (42, 40, 2 * 21 * 21)
    assert q == pytest.approx(19 / 42, abs=1e-15)


def test_modularity_path_split_by_hand():
    g = I.path(5)
    assert O.modularity(g, np.array([0, 0, 4, 0, 0], dtype=np.int32)) == pytest.approx(-0.125, abs=1e-15)
    assert O.modularity(g, np.array([0, 0, 2, 3, 3], dtype=np.int32)) == pytest.approx(0.15625, abs=1e-15)


def test_modularity_special_cases():
    g = I.random_graph(50, 0.1, seed=7)
    assert O.modularity(g, np.zeros(g.n, dtype=np.int32)) == pytest.approx(0.0, abs=1e-15)
    deg = np.diff(g.offsets).astype(np.float64)
    single = O.modularity(g, np.arange(g.n, dtype=np.int32))
    assert single == pytest.approx(-(deg ** 2).sum() / deg.sum() ** 2, abs=1e-15)
    empty = I.Graph(np.zeros(4, dtype=np.int64), np.zeros(0, dtype=np.int32))
    assert O.modularity(empty, np.arange(3, dtype=np.int32)) == 0.0


def test_modularity_matches_networkx_and_pair_sum():
    nx = pytest.importorskip("networkx")
    rng = np.random.default_rng(5)
    for trial in range(40):
        n = int(rng.integers(2, 40))
        g = I.random_graph(n, float(rng.uniform(0.05, 0.4)), seed=300 + trial)
        if g.nnz == 0:
            continue
        g.weights = I.symmetric_weights(g, seed=trial, wmax=7)
        labels = rng.integers(0, max(1, n // 4), n).astype(np.int32)
        q = O.modularity(g, labels)
        G = nx.Graph()
        G.add_nodes_from(range(n))
        src = np.repeat(np.arange(n), np.diff(g.offsets))
        for a, b, w in zip(src, g.cols, g.weights):
            if a < b:
                G.add_edge(int(a), int(b), weight=int(w))
        comms = [set(np.nonzero(labels == c)[0].tolist()) for c in np.unique(labels)]
        assert q == pytest.approx(nx.community.modularity(G, comms, weight="weight"), abs=1e-12)
        # first form of Eq. 1 over all ordered pairs: (1/2m) sum [A_ij - K_i K_j / 2m] delta
        A = dense(g).astype(np.float64)
        K = A.sum(axis=1)
        two_m = K.sum()
        delta = labels[:, None] == labels[None, :]
        assert q == pytest.approx(((A - np.outer(K, K) / two_m) * delta).sum() / two_m, abs=1e-12)
        assert -0.5 <= q <= 1.0


# ---------------------------------------------------------- Algorithm 4
def test_disconnected_checker_by_hand_and_vs_scipy():
    g = I.path(5)
    k, D = O.disconnected(g, np.array([0, 0, 2, 0, 0], dtype=np.int32))
    assert k == 1 and D[0] == 1 and D.sum() == 1
    rng = np.random.default_rng(6)
    for trial in range(100):
        g = I.random_graph(int(rng.integers(1, 50)), 0.1, seed=400 + trial)
        labels = rng.integers(0, min(5, g.n), g.n).astype(np.int32)
        pieces = components_split(g, labels)
        want = sum(1 for c in np.unique(labels) if np.unique(pieces[labels == c]).size > 1)
        assert O.disconnected(g, labels)[0] == want


# ---------------------------------------------------------- invariants I1-I5
@pytest.mark.parametrize("maker", [
    lambda: I.sbm_planted(2000, 100, 12.0, 3.0, seed=3),
    lambda: I.rmat(11, 8, seed=2),
    lambda: I.lattice_chains(40, 40, n_chains=50, seed=4),
])
def test_invariants_of_gsl_lpa(maker):
    g = maker()
    lab, t, dn = O.lpa_sync(g, 0.05, 20)
    out = O.split_bfs(g, lab)
    v = np.arange(g.n)
    assert O.disconnected(g, out)[0] == 0                               # I1
    src = np.repeat(v, np.diff(g.offsets))
    assert np.array_equal(out[src] == out[g.cols], lab[src] == lab[g.cols])  # I2: refines, cuts no intra edge
    assert (out <= v).all() and np.array_equal(out[out], out)           # I3
    assert O.modularity(g, out) >= O.modularity(g, lab) - 1e-12         # I5


def test_pruned_frontier_reading_is_exact():
    # Eq. 2 depends on neighbour labels only: recomputing only the vertices
    # next to a change (and the changed vertices) gives the same labels as
    # recomputing everything.
    rng = np.random.default_rng(8)
    for trial in range(20):
        g = I.random_graph(int(rng.integers(5, 80)), 0.08, seed=500 + trial)
        A = dense(g)
        cur = np.arange(g.n, dtype=np.int32)
        frontier = np.ones(g.n, dtype=bool)
        for _ in range(8):
            full = dense_sweep(A, cur)
            part = np.where(frontier, full, cur)
            assert np.array_equal(part, full)
            changed = part != cur
            frontier = changed | ((A > 0) & changed[None, :]).any(axis=1)
            cur = part


def test_sampled_sweep_equals_full_sweep_on_the_sample():
    rng = np.random.default_rng(21)
    for seed in range(4):
        g = I.rmat(9, 8, seed=seed)
        w = I.symmetric_weights(g, seed, 5) if seed % 2 else None
        h = I.Graph(g.offsets, g.cols, w)
        prev = rng.integers(0, g.n // 8, g.n).astype(np.int32)
        full, _ = O.sync_sweep(h, prev)
        sel = rng.permutation(g.n)[:100]
        assert np.array_equal(O.sync_sweep_at(h, prev, sel), full[sel])
    with pytest.raises(ValueError):
        O.sync_sweep_at(h, prev, [g.n])


# --------------------------------------- float32 weights with float64 sums
def dense_float_sweep(g, wf, prev):
    n = g.n
    A = np.zeros((n, n), dtype=np.float64)
    src = np.repeat(np.arange(n), np.diff(g.offsets))
    np.add.at(A, (src, g.cols), wf.astype(np.float64))
    np.fill_diagonal(A, 0.0)
    Y = np.zeros((n, n), dtype=np.float64)
    Y[np.arange(n), prev] = 1.0
    S = A @ Y
    has = A.sum(axis=1) > 0
    return np.where(has, np.argmax(S, axis=1), prev).astype(np.int32), S


def test_float_sweep_matches_dense_product():
    rng = np.random.default_rng(41)
    for trial in range(60):
        n = int(rng.integers(2, 30))
        g = I.random_graph(n, float(rng.uniform(0.1, 0.6)), seed=500 + trial)
        if g.nnz == 0:
            continue
        prev = rng.integers(0, max(1, n // 3), n).astype(np.int32)
        wf = float_weights(g, trial, dyadic=True)   # exact sums: the argmax is exact too
        got, dn = O.sync_sweep_f32(g, wf, prev)
        want, _ = dense_float_sweep(g, wf, prev)
        assert np.array_equal(got, want) and dn == int((got != prev).sum())
        wf = float_weights(g, trial, dyadic=False)  # rounding may differ: compare clear winners only
        got, _ = O.sync_sweep_f32(g, wf, prev)
        want, S = dense_float_sweep(g, wf, prev)
        top2 = -np.sort(-S, axis=1)[:, :2] if n > 1 else np.zeros((n, 2))
        clear = (top2[:, 0] - top2[:, 1]) > 1e-9 * np.maximum(1.0, top2[:, 0])
        assert np.array_equal(got[clear], want[clear])


def test_float_self_loop_is_ignored_by_hand():
    # vertex 0: self-loop of weight 10 plus edge to 1 (weight 0.5); vertex 2 isolated
    A = np.zeros((3, 3), dtype=np.int64)
    A[0, 0] = 10
    A[0, 1] = A[1, 0] = 1
    g = graph_from_adj(A)
    wf = np.where(g.cols == np.repeat(np.arange(3), np.diff(g.offsets)), 10.0, 0.5).astype(np.float32)
    nxt, dn = O.sync_sweep_f32(g, wf, np.array([0, 1, 2], dtype=np.int32))
    assert nxt.tolist() == [1, 0, 2] and dn == 2


def test_float_lpa_with_integer_weights_equals_integer_lpa():
    for seed in range(4):
        g = I.rmat(9, 8, seed=seed)
        wi = I.symmetric_weights(g, seed, 6)
        h = I.Graph(g.offsets, g.cols, wi)
        lab_i, t_i, dn_i = O.lpa_sync(h, 0.05, 20)
        lab_f, t_f, dn_f = O.lpa_sync_f32(g, wi.astype(np.float32), 0.05, 20)
        assert t_i == t_f and np.array_equal(lab_i, lab_f) and np.array_equal(dn_i, dn_f)
        assert O.modularity_f64(g, wi.astype(np.float32), lab_i) == pytest.approx(O.modularity(h, lab_i), abs=1e-12)


def test_float_lpa_with_dyadic_weights_equals_integer_lpa_on_scaled_weights():
    """Weights that are multiples of 2^-S with small row totals: every float64
    partial sum is exact, so the float oracle's labels equal the integer
    oracle's on the weights times 2^S (the form the library runs such
    weights in).  S = 3 (k/8) and S = 20 (1 + k/2^20)."""
    rng = np.random.default_rng(5)
    for g in (I.sbm_planted(3000, 60, 10.0, 2.0, seed=6), I.rmat(11, 8, seed=4)):
        src = np.repeat(np.arange(g.n), np.diff(g.offsets))
        key = np.minimum(src, g.cols).astype(np.int64) * g.n + np.maximum(src, g.cols)
        uniq, inv = np.unique(key, return_inverse=True)
        for shift, vals in ((3, rng.integers(1, 33, uniq.shape[0]) / 8.0),
                            (20, 1.0 + rng.integers(0, 1 << 20, uniq.shape[0]) / float(1 << 20))):
            wf = vals[inv].astype(np.float32)
            wi = (wf.astype(np.float64) * (1 << shift)).astype(np.int64)
            assert np.array_equal(wi.astype(np.float64), wf.astype(np.float64) * (1 << shift))
            assert wi.max() < (1 << 31)
            gi = I.Graph(g.offsets, g.cols, wi.astype(np.int32), name=g.name + "-scaled")
            lf, tf, dnf = O.lpa_sync_f32(g, wf, 0.05, 20)
            li, ti, dni = O.lpa_sync(gi, 0.05, 20)
            assert tf == ti and np.array_equal(dnf, dni) and np.array_equal(lf, li), (g.name, shift)


def test_own_label_majority_keeps_the_label():
    """The own-label majority shortcut: a vertex whose own label holds more
    than half of its row's weight (the vertex itself excluded) keeps it in
    a synchronous sweep; so does one whose own label holds more than half of
    an upper bound of that weight -- its entry count d with unit weights, or
    its weighted degree including self-loops.  Checked on random labellings
    concentrated enough that many vertices qualify."""
    rng = np.random.default_rng(12)
    base = I.rmat(10, 12, seed=7)
    for w in (False, True):
        wi = I.symmetric_weights(base, 3, 9) if w else np.ones(base.nnz, np.int32)
        g = I.Graph(base.offsets, base.cols, wi if w else None)
        src = np.repeat(np.arange(g.n), np.diff(g.offsets))
        checked = 0
        for trial in range(6):
            prev = rng.integers(0, 3 + trial, g.n).astype(np.int32)
            nxt, _ = O.sync_sweep(g, prev)
            same = prev[g.cols] == prev[src]
            notself = g.cols != src
            own = np.bincount(src, weights=wi * (same & notself), minlength=g.n)
            tot = np.bincount(src, weights=wi * notself, minlength=g.n)
            bound = np.bincount(src, weights=wi, minlength=g.n)   # includes self-loop entries
            for cond in (2 * own > tot, 2 * own > bound):
                assert np.array_equal(nxt[cond], prev[cond])
                checked += int(cond.sum())
        assert checked > 100


def test_first_sweep_of_increasing_rows_takes_the_first_other_entry():
    """Reading 12: from the identity labels with unit weights, a strictly
    increasing row holds every label once, so Eq. 2's tie rule picks its
    smallest neighbour other than the vertex: the first entry, or the second
    when the first is a self-loop."""
    g0 = I.rmat(11, 8, seed=8)
    # add self-loops to a few rows, keeping them strictly increasing
    rng = np.random.default_rng(8)
    pick = set(rng.choice(g0.n, 40, replace=False).tolist())
    rows = []
    for v in range(g0.n):
        r = g0.cols[g0.offsets[v]:g0.offsets[v + 1]]
        if v in pick:
            r = np.unique(np.append(r, v))
        rows.append(r.astype(np.int32))
    off = np.concatenate([[0], np.cumsum([len(r) for r in rows])]).astype(np.int64)
    g = I.Graph(off, np.concatenate(rows))
    got, _ = O.sync_sweep(g, np.arange(g.n, dtype=np.int32))
    want = np.arange(g.n, dtype=np.int32)
    for v in range(g.n):
        r = g.cols[g.offsets[v]:g.offsets[v + 1]]
        assert (np.diff(r) > 0).all()
        r = r[r != v]
        if r.size:
            want[v] = r[0]
    assert np.array_equal(got, want)


def test_float_modularity_matches_networkx():
    nx = pytest.importorskip("networkx")
    rng = np.random.default_rng(43)
    for trial in range(30):
        n = int(rng.integers(2, 40))
        g = I.random_graph(n, float(rng.uniform(0.05, 0.4)), seed=700 + trial)
        if g.nnz == 0:
            continue
        wf = float_weights(g, trial, dyadic=False)
        labels = rng.integers(0, max(1, n // 4), n).astype(np.int32)
        G = nx.Graph()
        G.add_nodes_from(range(n))
        src = np.repeat(np.arange(n), np.diff(g.offsets))
        for a, b, w in zip(src, g.cols, wf):
            if a < b:
                G.add_edge(int(a), int(b), weight=float(w))
        comms = [set(np.nonzero(labels == c)[0].tolist()) for c in np.unique(labels)]
        assert O.modularity_f64(g, wf, labels) == pytest.approx(nx.community.modularity(G, comms, weight="weight"),
                                                                abs=1e-12)


def test_float_weights_must_be_finite_and_positive():
    g = I.path(4)
    for bad in (0.0, -1.0, np.nan, np.inf):
        wf = np.ones(g.nnz, dtype=np.float32)
        wf[1] = bad
        with pytest.raises(ValueError):
            O.sync_sweep_f32(g, wf, np.arange(4, dtype=np.int32))
