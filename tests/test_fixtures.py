"""The 40-vertex fixture: synchronous LPA leaves a community disconnected
(the situation of Fig. 1) and the split of Algorithm 2 repairs it."""
import numpy as np
from scipy.sparse.csgraph import connected_components
import scipy.sparse as sp

import oracle as O
from fixtures import load_disconnected40


def _pieces(g, labels):
    src = np.repeat(np.arange(g.n), np.diff(g.offsets))
    keep = labels[src] == labels[g.cols]
    M = sp.csr_matrix((np.ones(keep.sum()), (src[keep], g.cols[keep])), shape=(g.n, g.n))
    return connected_components(M, directed=False)


def test_fixture_is_disconnected_then_repaired():
    g, rec = load_disconnected40()
    lab = rec["lpa"].astype(np.int32)
    # independent of the oracle: count communities whose intra-community
    # subgraph has more than one connected component
    k, comp = _pieces(g, lab)
    split_comms = sum(1 for c in np.unique(lab) if np.unique(comp[lab == c]).size > 1)
    assert split_comms == rec["disconnected_before"] >= 1
    out = rec["split"].astype(np.int32)
    k2, comp2 = _pieces(g, out)
    assert all(np.unique(comp2[out == c]).size == 1 for c in np.unique(out))


def test_oracle_reproduces_fixture():
    g, rec = load_disconnected40()
    lab, t, dn = O.lpa_sync(g, rec["tolerance"], rec["max_iters"])
    assert t == rec["sweeps"] and np.array_equal(dn, rec["dn"]) and np.array_equal(lab, rec["lpa"])
    assert np.array_equal(O.split_bfs(g, lab), rec["split"])
    assert O.modularity(g, O.split_bfs(g, lab)) == rec["modularity_after"]
