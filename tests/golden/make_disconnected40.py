"""Writes disconnected40.txt: a 40-vertex graph on which synchronous LPA
(tolerance 0.05, at most 20 sweeps) leaves at least one community internally
disconnected -- the situation of Fig. 1 (a vertex that held its community
together moves to a heavier neighbouring label).  The drawing of Fig. 1 is not
available, so the graph is the first hit of a seeded search over 40-vertex
planted-partition graphs, and the expected labels are the oracle's.

Run from the repository root:  python tests/golden/make_disconnected40.py
Calls only inputs/ (graph candidates) and oracle/ (labels).
"""
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import inputs as I  # noqa: E402
import oracle as O  # noqa: E402

P_IN, P_OUT = 0.4, 0.08
OUT = os.path.join(os.path.dirname(os.path.abspath(__file__)), "disconnected40.txt")


def search():
    for seed in range(100000):
        nb = 4 + seed % 5
        bs = (np.arange(nb + 1, dtype=np.int64) * 40) // nb
        g = I.sbm(40, bs, P_IN, P_OUT, seed=seed, threads=1)
        lab, t, dn = O.lpa_sync(g, 0.05, 20)
        k, _ = O.disconnected(g, lab)
        if k >= 1 and t < 20:   # stopped by the tolerance test, still disconnected
            return seed, nb, g, lab, t, dn
    raise RuntimeError("no hit")


def main():
    seed, nb, g, lab, t, dn = search()
    out = O.split_bfs(g, lab)
    k_before, _ = O.disconnected(g, lab)
    k_after, _ = O.disconnected(g, out)
    q_before, q_after = O.modularity(g, lab), O.modularity(g, out)
    src = np.repeat(np.arange(g.n), np.diff(g.offsets))
    edges = [(int(a), int(b)) for a, b in zip(src, g.cols) if a < b]
    with open(OUT, "w") as f:
        f.write("# 40-vertex graph where synchronous LPA leaves a community disconnected (cf. Fig. 1).\n")
        f.write("# Written by tests/golden/make_disconnected40.py from inputs.sbm(40, %d equal blocks,\n" % nb)
        f.write("# p_in=%g, p_out=%g, seed=%d); labels are the CPU oracle's (Algorithm 3, Algorithm 2).\n" % (P_IN, P_OUT, seed))
        f.write("n 40\n")
        f.write("tolerance 0.05\nmax_iters 20\n")
        f.write("sweeps %d\n" % t)
        f.write("dn %s\n" % " ".join(str(int(x)) for x in dn))
        f.write("disconnected_before %d\ndisconnected_after %d\n" % (k_before, k_after))
        f.write("modularity_before %.17g\nmodularity_after %.17g\n" % (q_before, q_after))
        f.write("lpa %s\n" % " ".join(str(int(x)) for x in lab))
        f.write("split %s\n" % " ".join(str(int(x)) for x in out))
        for a, b in edges:
            f.write("e %d %d\n" % (a, b))
    print("seed", seed, "blocks", nb, "sweeps", t, "dN", dn.tolist(), "disconnected", k_before, "->", k_after)


if __name__ == "__main__":
    main()
