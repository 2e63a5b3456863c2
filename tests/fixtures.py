"""Loaders for the text fixtures under tests/golden/."""
import os

import numpy as np

import inputs as I

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def load_disconnected40():
    """The 40-vertex graph of disconnected40.txt and its recorded values."""
    rec = {"edges": []}
    with open(os.path.join(GOLDEN, "disconnected40.txt")) as f:
        for line in f:
            if line.startswith("#") or not line.strip():
                continue
            key, *vals = line.split()
            if key == "e":
                rec["edges"].append((int(vals[0]), int(vals[1])))
            elif key in ("lpa", "split", "dn"):
                rec[key] = np.array([int(v) for v in vals], dtype=np.int64)
            elif key in ("modularity_before", "modularity_after", "tolerance"):
                rec[key] = float(vals[0])
            else:
                rec[key] = int(vals[0])
    g = I.from_edges(rec["n"], rec["edges"], name="disconnected40")
    return g, rec


def float_weights(g, seed, dyadic=True):
    """Symmetric float32 weights: multiples of 1/8 in [0.125, 4] (sums exact
    in float64 in any order) or arbitrary values in (0.01, 3)."""
    rng = np.random.default_rng(seed)
    src = np.repeat(np.arange(g.n), np.diff(g.offsets))
    lo = np.minimum(src, g.cols).astype(np.int64)
    hi = np.maximum(src, g.cols).astype(np.int64)
    key = lo * g.n + hi
    uniq, inv = np.unique(key, return_inverse=True)
    vals = (rng.integers(1, 33, uniq.shape[0]) / 8.0) if dyadic else rng.uniform(0.01, 3.0, uniq.shape[0])
    return vals[inv].astype(np.float32)


# ------------------------------------------------------------------
# Oracle jobs for process pools (spawn context).  They build their own
# graph (loaded from the benchmark's .npy cache or generated from its
# seed), so that nothing but a small spec crosses the process boundary.
def graph_from_spec(spec):
    """spec = ("npy", offsets_path, cols_path, name) | ("lattice",) | ("batched", g)."""
    if spec[0] == "npy":
        return I.Graph(np.load(spec[1], mmap_mode="r"), np.load(spec[2], mmap_mode="r"), name=spec[3])
    if spec[0] == "lattice":
        return I.lattice_chains(threads=4)
    if spec[0] == "batched":
        return I.batched_sbm(spec[1], threads=1)
    raise ValueError(spec)


def oracle_job(spec, kind, tol=0.05, max_iters=20):
    """kind "sync": Algorithm 3 with Jacobi sweeps then Algorithm 2 ->
    (lpa labels, sweeps, dN per sweep, split labels, Q of the split labels);
    kind "seq": Algorithm 3 as printed (one thread, in place) then
    Algorithm 2 -> the same tuple."""
    import oracle as O
    g = graph_from_spec(spec)
    fn = O.lpa_sync if kind == "sync" else O.lpa_seq
    lab, t, dn = fn(g, tol, max_iters)
    split = O.split_bfs(g, lab)
    return lab, t, dn, split, O.modularity(g, split)


def oracle_batched_check(job):
    """Graphs k0..k1-1 of the batched workload through the oracle (GSL-LPA:
    Jacobi LPA then Algorithm 2), compared with the GPU's labels stored in
    the .npy file at labels_path (local ids, graph k at vptr[k]..vptr[k+1])
    and its sweep counts.  Returns [(k, oracle sweeps, labels equal,
    sweeps equal)]."""
    import oracle as O
    k0, k1, labels_path, vptr, iters = job
    lab = np.load(labels_path, mmap_mode="r")
    out = []
    for k in range(k0, k1):
        g = I.batched_sbm(k, threads=1)
        assert g.n == vptr[k + 1 - k0] - vptr[k - k0], k
        want, t, _ = O.gsl_lpa(g, 0.05, 20)
        got = lab[vptr[k - k0]:vptr[k + 1 - k0]]
        out.append((k, t, bool(np.array_equal(got, want)), int(iters[k - k0]) == t))
    return out


def record(kind, **fields):
    """Appends one JSON line to the file named by GSL_TEST_RECORD (when set):
    measured values that a test checks and a reader may want to cite."""
    import json
    path = os.environ.get("GSL_TEST_RECORD")
    if not path:
        return
    with open(path, "a") as f:
        f.write(json.dumps({"kind": kind, **fields}) + "\n")
