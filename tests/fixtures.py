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
