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
