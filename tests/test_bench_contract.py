"""The benchmark's reference arm (the CPU oracle timed on the host) prints
one JSON line with the keys the benchmark contract names; it needs no GPU."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_reference_arm_json_line(tmp_path):
    env = dict(os.environ, GSL_BENCH_CACHE=str(tmp_path))
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
                        "--warmup", "0"], capture_output=True, text=True, timeout=600, env=env, cwd=ROOT)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [l for l in r.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference"
    for k in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "higher_is_better", "scaling", "vs_baseline",
              "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert k in d, k
    assert d["value"] > 0 and d["unit"] == "edges/s" and d["higher_is_better"] is True
    assert d["steps"] == 1 and d["warmup"] == 0 and d["n_gpus"] == 1
    assert "workload" in d["config"]
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["value"] == d["value"] and cb["sample"]
    assert d["e2e"] == {"value": d["value"], "unit": d["unit"], "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}


def _bench():
    sys.path.insert(0, ROOT)
    import bench
    return bench


def _slot(name, ms, nbytes, launches=1):
    return {"name": name, "ms": ms, "bytes": nbytes, "launches": launches, "kernels": launches, "vertices": 0,
            "entries": 0}


def test_dominant_roofline_arithmetic(monkeypatch):
    """The slot with the largest device time is the dominant one; achieved
    = its algorithmic bytes over its time, frac = achieved / peak; slots
    without bytes are ignored."""
    b = _bench()
    from paper_2403_01261_gb300 import _build
    monkeypatch.setattr(_build, "source_hash", lambda: "no-such-hash")
    prof = [_slot("sweep_block", 20.0, 40e9, launches=4), _slot("sweep_hub", 10.0, 50e9), _slot("idle", 30.0, 0.0)]
    r = b.dominant_roofline(prof, (1000.0, "measured"))
    assert r["kernel"] == "sweep_block" and r["bound"] == "hbm" and r["unit"] == "GB/s"
    assert abs(r["achieved"] - 2000.0) < 1e-9 and abs(r["frac"] - 2.0) < 1e-12
    assert r["bytes_per_launch"] == 10e9 and r["ms_per_launch"] == 5.0 and r["launches"] == 4
    assert r["traffic"] is None and r["peak_source"] == "measured"
    assert b.dominant_roofline([_slot("x", 0.0, 1.0)], (1.0, "fallback")) is None


def test_roofline_traffic_only_for_the_profiled_library(monkeypatch):
    """profiles/traffic.json is used only when its source hash is the built
    library's; any other hash gives traffic null."""
    b = _bench()
    from paper_2403_01261_gb300 import _build
    rec = json.load(open(os.path.join(ROOT, "profiles", "traffic.json")))
    prof = [_slot("sweep_block", 10.0, 1e9)]
    monkeypatch.setattr(_build, "source_hash", lambda: rec["source_hash"])
    assert b.dominant_roofline(prof, (1.0, "measured"))["traffic"] == rec["per_launch"]["sweep_block"]
    monkeypatch.setattr(_build, "source_hash", lambda: rec["source_hash"] + "x")
    assert b.dominant_roofline(prof, (1.0, "measured"))["traffic"] is None


def test_phase_roofline_split_and_step():
    """The sweep phase counts every slot but the split and modularity; the
    step counts every slot but modularity over the measured step time."""
    b = _bench()
    prof = [_slot("sweep_block", 4.0, 8e9), _slot("majority_filter", 6.0, 2e9), _slot("split_unionfind", 5.0, 5e9),
            _slot("split_count_renumber", 1.0, 1e9), _slot("modularity", 2.0, 9e9)]
    r = b.phase_roofline(prof, 100.0, steps=2, step_ms=10.0)
    assert abs(r["sweep_phase"]["achieved"] - 1000.0) < 1e-9          # 10 GB over 10 ms
    assert r["sweep_phase"]["bytes_per_step"] == 5e9 and r["sweep_phase"]["ms_per_step"] == 5.0
    assert abs(r["sweep_phase"]["frac"] - 10.0) < 1e-12
    assert abs(r["step"]["achieved"] - 800.0) < 1e-9                  # 16 GB / 2 steps over 10 ms
    assert r["step"]["bytes_per_step"] == 8e9 and r["step"]["ms_per_step"] == 10.0
    assert b.phase_roofline([], 1.0, steps=1, step_ms=0.0) == {}


def test_pack_graphs_is_the_disjoint_union():
    """The batched workload's packing: graph k's vertices are vptr[k]..,
    its rows and columns shifted by its vertex and entry offsets; graphs
    with no vertex or no entry keep their place; connected components of
    the union never cross graphs."""
    import numpy as np
    import inputs as I
    b = _bench()
    parts = [I.path(4), I.from_edges(3, [], name="empty"), I.from_edges(0, [], name="none"), I.two_cliques_bridge(5)]
    off, col, vptr = b.pack_graphs([(g.offsets, g.cols) for g in parts])
    assert vptr.tolist() == [0, 4, 7, 7, 17]
    assert off.shape[0] == 18 and off[0] == 0 and off[-1] == col.shape[0] == sum(g.cols.shape[0] for g in parts)
    for k, g in enumerate(parts):
        v0, v1 = int(vptr[k]), int(vptr[k + 1])
        assert np.array_equal(off[v0:v1 + 1] - off[v0], g.offsets)
        seg = col[off[v0]:off[v1]]
        assert np.array_equal(seg - v0, g.cols) and ((seg >= v0) & (seg < v1)).all()
