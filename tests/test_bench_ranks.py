"""The benchmark's multi-rank host path, run as two gloo ranks on the CPU.

Under torchrun every rank solves its own replica of the workload: rank 0
generates the graph into the cache while the others wait at a barrier,
every rank then reads the same files, the step time is the maximum over
ranks and the value counts every rank's units.  No GPU is involved.
"""
import json
import os
import socket
import subprocess
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

WORKER = r"""
import json, os, sys
sys.path.insert(0, sys.argv[1])
import numpy as np
import torch.distributed as dist
import bench
rank, world, local = bench.rank_env()
dist.init_process_group("gloo")
off, col = bench.workload_graph(9, 8, sys.argv[2], rank, world)
ms = bench.max_over_ranks(10.0 + 5.0 * rank, world)
out = {"rank": rank, "world": world, "n": int(off.shape[0] - 1), "nnz": int(col.shape[0]),
       "sum": int(np.asarray(col, dtype=np.int64).sum()), "ms": ms,
       "value": bench.replicas_value(world, int(col.shape[0]), ms)}
with open(os.path.join(sys.argv[2], f"rank{rank}.json"), "w") as f:
    json.dump(out, f)
dist.barrier()
dist.destroy_process_group()
"""


def free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def test_two_gloo_ranks_share_the_workload_and_take_the_slowest_time(tmp_path):
    pytest.importorskip("torch.distributed")
    script = tmp_path / "worker.py"
    script.write_text(WORKER)
    port = free_port()
    procs = []
    for rank in range(2):
        env = dict(os.environ, RANK=str(rank), WORLD_SIZE="2", LOCAL_RANK=str(rank), MASTER_ADDR="127.0.0.1",
                   MASTER_PORT=str(port))
        procs.append(subprocess.Popen([sys.executable, str(script), ROOT, str(tmp_path)], env=env))
    for p in procs:
        assert p.wait(timeout=300) == 0
    res = [json.load(open(tmp_path / f"rank{r}.json")) for r in range(2)]
    assert res[0]["n"] == res[1]["n"] == 512 and res[0]["nnz"] == res[1]["nnz"] > 0
    assert res[0]["sum"] == res[1]["sum"]                  # the same replica on every rank
    assert res[0]["ms"] == res[1]["ms"] == 15.0              # the slowest rank's time
    assert res[0]["value"] == pytest.approx(2 * res[0]["nnz"] / 15e-3)


def test_single_rank_helpers():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(3.5, 1) == 3.5
    assert bench.replicas_value(4, 1000, 2.0) == pytest.approx(2e6)


def test_reference_arm_on_other_ranks_exits_without_work(monkeypatch, capsys):
    sys.path.insert(0, ROOT)
    import bench
    monkeypatch.setenv("RANK", "1")
    monkeypatch.setenv("WORLD_SIZE", "2")

    class Args:
        pass
    assert bench.run_reference(Args()) == 0
    assert capsys.readouterr().out == ""
