"""Contexts with different block shapes used from several host threads at
once (as the server's workers do): each thread's results equal the
oracle's.  The launch caches and shared-memory limits are shared by the
process, so this exercises them under concurrency."""
import threading

import numpy as np
import pytest
import torch

import inputs as I
import oracle as O

pytestmark = pytest.mark.gpu
DEV = "cuda:0"


def _graph():
    rng = np.random.default_rng(11)
    base = I.sbm_planted(60_000, 300, 12.0, 3.0, seed=11)
    src = np.repeat(np.arange(base.n), np.diff(base.offsets))
    keep = src < base.cols
    u, v = [src[keep]], [base.cols[keep]]
    for h, deg in enumerate((45_000, 20_000, 3_000)):
        nb = rng.choice(base.n, deg, replace=False)
        u.append(np.full(deg, base.n + h))
        v.append(nb)
    return I.csr_from_pairs(base.n + 3, np.concatenate(u), np.concatenate(v), name="sbm60k-hubs")


def test_contexts_on_several_threads(gpu_lib):
    g = _graph()
    want = O.gsl_lpa(g, 0.05, 20)[0]
    shapes = [(512, 12288), (256, 6144), (128, 2048), (512, 8192)]
    errors = []

    def work(shape):
        try:
            c = gpu_lib.Context(0)
            c.set_block_config(*shape)
            stream = torch.cuda.Stream(device=DEV)
            with torch.cuda.stream(stream):
                off = torch.from_numpy(g.offsets).to(DEV)
                col = torch.from_numpy(g.cols).to(DEV)
                for _ in range(4):
                    got = c.gsllpa(off, col, stream=stream)
                    stream.synchronize()
                    if not np.array_equal(got.cpu().numpy(), want):
                        errors.append(("labels differ", shape))
        except Exception as e:   # noqa: BLE001 -- reported below
            errors.append((repr(e), shape))

    threads = [threading.Thread(target=work, args=(s,)) for s in shapes]
    for t in threads:
        t.start()
    for t in threads:
        t.join()
    assert not errors, errors
