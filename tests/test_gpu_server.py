"""Request server: continuous batching returns each graph's solo result,
alone and in a mix of concurrent requests."""
import threading

import numpy as np
import pytest

import inputs as I
import oracle as O

pytestmark = pytest.mark.gpu


def pool(seed=0, count=40):
    rng = np.random.default_rng(seed)
    gs = []
    for k in range(count):
        if k % 3 == 0:
            gs.append(I.batched_sbm(k, n_lo=100, n_hi=20000))
        elif k % 3 == 1:
            gs.append(I.rmat(int(rng.integers(8, 14)), 16, seed=k))
        else:
            gs.append(I.random_graph(int(rng.integers(1, 200)), 0.05, seed=k))
    return gs


def test_server_results_equal_solo_oracle(gpu_lib):
    gs = pool()
    want = [O.gsl_lpa(g, 0.05, 20)[0] for g in gs]
    srv = gpu_lib.Server(slots=3, slot_vertices=60_000, slot_entries=2_000_000, max_batch_graphs=8)
    # alone: one request at a time
    for g, w in zip(gs[:6], want[:6]):
        rid = srv.submit(g.offsets, g.cols)
        assert np.array_equal(srv.wait(rid), w)
    # in the mix: all requests from several submitting threads at once
    ids = [None] * len(gs)

    def submit(part):
        for k in part:
            ids[k] = srv.submit(gs[k].offsets, gs[k].cols)

    th = [threading.Thread(target=submit, args=(range(p, len(gs), 4),)) for p in range(4)]
    for t in th:
        t.start()
    for t in th:
        t.join()
    infos = []
    for k, rid in enumerate(ids):
        lab, info = srv.wait(rid, info=True)
        assert np.array_equal(lab, want[k]), gs[k].name
        infos.append(info)
    st = srv.stats()
    assert st["completed"] == len(gs) + 6 and st["queued"] == 0
    assert max(i["batch_graphs"] for i in infos) > 1          # requests were batched together
    assert st["max_concurrent_batches"] >= 1
    srv.close()


def test_server_rejects_graph_that_never_fits(gpu_lib):
    srv = gpu_lib.Server(slots=1, slot_vertices=100, slot_entries=1000)
    g = I.path(500)
    with pytest.raises(gpu_lib.GslError) as e:
        srv.submit(g.offsets, g.cols)
    assert e.value.code == 3
    small = I.path(50)
    assert np.array_equal(srv.wait(srv.submit(small.offsets, small.cols)), O.gsl_lpa(small, 0.05, 20)[0])
    srv.close()


def test_server_async_mode_invariants(gpu_lib):
    gs = pool(seed=3, count=12)
    srv = gpu_lib.Server(slots=2, slot_vertices=60_000, slot_entries=2_000_000, mode=1)
    ids = [srv.submit(g.offsets, g.cols) for g in gs]
    for g, rid in zip(gs, ids):
        lab = srv.wait(rid)
        v = np.arange(g.n)
        assert (lab <= v).all() and np.array_equal(lab[lab], lab)
        assert O.disconnected(g, lab)[0] == 0
    srv.close()


def test_server_large_requests_run_alone(gpu_lib):
    """A request of 2^22 entries or more runs alone through the single-graph
    path, between batched small ones; every result is its solo result."""
    big = I.rmat(17, 24, seed=8)
    assert big.nnz >= 1 << 22
    small = [I.batched_sbm(k, n_lo=500, n_hi=3000) for k in range(6)]
    gs = [small[0], big, small[1], small[2], big, small[3], small[4], small[5]]
    want = [O.gsl_lpa(g, 0.05, 20)[0] for g in gs]
    srv = gpu_lib.Server(slots=2, slot_vertices=400_000, slot_entries=8_000_000, max_batch_graphs=8)
    ids = [srv.submit(g.offsets, g.cols) for g in gs]
    infos = []
    for k, rid in enumerate(ids):
        lab, info = srv.wait(rid, info=True)
        assert np.array_equal(lab, want[k]), gs[k].name
        infos.append(info)
    assert all(infos[k]["batch_graphs"] == 1 for k in (1, 4))
    assert infos[1]["sweeps"] == O.lpa_sync(big, 0.05, 20)[1]
    srv.close()
