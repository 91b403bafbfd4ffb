"""The serving loop: queries submitted concurrently (and in bursts that get
batched) must return exactly what the same query returns alone."""
import threading
import time

import numpy as np
import pytest

import kclgen

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def kcl():
    import paper_2203_13512_gb300 as kcl
    return kcl


@pytest.mark.parametrize("slots", [1, 4])
def test_served_results_equal_results_alone(kcl, slots):
    graphs = [kcl.kcl_load_csr(*kclgen.rmat20(seed=s, scale=12)) for s in (1, 2)]
    graphs += [kcl.kcl_load_csr(*kclgen.batch_graph(i)[:2]) for i in range(6)]
    srv = kcl.kcl_server_create(slots=slots, scratch_budget_bytes=8 << 30, small_nnz=1 << 20)
    ids = [kcl.kcl_server_add_graph(srv, g) for g in graphs]
    rng = np.random.default_rng(slots)
    queries = [(int(rng.integers(len(ids))), int(rng.integers(3, 8)),
                "color" if rng.random() < 0.5 else "degree", bool(rng.random() < 0.5))
               for _ in range(120)]
    queries += queries[:10]  # repeated queries share results
    tickets = [None] * len(queries)

    def submitter(lo, hi):
        for i in range(lo, hi):
            gi, k, o, lst = queries[i]
            tickets[i] = kcl.kcl_server_submit(srv, ids[gi], k, o, lst)
            if i % 7 == 0:
                time.sleep(0.001)

    th = [threading.Thread(target=submitter, args=(a, min(a + 33, len(queries))))
          for a in range(0, len(queries), 33)]
    for t in th:
        t.start()
    for t in th:
        t.join()
    results = [kcl.kcl_server_wait(srv, t) for t in tickets]
    srv.destroy()
    for (gi, k, o, lst), r in zip(queries, results):
        assert r["status"] == 0
        assert r["submit_s"] <= r["start_s"] <= r["done_s"]
        if lst:
            c, s, _, _ = kcl.kcl_list(graphs[gi], k, o, None)
            assert (r["count"], r["checksum"]) == (c, s)
        else:
            assert r["count"] == kcl.kcl_count(graphs[gi], k, o)


def test_burst_is_batched_and_slots_overlap(kcl):
    """Four heavy queries occupy the four slots at once (their [start, done]
    intervals overlap on the device); a burst of small-graph queries that
    arrives meanwhile waits in the queue and is answered by batched passes
    (some result reports batch > 1).  Every result equals the query alone."""
    heavy = [kcl.kcl_load_csr(*kclgen.rmat20(seed=s, scale=12)) for s in (1, 2)]
    small = []
    i = 0
    while len(small) < 6:
        rp, col, _ = kclgen.batch_graph(i)
        i += 1
        if len(col) <= 20000:
            small.append(kcl.kcl_load_csr(rp, col))
    srv = kcl.kcl_server_create(slots=4, scratch_budget_bytes=8 << 30, small_nnz=20000)
    hid = [kcl.kcl_server_add_graph(srv, g) for g in heavy]
    sid = [kcl.kcl_server_add_graph(srv, g) for g in small]
    hq = [(hid[j % 2], heavy[j % 2], 6 + j % 2, "color" if j < 2 else "degree") for j in range(4)]
    ht = [kcl.kcl_server_submit(srv, gid, k, o, True) for gid, _, k, o in hq]
    sq = [(j % len(small), 3 + j % 5, "color" if j % 3 else "degree") for j in range(30)]
    st = [kcl.kcl_server_submit(srv, sid[gi], k, o, False) for gi, k, o in sq]
    hr = [kcl.kcl_server_wait(srv, t) for t in ht]
    sr = [kcl.kcl_server_wait(srv, t) for t in st]
    srv.destroy()
    assert all(r["status"] == 0 for r in hr + sr)
    spans = sorted((r["start_s"], r["done_s"]) for r in hr)
    assert any(spans[j][0] < spans[j - 1][1] for j in range(1, len(spans))), spans
    assert max(r["batch"] for r in sr) > 1
    for (_, g, k, o), r in zip(hq, hr):
        assert (r["count"], r["checksum"]) == kcl.kcl_list(g, k, o, None)[:2]
    for (gi, k, o), r in zip(sq, sr):
        assert r["count"] == kcl.kcl_count(small[gi], k, o)


def test_graph_view_shares_the_graph(kcl):
    g = kcl.kcl_load_csr(*kclgen.rmat20(seed=5, scale=11))
    v = kcl.kcl_graph_view(g)
    for k in (3, 4, 5):
        assert kcl.kcl_count(v, k, "color") == kcl.kcl_count(g, k, "color")
    v.free()
    assert kcl.kcl_count(g, 4, "degree") == kcl.kcl_count(g, 4, "color")


def test_server_time_limit(kcl):
    """A pass that outlasts the server's time limit finishes with
    KCL_ETIMEOUT (R-MAT scale 16, k = 7: seconds of work against 1 ms);
    light queries submitted with it still complete exactly."""
    heavy = kcl.kcl_load_csr(*kclgen.rmat20(seed=1, scale=16))
    light = kcl.kcl_load_csr(*kclgen.batch_graph(1)[:2])
    want = kcl.kcl_count(light, 4, "color")
    srv = kcl.kcl_server_create(slots=2, scratch_budget_bytes=8 << 30, small_nnz=1 << 14)
    hid = kcl.kcl_server_add_graph(srv, heavy)
    lid = kcl.kcl_server_add_graph(srv, light)
    kcl.kcl_server_set_time_limit(srv, 1)
    rh = kcl.kcl_server_wait(srv, kcl.kcl_server_submit(srv, hid, 7, "color"))
    assert rh["status"] == kcl.KCL_ETIMEOUT
    kcl.kcl_server_set_time_limit(srv, 0)
    rl = kcl.kcl_server_wait(srv, kcl.kcl_server_submit(srv, lid, 4, "color"))
    srv.destroy()
    assert rl["status"] == 0 and rl["count"] == want
