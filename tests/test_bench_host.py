"""Host-side logic of bench.py that needs no GPU: attribution of the
oracle's per-out-degree work to one listing launch, the choice of the
dominant launch, and the max-over-ranks reduction of replica timings
(world size 2 over gloo)."""
import os
import socket

import pytest
import torch.multiprocessing as mp

import bench


def test_class_work_buckets():
    e = {"work_by_outdeg": {"2": 1, "3": 2, "4": 4, "5": 8, "6": 16, "7": 32, "8": 64, "9": 128}}
    # class 0 of k = 4 (3 <= d+ <= 32) holds buckets 2..5; later classes one each
    assert bench.class_work(e, 3, 32) == 15
    assert bench.class_work(e, 33, 64) == 16
    assert bench.class_work(e, 129, 256) == 64
    assert bench.class_work(e, 257, 300) == 128
    assert bench.class_work({}, 3, 32) is None
    assert bench.class_work({"work": 5}, 3, 32) is None


def _call(k, o, m, listing_ms, classes):
    ms = {"pre_core": 0.1, "pre_list": 1.0, "orientation": 2.0, "listing": listing_ms,
          "total": listing_ms + 3.1}
    la = {"pre_core": 1, "pre_list": 1, "orientation": 5, "listing": len(classes), "total": 0}
    cl = [{"lo": lo, "hi": hi, "roots": r, "ms": t} for lo, hi, r, t in classes]
    return (k, o, m, 0, ms, la, cl)


PEAKS = {"num_sms": 152, "sm_clock_mhz": 2070.0, "bitjoin_words_per_sm_clk": 15.7,
         "mix64_per_sm_clk": 3.9}


def test_roofline_picks_the_longest_launch(monkeypatch):
    work = {"k=5 degree": {"work": 300, "bitrow_words_by_outdeg": {"5": 100, "9": 200}},
            "k=5 color": {"work": 50, "work_by_outdeg": {"5": 50}}}
    monkeypatch.setattr(bench, "_load_work", lambda: work)
    calls = [_call(5, "color", "count", 10.0, [(4, 32, 10, 10.0)]),
             _call(5, "degree", "count", 30.0, [(4, 32, 10, 5.0), (257, 512, 3, 25.0)])] * 2
    r = bench.roofline(calls, 2, PEAKS, 2000.0)
    assert r["bound"] == "alu" and r["unit"] == "Gword/s"
    assert "257 <= d+ <= 512" in r["kernel"]
    assert r["work_per_launch"] == 200 and r["avg_ms"] == 25.0
    assert abs(r["achieved"] - 200 / 25e-3 / 1e9) < 1e-12
    assert abs(r["frac"] - r["achieved"] / r["peak"]) < 1e-12
    # measured BitJoin word rate x SMs x sampled clock
    assert abs(r["peak"] - 152 * 15.7 * 2000e6 / 1e9) < 1e-9
    assert "measured" in r["peak_source"]


def test_roofline_listing_counts_cliques(monkeypatch):
    work = {"k=4 color": {"work": 50, "work_by_outdeg": {"5": 50},
                          "count_by_outdeg": {"5": 7000, "9": 9000}}}
    monkeypatch.setattr(bench, "_load_work", lambda: work)
    calls = [_call(4, "color", "list", 40.0, [(3, 32, 10, 10.0), (257, 512, 3, 30.0)]),
             _call(4, "color", "count", 5.0, [(3, 32, 10, 5.0)])]
    r = bench.roofline(calls, 1, PEAKS, 2070.0)
    assert r["unit"] == "Gclique/s" and r["work_per_launch"] == 9000
    # k SplitMix64 rounds per clique at the measured round rate
    assert abs(r["peak"] - 152 * 3.9 / 4 * 2070e6 / 1e9) < 1e-9
    assert bench.roofline(calls, 1, PEAKS, 2070.0, modes=("nothing",)) is None


def test_frontend_roofline_bytes():
    calls = [_call(4, "color", "count", 5.0, [(3, 32, 10, 5.0)]),
             _call(4, "degree", "count", 5.0, [(3, 32, 10, 5.0)])]
    n, nnz = 1000, 8000
    f = bench.frontend_roofline(calls, 1, n, nnz)
    C = 8 * (n + 1) + 4 * nnz
    assert f["k=4 degree count"]["pre_list"]["bytes"] == C + n
    assert f["k=4 color count"]["orientation"]["bytes"] == 3 * (C + 5 * n) + 4 * (n + 1) + 2 * nnz
    o = f["k=4 degree count"]["orientation"]
    assert abs(o["frac"] - o["bytes"] / 2e-3 / 1e9 / f["peak_GB_s"]) < 1e-12


def test_golden_check_raises_on_mismatch():
    gold = {"k=4 color": {"count": 10, "checksum": 77}, "k=5 color": {"count": 3}}
    ok = [(4, "color", "count", 10, None), (4, "color", "list", 10, 77), (5, "color", "count", 3, None)]
    assert bench.check_golden(ok, gold) == ["k=4 color count count", "k=4 color list checksum",
                                            "k=4 color list count", "k=5 color count count"]
    with pytest.raises(AssertionError):
        bench.check_golden([(4, "color", "list", 10, 78)], gold)
    with pytest.raises(AssertionError):
        bench.check_golden([(5, "color", "count", 4, None)], gold)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        out[rank] = bench.max_over_ranks([1.0 + rank, 10.0 - rank], world)
    finally:
        dist.destroy_process_group()


def test_max_over_ranks_two_gloo_ranks():
    ctx = mp.get_context("spawn")
    with ctx.Manager() as mgr:
        out = mgr.dict()
        port = _free_port()
        ps = [ctx.Process(target=_rank, args=(r, 2, port, out)) for r in range(2)]
        for p in ps:
            p.start()
        for p in ps:
            p.join(120)
        assert all(p.exitcode == 0 for p in ps)
        assert out[0] == out[1] == [2.0, 10.0]


def test_max_over_ranks_single_rank():
    assert bench.max_over_ranks([3.0, 4.0], 1) == [3.0, 4.0]


# ------------------------------------------ batched / served forms' host loop
class _FakeGraph:
    def __init__(self, key):
        self.key = key

    def free(self):
        pass


def _answer(key, k):
    return (key * 1000 + k, (key * 7919 + 31 * k) & 0xFFFF)


class _FakeLib:
    """Stands in for the CUDA library so the forms' control flow (timing,
    result comparison, report) runs on the CPU; results are a function of
    (graph, k), and `wrong` names queries the fake server answers wrongly."""

    class KclError(Exception):
        def __init__(self, status):
            super().__init__(status)
            self.status = status

    def __init__(self, wrong=()):
        self.n = 0
        self.wrong = set(wrong)

    def kcl_load_csr(self, rp, col):
        self.n += 1
        return _FakeGraph(len(rp) * 100003 + len(col))

    def kcl_set_time_limit(self, g, ms):
        pass

    def kcl_count(self, g, k, o):
        return _answer(g.key, k)[0]

    def kcl_list(self, g, k, o, ring, wrap=False):
        c, h = _answer(g.key, k)
        return c, h, 0, False

    def kcl_batch_create(self):
        return _FakeGraph(0)

    def kcl_count_batch(self, b, gs, ks, ords, checksums=False):
        res = [_answer(g.key, k) for g, k in zip(gs, ks)]
        cks = [h for _, h in res] if checksums else None
        counts = [c + (1 if (g.key, k) in self.wrong else 0) for (c, _), g, k in zip(res, gs, ks)]
        return counts, cks

    def kcl_server_create(self, slots, scratch_budget_bytes, small_nnz):
        import time as _t
        srv = _FakeGraph(0)
        srv.t0, srv.graphs, srv.tickets = _t.perf_counter(), [], []
        srv.destroy = lambda: None
        return srv

    def kcl_server_set_time_limit(self, srv, ms):
        pass

    def kcl_server_add_graph(self, srv, g):
        srv.graphs.append(g)
        return len(srv.graphs) - 1

    def kcl_server_clock(self, srv):
        import time as _t
        return _t.perf_counter() - srv.t0

    def kcl_server_submit(self, srv, gid, k, o, lst=False):
        srv.tickets.append((gid, k, lst, self.kcl_server_clock(srv)))
        return len(srv.tickets) - 1

    def kcl_server_wait(self, srv, t):
        gid, k, lst, sub = srv.tickets[t]
        g = srv.graphs[gid]
        c, h = _answer(g.key, k)
        if (g.key, k) in self.wrong:
            c += 1
        now = self.kcl_server_clock(srv)
        return {"status": 0, "count": c, "checksum": h if lst else 0, "submit_s": sub,
                "start_s": sub, "done_s": max(now, sub + 1e-6), "batch": 1}


def _use_fake(monkeypatch, lib):
    import sys
    import types

    import torch
    mod = types.ModuleType("paper_2203_13512_gb300")
    for name in dir(lib):
        if not name.startswith("__"):
            setattr(mod, name, getattr(lib, name))
    monkeypatch.setitem(sys.modules, "paper_2203_13512_gb300", mod)
    monkeypatch.setattr(torch.cuda, "synchronize", lambda *a, **k: None)


def test_batch_form_reports_mismatches(monkeypatch):
    import kclgen
    _use_fake(monkeypatch, _FakeLib())
    out = bench.batch_form(4, quiet=True)
    assert out["bit_exact"] and out["config"]["graphs"] == 4 and out["speedup"] > 0
    summ = bench.batched_summary(out)
    assert summ["graphs"] == 4 and summ["bit_exact"] and "mismatches" not in summ
    rp, col, _ = kclgen.batch_graph(2)
    key = len(rp) * 100003 + len(col)
    k = kclgen.batch_graph(2)[2]
    _use_fake(monkeypatch, _FakeLib(wrong={(key, k)}))
    out = bench.batch_form(4, quiet=True)
    assert not out["bit_exact"] and out["mismatches"] == 2  # both orderings
    assert out["mismatch_examples"][0]["graph"] == 2
    assert bench.batched_summary(out)["mismatches"] == 2


def test_serve_form_compares_and_reports(monkeypatch):
    kw = dict(rmat_ids=range(1, 3), batch_ids=range(33, 35), rmat_scale=lambda i: 8, quiet=True)
    _use_fake(monkeypatch, _FakeLib())
    out = bench.serve_form(24, [1e5], 50, **kw)
    r = out["rates"]["100000.0"]
    assert out["bit_exact"] and out["results_compared"] == 24
    assert out["results_compared_equal"] == 24 and r["served"]["completed"] == 24
    summ = bench.served_summary(out, 1e5, 50)
    assert summ["bit_exact"] and summ["results_compared"] == 24 and summ["mismatches"] is None
    assert "2 R-MAT graphs (scales 8..8) + 2 batched-workload graphs" in summ["sample"]
    import kclgen
    rp, col = kclgen.rmat20(seed=1, scale=8)
    _use_fake(monkeypatch, _FakeLib(wrong={(len(rp) * 100003 + len(col), k) for k in range(3, 11)}))
    out = bench.serve_form(24, [1e5], 50, **kw)
    assert not out["bit_exact"] and out["mismatches"]
    assert out["results_compared_equal"] < out["results_compared"] == 24
    assert not bench.served_summary(out, 1e5, 50)["bit_exact"]
