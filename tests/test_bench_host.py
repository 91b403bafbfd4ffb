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


def test_roofline_picks_the_longest_launch(monkeypatch):
    work = {"k=5 degree": {"work": 300, "work_by_outdeg": {"5": 100, "9": 200}},
            "k=5 color": {"work": 50, "work_by_outdeg": {"5": 50}}}
    monkeypatch.setattr(bench, "_load_work", lambda: work)
    calls = [_call(5, "color", "count", 10.0, [(4, 32, 10, 10.0)]),
             _call(5, "degree", "count", 30.0, [(4, 32, 10, 5.0), (257, 512, 3, 25.0)])] * 2
    r = bench.roofline(calls, 2)
    assert r["bound"] == "alu" and r["unit"] == "Gelem/s"
    assert "257 <= d+ <= 512" in r["kernel"]
    assert r["work_per_launch"] == 200 and r["avg_ms"] == 25.0
    assert abs(r["achieved"] - 200 / 25e-3 / 1e9) < 1e-12
    assert abs(r["frac"] - r["achieved"] / r["peak"]) < 1e-12
    # SDegree's peak counts 64 compares per SM and clock, BitCol's 16 POPC
    calls = [_call(5, "color", "count", 30.0, [(4, 32, 10, 30.0)])]
    rc = bench.roofline(calls, 1)
    assert abs(r["peak"] / rc["peak"] - 4.0) < 1e-12


def test_roofline_listing_counts_cliques(monkeypatch):
    work = {"k=4 color": {"work": 50, "work_by_outdeg": {"5": 50},
                          "count_by_outdeg": {"5": 7000, "9": 9000}}}
    monkeypatch.setattr(bench, "_load_work", lambda: work)
    calls = [_call(4, "color", "list", 40.0, [(3, 32, 10, 10.0), (257, 512, 3, 30.0)]),
             _call(4, "color", "count", 5.0, [(3, 32, 10, 5.0)])]
    r = bench.roofline(calls, 1)
    assert r["unit"] == "Gclique/s" and r["work_per_launch"] == 9000
    # k SplitMix64 rounds per clique at 6 IMADs each, 64 IMADs per SM and clock
    assert abs(r["peak"] - 152 * 64 / 24 * 2070e6 / 1e9) < 1e-6
    rc = bench.roofline(calls, 1, modes=("count",))
    assert rc["unit"] == "Gword/s" and rc["work_per_launch"] == 50


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
