"""Parity of the CUDA path (through the C ABI) with the CPU oracle.

Counts, checksums, listed cliques, per-root counts and the front-end stages
must match exactly: the whole computation is integer work.
"""
import math
import os

import numpy as np
import pytest

import kclgen
import oracle
from tests.graphs import complete, csr_from_edges, gnp

pytestmark = pytest.mark.gpu

ORDS = ("degree", "color")


@pytest.fixture(scope="module")
def kcl():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    import paper_2203_13512_gb300 as kcl
    return kcl


def _ring(kcl, k, cap):
    import torch
    return torch.zeros(cap * k, dtype=torch.int32, device="cuda")


def _listed(ring, k, written):
    a = ring[: written * k].cpu().numpy().astype(np.uint32).reshape(-1, k)
    return sorted(tuple(int(x) for x in r) for r in a)


def _oracle_mode(ordering):
    return oracle.sdegree if ordering == "degree" else oracle.bitcol


# ------------------------------------------------------------ worked example
@pytest.mark.parametrize("ordering", ORDS)
def test_worked_example_counts_and_listing(kcl, fig1, ordering):
    rp, col = fig1
    g = kcl.kcl_load_csr(rp, col)
    for k in (3, 4, 5, 6):
        ref_c, ref_s, ref_l = oracle.plain(rp, col, k, list_cap=1000)
        assert kcl.kcl_count(g, k, ordering) == ref_c
        ring = _ring(kcl, k, 1000)
        c, s, w, trunc = kcl.kcl_list(g, k, ordering, ring)
        assert (c, s, w, trunc) == (ref_c, ref_s, ref_c, False)
        assert _listed(ring, k, w) == sorted(tuple(int(x) for x in r) for r in ref_l)
    # Example 1: the three 4-cliques
    ring = _ring(kcl, 4, 8)
    c, s, w, _ = kcl.kcl_list(g, 4, ordering, ring)
    assert _listed(ring, 4, w) == [(1, 2, 3, 4), (1, 2, 4, 6), (9, 10, 11, 12)]


def test_worked_example_stages(kcl, fig1):
    rp, col = fig1
    g = kcl.kcl_load_csr(rp, col)
    k = 4
    core = oracle.precore(rp, col, k)
    pl = oracle.prelist(rp, col, k, core)
    for ordering, mode in (("degree", 0), ("color", 1)):
        st = kcl.kcl_stage_info(g, k, ordering)
        assert np.array_equal(st["alive_core"], core)          # Example 2
        assert np.array_equal(st["alive_final"], pl["alive"])  # Example 3
        assert st["prelist_count"] == pl["count"] == 1
        assert np.array_equal(st["outdeg"], oracle.outdegrees(rp, col, pl["alive"], mode))
    # Example 4's DAG: d+ = v1:0 v2:4 v3:2 v4:2 v5:3 v6:1
    st = kcl.kcl_stage_info(g, k, "degree")
    assert [int(st["outdeg"][v]) for v in range(1, 7)] == [0, 4, 2, 2, 3, 1]
    st = kcl.kcl_stage_info(g, k, "color")
    rounds, _ = oracle.degeneracy_rounds(rp, col, pl["alive"])
    assert np.array_equal(st["key"], rounds)


# ----------------------------------------------------------- random graphs
@pytest.mark.parametrize("seed", range(10))
def test_random_small_graphs(kcl, seed):
    rng = np.random.default_rng(300 + seed)
    n = int(rng.integers(5, 41))
    p = float(rng.choice([0.15, 0.35, 0.55, 0.75, 0.9]))
    rp, col = gnp(n, p, 500 + seed)
    g = kcl.kcl_load_csr(rp, col)
    for k in range(3, 9):
        ref = oracle.plain(rp, col, k)
        for ordering in ORDS:
            c, s, _, _ = kcl.kcl_list(g, k, ordering, None)
            assert (c, s) == ref, (k, ordering)
            assert kcl.kcl_count(g, k, ordering) == ref[0]


# ----------------------------------------------- small Chung-Lu workload
@pytest.fixture(scope="module")
def small_workload():
    return kclgen.chung_lu_planted_small(seed=1)


@pytest.mark.parametrize("ordering", ORDS)
def test_small_workload_counts_checksums_per_root(kcl, small_workload, ordering):
    import torch
    rp, col = small_workload
    g = kcl.kcl_load_csr(rp, col)
    n = len(rp) - 1
    for k in range(3, 10):
        ref_c, ref_s = oracle.plain(rp, col, k)
        assert kcl.kcl_count(g, k, ordering) == ref_c
        c, s, _, _ = kcl.kcl_list(g, k, ordering, None)
        assert (c, s) == (ref_c, ref_s)
        pr = torch.zeros(n, dtype=torch.int64, device="cuda")
        tot, pre = kcl.kcl_count_per_root(g, k, ordering, pr)
        o = _oracle_mode(ordering)(rp, col, k, per_root=True)
        assert tot == ref_c
        assert np.array_equal(pr.cpu().numpy().astype(np.uint64), o["per_root"])


@pytest.mark.parametrize("ordering", ORDS)
def test_small_workload_listing_is_the_clique_set(kcl, small_workload, ordering):
    rp, col = small_workload
    g = kcl.kcl_load_csr(rp, col)
    for k in (5, 7):
        ref_c, ref_s, ref_l = oracle.plain(rp, col, k, list_cap=200000)
        ring = _ring(kcl, k, ref_c + 5)
        c, s, w, trunc = kcl.kcl_list(g, k, ordering, ring)
        assert (c, s, w, trunc) == (ref_c, ref_s, ref_c, False)
        assert _listed(ring, k, w) == sorted(tuple(int(x) for x in r) for r in ref_l)


# ------------------------------------------------ every out-degree class
@pytest.mark.parametrize("size,p", [(40, 0.9), (70, 0.8), (110, 0.7), (170, 0.6), (260, 0.45)])
def test_planted_communities_span_the_classes(kcl, size, p):
    rp, col = kclgen.chung_lu(3000, 12000, 2.3, groups=3, group_size=(size, size), group_p=p,
                              seed=size)
    g = kcl.kcl_load_csr(rp, col)
    for k in (3, 4, 5):
        ref = oracle.plain(rp, col, k)
        for ordering in ORDS:
            c, s, _, _ = kcl.kcl_list(g, k, ordering, None)
            assert (c, s) == ref, (k, ordering)


@pytest.mark.parametrize("ordering", ORDS)
def test_class_timing_matches_oracle_outdegrees(kcl, ordering):
    """The per-class split of the listing stage (used to attribute the
    oracle's per-out-degree work to one launch) covers exactly the roots the
    oracle expands, class by class."""
    rp, col = kclgen.chung_lu(3000, 12000, 2.3, groups=3, group_size=(260, 260), group_p=0.45,
                              seed=260)
    g = kcl.kcl_load_csr(rp, col)
    kcl.kcl_enable_timing(g, True)
    for k in (3, 5):
        kcl.kcl_count(g, k, ordering)
        ms, la, classes = kcl.kcl_last_timing(g)
        pl = oracle.prelist(rp, col, k, oracle.precore(rp, col, k))
        od = oracle.outdegrees(rp, col, pl["alive"], 0 if ordering == "degree" else 1).astype(np.int64)
        od = od[(pl["alive"] != 0) & (od >= k - 1)]
        assert classes and sum(c["roots"] for c in classes) == len(od)
        launched = 0
        for c in classes:
            assert c["roots"] == int(np.count_nonzero((od >= c["lo"]) & (od <= c["hi"])))
            assert (c["ms"] > 0) == (c["roots"] > 0)
            launched += c["roots"] > 0
        assert launched == la["listing"]
        assert sum(c["ms"] for c in classes) <= ms["listing"] * 1.01 + 0.05


def _near_complete(n):
    """K_n minus the edge {0, 1}: C(n,k) - C(n-2,k-2) k-cliques, and no
    Pre-List shortcut (the component is not a clique)."""
    return csr_from_edges(n, [(u, v) for u in range(n) for v in range(u + 1, n) if (u, v) != (0, 1)])


@pytest.mark.parametrize("n", [300, 700, 1300])
def test_large_outdegree_arena_classes(kcl, n):
    """K_n minus one edge: out-degrees up to n-1 reach the arena classes of
    both paths (BitCol W = 32..64, SDegree's literal form above 1024).  Counts
    against the closed form; k = 3 counts and checksums against the oracle
    (up to 3.6e8 triangles at n = 1300, seconds on the CPU)."""
    rp, col = _near_complete(n)
    g = kcl.kcl_load_csr(rp, col)
    ref3 = oracle.plain(rp, col, 3)
    assert ref3[0] == math.comb(n, 3) - (n - 2)
    # above 1024 SDegree runs the literal Algorithm 5 on global out-lists,
    # whose cost on a near-clique grows as n^k: keep k = 3 there
    for k in ((3, 4) if n <= 1024 else (3,)):
        want = math.comb(n, k) - math.comb(n - 2, k - 2)
        res = {o: kcl.kcl_list(g, k, o, None)[:2] for o in ORDS}
        assert res["degree"][0] == want and res["color"][0] == want
        assert kcl.kcl_count(g, k, "degree") == want and kcl.kcl_count(g, k, "color") == want
        if k == 3:
            assert res["degree"] == ref3 and res["color"] == ref3
        else:  # no oracle checksum at this size: both paths must agree
            assert res["degree"][1] == res["color"][1]


# ------------------------------------------------------------- edge cases
def test_edge_cases(kcl):
    # empty graph, no edges, single edge
    for n, edges in ((0, []), (5, []), (2, [(0, 1)])):
        rp, col = csr_from_edges(n, edges)
        g = kcl.kcl_load_csr(rp, col)
        for o in ORDS:
            assert kcl.kcl_count(g, 3, o) == 0
            assert kcl.kcl_list(g, 3, o, None)[:3] == (0, 0, 0)
    # K_k alone: Pre-List reports it; K_n with n < k: nothing
    for n, k in ((3, 3), (8, 8), (12, 5), (6, 9)):
        rp, col = complete(n)
        g = kcl.kcl_load_csr(rp, col)
        ref = oracle.plain(rp, col, k)
        for o in ORDS:
            assert kcl.kcl_list(g, k, o, None)[:2] == ref
    # the largest k: K_33 has C(33, 32) = 33 cliques of size 32 (closed form;
    # the plain recursion would visit ~2^33 partial cliques here)
    import itertools
    rp, col = complete(33)
    g = kcl.kcl_load_csr(rp, col)
    want = (33, sum(oracle.clique_hash(c) for c in itertools.combinations(range(33), 32)) % (1 << 64))
    for o in ORDS:
        assert kcl.kcl_list(g, 32, o, None)[:2] == want
    # k bounds
    rp, col = complete(5)
    g = kcl.kcl_load_csr(rp, col)
    for bad_k in (0, 1, 2, 33):
        with pytest.raises(kcl.KclError) as e:
            kcl.kcl_count(g, bad_k, "color")
        assert e.value.status == kcl.KCL_EINVAL


def test_malformed_graphs_rejected(kcl):
    bad = [
        (np.array([0, 1, 1], np.uint64), np.array([1], np.uint32)),              # asymmetric
        (np.array([0, 1, 2], np.uint64), np.array([0, 1], np.uint32)),           # self-loops
        (np.array([0, 2, 4], np.uint64), np.array([1, 1, 0, 0], np.uint32)),     # duplicates
        (np.array([0, 2, 3, 4], np.uint64), np.array([2, 1, 0, 0], np.uint32)),  # unsorted
        (np.array([0, 1, 2], np.uint64), np.array([5, 0], np.uint32)),           # out of range
        (np.array([1, 1, 2], np.uint64), np.array([1, 0], np.uint32)),           # row_ptr[0] != 0
    ]
    for rp, col in bad:
        with pytest.raises(kcl.KclError) as e:
            kcl.kcl_load_csr(rp, col)
        assert e.value.status == kcl.KCL_EINVAL


def test_ring_truncation_and_wrap(kcl, small_workload):
    rp, col = small_workload
    g = kcl.kcl_load_csr(rp, col)
    k = 5
    ref_c, ref_s = oracle.plain(rp, col, k)
    for o in ORDS:
        ring = _ring(kcl, k, 1000)
        c, s, w, trunc = kcl.kcl_list(g, k, o, ring, wrap=False)
        assert (c, s, w, trunc) == (ref_c, ref_s, 1000, True)
        got = _listed(ring, k, w)
        assert len(set(got)) == 1000
        ring = _ring(kcl, k, 777)
        c, s, w, trunc = kcl.kcl_list(g, k, o, ring, wrap=True)
        assert (c, s, w, trunc) == (ref_c, ref_s, 777, False)


def test_device_resident_input(kcl, small_workload):
    import torch
    rp, col = small_workload
    g = kcl.kcl_load_csr(torch.from_numpy(rp.astype(np.int64)).cuda(),
                         torch.from_numpy(col.astype(np.int32)).cuda())
    assert kcl.kcl_count(g, 5, "color") == oracle.plain(rp, col, 5)[0]


# --------------------------------------------------- degeneracy peel rounds
@pytest.mark.parametrize("which", ["small", "rmat14"])
def test_degeneracy_rounds_match_oracle(kcl, small_workload, which):
    rp, col = small_workload if which == "small" else kclgen.rmat20(seed=3, scale=14)
    g = kcl.kcl_load_csr(rp, col)
    for k in (3, 6):
        st = kcl.kcl_stage_info(g, k, "color")
        pl = oracle.prelist(rp, col, k, oracle.precore(rp, col, k))
        rounds, _ = oracle.degeneracy_rounds(rp, col, pl["alive"])
        assert np.array_equal(st["key"], rounds)
        assert np.array_equal(st["outdeg"], oracle.outdegrees(rp, col, pl["alive"], 1))
        st = kcl.kcl_stage_info(g, k, "degree")
        assert np.array_equal(st["outdeg"], oracle.outdegrees(rp, col, pl["alive"], 0))


# ------------------------------------- the bench workload at full size
@pytest.fixture(scope="module")
def rmat20():
    return kclgen.rmat20(seed=1)


def _golden_rmat20():
    import json
    import os
    p = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "rmat20_work.json")
    if not os.path.exists(p):
        return {}
    with open(p) as f:
        return json.load(f)


@pytest.mark.parametrize("k", [4, 5])
def test_rmat20_full_size_counts(kcl, rmat20, k):
    """Full-size R-MAT scale 20 in the bench's launch configuration: exact
    counts equal the oracle's stored full-size counts (written by
    tests/golden/make_rmat20_work.py) and agree across the two orderings;
    sampled roots match the oracle's per-root counts."""
    import torch
    rp, col = rmat20
    n = len(rp) - 1
    g = kcl.kcl_load_csr(rp, col)
    counts = {o: kcl.kcl_count(g, k, o) for o in ORDS}
    assert counts["degree"] == counts["color"]
    gold = _golden_rmat20()
    for o in ORDS:
        key = "k=%d %s" % (k, o)
        if key in gold:
            assert counts[o] == gold[key]["count"], key
        if key in gold and "checksum" in gold[key]:  # the oracle's full listing checksum
            c, s, _, _ = kcl.kcl_list(g, k, o, None)
            assert (c, s) == (gold[key]["count"], gold[key]["checksum"]), key
    # per-root parity on a seeded sample: the heaviest roots plus random ones
    for o in ORDS:
        pr = torch.zeros(n, dtype=torch.int64, device="cuda")
        tot, pre = kcl.kcl_count_per_root(g, k, o, pr)
        assert tot == counts[o]
        per = pr.cpu().numpy().astype(np.uint64)
        assert int(per.sum()) + pre == tot
        od = kcl.kcl_stage_info(g, k, o)["outdeg"]
        heavy = np.argsort(od)[-3:]
        rng = np.random.default_rng(k)
        sample = np.unique(np.concatenate([heavy, rng.integers(0, n, 40)])).astype(np.uint32)
        fn = _oracle_mode(o)
        ref = fn(rp, col, k, roots=sample, per_root=True, count_only=True)["per_root"]
        assert np.array_equal(per[sample], ref[sample]), o


# ------------------------------------------- leaf forms and the autotuner
@pytest.mark.parametrize("gallop", [0, 4_000_000_000])
def test_sdegree_leaf_forms_agree(kcl, small_workload, gallop):
    """SDegree's leaf by merges only (0) and by galloping only (a threshold
    no estimate reaches): identical counts, checksums and listings."""
    rp, col = small_workload
    g = kcl.kcl_load_csr(rp, col)
    kcl.kcl_set_tuning(g, {"sdegree_gallop": [gallop] * kcl.KCL_MAX_CLASSES,
                           "sdegree_gallop_list": [gallop] * kcl.KCL_MAX_CLASSES})
    for k in (3, 4, 6):
        ref_c, ref_s = oracle.plain(rp, col, k)
        assert kcl.kcl_count(g, k, "degree") == ref_c
        assert kcl.kcl_list(g, k, "degree", None)[:2] == (ref_c, ref_s)
    dense = kclgen.chung_lu(3000, 12000, 2.3, groups=3, group_size=(260, 260), group_p=0.45, seed=260)
    g2 = kcl.kcl_load_csr(*dense)
    kcl.kcl_set_tuning(g2, {"sdegree_gallop": [gallop] * kcl.KCL_MAX_CLASSES,
                            "sdegree_gallop_list": [gallop] * kcl.KCL_MAX_CLASSES})
    for k in (4, 5):
        ref = oracle.plain(*dense, k)
        assert kcl.kcl_list(g2, k, "degree", None)[:2] == ref


def test_autotune_keeps_results(kcl, small_workload):
    rp, col = small_workload
    g = kcl.kcl_load_csr(rp, col)
    kcl.kcl_autotune(g, 5, "degree")
    t = kcl.kcl_autotune(g, 4, "degree", listing=True)
    assert kcl.kcl_get_tuning(g) == t
    assert all(v in (0, 40, 80, 160, 400) for v in t["sdegree_gallop"] + t["sdegree_gallop_list"])
    assert all(v in (0, 4, 64, 0xFFFFFFFF) for v in t["sdegree_bitmap"])
    assert all(v in (0, 4, 8) for v in t["sdegree_cta_warps"] + t["bitcol_cta_warps"])
    assert all(v in (0, 2, 8, 32) for v in t["sdegree_split"] + t["bitcol_split"])
    assert kcl.kcl_count(g, 5, "degree") == oracle.plain(rp, col, 5)[0]
    assert kcl.kcl_list(g, 4, "degree", None)[:2] == oracle.plain(rp, col, 4)
    tc = kcl.kcl_autotune(g, 5, "color")
    mine = ("bitcol_cta_warps", "bitcol_split")
    assert {f: tc[f] for f in tc if f not in mine} == {f: t[f] for f in t if f not in mine}
    assert kcl.kcl_count(g, 5, "color") == oracle.plain(rp, col, 5)[0]


# ------------------------------------------------------ ablation switches
@pytest.mark.parametrize("flags", [1, 2, 4, 7])
def test_ablation_switches_keep_results(kcl, small_workload, flags):
    """Pre-Core, Pre-List and the colour prune off (alone and together):
    counts, checksums and per-root sums stay exact."""
    rp, col = small_workload
    g = kcl.kcl_load_csr(rp, col)
    kcl.kcl_set_options(g, flags)
    assert kcl.kcl_get_options(g) == flags
    for k in (3, 5, 8):
        ref = oracle.plain(rp, col, k)
        for o in ORDS:
            assert kcl.kcl_count(g, k, o) == ref[0], (k, o)
            assert kcl.kcl_list(g, k, o, None)[:2] == ref, (k, o)
    st = kcl.kcl_stage_info(g, 5, "color")
    if flags & kcl.KCL_OPT_NO_PRECORE and flags & kcl.KCL_OPT_NO_PRELIST:
        assert st["alive_final"].all() and st["prelist_count"] == 0


def test_ablation_rejects_unknown_bits(kcl, fig1):
    g = kcl.kcl_load_csr(*fig1)
    with pytest.raises(kcl.KclError):
        kcl.kcl_set_options(g, 8)


def test_scratch_bytes_grow_with_the_call(kcl, small_workload):
    rp, col = small_workload
    g = kcl.kcl_load_csr(rp, col)
    assert kcl.kcl_scratch_bytes(g)[1] == 0  # loading validates with the workspace; no arena yet
    kcl.kcl_count(g, 4, "degree")
    ws, ar = kcl.kcl_scratch_bytes(g)
    n, nnz = len(rp) - 1, len(col)
    assert 70 * n + 2 * nnz <= ws <= 90 * n + 2 * nnz + (1 << 16)
    assert ar > 0


@pytest.mark.parametrize("bitmap", [1, 0xFFFFFFFF])
def test_sdegree_bitrow_and_list_forms_agree(kcl, bitmap):
    """SDegree on bit-rows (threshold 1: whenever the rows fit; warp-per-root
    and CTA classes) and on lists only: identical counts and checksums."""
    tune = {"sdegree_bitmap": [bitmap] * kcl.KCL_MAX_CLASSES}
    for n in (40, 100, 300, 700):
        rp, col = _near_complete(n)
        g = kcl.kcl_load_csr(rp, col)
        kcl.kcl_set_tuning(g, tune)
        for k in (4, 5, 7) if n <= 100 else (4, 5) if n <= 300 else (4,):
            want = math.comb(n, k) - math.comb(n - 2, k - 2)
            assert kcl.kcl_count(g, k, "degree") == want
            assert kcl.kcl_list(g, k, "degree", None)[0] == want
    for size, p in ((170, 0.6), (260, 0.45)):
        rp, col = kclgen.chung_lu(3000, 12000, 2.3, groups=3, group_size=(size, size), group_p=p,
                                  seed=size)
        g = kcl.kcl_load_csr(rp, col)
        kcl.kcl_set_tuning(g, tune)
        for k in (4, 5, 6):
            ref = oracle.plain(rp, col, k)
            assert kcl.kcl_count(g, k, "degree") == ref[0]
            assert kcl.kcl_list(g, k, "degree", None)[:2] == ref


@pytest.mark.parametrize("warps", [1, 3])
def test_warps_per_root_keep_results(kcl, warps):
    """One warp per root (NodeParallel) and three: identical results in both
    orderings' CTA classes, counting and listing."""
    tune = {"sdegree_cta_warps": [warps] * kcl.KCL_MAX_CLASSES,
            "bitcol_cta_warps": [warps] * kcl.KCL_MAX_CLASSES}
    for size, p in ((170, 0.6), (260, 0.45)):
        rp, col = kclgen.chung_lu(3000, 12000, 2.3, groups=3, group_size=(size, size), group_p=p,
                                  seed=size)
        g = kcl.kcl_load_csr(rp, col)
        kcl.kcl_set_tuning(g, tune)
        for k in (3, 4, 5):
            ref = oracle.plain(rp, col, k)
            for o in ORDS:
                assert kcl.kcl_count(g, k, o) == ref[0], (k, o)
                assert kcl.kcl_list(g, k, o, None)[:2] == ref, (k, o)


# ------------------------------------------- a5: the per-root colouring
def _induced_out_subgraph(rp, col, key, alive, u):
    """N+_u in the DAG eta = (key, id) over alive vertices (ascending id) and
    the CSR of G_u, the subgraph it induces (local index = rank in N+_u)."""
    nb = [int(w) for w in col[rp[u]:rp[u + 1]]
          if alive[w] and (int(key[u]), u) < (int(key[w]), int(w))]
    pos = {w: i for i, w in enumerate(nb)}
    edges = []
    for i, a in enumerate(nb):
        for w in col[rp[a]:rp[a + 1]]:
            j = pos.get(int(w))
            if j is not None and j > i:
                edges.append((i, j))
    return nb, csr_from_edges(len(nb), edges)


def test_colouring_of_example6(kcl, fig1):
    """G_r equal to the Example 6 graph (v1..v6 of Figure 1): root r = 0 is
    adjacent to v1..v6, and each v_i also to its own K_8, so r leaves in the
    first peel round and N+_r = {v1..v6}.  The GPU's colours are Example 6's
    (v1..v6 -> 1, 2, 3, 4, 2, 3; tests/golden/table2_bitmaps.txt)."""
    rp0, col0 = fig1
    ex6 = [(u, int(v)) for u in range(1, 7) for v in col0[rp0[u]:rp0[u + 1]] if u < v <= 6]
    edges = list(ex6) + [(0, v) for v in range(1, 7)]
    nxt = 7
    for v in range(1, 7):
        block = list(range(nxt, nxt + 8))
        edges += [(a, b) for i, a in enumerate(block) for b in block[i + 1:]]
        edges += [(v, a) for a in block]
        nxt += 8
    rp, col = csr_from_edges(nxt, edges)
    g = kcl.kcl_load_csr(rp, col)
    colours = {}
    with open(os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden",
                           "table2_bitmaps.txt")) as f:
        for line in f:
            p = line.split("#", 1)[0].split()
            if p and p[0] == "colour":
                colours[int(p[1])] = int(p[2])
    for k in (3, 4):
        nb, co = kcl.kcl_root_colouring(g, k, 0)
        assert list(nb) == [1, 2, 3, 4, 5, 6]
        assert [int(c) for c in co] == [colours[v] for v in range(1, 7)]
        _, ex_rp_col = _induced_out_subgraph(rp, col, kcl.kcl_stage_info(g, k, "color")["key"],
                                             np.ones(nxt, np.uint8), 0)
        assert list(oracle.colour_graph(*ex_rp_col)[1]) == list(co)


@pytest.mark.parametrize("scale,k", [(16, 4), (20, 5)])
def test_colouring_matches_oracle_on_sampled_roots(kcl, scale, k):
    """The colour of every out-neighbour of 55 seeded roots (the 5 largest
    out-degrees and 50 drawn at random) equals oracle.colour_graph on G_u
    built from the oracle's own front end (Pre-Core, Pre-List, bulk peel)."""
    rp, col = kclgen.rmat20(seed=1, scale=scale)
    g = kcl.kcl_load_csr(rp, col)
    pl = oracle.prelist(rp, col, k, oracle.precore(rp, col, k))
    key, _ = oracle.degeneracy_rounds(rp, col, pl["alive"])
    od = oracle.outdegrees(rp, col, pl["alive"], 1).astype(np.int64)
    roots = np.nonzero((pl["alive"] != 0) & (od >= k - 1))[0]
    rng = np.random.default_rng(scale)
    sample = list(roots[np.argsort(-od[roots], kind="stable")[:5]])
    sample += list(rng.choice(roots, 50, replace=False))
    for u in sample:
        u = int(u)
        nb, (grp, gcol) = _induced_out_subgraph(rp, col, key, pl["alive"], u)
        got_nb, got_co = kcl.kcl_root_colouring(g, k, u)
        assert list(got_nb) == nb, u
        _, want = oracle.colour_graph(grp, gcol)
        assert np.array_equal(got_co, want), u


def test_rmat20_k6_sampled_roots(kcl, rmat20):
    """k = 6 on the full-size R-MAT scale 20 graph (2.8e13 cliques, beyond
    the oracle): the two orderings agree on the count, and the per-root
    counts of the seeded sample stored by tests/golden/make_rmat20_work.py
    (the 3 heaviest roots, 40 at random, 2 per out-degree bucket) equal the
    oracle's."""
    import torch
    gold = _golden_rmat20()
    rp, col = rmat20
    n = len(rp) - 1
    g = kcl.kcl_load_csr(rp, col)
    totals = {}
    for o in ORDS:
        e = gold.get("k=6 %s" % o, {}).get("sample")
        assert e, "golden sample missing for k=6 %s" % o
        pr = torch.zeros(n, dtype=torch.int64, device="cuda")
        tot, pre = kcl.kcl_count_per_root(g, 6, o, pr)
        per = pr.cpu().numpy().astype(np.uint64)
        assert int(per.sum()) + pre == tot
        roots = np.array(e["roots"], np.int64)
        assert [int(x) for x in per[roots]] == e["per_root"], o
        od = kcl.kcl_stage_info(g, 6, o)["outdeg"]
        assert [int(x) for x in od[roots]] == e["outdeg"], o
        totals[o] = tot
    assert totals["degree"] == totals["color"]


@pytest.mark.parametrize("split", [1, 3])
def test_work_splitting_keeps_results(kcl, split):
    """Heavy roots shared between CTAs (a CTA that runs out of roots rebuilds
    a root still in progress and takes over first-level children while at
    least `split` are left): counts, checksums, listings and per-root counts
    are those of the oracle, in both orderings."""
    import torch
    tune = {"sdegree_split": [split] * kcl.KCL_MAX_CLASSES,
            "bitcol_split": [split] * kcl.KCL_MAX_CLASSES}
    graphs = [kclgen.chung_lu(3000, 12000, 2.3, groups=3, group_size=(sz, sz), group_p=p, seed=sz)
              for sz, p in ((170, 0.6), (260, 0.45))]
    graphs.append(_near_complete(300))
    for rp, col in graphs:
        g = kcl.kcl_load_csr(rp, col)
        kcl.kcl_set_tuning(g, tune)
        n = len(rp) - 1
        for k in (4, 5):
            ref = oracle.plain(rp, col, k)
            for o in ORDS:
                assert kcl.kcl_count(g, k, o) == ref[0], (k, o)
                assert kcl.kcl_list(g, k, o, None)[:2] == ref, (k, o)
                pr = torch.zeros(n, dtype=torch.int64, device="cuda")
                kcl.kcl_count_per_root(g, k, o, pr)
                want = _oracle_mode(o)(rp, col, k, per_root=True, count_only=True)["per_root"]
                assert np.array_equal(pr.cpu().numpy().astype(np.uint64), want), (k, o)
    # the listed records themselves (4.7e6 4-cliques, compared as sorted rows)
    rp, col = graphs[0]
    g = kcl.kcl_load_csr(rp, col)
    kcl.kcl_set_tuning(g, tune)
    ref_c, ref_s, ref_l = oracle.plain(rp, col, 4, list_cap=5_000_000)
    want = ref_l[np.lexsort(ref_l.T[::-1])]
    for o in ORDS:
        ring = _ring(kcl, 4, ref_c + 3)
        c, s, w, trunc = kcl.kcl_list(g, 4, o, ring)
        assert (c, s, w, trunc) == (ref_c, ref_s, ref_c, False)
        got = ring[: w * 4].cpu().numpy().astype(np.uint32).reshape(-1, 4)
        assert np.array_equal(got[np.lexsort(got.T[::-1])], want), o


def test_time_limit_stops_a_long_call(kcl):
    """kcl_set_time_limit: a call whose listing stage outlasts the limit
    returns KCL_ETIMEOUT (R-MAT scale 16, k = 7: seconds of work against a
    1 ms limit), the handle stays usable, and a generous limit leaves the
    results unchanged."""
    rp, col = kclgen.rmat20(seed=1, scale=16)
    g = kcl.kcl_load_csr(rp, col)
    ref = kcl.kcl_count(g, 5, "color")
    for o in ORDS:
        kcl.kcl_set_time_limit(g, 1)
        with pytest.raises(kcl.KclError) as e:
            kcl.kcl_count(g, 7, o)
        assert e.value.status == kcl.KCL_ETIMEOUT
        with pytest.raises(kcl.KclError):
            kcl.kcl_list(g, 7, o, None)
        kcl.kcl_set_time_limit(g, 600_000)
        assert kcl.kcl_count(g, 5, o) == ref
        kcl.kcl_set_time_limit(g, 0)
        assert kcl.kcl_count(g, 5, o) == ref
