"""The oracle against the paper's worked examples (Examples 1-7, Table II).

The graph is in tests/golden/fig1_graph.txt (with the provenance of each
edge); Table II and Example 6 are in tests/golden/table2_bitmaps.txt.
"""
import os

import numpy as np

import oracle
from tests.graphs import GOLDEN, adjacency_sets, csr_from_edges


def _table2():
    B, colour, order = {}, {}, None
    with open(os.path.join(GOLDEN, "table2_bitmaps.txt")) as f:
        for line in f:
            line = line.split("#", 1)[0].strip()
            if not line:
                continue
            p = line.split()
            if p[0] == "colour":
                colour[int(p[1])] = int(p[2])
            elif p[0] == "order":
                order = [int(x) for x in p[1:]]
            else:
                B[int(p[0])] = [int(x) for x in p[1:]]
    return B, colour, order


def _fig7_graph(fig1):
    """The six-vertex graph of Example 6 / Table II, ids v1..v6 -> 0..5."""
    rp, col = fig1
    adj = adjacency_sets(rp, col)
    edges = [(u - 1, v - 1) for u in range(1, 7) for v in adj[u] if u < v <= 6]
    return csr_from_edges(6, edges)


def test_example1_three_4cliques(fig1):
    rp, col = fig1
    cnt, cks, cl = oracle.plain(rp, col, 4, list_cap=16)
    got = sorted(tuple(int(x) for x in r) for r in cl)
    assert got == [(1, 2, 3, 4), (1, 2, 4, 6), (9, 10, 11, 12)]
    assert cnt == 3
    assert cks == sum(oracle.clique_hash(c) for c in got) % (1 << 64)
    for fn in (oracle.sdegree, oracle.bitcol):
        r = fn(rp, col, 4, list_cap=16)
        assert r["count"] == 3 and r["checksum"] == cks
        assert sorted(tuple(int(x) for x in c) for c in r["cliques"]) == got


def test_example2_precore_removes_v8_then_v7(fig1):
    rp, col = fig1
    alive = oracle.precore(rp, col, 4)
    dead = sorted(int(v) for v in np.nonzero(alive == 0)[0])
    assert dead == [0, 7, 8]  # 0 is the unused isolated id


def test_example3_prelist_removes_the_4clique(fig1):
    rp, col = fig1
    alive = oracle.precore(rp, col, 4)
    r = oracle.prelist(rp, col, 4, alive, list_cap=4)
    assert r["removed"] == 1
    assert r["count"] == 1
    assert [tuple(int(x) for x in c) for c in r["cliques"]] == [(9, 10, 11, 12)]
    left = sorted(int(v) for v in np.nonzero(r["alive"])[0])
    assert left == [1, 2, 3, 4, 5, 6]


def test_example4_sdegree_trace(fig1):
    rp, col = fig1
    alive = oracle.prelist(rp, col, 4, oracle.precore(rp, col, 4))["alive"]
    od = oracle.outdegrees(rp, col, alive, 0)
    assert {v: int(od[v]) for v in range(1, 7)} == {1: 0, 2: 4, 3: 2, 4: 2, 5: 3, 6: 1}
    r = oracle.sdegree(rp, col, 4, list_cap=8, trace_cap=4096)
    calls = r["trace"]
    # only v2 and v5 start SDegreeList; from v2 only v3 and v4 recurse;
    # at v3 the candidate set is {v1, v4}
    assert calls == [
        (3, [2], [1, 3, 4, 6]),
        (2, [2, 3], [1, 4]),
        (2, [2, 4], [1, 6]),
        (3, [5], [1, 3, 6]),
    ]
    assert sorted(tuple(int(x) for x in c) for c in r["cliques"]) == [
        (1, 2, 3, 4), (1, 2, 4, 6), (9, 10, 11, 12)]


def test_example6_colouring_order_and_colours(fig1):
    B, colour, order = _table2()
    rp, col = _fig7_graph(fig1)
    o, c = oracle.colour_graph(rp, col)
    assert [int(x) + 1 for x in o] == order
    assert {v + 1: int(c[v]) for v in range(6)} == colour
    # Section VII-A: v4 has four out-neighbours but colour 4, so it cannot
    # root a 5-clique
    assert colour[4] == 4


def test_table2_bitmaps_L3(fig1):
    B, colour, _ = _table2()
    rp, col = _fig7_graph(fig1)
    c, bits = oracle.bitencode_graph(rp, col, 3)
    assert bits.shape == (6, 2)
    for v in range(1, 7):
        assert [int(x) for x in bits[v - 1]] == B[v], v
    # BitJoin(B(v3), B(v4)) = <3, 0> = {v1, v2}
    assert [int(a) & int(b) for a, b in zip(bits[2], bits[3])] == [3, 0]


def test_bitmap_word_size_does_not_change_results(fig1):
    rp, col = fig1
    ref = oracle.plain(rp, col, 3)
    for L in (1, 3, 5, 24, 32):
        r = oracle.bitcol(rp, col, 3, L=L)
        assert (r["count"], r["checksum"]) == ref


def test_example4_merge_work(fig1):
    """Lemma 2's cost model on Example 4, by hand from the trace above and the
    pinned out-degrees d+ = {v1: 0, v2: 4, v3: 2, v4: 2, v5: 3, v6: 1}: a
    candidate v of a call at level l is merged (|C| + d+_v elements) unless
    d+_v <= l - 2.
      (3, [2], {1,3,4,6}): v3 4+2, v4 4+2 (v1, v6 pruned)  -> 12, 2 joins
      (2, [2,3], {1,4}):   v4 2+2                          ->  4, 1 join
      (2, [2,4], {1,6}):   v6 2+1                          ->  3, 1 join
      (3, [5], {1,3,6}):   v3 3+2                          ->  5, 1 join
    The roofline of the degree-ordered path counts exactly these elements."""
    rp, col = fig1
    r = oracle.sdegree(rp, col, 4, count_only=True)
    assert r["counters"]["merge_elems"] == 12 + 4 + 3 + 5
    assert r["counters"]["intersections"] == 5
    assert r["counters"]["roots"] == 2 and r["counters"]["max_outdeg"] == 4
    # every root has d+ <= 32: one bitmap word per merge join
    assert r["counters"]["bitrow_words"] == 5
