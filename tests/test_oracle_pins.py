"""The oracle pinned to things other than itself: brute force, closed forms,
published hash test vectors, invariants and the paper's bounds."""
import itertools

import numpy as np
import pytest

import kclgen
import oracle
from tests.graphs import (GOLD, M64, brute_cliques_bitmask, brute_cliques_subsets, comb,
                          complete, csr_from_edges, disjoint_union, elementary_symmetric, gnp,
                          relabel, turan)


def _checksum(cliques):
    return sum(oracle.clique_hash(c) for c in cliques) % (1 << 64)


# ------------------------------------------------------------------ hash
def test_splitmix64_published_outputs():
    # SplitMix64 seeded with 0 (Steele, Lea & Flood): the first three outputs
    # are the finaliser applied to 1, 2 and 3 times the golden gamma.
    assert oracle.mix64(GOLD) == 0xE220A8397B1DCDAF
    assert oracle.mix64((2 * GOLD) & M64) == 0x6E789E6AA1B965F4
    assert oracle.mix64((3 * GOLD) & M64) == 0x06C45D188009454F


def test_clique_hash_is_the_stated_chain():
    # H(v_1..v_k) chains the finaliser over GOLD ^ k then each sorted id;
    # the published outputs give the first link for k = 0 (empty tuple).
    assert oracle.clique_hash([]) == 0xE220A8397B1DCDAF
    assert oracle.clique_hash([5, 3, 9]) == oracle.clique_hash([3, 5, 9])


# ------------------------------------------------------------ brute force
@pytest.mark.parametrize("seed", range(12))
def test_plain_vs_subset_brute_force(seed):
    rng = np.random.default_rng(100 + seed)
    n = int(rng.integers(4, 17))
    p = float(rng.choice([0.1, 0.3, 0.5, 0.7, 0.9]))
    rp, col = gnp(n, p, seed)
    for k in range(1, min(n, 9) + 1):
        ref = brute_cliques_subsets(rp, col, k)
        cnt, cks, cl = oracle.plain(rp, col, k, list_cap=len(ref) + 1)
        assert cnt == len(ref)
        assert sorted(tuple(int(x) for x in r) for r in cl) == ref
        assert cks == _checksum(ref)


@pytest.mark.parametrize("seed", range(8))
def test_all_modes_vs_bitmask_brute_force(seed):
    rng = np.random.default_rng(200 + seed)
    n = int(rng.integers(18, 41))
    p = float(rng.choice([0.2, 0.4, 0.6, 0.8]))
    rp, col = gnp(n, p, 1000 + seed)
    for k in range(3, 9):
        ref = brute_cliques_bitmask(rp, col, k)
        want = (len(ref), _checksum(ref))
        assert oracle.plain(rp, col, k) == want
        for pre in (True, False):
            for r in (oracle.sdegree(rp, col, k, preprocess=pre),
                      oracle.bitcol(rp, col, k, preprocess=pre, L=24),
                      oracle.bitcol(rp, col, k, preprocess=pre, L=32),
                      oracle.bitcol(rp, col, k, preprocess=pre, L=7)):
                assert (r["count"], r["checksum"]) == want, (k, pre)


def test_listing_has_no_duplicates_and_only_cliques():
    rp, col = kclgen.chung_lu(300, 2000, 2.3, groups=3, group_size=(9, 12), seed=5)
    adj = [set(col[rp[u]:rp[u + 1]].tolist()) for u in range(len(rp) - 1)]
    for k in (3, 4, 6):
        for r in (oracle.sdegree(rp, col, k, list_cap=10**6), oracle.bitcol(rp, col, k, list_cap=10**6)):
            tuples = [tuple(int(x) for x in c) for c in r["cliques"]]
            assert len(tuples) == r["count"] == len(set(tuples))
            for t in tuples:
                assert list(t) == sorted(t)
                assert all(b in adj[a] for a, b in itertools.combinations(t, 2))


# ----------------------------------------------------------- closed forms
@pytest.mark.parametrize("n", [1, 3, 5, 9, 14])
def test_complete_graph_binomial(n):
    rp, col = complete(n)
    for k in range(1, n + 2):
        want = comb(n, k)
        assert oracle.plain(rp, col, k)[0] == want
        if k >= 3:
            assert oracle.sdegree(rp, col, k)["count"] == want
            assert oracle.bitcol(rp, col, k)["count"] == want


@pytest.mark.parametrize("parts", [(3, 3, 3), (2, 4, 1, 5), (5, 5), (1, 1, 1, 1, 1, 1), (4, 2, 3, 3, 2)])
def test_turan_graph_elementary_symmetric(parts):
    rp, col = turan(parts)
    for k in range(3, len(parts) + 2):
        want = elementary_symmetric(parts, k)
        assert oracle.plain(rp, col, k)[0] == want
        assert oracle.sdegree(rp, col, k)["count"] == want
        assert oracle.bitcol(rp, col, k)["count"] == want


def test_empty_and_matching_graphs():
    rp, col = csr_from_edges(10, [])
    assert oracle.plain(rp, col, 3) == (0, 0)
    rp, col = csr_from_edges(10, [(2 * i, 2 * i + 1) for i in range(5)])
    assert oracle.plain(rp, col, 2)[0] == 5
    for k in (3, 4):
        assert oracle.sdegree(rp, col, k)["count"] == 0
        assert oracle.bitcol(rp, col, k)["count"] == 0


@pytest.mark.parametrize("seed", range(3))
def test_triangles_equal_trace_a_cubed_over_six(seed):
    rp, col = kclgen.chung_lu(400, 3000, 2.2, groups=2, group_size=(8, 10), seed=seed + 7)
    n = len(rp) - 1
    A = np.zeros((n, n), dtype=np.int64)
    for u in range(n):
        A[u, col[rp[u]:rp[u + 1]]] = 1
    tri = int(np.trace(A @ A @ A)) // 6
    assert oracle.plain(rp, col, 3)[0] == tri
    assert oracle.sdegree(rp, col, 3)["count"] == tri
    assert oracle.bitcol(rp, col, 3)["count"] == tri
    assert oracle.plain(rp, col, 2)[0] == len(col) // 2


# ---------------------------------------------------------------- readings
def test_precore_keeps_the_k_minus_1_core():
    # K_k alone must give one k-clique: a "degree >= k" threshold would wipe it
    for k in (3, 5, 8):
        rp, col = complete(k)
        assert oracle.precore(rp, col, k).all()
        assert oracle.sdegree(rp, col, k)["count"] == 1
        assert oracle.bitcol(rp, col, k)["count"] == 1


def test_prelist_uses_directed_edge_count():
    # A 5-cycle has degree sum 10 = 5*4/2; only the directed count
    # n_c (n_c - 1) = 20 identifies cliques, so it must not be reported.
    rp, col = csr_from_edges(5, [(i, (i + 1) % 5) for i in range(5)])
    r = oracle.prelist(rp, col, 3, np.ones(5, np.uint8))
    assert r["removed"] == 0 and r["count"] == 0 and r["alive"].all()
    rp, col = complete(6)
    r = oracle.prelist(rp, col, 3, np.ones(6, np.uint8))
    assert r["removed"] == 1 and r["count"] == comb(6, 3) and not r["alive"].any()


def test_prelist_component_smaller_than_k():
    rp, col = complete(3)
    r = oracle.prelist(rp, col, 5, np.ones(3, np.uint8))
    assert r["removed"] == 1 and r["count"] == 0


def _core_numbers(rp, col):
    """Textbook one-at-a-time min-degree peel (Batagelj-Zaversnik order)."""
    n = len(rp) - 1
    adj = [set(col[rp[u]:rp[u + 1]].tolist()) for u in range(n)]
    deg = [len(a) for a in adj]
    gone = [False] * n
    core = [0] * n
    cur = 0
    for _ in range(n):
        u = min((v for v in range(n) if not gone[v]), key=lambda v: deg[v])
        cur = max(cur, deg[u])
        core[u] = cur
        gone[u] = True
        for v in adj[u]:
            if not gone[v]:
                deg[v] -= 1
    return core


@pytest.mark.parametrize("seed", range(4))
def test_degeneracy_rounds_give_degeneracy_bounded_outdegree(seed):
    rp, col = kclgen.chung_lu(250, 1800, 2.3, groups=2, group_size=(7, 11), seed=seed + 20)
    n = len(rp) - 1
    alive = np.ones(n, np.uint8)
    rounds, beta = oracle.degeneracy_rounds(rp, col, alive)
    core = _core_numbers(rp, col)
    assert beta == max(core)
    od = oracle.outdegrees(rp, col, alive, 1)
    assert int(od.max()) <= beta
    # the (k-1)-core of Pre-Core is the set of vertices with core number >= k-1
    for k in (3, 5, 8):
        assert [int(x) for x in oracle.precore(rp, col, k)] == [1 if c >= k - 1 else 0 for c in core]


def test_colouring_is_proper_and_greedy():
    rp, col = kclgen.chung_lu(120, 900, 2.2, groups=2, group_size=(10, 12), seed=3)
    order, colour = oracle.colour_graph(rp, col)
    n = len(rp) - 1
    deg = np.diff(rp.astype(np.int64))
    keys = [(-int(deg[v]), v) for v in order]
    assert keys == sorted(keys)
    pos = {int(v): i for i, v in enumerate(order)}
    for u in range(n):
        nb = col[rp[u]:rp[u + 1]]
        assert all(colour[u] != colour[v] for v in nb)
        earlier = {int(colour[v]) for v in nb if pos[int(v)] < pos[u]}
        assert int(colour[u]) == min(c for c in range(1, n + 2) if c not in earlier)


# --------------------------------------------------------------- invariants
@pytest.mark.parametrize("seed", range(3))
def test_relabelling_and_disjoint_union(seed):
    g = kclgen.chung_lu(200, 1500, 2.3, groups=2, group_size=(8, 10), seed=40 + seed)
    h = kclgen.chung_lu(150, 900, 2.5, groups=1, group_size=(9, 9), seed=50 + seed)
    n = len(g[0]) - 1
    perm = np.random.default_rng(seed).permutation(n)
    gp = relabel(g, perm)
    u = disjoint_union(g, h)
    for k in (3, 4, 6):
        c, s, cl = oracle.plain(*g, k, list_cap=10**6)
        cp, sp = oracle.plain(*gp, k)
        assert cp == c
        assert sp == _checksum([[int(perm[x]) for x in t] for t in cl])
        ch = oracle.plain(*h, k)[0]
        assert oracle.plain(*u, k)[0] == c + ch
        assert oracle.sdegree(*u, k)["count"] == c + ch


@pytest.mark.parametrize("k", [3, 5, 7])
def test_per_root_counts_sum_to_total(k):
    rp, col = kclgen.chung_lu(500, 3000, 2.3, groups=4, group_size=(8, 14), seed=k)
    total = oracle.plain(rp, col, k)[0]
    for fn in (oracle.sdegree, oracle.bitcol):
        r = fn(rp, col, k, per_root=True)
        pre = oracle.prelist(rp, col, k, oracle.precore(rp, col, k))["count"]
        assert int(r["per_root"].sum()) + pre == total == r["count"]
        # per-root mode on a subset reproduces the same per-root values
        roots = [int(v) for v in np.nonzero(r["per_root"])[0][:7]]
        sub = fn(rp, col, k, roots=roots, per_root=True)
        assert sub["count"] == sum(int(r["per_root"][v]) for v in roots)


def test_sdegree_work_within_theorem_bound():
    # Theorem 3: SDegreeList costs at most 6 k m (Delta/2)^(k-2) element steps
    rp, col = kclgen.chung_lu(800, 6000, 2.3, groups=3, group_size=(9, 13), seed=9)
    m = len(col) // 2
    for k in (3, 4, 5, 6):
        r = oracle.sdegree(rp, col, k, preprocess=False)
        d = r["counters"]["max_outdeg"]
        assert r["counters"]["merge_elems"] <= 6 * k * m * (d / 2) ** (k - 2)


def test_bitcol_outdegree_bounded_by_degeneracy():
    rp, col = kclgen.chung_lu(600, 5000, 2.2, groups=3, group_size=(10, 15), seed=11)
    _, beta = oracle.degeneracy_rounds(rp, col)
    r = oracle.bitcol(rp, col, 4, preprocess=False)
    assert r["counters"]["max_outdeg"] <= beta


def test_small_workload_all_modes_agree():
    rp, col = kclgen.chung_lu_planted_small(seed=1)
    want = oracle.plain(rp, col, 5)
    assert want[0] >= 20 * comb(12, 5)
    assert (oracle.sdegree(rp, col, 5)["count"], oracle.sdegree(rp, col, 5)["checksum"]) == want
    r = oracle.bitcol(rp, col, 5)
    assert (r["count"], r["checksum"]) == want


@pytest.mark.parametrize("k", [3, 4, 6])
def test_count_only_mode_matches_enumeration(k):
    # the count-only mode (used to count algorithmic work on large inputs)
    # must walk the same recursion: same count, counters and per-root values
    rp, col = kclgen.chung_lu(700, 5000, 2.3, groups=3, group_size=(10, 16), seed=30 + k)
    for fn, kw in ((oracle.sdegree, {}), (oracle.bitcol, {"L": 32}), (oracle.bitcol, {"L": 24})):
        full = fn(rp, col, k, per_root=True, **kw)
        fast = fn(rp, col, k, per_root=True, count_only=True, **kw)
        assert fast["count"] == full["count"] == oracle.plain(rp, col, k)[0]
        assert fast["counters"] == full["counters"]
        assert np.array_equal(fast["per_root"], full["per_root"])


@pytest.mark.parametrize("L,k,joins,words", [(32, 3, 10, 10), (32, 4, 16, 16), (3, 4, 16, 30)])
def test_bitjoin_work_closed_form_on_K6(L, k, joins, words):
    """BitCol's work counters on K_6 without preprocessing, derived by hand.
    Every vertex has degree 5, so the bulk peel removes all of them in round
    0 and the DAG is by id: root u has h = 5 - u out-neighbours, G_u is K_h,
    the greedy colouring gives local vertex i colour i + 1 and B(i) = {0..i-1}.
    k = 3: the roots with h >= 2 join every v >= 1 once: sum (h - 1) over
    h = 2..5 = 10 joins.  k = 4: roots with h >= 3; each v >= 2 is joined at
    level 3 and its C' = {0..v-1} (size v >= 2) recurses with v - 1 joins, so
    a root costs sum_{v=2}^{h-1} v: 9 + 5 + 2 = 16 joins.  Each join touches
    ceil(h / L) words: 16 at L = 32; 9*2 + 5*2 + 2*1 = 30 at L = 3."""
    rp, col = complete(6)
    r = oracle.bitcol(rp, col, k, preprocess=False, L=L, count_only=True)
    assert r["count"] == comb(6, k)
    assert r["counters"]["intersections"] == joins
    assert r["counters"]["bitjoin_words"] == words


# ------------------------------------------------------------ validation
def _valid_by_definition(n, rp, col):
    """Problem input (Section III-A): an undirected simple graph as CSR --
    offsets start at 0 and never decrease, every id < n, no self-loop, each
    row strictly ascending (no duplicate), and v in row u iff u in row v."""
    if rp[0] != 0 or any(rp[i + 1] < rp[i] for i in range(n)):
        return False
    rows = [list(col[rp[u]:rp[u + 1]]) for u in range(n)]
    for u, r in enumerate(rows):
        if any(v >= n or v == u for v in r):
            return False
        if any(r[i] >= r[i + 1] for i in range(len(r) - 1)):
            return False
    return all(u in rows[v] for u, r in enumerate(rows) for v in r)


def test_validate_rejects_each_kind_of_malformed_input():
    bad = {
        "asymmetric": ([0, 1, 1], [1]),
        "self-loops": ([0, 1, 2], [0, 1]),
        "duplicate edge": ([0, 2, 4], [1, 1, 0, 0]),
        "unsorted row": ([0, 2, 3, 4], [2, 1, 0, 0]),
        "id out of range": ([0, 1, 2], [5, 0]),
        "row_ptr[0] != 0": ([1, 1, 2], [1, 0]),
        "decreasing row_ptr": ([0, 2, 1, 3], [1, 2, 0]),
    }
    for what, (rp, col) in bad.items():
        rp = np.array(rp, np.uint64)
        col = np.array(col, np.uint32)
        assert not oracle.validate(rp, col), what
    good = [csr_from_edges(0, []), csr_from_edges(4, []), csr_from_edges(3, [(0, 1), (1, 2)]),
            complete(6), gnp(30, 0.3, 5)]
    for rp, col in good:
        assert oracle.validate(rp, col)


def test_validate_matches_the_definition_on_every_tiny_input():
    """Brute force: all 0/1 adjacency matrices on 3 vertices (self-loops and
    asymmetric pairs included), and random row orders / duplicated entries on
    4-5 vertices, judged against the definition written out above."""
    for bits in range(1 << 9):
        n = 3
        rows = [[v for v in range(n) if bits >> (3 * u + v) & 1] for u in range(n)]
        rp = np.cumsum([0] + [len(r) for r in rows]).astype(np.uint64)
        col = np.array([v for r in rows for v in r], np.uint32)
        assert oracle.validate(rp, col) == _valid_by_definition(n, rp, col), bits
    rng = np.random.default_rng(9)
    for _ in range(400):
        n = int(rng.integers(4, 6))
        a = rng.random((n, n)) < 0.5
        if rng.random() < 0.5:
            a = a | a.T
        rows = [list(np.nonzero(a[u])[0]) for u in range(n)]
        for r in rows:
            if r and rng.random() < 0.2:
                r.append(r[int(rng.integers(len(r)))])
            if rng.random() < 0.2:
                rng.shuffle(r)
            if rng.random() < 0.7:
                r.sort()
        rp = np.cumsum([0] + [len(r) for r in rows]).astype(np.uint64)
        col = np.array([v for r in rows for v in r], np.uint32)
        assert oracle.validate(rp, col) == _valid_by_definition(n, rp, col)


@pytest.mark.parametrize("n", [40, 70])
def test_sdegree_bitrow_words_closed_form_on_Kn(n):
    """SDegree's bitmap-width work counter on K_n (k = 3, no preprocessing),
    derived by hand.  All degrees are equal, so the degree DAG is by id: root
    u has d+ = n-1-u out-neighbours v > u and is a root when d+ >= 2 (u <=
    n-3).  Its call is at level 2, where a candidate v is merged unless
    d+_v <= 0 (v = n-1): n-2-u joins, (n-2)(n-1)/2 in all.  Each join at root
    u counts ceil((n-1-u) / 32) words."""
    rp, col = complete(n)
    r = oracle.sdegree(rp, col, 3, preprocess=False, count_only=True)
    joins = sum(n - 2 - u for u in range(n - 2))
    assert joins == (n - 2) * (n - 1) // 2
    words = sum((n - 2 - u) * -(-(n - 1 - u) // 32) for u in range(n - 2))
    assert r["count"] == comb(n, 3)
    assert r["counters"]["intersections"] == joins
    assert r["counters"]["bitrow_words"] == words
