"""The seeded input generators (kclgen): every graph is a valid symmetric
CSR, sizes follow the stated recipes, the same seed gives the same graph,
and planted structure is present.  These inputs feed both the oracle and
the CUDA path."""
import numpy as np
import pytest

import kclgen
import oracle


def _edges(rp, col):
    rp = rp.astype(np.int64)
    u = np.repeat(np.arange(len(rp) - 1), np.diff(rp))
    return u, col.astype(np.int64)


@pytest.mark.parametrize("make", [
    lambda: kclgen.chung_lu(3000, 20000, 2.3, groups=3, group_size=(10, 20), group_p=0.8, seed=4),
    lambda: kclgen.chung_lu(2000, 15000, 2.1, 300.0, seed=5),
    lambda: kclgen.rmat20(seed=2, scale=12),
    lambda: kclgen.planted_only(500, 4, (5, 9), seed=6),
    lambda: kclgen.batch_graph(7)[:2],
])
def test_graphs_are_valid_symmetric_csr(make):
    rp, col = make()
    assert rp.dtype == np.uint64 and col.dtype == np.uint32
    assert int(rp[0]) == 0 and int(rp[-1]) == len(col)
    assert oracle.validate(rp, col)
    u, v = _edges(rp, col)
    assert not np.any(u == v)
    # every row strictly ascending
    same = u[1:] == u[:-1]
    assert np.all(v[1:][same] > v[:-1][same])


def test_rmat_has_exactly_the_requested_unique_edges():
    for scale in (8, 10, 12):
        rp, col = kclgen.rmat20(seed=3, scale=scale)
        assert len(rp) - 1 == 1 << scale
        assert len(col) == 2 * 16 << scale


def test_same_seed_same_graph_other_seed_other_graph():
    a = kclgen.chung_lu(1000, 8000, 2.3, groups=2, group_size=(8, 12), seed=11)
    b = kclgen.chung_lu(1000, 8000, 2.3, groups=2, group_size=(8, 12), seed=11)
    c = kclgen.chung_lu(1000, 8000, 2.3, groups=2, group_size=(8, 12), seed=12)
    assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1])
    assert not (len(a[1]) == len(c[1]) and np.array_equal(a[1], c[1]))
    r1, r2 = kclgen.rmat20(seed=9, scale=10), kclgen.rmat20(seed=9, scale=10)
    assert np.array_equal(r1[1], r2[1])


def test_planted_cliques_are_present():
    # 20 planted 12-cliques: at least 20 12-cliques, and C(12, 5) 5-cliques each
    rp, col = kclgen.chung_lu_planted_small(seed=1)
    assert len(rp) - 1 == 10_000
    assert oracle.plain(rp, col, 12)[0] >= 20
    assert oracle.plain(rp, col, 5)[0] >= 20 * 792
    # planted groups alone at density 1: sum of C(s, k) over the groups
    rp, col = kclgen.planted_only(400, 3, (6, 6), seed=2)
    c3 = oracle.plain(rp, col, 3)[0]
    assert c3 >= 3 * 20  # overlapping groups can only add triangles


def test_batch_recipe_ranges():
    for i in range(0, 64, 7):
        rp, col, k = kclgen.batch_graph(i)
        n = len(rp) - 1
        assert 50 <= n <= 20000 and 3 <= k <= 9
        assert oracle.validate(rp, col)


def test_splitmix64_seeds_are_distinct():
    seen = {kclgen.splitmix64(1, i) for i in range(1000)}
    assert len(seen) == 1000
