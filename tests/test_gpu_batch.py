"""The batched form (kcl_count_batch) against per-graph calls and the oracle:
each graph's count and checksum must be the same alone and in the batch."""
import numpy as np
import pytest

import kclgen
import oracle

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def kcl():
    import paper_2203_13512_gb300 as kcl
    return kcl


def _small_batch(count, seed):
    rng = np.random.default_rng(seed)
    graphs = []
    for i in range(count):
        n = int(rng.integers(5, 400))
        m = int(n * rng.uniform(2, 12))
        groups = int(rng.integers(0, 4))
        rp, col = kclgen.chung_lu(n, m, 2.3, groups=groups, group_size=(6, 14), seed=seed * 1000 + i)
        graphs.append((rp, col, int(rng.integers(3, 10))))
    return graphs


def test_batch_matches_oracle_and_single_calls(kcl):
    data = _small_batch(48, 7)
    # include degenerate members: empty graph, a single clique (Pre-List)
    data.append((*kclgen.from_edges(0, []), 3))
    data.append((*kclgen.from_edges(9, [(u, v) for u in range(9) for v in range(u + 1, 9)]), 5))
    gs = [kcl.kcl_load_csr(rp, col) for rp, col, _ in data]
    ks = [k for _, _, k in data]
    ords = ["degree" if i % 2 else "color" for i in range(len(data))]
    b = kcl.kcl_batch_create()
    counts, cks = kcl.kcl_count_batch(b, gs, ks, ords, checksums=True)
    counts2, none = kcl.kcl_count_batch(b, gs, ks, ords)
    assert none is None and counts2 == counts
    for i, (rp, col, k) in enumerate(data):
        ref = oracle.plain(rp, col, k)
        assert (counts[i], cks[i]) == ref, i
        assert kcl.kcl_list(gs[i], k, ords[i], None)[:2] == ref
    b.free()


def test_batch_of_the_batched_workload_generator(kcl):
    # the first graphs of the 8,192-graph workload, both orderings
    data = [kclgen.batch_graph(i) for i in range(24)]
    gs = [kcl.kcl_load_csr(rp, col) for rp, col, _ in data]
    ks = [k for _, _, k in data]
    b = kcl.kcl_batch_create()
    for o in ("color", "degree"):
        counts, cks = kcl.kcl_count_batch(b, gs, ks, [o] * len(gs), checksums=True)
        for i, (rp, col, k) in enumerate(data):
            assert (counts[i], cks[i]) == oracle.plain(rp, col, k), (o, i)
    b.free()


_ORACLE_CACHE = {}
# graphs of 33..64 whose k >= 8 counts (5e7 - 2e8 cliques) take the oracle
# 4-22 s each: there the batch is checked against single calls only
_HEAVY = {34, 41, 44, 46, 56}


@pytest.mark.parametrize("ordering", ["color", "degree"])
def test_batch_of_served_queries(kcl, ordering):
    """Batches as the server forms them: graphs 33..64 of the batched
    workload, each query's own k in 3..10 (so one graph can appear twice with
    different k, or twice with the same k), 64 queries per pass; every
    member's count and checksum must equal a single call's and, but for the
    heavy cases above, the oracle's."""
    graphs = {i: kclgen.batch_graph(i)[:2] for i in range(33, 65)}
    loaded = {i: kcl.kcl_load_csr(*graphs[i]) for i in graphs}
    rng = np.random.default_rng(11)
    b = kcl.kcl_batch_create()
    single = {}
    for trial in range(6):
        qs = [(int(rng.integers(33, 65)), int(rng.integers(3, 11))) for _ in range(64)]
        if trial == 0:
            qs[5] = (47, 8)
        counts, cks = kcl.kcl_count_batch(b, [loaded[i] for i, _ in qs], [k for _, k in qs],
                                          [ordering] * len(qs), checksums=True)
        for j, (i, k) in enumerate(qs):
            if (i, k) not in single:
                single[(i, k)] = kcl.kcl_list(loaded[i], k, ordering, None)[:2]
                if not (i in _HEAVY and k >= 8):
                    if (i, k) not in _ORACLE_CACHE:
                        _ORACLE_CACHE[(i, k)] = oracle.plain(*graphs[i], k)
                    assert single[(i, k)] == _ORACLE_CACHE[(i, k)], ("single", i, k)
            assert (counts[j], cks[j]) == single[(i, k)], (trial, j, i, k, counts[j], cks[j],
                                                          single[(i, k)])
    b.free()
    for g in loaded.values():
        g.free()
