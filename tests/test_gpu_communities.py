"""Dense planted communities on a heavy-tailed base graph: the shape of the
4M-vertex community workload (exponent 2.1, communities of 60-300 vertices at
density 0.8) at reduced scale, against the oracle.  Counts and listing
checksums are exact."""
import numpy as np
import pytest

import kclgen
import oracle

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def kcl():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    import paper_2203_13512_gb300 as kcl
    return kcl


@pytest.fixture(scope="module")
def twin():
    """n = 100,000, 1e6 drawn pairs, exponent 2.1, degree cap 300, and 40
    communities of 60-90 vertices at density 0.8 (3.4e8 6-cliques)."""
    return kclgen.chung_lu(100_000, 1_000_000, 2.1, 300.0, groups=40, group_size=(60, 90),
                           group_p=0.8, seed=1)


@pytest.fixture(scope="module")
def small_twin():
    """n = 20,000, 2e5 drawn pairs, 10 communities: small enough for the
    oracle's listing checksum at k = 5, 6."""
    return kclgen.chung_lu(20_000, 200_000, 2.1, 300.0, groups=10, group_size=(60, 90),
                           group_p=0.8, seed=2)


def test_twin_counts_both_orderings(kcl, twin):
    rp, col = twin
    g = kcl.kcl_load_csr(rp, col)
    want = oracle.bitcol(rp, col, 6, L=32, count_only=True)["count"]
    assert kcl.kcl_count(g, 6, "color") == want
    assert kcl.kcl_count(g, 6, "degree") == want


@pytest.mark.parametrize("k", [5, 6])
def test_small_twin_listing_checksums(kcl, small_twin, k):
    rp, col = small_twin
    g = kcl.kcl_load_csr(rp, col)
    want = oracle.plain(rp, col, k)
    for o in ("color", "degree"):
        c, s, _, _ = kcl.kcl_list(g, k, o, None)
        assert (c, s) == want, o


def test_twin_per_root_sample(kcl, twin):
    """Per-root counts at k = 7 on a seeded sample of roots (the full count
    is beyond the oracle's budget here)."""
    import torch
    rp, col = twin
    n = len(rp) - 1
    g = kcl.kcl_load_csr(rp, col)
    pr = torch.zeros(n, dtype=torch.int64, device="cuda")
    kcl.kcl_count_per_root(g, 7, "color", pr)
    got = pr.cpu().numpy().astype(np.uint64)
    roots = np.random.default_rng(1).choice(n, 400, replace=False).astype(np.uint32)
    ref = oracle.bitcol(rp, col, 7, L=32, roots=roots, per_root=True)["per_root"]
    assert np.array_equal(got[roots], ref[roots])
