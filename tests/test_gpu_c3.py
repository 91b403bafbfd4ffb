"""The community workload (Chung-Lu, exponent 2.1, dense planted
communities at density 0.8) against the oracle's stored values
(tests/golden/c3.json, written by tests/golden/make_c3.py):

  - the reduced twin (n = 400,000, 4e6 drawn pairs, degree cap 300, 200
    communities of 60-120 vertices): the exact k = 6 count, both orderings;
  - the full-size graph (n = 4,000,000, 1.2e8 drawn pairs, degree cap
    40,000, 2,000 communities of 60-300): per-root k = 6 counts of 200
    seeded roots, through kcl_count_roots (the graph's hub core puts its full
    count beyond the oracle, and beyond a test's time)."""
import json
import os

import numpy as np
import pytest

import kclgen

pytestmark = pytest.mark.gpu

GOLD = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "c3.json")


@pytest.fixture(scope="module")
def kcl():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    import paper_2203_13512_gb300 as kcl
    return kcl


@pytest.fixture(scope="module")
def gold():
    with open(GOLD) as f:
        return json.load(f)


def test_twin_k6_count(kcl, gold):
    t = gold["twin"]
    p = t["params"]
    rp, col = kclgen.chung_lu(p["n"], p["m"], p["gamma"], p["cap"], groups=p["groups"],
                              group_size=tuple(p["group_size"]), group_p=p["group_p"], seed=p["seed"])
    g = kcl.kcl_load_csr(rp, col)
    kcl.kcl_set_time_limit(g, 600_000)
    for o in ("color", "degree"):
        assert kcl.kcl_count(g, t["k"], o) == t["count"], o


def test_full_size_sampled_roots(kcl, gold):
    import torch
    e = gold["sample"]
    rp, col = kclgen.chung_lu_communities(seed=1)
    n = len(rp) - 1
    g = kcl.kcl_load_csr(rp, col)
    kcl.kcl_set_time_limit(g, 600_000)
    roots = np.array(e["roots"], np.uint32)
    pr = torch.zeros(n, dtype=torch.int64, device="cuda")
    tot = kcl.kcl_count_roots(g, e["k"], "color", roots, pr)
    per = pr.cpu().numpy().astype(np.uint64)
    assert [int(x) for x in per[roots]] == e["per_root"]
    assert tot == sum(e["per_root"]) and int(per.sum()) == tot
    od = kcl.kcl_stage_info(g, e["k"], "color")["outdeg"]
    assert [int(x) for x in od[roots]] == e["outdeg"]
