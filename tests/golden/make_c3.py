"""Write tests/golden/c3.json with the oracle only: parity values for the
community workload (Chung-Lu, exponent 2.1, expected degree capped at 40,000,
communities of dense planted vertices at density 0.8).

  twin    -- the reduced twin: n = 400,000, 4e6 drawn pairs, exponent 2.1,
             degree cap 300, 200 communities of 60-120 vertices at density
             0.8, seed 1: the exact k = 6 count (oracle BitCol, count-only,
             sharded over the roots by out-degree bucket) and the Pre-List
             count;
  sample  -- the full-size graph (kclgen.chung_lu_communities(seed=1): n =
             4,000,000, 1.2e8 drawn pairs, 2,000 communities of 60-300): the
             k = 6 per-root counts of 200 roots drawn uniformly (numpy
             default_rng(6)) from the roots with out-degree 5..64 in the
             degeneracy DAG, where the oracle's work per root is small (the
             graph's hub core puts its full count beyond the oracle).
Usage: python tests/golden/make_c3.py [twin | sample ...]
"""
import json
import multiprocessing as mp
import os
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
OUT = os.path.join(HERE, "c3.json")
SHARDS = 8
if ROOT not in sys.path:  # spawned workers re-run this module's top level
    sys.path.insert(0, ROOT)

TWIN = dict(n=400_000, m=4_000_000, gamma=2.1, cap=300.0, groups=200, group_size=(60, 120),
            group_p=0.8, seed=1)


def twin_graph():
    import kclgen
    t = TWIN
    return kclgen.chung_lu(t["n"], t["m"], t["gamma"], t["cap"], groups=t["groups"],
                           group_size=t["group_size"], group_p=t["group_p"], seed=t["seed"])


def _twin_plan(k):
    import numpy as np

    import oracle
    rp, col = twin_graph()
    pl = oracle.prelist(rp, col, k, oracle.precore(rp, col, k))
    od = oracle.outdegrees(rp, col, pl["alive"], 1).astype(np.int64)
    roots = np.nonzero((pl["alive"] != 0) & (od >= k - 1))[0]
    roots = roots[np.argsort(-od[roots], kind="stable")].astype(np.uint32)
    return pl["count"], roots


def _twin_shard(task):
    import oracle
    k, roots = task
    rp, col = twin_graph()
    return oracle.bitcol(rp, col, k, L=32, roots=roots, count_only=True)["count"]


def main_twin(data, k=6):
    ctx = mp.get_context("spawn")
    t0 = time.time()
    with ctx.Pool(SHARDS) as pool:
        pre, roots = pool.apply(_twin_plan, (k,))
        tasks = [(k, roots[s::SHARDS * 4]) for s in range(SHARDS * 4)]
        count = pre + sum(pool.imap_unordered(_twin_shard, tasks))
    data["twin"] = {"params": {**TWIN, "group_size": list(TWIN["group_size"])},
                    "k": k, "count": count, "prelist_count": pre,
                    "oracle_wall_seconds": round(time.time() - t0, 1)}
    print("twin k=%d" % k, count, flush=True)


def main_sample(data, k=6):
    import numpy as np

    import kclgen
    import oracle
    rp, col = kclgen.chung_lu_communities(seed=1)
    pl = oracle.prelist(rp, col, k, oracle.precore(rp, col, k))
    od = oracle.outdegrees(rp, col, pl["alive"], 1).astype(np.int64)
    cand = np.nonzero((pl["alive"] != 0) & (od >= k - 1) & (od <= 64))[0]
    roots = np.sort(np.random.default_rng(6).choice(cand, 200, replace=False)).astype(np.uint32)
    r = oracle.bitcol(rp, col, k, L=32, roots=roots, per_root=True, count_only=True)
    data["sample"] = {"k": k, "roots": [int(x) for x in roots],
                      "outdeg": [int(od[x]) for x in roots],
                      "per_root": [int(r["per_root"][x]) for x in roots]}
    print("sample k=%d" % k, len(roots), "roots", int(sum(data["sample"]["per_root"])), flush=True)


def main():
    what = sys.argv[1:] or ["twin", "sample"]
    data = {}
    if os.path.exists(OUT):
        with open(OUT) as f:
            data = json.load(f)
    for w in what:
        {"twin": main_twin, "sample": main_sample}[w](data)
        with open(OUT, "w") as f:
            json.dump(data, f, indent=1)


if __name__ == "__main__":
    main()
