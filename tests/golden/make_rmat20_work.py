"""Write tests/golden/rmat20_work.json with the oracle only.

For the R-MAT scale-20 workload (kclgen.rmat20(seed=1): integer-only sampling,
so the graph is identical on every host) and each (k, ordering) pair, the
oracle's count-only mode gives:
  count  -- the exact number of k-cliques (a full-size parity value), and
  work   -- the algorithmic work of the listing recursion: BitJoin words with a
            32-bit word for BitCol (Algorithm 6), merge-join elements
            sum(|C| + d+_v) for SDegree (Algorithm 5, the cost model of
            Lemma 2),
  work_by_outdeg / roots_by_outdeg / count_by_outdeg -- the same work, the
            number of expanded roots and the k-cliques they list, split by
            the root's out-degree d+_u in power-of-two buckets: key "b" holds
            the roots with 2^(b-1) < d+_u <= 2^b.
The roots are split into buckets (and each bucket into interleaved shards)
so that the oracle runs on every core; the count adds the Pre-List cliques
(Algorithm 4), which the per-root runs leave out.
Usage: python tests/golden/make_rmat20_work.py [k ...]
"""
import json
import multiprocessing as mp
import os
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
OUT = os.path.join(HERE, "rmat20_work.json")
SHARDS = 8


def _graph():
    sys.path.insert(0, ROOT)
    import kclgen
    return kclgen.rmat20(seed=1)


def plan(job):
    """Pre-List count and the roots of each out-degree bucket."""
    import numpy as np
    import oracle
    k, ordering = job
    rp, col = _graph()
    alive = oracle.precore(rp, col, k)
    pl = oracle.prelist(rp, col, k, alive)
    od = oracle.outdegrees(rp, col, pl["alive"], 0 if ordering == "degree" else 1)
    od = od.astype(np.int64)
    roots = np.nonzero((pl["alive"] != 0) & (od >= k - 1))[0]
    b = np.ceil(np.log2(np.maximum(od[roots], 1))).astype(np.int64)
    buckets = {}
    for bb in np.unique(b):
        r = roots[b == bb].astype(np.uint32)
        # heaviest roots first so that interleaved shards get equal shares
        r = r[np.argsort(-od[r], kind="stable")]
        buckets[int(bb)] = r
    return pl["count"], buckets


def one(task):
    import oracle
    k, ordering, bucket, roots = task
    rp, col = _graph()
    if ordering == "color":
        r = oracle.bitcol(rp, col, k, L=32, roots=roots, count_only=True)
        work = r["counters"]["bitjoin_words"]
    else:
        r = oracle.sdegree(rp, col, k, roots=roots, count_only=True)
        work = r["counters"]["merge_elems"]
    return (k, ordering), bucket, r["count"], work, r["counters"]


def main():
    ks = [int(a) for a in sys.argv[1:]] or [4, 5]
    jobs = [(k, o) for k in ks for o in ("color", "degree")]
    data = {}
    if os.path.exists(OUT):
        with open(OUT) as f:
            data = json.load(f)
    ctx = mp.get_context("spawn")
    t0 = time.time()
    with ctx.Pool(min(SHARDS, os.cpu_count() or 1)) as pool:
        plans = dict(zip(jobs, pool.map(plan, jobs)))
        tasks = []
        for job, (_, buckets) in plans.items():
            for b, r in buckets.items():
                ns = SHARDS if len(r) >= 64 else 1
                tasks += [(job[0], job[1], b, r[s::ns]) for s in range(ns)]
        tasks.sort(key=lambda t: (-t[0], t[1] == "color", -t[2]))
        acc = {job: {"count": plans[job][0], "work": 0, "counters": {}, "work_by_outdeg": {},
                     "roots_by_outdeg": {}, "count_by_outdeg": {}} for job in jobs}
        left = {job: sum(1 for t in tasks if (t[0], t[1]) == job) for job in jobs}
        for job, b, cnt, work, ctr in pool.imap_unordered(one, tasks):
            a = acc[job]
            a["count"] += cnt
            a["work"] += work
            for name, v in ctr.items():
                a["counters"][name] = (max(a["counters"].get(name, 0), v) if name == "max_outdeg"
                                       else a["counters"].get(name, 0) + v)
            key = str(b)
            a["work_by_outdeg"][key] = a["work_by_outdeg"].get(key, 0) + work
            a["roots_by_outdeg"][key] = a["roots_by_outdeg"].get(key, 0) + ctr["roots"]
            a["count_by_outdeg"][key] = a["count_by_outdeg"].get(key, 0) + cnt
            left[job] -= 1
            if left[job] == 0:
                a["oracle_wall_seconds"] = round(time.time() - t0, 1)
                a["work_by_outdeg"] = dict(sorted(a["work_by_outdeg"].items(), key=lambda x: int(x[0])))
                a["roots_by_outdeg"] = dict(sorted(a["roots_by_outdeg"].items(), key=lambda x: int(x[0])))
                a["count_by_outdeg"] = dict(sorted(a["count_by_outdeg"].items(), key=lambda x: int(x[0])))
                data["k=%d %s" % job] = a
                print("k=%d %s" % job, a, flush=True)
                with open(OUT, "w") as f:
                    json.dump(dict(sorted(data.items())), f, indent=1)


if __name__ == "__main__":
    main()
