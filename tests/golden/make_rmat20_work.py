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
  bitrow_words_by_outdeg (SDegree) -- per bucket, the merge joins of
            Algorithm 5 each costed at ceil(d+_root / 32) words: the words a
            bitmap over the root's out-neighbourhood touches per join.
The roots are split into buckets (and each bucket into interleaved shards)
so that the oracle runs on every core; the count adds the Pre-List cliques
(Algorithm 4), which the per-root runs leave out.

--checksum: also the listing checksum of every k-clique (the oracle's
  listing mode, each clique hashed; additive mod 2^64, so it is summed over
  the same shards plus the Pre-List cliques' checksum).  Each ordering's
  oracle computes it on its own: the two values must agree.
--sample: per-root counts of a seeded sample of roots -- the three with the
  largest out-degree, 40 drawn uniformly from all roots and 2 from every
  out-degree bucket (numpy default_rng(1000 + k)) -- stored as
  "sample": {"roots": [...], "per_root": [...]} for a (k, ordering) whose
  full count is beyond the oracle.
Usage: python tests/golden/make_rmat20_work.py [--checksum | --sample | --color | --degree] [k ...]
       python tests/golden/make_rmat20_work.py --c1   (the small Chung-Lu workload, k = 5)
(--color / --degree: counts and work of that ordering only.)
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
if ROOT not in sys.path:  # spawned workers re-run this module's top level
    sys.path.insert(0, ROOT)


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



def one_checksum(task):
    import oracle
    k, ordering, roots = task
    rp, col = _graph()
    fn = oracle.bitcol if ordering == "color" else oracle.sdegree
    r = fn(rp, col, k, roots=roots)
    return (k, ordering), r["count"], r["checksum"]


def prelist_checksum(k):
    import oracle
    rp, col = _graph()
    pl = oracle.prelist(rp, col, k, oracle.precore(rp, col, k))
    return pl["count"], pl["checksum"]


def main_checksum(ks):
    """Full listing checksums, sharded over roots like the counts."""
    with open(OUT) as f:
        data = json.load(f)
    jobs = [(k, o) for k in ks for o in ("color", "degree")]
    ctx = mp.get_context("spawn")
    with ctx.Pool(min(SHARDS, os.cpu_count() or 1)) as pool:
        plans = dict(zip(jobs, pool.map(plan, jobs)))
        pre = dict(zip(ks, pool.map(prelist_checksum, ks)))
        tasks = []
        for job, (_, buckets) in plans.items():
            for b, r in buckets.items():
                ns = SHARDS if len(r) >= 64 else 1
                tasks += [(job[0], job[1], r[s::ns]) for s in range(ns)]
        acc = {job: [pre[job[0]][0], pre[job[0]][1]] for job in jobs}
        for job, cnt, cks in pool.imap_unordered(one_checksum, tasks):
            acc[job][0] += cnt
            acc[job][1] = (acc[job][1] + cks) % (1 << 64)
    for job, (cnt, cks) in acc.items():
        key = "k=%d %s" % job
        assert cnt == data[key]["count"], (key, cnt)
        data[key]["checksum"] = cks
        print(key, cnt, hex(cks), flush=True)
    for k in ks:
        assert acc[(k, "color")][1] == acc[(k, "degree")][1], "orderings disagree at k=%d" % k
    with open(OUT, "w") as f:
        json.dump(dict(sorted(data.items())), f, indent=1)


def sample_roots(job):
    """The seeded root sample of one (k, ordering)."""
    import numpy as np
    import oracle
    k, ordering = job
    rp, col = _graph()
    pl = oracle.prelist(rp, col, k, oracle.precore(rp, col, k))
    od = oracle.outdegrees(rp, col, pl["alive"], 0 if ordering == "degree" else 1).astype(np.int64)
    roots = np.nonzero((pl["alive"] != 0) & (od >= k - 1))[0]
    rng = np.random.default_rng(1000 + k)
    pick = list(roots[np.argsort(-od[roots], kind="stable")[:3]])
    pick += list(rng.choice(roots, 40, replace=False))
    b = np.ceil(np.log2(np.maximum(od[roots], 1))).astype(np.int64)
    for bb in np.unique(b):
        r = roots[b == bb]
        pick += list(rng.choice(r, min(2, len(r)), replace=False))
    return sorted(set(int(x) for x in pick)), [int(od[x]) for x in sorted(set(int(x) for x in pick))]


def one_sample(task):
    import numpy as np
    import oracle
    k, ordering, roots = task
    rp, col = _graph()
    fn = oracle.bitcol if ordering == "color" else oracle.sdegree
    r = fn(rp, col, k, roots=np.array(roots, np.uint32), per_root=True, count_only=True)
    return (k, ordering), {int(x): int(r["per_root"][x]) for x in roots}


def main_sample(ks):
    data = {}
    if os.path.exists(OUT):
        with open(OUT) as f:
            data = json.load(f)
    jobs = [(k, o) for k in ks for o in ("color", "degree")]
    ctx = mp.get_context("spawn")
    with ctx.Pool(min(SHARDS, os.cpu_count() or 1)) as pool:
        picks = dict(zip(jobs, pool.map(sample_roots, jobs)))
        tasks = []
        for job, (roots, ods) in picks.items():
            heavy = [r for r, d in sorted(zip(roots, ods), key=lambda x: -x[1])[:3]]
            rest = [r for r in roots if r not in heavy]
            tasks += [(job[0], job[1], [h]) for h in heavy]
            tasks += [(job[0], job[1], rest[s::4]) for s in range(4)]
        got = {job: {} for job in jobs}
        for job, part in pool.imap_unordered(one_sample, tasks):
            got[job].update(part)
    for job in jobs:
        key = "k=%d %s" % job
        roots = picks[job][0]
        entry = data.setdefault(key, {})
        entry["sample"] = {"roots": roots, "outdeg": picks[job][1],
                           "per_root": [got[job][r] for r in roots]}
        print(key, len(roots), "sampled roots", flush=True)
    with open(OUT, "w") as f:
        json.dump(dict(sorted(data.items())), f, indent=1)


def main_c1():
    """The small Chung-Lu workload (n = 10,000, 50,000 drawn pairs, exponent
    2.5, 20 planted 12-cliques, seed 1) at k = 5: the oracle's count and
    checksum, stored as "c1 k=5"."""
    import kclgen
    import oracle
    rp, col = kclgen.chung_lu_planted_small(seed=1)
    cnt, cks = oracle.plain(rp, col, 5)
    data = {}
    if os.path.exists(OUT):
        with open(OUT) as f:
            data = json.load(f)
    data["c1 k=5"] = {"count": cnt, "checksum": cks, "n": len(rp) - 1, "undirected_edges": len(col) // 2}
    with open(OUT, "w") as f:
        json.dump(dict(sorted(data.items())), f, indent=1)
    print("c1 k=5", cnt, hex(cks))


def main():
    args = sys.argv[1:]
    if args and args[0] == "--c1":
        return main_c1()
    if args and args[0] == "--checksum":
        return main_checksum([int(a) for a in args[1:]] or [4])
    if args and args[0] == "--sample":
        return main_sample([int(a) for a in args[1:]] or [6])
    orderings = ("color", "degree")
    if args and args[0] in ("--color", "--degree"):
        orderings = (args[0][2:],)
        args = args[1:]
    ks = [int(a) for a in args] or [4, 5]
    jobs = [(k, o) for k in ks for o in orderings]
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
            if job[1] == "degree":
                bw = a.setdefault("bitrow_words_by_outdeg", {})
                bw[key] = bw.get(key, 0) + ctr["bitrow_words"]
            left[job] -= 1
            if left[job] == 0:
                a["oracle_wall_seconds"] = round(time.time() - t0, 1)
                a["work_by_outdeg"] = dict(sorted(a["work_by_outdeg"].items(), key=lambda x: int(x[0])))
                a["roots_by_outdeg"] = dict(sorted(a["roots_by_outdeg"].items(), key=lambda x: int(x[0])))
                a["count_by_outdeg"] = dict(sorted(a["count_by_outdeg"].items(), key=lambda x: int(x[0])))
                if "bitrow_words_by_outdeg" in a:
                    a["bitrow_words_by_outdeg"] = dict(sorted(a["bitrow_words_by_outdeg"].items(),
                                                              key=lambda x: int(x[0])))
                old = data.get("k=%d %s" % job, {})
                for keep in ("checksum", "sample"):  # written by the other modes
                    if keep in old:
                        a[keep] = old[keep]
                data["k=%d %s" % job] = a
                print("k=%d %s" % job, a, flush=True)
                with open(OUT, "w") as f:
                    json.dump(dict(sorted(data.items())), f, indent=1)


if __name__ == "__main__":
    main()
