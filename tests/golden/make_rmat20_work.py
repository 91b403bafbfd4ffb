"""Write tests/golden/rmat20_work.json with the oracle only.

For the R-MAT scale-20 workload (kclgen.rmat20(seed=1): integer-only sampling,
so the graph is identical on every host) and each (k, ordering) pair, the
oracle's count-only mode gives:
  count  -- the exact number of k-cliques (a full-size parity value), and
  work   -- the algorithmic work of the listing recursion: BitJoin words with a
            32-bit word for BitCol (Algorithm 6), merge-join elements
            sum(|C| + d+_v) for SDegree (Algorithm 5, the cost model of
            Lemma 2).
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


def one(job):
    sys.path.insert(0, ROOT)
    import kclgen
    import oracle
    k, ordering = job
    rp, col = kclgen.rmat20(seed=1)
    t = time.time()
    if ordering == "color":
        r = oracle.bitcol(rp, col, k, L=32, count_only=True)
        work = r["counters"]["bitjoin_words"]
    else:
        r = oracle.sdegree(rp, col, k, count_only=True)
        work = r["counters"]["merge_elems"]
    return "k=%d %s" % (k, ordering), {"count": r["count"], "work": work,
                                      "counters": r["counters"],
                                      "oracle_seconds": round(time.time() - t, 1)}


def main():
    ks = [int(a) for a in sys.argv[1:]] or [4, 5]
    jobs = [(k, o) for k in ks for o in ("color", "degree")]
    data = {}
    if os.path.exists(OUT):
        with open(OUT) as f:
            data = json.load(f)
    with mp.get_context("spawn").Pool(min(len(jobs), os.cpu_count() or 1)) as pool:
        for key, val in pool.imap_unordered(one, jobs):
            data[key] = val
            print(key, val, flush=True)
            with open(OUT, "w") as f:
                json.dump(dict(sorted(data.items())), f, indent=1)


if __name__ == "__main__":
    main()
