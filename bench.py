"""Benchmark: k-cliques/s of the GB300 k-clique library on the R-MAT scale-20
workload (2^20 vertices, 16*2^20 unique undirected edges, a=0.57 b=0.19
c=0.19 d=0.05, seed 1), SDegree (degree ordering) and BitCol (colour
ordering), counting mode and listing mode.

One step = every (k, ordering, mode) call of STEP_PLAN on the resident
graph: Pre-Core, Pre-List, orientation and the listing kernels run inside
each call; the listing calls write every clique (k uint32 ids) into a 4 GiB
device ring that wraps, and return the exact count and checksum.  `value` =
sum of the k-clique counts of the step / device time of the step (CUDA
events on the stream the library runs on).  `e2e` = the same metric through
the C ABI from pinned host buffers: graph copy-in (validated on the device),
the step's calls and the read-back of every count/checksum.  Every count and
checksum is checked against the oracle's stored full-size values
(tests/golden/rmat20_work.json); a mismatch aborts the run.

After the timed steps, the k = 6 counts (both orderings) are timed once each
(`c2_k6`: 2.8e13 cliques, seconds per call, so not part of the step); k = 7
is out of reach of a bench run (12 s per call already at scale 17).

The roofline denominators are measured by kcl_measure_int_peaks (per-SM
rates of the BitJoin word, the SplitMix64 round, ...) times the SM count
and the SM clock sampled during the timed region; the front-end passes are
reported against the measured HBM copy bandwidth (MEASURED_PEAKS.json).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

--impl reference times the CPU oracle (oracle/, all host cores) on a
bounded sample of the same plan: a fixed set of roots of each call's DAG.
Multi-GPU: the path does not shard (one graph per GPU); N ranks run
independent replicas and `value` is the total over ranks / the slowest rank.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

SCALE = 20
STEP_PLAN = [  # (k, ordering, mode)
    (4, "color", "count"), (5, "color", "count"), (4, "degree", "count"), (5, "degree", "count"),
    (4, "color", "list"), (4, "degree", "list"),
]
K6_PLAN = [(6, "color", "count"), (6, "degree", "count")]
METRIC = "k-cliques/s (bit-exact counts; R-MAT scale 20, SDegree + BitCol)"
L2_BYTES = 129 * 2 ** 20
RING_BYTES = 4 << 30  # listing ring (wraps)


def _peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            return json.load(f), "measured"
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "sm_max_mhz": 2070.0}, "fallback"


class ClockSampler:
    """nvidia-smi clock / throttle sampling during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), "--query-gpu=" + self.FIELDS,
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        with open(self.path) as f:
            for line in f:
                p = [x.strip() for x in line.split(",")]
                if len(p) < 9:
                    continue
                try:
                    sm.append(float(p[1]))
                    mx.append(float(p[2]))
                except ValueError:
                    continue
                for name, val in zip(names, p[5:9]):
                    if val.lower().startswith("active"):
                        reasons.add(name)
        os.unlink(self.path)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def workload():
    import kclgen
    rp, col = kclgen.rmat20(seed=1, scale=SCALE)
    return rp, col


# --------------------------------------------------------------- our arm
def check_golden(per_call, golden):
    """Every count (and listing checksum) of the plan against the oracle's
    stored full-size values; raises on a mismatch.  Returns the checked keys."""
    checked = []
    for (k, o, m, c, s) in per_call:
        e = golden.get("k=%d %s" % (k, o))
        if not e:
            continue
        if c != e["count"]:
            raise AssertionError("k=%d %s %s: count %d, oracle %d" % (k, o, m, c, e["count"]))
        checked.append("k=%d %s %s count" % (k, o, m))
        if s is not None and "checksum" in e:
            if s != e["checksum"]:
                raise AssertionError("k=%d %s: checksum %#x, oracle %#x" % (k, o, s, e["checksum"]))
            checked.append("k=%d %s %s checksum" % (k, o, m))
    return sorted(set(checked))


def run_ours(args, rank, world):
    import numpy as np
    import torch

    import paper_2203_13512_gb300 as kcl

    dev = rank % max(torch.cuda.device_count(), 1)
    torch.cuda.set_device(dev)
    stream = torch.cuda.current_stream()
    rp, col = workload()
    n, nnz = len(rp) - 1, len(col)
    golden = _load_work()
    peaks = kcl.kcl_measure_int_peaks()
    g = kcl.kcl_load_csr(rp, col)
    # the library's autotuner picks, per out-degree class, SDegree's
    # bitmap-versus-list threshold and leaf form and both paths' warps per
    # subproblem, on the heaviest calls (untimed, like the warm-up)
    kcl.kcl_autotune(g, max(k for k, o, m in STEP_PLAN if o == "degree" and m == "count"), "degree")
    kcl.kcl_autotune(g, max(k for k, o, m in STEP_PLAN if o == "color" and m == "count"), "color")
    tuning = kcl.kcl_autotune(g, max(k for k, o, m in STEP_PLAN if o == "degree" and m == "list"),
                              "degree", listing=True)
    kcl.kcl_enable_timing(g, True)

    flush = torch.empty(2 * L2_BYTES // 4, dtype=torch.int32, device="cuda")
    ring = torch.empty(RING_BYTES // 4, dtype=torch.int32, device="cuda")

    def step(graph, collect=None, results=None):
        total = 0
        for k, o, mode in STEP_PLAN:
            s = None
            if mode == "count":
                c = kcl.kcl_count(graph, k, o)
            else:
                r = ring[: (ring.numel() // k) * k]
                c, s, w, _ = kcl.kcl_list(graph, k, o, r, wrap=True)
                assert w == min(c, r.numel() // k)
            total += c
            if results is not None:
                results.append((k, o, mode, c, s))
            if collect is not None:
                ms, la, cl = kcl.kcl_last_timing(graph)
                collect.append((k, o, mode, c, ms, la, cl))
        return total

    for i in range(args.warmup):
        res0 = []
        step(g, results=res0)
        if i == 0:
            checked = check_golden(res0, golden)
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()

    clocks = ClockSampler(dev)
    clocks.start()
    per_call, results = [], []
    dev_ms = 0.0
    cliques = 0
    for _ in range(args.steps):
        flush.fill_(1)  # evict L2 between timed steps (untimed)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record(stream)
        cliques += step(g, per_call, results)
        e1.record(stream)
        e1.synchronize()
        dev_ms += e0.elapsed_time(e1)
    torch.cuda.synchronize()
    # k = 6 in both orderings, one timed call each (seconds per call)
    k6 = {}
    if not args.no_k6:
        for k, o, _ in K6_PLAN:
            flush.fill_(1)
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            c = kcl.kcl_count(g, k, o)
            e1.record(stream)
            e1.synchronize()
            ms, la, cl = kcl.kcl_last_timing(g)
            k6[o] = {"count": c, "ms": e0.elapsed_time(e1), "listing_ms": ms["listing"],
                     "classes": [[x["lo"], x["hi"], x["roots"], round(x["ms"], 2)] for x in cl
                                 if x["roots"]]}
    clk = clocks.stop()
    check_golden(results, golden)

    # e2e: pinned host CSR -> C ABI (copy, validate, all calls) -> counts back
    rp_pin = torch.from_numpy(rp.view(np.int64)).pin_memory()
    col_pin = torch.from_numpy(col.view(np.int32)).pin_memory()
    e2e_ms = 0.0
    e2e_steps = max(1, min(args.steps, 3))
    for _ in range(e2e_steps):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        g2 = kcl.kcl_load_csr(rp_pin.numpy().view(np.uint64), col_pin.numpy().view(np.uint32))
        kcl.kcl_set_tuning(g2, tuning)
        step(g2)
        g2.free()
        torch.cuda.synchronize()
        e2e_ms += (time.perf_counter() - t0) * 1e3
    h2d = (n + 1) * 8 + nnz * 4
    d2h = 16 * len(STEP_PLAN)

    dev_ms, e2e_ms = max_over_ranks([dev_ms, e2e_ms], world)
    cliques_all = cliques * world
    value = cliques_all / (dev_ms / 1e3)
    e2e_value = (cliques // args.steps) * e2e_steps * world / (e2e_ms / 1e3)

    sm_mhz = clk.get("sm_mhz") or peaks["sm_clock_mhz"]
    roof = roofline(per_call, args.steps, peaks, sm_mhz)
    launches = sum(sum(pc[5].values()) - pc[5]["total"] for pc in per_call) // args.steps
    res = {
        "metric": METRIC, "value": value, "unit": "k-cliques/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": dev_ms / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u32/u64",
        "data": "synthetic (seeded R-MAT generator, no dataset)",
        "config": {"workload": "rmat-scale20-ef16", "n": n, "undirected_edges": nnz // 2,
                   "plan": ["k=%d %s %s" % p for p in STEP_PLAN],
                   "listing_ring": "%d GiB device ring, wrap=1, k uint32 ids per clique" %
                                   (RING_BYTES >> 30),
                   "l2": "inputs (%.0f MB CSR) larger than L2; L2 also flushed between steps"
                         % ((n + 1) * 8 / 1e6 + nnz * 4 / 1e6),
                   "parallelism": "replicas" if world > 1 else "single-gpu",
                   "tuning": tuning},
        "counts": {"k=%d %s %s" % pc[:3]: pc[3] for pc in per_call[: len(STEP_PLAN)]},
        "oracle_checked": checked,
        "e2e": {"value": e2e_value, "unit": "k-cliques/s", "h2d_bytes_per_step": h2d,
                "d2h_bytes_per_step": d2h},
        "gpu_launches": launches,
        "clocks": clk,
        "roofline": roof,
        "roofline_counting": roofline(per_call, args.steps, peaks, sm_mhz, modes=("count",)),
        "roofline_listing": roofline(per_call, args.steps, peaks, sm_mhz, modes=("list",)),
        "roofline_frontend": frontend_roofline(per_call, args.steps, n, nnz),
        "int_peaks": peaks,
        "stage_ms": stage_summary(per_call, args.steps),
    }
    if not args.no_c1:
        res["c1"] = run_c1(golden)
    if k6:
        tot = sum(v["count"] for v in k6.values())
        res["c2_k6"] = {"orderings": k6, "orderings_agree": len({v["count"] for v in k6.values()}) == 1,
                        "k_cliques_per_s": tot / (sum(v["ms"] for v in k6.values()) / 1e3)}
    g.free()
    if not args.no_forms:
        # bounded samples of the batched and served forms (their own
        # --form lines run them at full size)
        bt = batch_form(args.summary_batch_graphs, quiet=True)
        res["batched"] = batched_summary(bt)
        sv = serve_form(args.summary_serve_queries, [10000.0], args.serve_limit_ms,
                        rmat_ids=range(1, 9), batch_ids=range(33, 57), rmat_scale=lambda i: 16,
                        quiet=True)
        res["served"] = served_summary(sv, 10000.0, args.serve_limit_ms)
    return res


def batched_summary(bt):
    """The default line's record of a bounded batched-form run."""
    out = {"graphs": bt["config"]["graphs"],
           "batched_graphs_per_s": bt["value"],
           "per_graph_graphs_per_s": bt["per_graph_value"],
           "speedup": bt["speedup"], "bit_exact": bt["bit_exact"],
           "sample": "graphs 0..%d of the batched workload, both orderings, "
                     "count + checksum" % (bt["config"]["graphs"] - 1)}
    if not bt["bit_exact"]:
        out["mismatches"] = bt.get("mismatches")
    return out


def served_summary(sv, rate, limit_ms):
    """The default line's record of a bounded served-form run at one rate."""
    r = sv["rates"][str(float(rate))]
    return {"queries": sv["config"]["queries"], "rate_per_s": rate,
            "time_limit_ms": limit_ms,
            "served": r["served"], "fifo": r["fifo"],
            "results_compared": sv["results_compared"],
            "results_compared_equal": sv["results_compared_equal"],
            "bit_exact": sv["bit_exact"],
            "mismatches": sv.get("mismatches"),
            "sample": "%d R-MAT graphs (scales %s) + %d batched-workload graphs, k 3..10, "
                      "Poisson arrivals at %g/s" % (sv["config"]["rmat_graphs"],
                                                     sv["config"]["rmat_scales"],
                                                     sv["config"]["batch_graphs"], rate)}


def run_c1(golden, repeats=20):
    """The small Chung-Lu workload (n = 10,000, 50,000 drawn pairs, exponent
    2.5, 20 planted 12-cliques, seed 1), k = 5, degree ordering: kcl_count and
    kcl_list (count + checksum) through the C ABI, median of `repeats` warm
    calls (host wall clock, each call synchronous); `e2e` also copies the
    graph in from host memory (validated on the device) and frees it.  The
    count and checksum must equal the oracle's (tests/golden)."""
    import kclgen
    import paper_2203_13512_gb300 as kcl
    rp, col = kclgen.chung_lu_planted_small(seed=1)
    want = golden.get("c1 k=5")
    g = kcl.kcl_load_csr(rp, col)
    for _ in range(3):
        kcl.kcl_count(g, 5, "degree")
        kcl.kcl_list(g, 5, "degree", None)
    tc, tl, te = [], [], []
    for _ in range(repeats):
        t = time.perf_counter()
        c = kcl.kcl_count(g, 5, "degree")
        tc.append(time.perf_counter() - t)
        t = time.perf_counter()
        c2, s, _, _ = kcl.kcl_list(g, 5, "degree", None)
        tl.append(time.perf_counter() - t)
        t = time.perf_counter()
        g2 = kcl.kcl_load_csr(rp, col)
        c3 = kcl.kcl_count(g2, 5, "degree")
        c4, s2, _, _ = kcl.kcl_list(g2, 5, "degree", None)
        g2.free()
        te.append(time.perf_counter() - t)
        if want and (c, c2, s, c3, c4, s2) != (want["count"], want["count"], want["checksum"],
                                                 want["count"], want["count"], want["checksum"]):
            raise AssertionError("C1: (%d, %d, %#x) differs from the oracle's (%d, %#x)" %
                                 (c, c2, s, want["count"], want["checksum"]))
    g.free()
    med = statistics.median
    return {"workload": "chung-lu-n10000-m50000-g2.5-20xK12 (seed 1), k=5, degree ordering",
            "count": c, "checksum": "%#x" % s, "oracle_checked": bool(want),
            "count_ms_median": 1e3 * med(tc), "list_ms_median": 1e3 * med(tl),
            "e2e_load_count_list_ms_median": 1e3 * med(te), "repeats": repeats}


def max_over_ranks(values, world):
    """Element-wise maximum of per-rank floats over the job (the slowest
    replica's times); the identity for one rank."""
    if world <= 1:
        return list(values)
    import torch
    import torch.distributed as dist
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor(list(values), dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return [float(x) for x in t.cpu()]


def stage_summary(per_call, steps):
    """Mean stage times per call family, and the listing stage split by
    out-degree class: [lo, hi, roots, ms] for each launched class."""
    out, cls = {}, {}
    for (k, o, m, c, ms, la, cl) in per_call:
        key = "k=%d %s %s" % (k, o, m)
        d = out.setdefault(key, {s: 0.0 for s in ms})
        for s, v in ms.items():
            d[s] += v / steps
        cc = cls.setdefault(key, {})
        for x in cl:
            if x["roots"]:
                cc.setdefault((x["lo"], x["hi"], x["roots"]), []).append(x["ms"])
    res = {k: {s: round(v, 3) for s, v in d.items()} for k, d in out.items()}
    for key, cc in cls.items():
        res[key]["classes"] = [[lo, hi, r, round(sum(t) / len(t), 3)]
                               for (lo, hi, r), t in sorted(cc.items())]
    return res


def roofline(per_call, steps, peaks, sm_mhz, modes=("count", "list")):
    """The dominant kernel: the single listing launch with the largest device
    time per step -- one out-degree class of the call family (among `modes`)
    whose listing stage is longest.  Its bound is the integer pipe; the peak
    is the measured per-SM rate of its unit (kcl_measure_int_peaks) x SMs x
    the SM clock sampled during the timed region:
      counting, BitCol: BitJoin words of Algorithm 6 (a 32-bit word of a
        bit-row ANDed with the candidate set and counted), peak = the
        measured BitJoin word rate;
      counting, SDegree: the merge joins of Algorithm 5 each costed at the
        width of a bitmap over the root's out-neighbourhood, ceil(d+/32)
        words (what the bit-row form computes), same peak;
      listing: cliques, each k SplitMix64 rounds of the checksum, peak = the
        measured round rate / k.
    `achieved` = the oracle's count of that unit for the roots of that class
    (tests/golden/rmat20_work.json, split by out-degree) / that launch's
    CUDA-event time."""
    work = _load_work()
    fam = {}
    for (k, o, m, c, ms, la, cl) in per_call:
        if m not in modes:
            continue
        f = fam.setdefault((k, o, m), {"listing": [], "classes": {}})
        f["listing"].append(ms["listing"])
        for ci, cc in enumerate(cl):
            f["classes"].setdefault((ci, cc["lo"], cc["hi"], cc["roots"]), []).append(cc["ms"])
    if not fam:
        return None
    (k, o, m), f = max(fam.items(), key=lambda kv: sum(kv[1]["listing"]))
    (ci, lo, hi, roots), times = max(f["classes"].items(), key=lambda kv: sum(kv[1]))
    avg_ms = sum(times) / len(times)
    entry = work.get("k=%d %s" % (k, o))
    sms = peaks["num_sms"]
    if m == "list":
        per_clk = peaks["mix64_per_sm_clk"] / k
        what, unit = "%.2f SplitMix64 rounds/clk/SM / %d per clique" % (peaks["mix64_per_sm_clk"], k), \
            "Gclique/s"
        wk = class_work(entry, lo, hi, field="count_by_outdeg")
    else:
        per_clk = peaks["bitjoin_words_per_sm_clk"]
        what = "%.2f BitJoin words/clk/SM" % per_clk
        unit = "Gword/s"
        wk = class_work(entry, lo, hi, field="work_by_outdeg" if o == "color" else "bitrow_words_by_outdeg")
    peak_g = sms * per_clk * sm_mhz * 1e6 / 1e9
    achieved = (wk / (avg_ms / 1e3) / 1e9) if wk else None
    kern = KERNEL_NAMES.get((o, m, ci), "listing launch of class %d" % ci)
    tr = TRAFFIC.get((k, o, m, ci))
    return {"kernel": "%s (k=%d %s %s, roots with %d <= d+ <= %d)" % (kern, k, o, m, lo, hi),
            "bound": "alu", "achieved": achieved, "peak": peak_g, "unit": unit,
            "frac": (achieved / peak_g) if achieved else None,
            "traffic": tr[0] if tr else None,
            "traffic_source": tr[1] if tr else None,
            "work_per_launch": wk, "roots": roots, "avg_ms": avg_ms,
            "listing_stage_ms": sum(f["listing"]) / len(f["listing"]),
            "peak_source": "measured: %d SMs x %s (kcl_measure_int_peaks) x %.0f MHz (sampled SM clock)"
                           % (sms, what, sm_mhz)}


def frontend_roofline(per_call, steps, n, nnz):
    """The front-end passes of the k = 4 counting calls against the measured
    HBM copy bandwidth.  Algorithmic bytes per pass (n vertices, nnz CSR
    entries, C = 8 (n + 1) + 4 nnz bytes of CSR):
      pre_core: read the row offsets, write alive + degrees: 8 (n + 1) + 5 n;
      pre_list: one pass over the CSR and alive: C + n;
      orientation, degree: two passes over the CSR, alive and keys (out-degree
        count, then fill) + the out-CSR written: 2 (C + 5 n) + 4 (n + 1) + 2 nnz;
      orientation, colour: the same + the peel's pass over the CSR and its
        degree/key arrays: 3 (C + 5 n) + 4 (n + 1) + 2 nnz."""
    peaks, src = _peaks()
    hbm = peaks.get("hbm_gbs", 6800.0)
    C = 8 * (n + 1) + 4 * nnz
    out = {}
    for o in ("color", "degree"):
        fam = [pc for pc in per_call if pc[0] == 4 and pc[1] == o and pc[2] == "count"]
        if not fam:
            continue
        ms = {st: sum(pc[4][st] for pc in fam) / len(fam) for st in ("pre_core", "pre_list", "orientation")}
        passes = 3 if o == "color" else 2
        byt = {"pre_core": 8 * (n + 1) + 5 * n, "pre_list": C + n,
               "orientation": passes * (C + 5 * n) + 4 * (n + 1) + 2 * nnz}
        out["k=4 %s count" % o] = {
            st: {"bytes": byt[st], "ms": round(ms[st], 3),
                 "GB_s": byt[st] / (ms[st] / 1e3) / 1e9 if ms[st] > 0 else None,
                 "frac": (byt[st] / (ms[st] / 1e3) / 1e9 / hbm) if ms[st] > 0 else None}
            for st in byt}
    out["peak_GB_s"] = hbm
    out["peak_source"] = "%s HBM copy bandwidth (MEASURED_PEAKS.json)" % src
    return out


# listing kernels of the out-degree classes (count mode), by (ordering, mode,
# class index); classes as in kcl_sdegree.cu / kcl_bitcol.cu
KERNEL_NAMES = {
    ("degree", "count", 0): "k_sdegree<0,0,1> (warp per root, d+ <= 32)",
    ("degree", "count", 1): "k_sdegree<0,0,1> (warp per root, d+ <= 64)",
    ("degree", "count", 2): "k_sdegree<0,0,1> (warp per root, d+ <= 128)",
    ("degree", "count", 3): "k_sdegree_cta<0> (CTA per root, d+ <= 256)",
    ("degree", "count", 4): "k_sdegree_cta<0> (CTA per root, d+ <= 512)",
    ("degree", "count", 5): "k_sdegree_cta<0> (CTA per root, d+ <= 1024)",
    ("color", "count", 0): "k_bitcol_warp<1,0>",
    ("color", "count", 1): "k_bitcol_warp<2,0>",
    ("color", "count", 2): "k_bitcol_warp<4,0>",
    ("color", "count", 3): "k_bitcol_cta<8,0,0,0>",
    ("color", "count", 4): "k_bitcol_cta<16,0,0,0>",
    ("color", "count", 5): "k_bitcol_cta<16,0,1,0>",
    ("degree", "list", 0): "k_sdegree_cta<1> (d+ <= 32)",
    ("degree", "list", 1): "k_sdegree_cta<1> (d+ <= 64)",
    ("degree", "list", 2): "k_sdegree_cta<1> (d+ <= 128)",
    ("degree", "list", 3): "k_sdegree_cta<1> (d+ <= 256)",
    ("degree", "list", 4): "k_sdegree_cta<1> (d+ <= 512)",
    ("degree", "list", 5): "k_sdegree_cta<1> (d+ <= 1024)",
    ("color", "list", 0): "k_bitcol_cta<4,1,0,0> (W=1)",
    ("color", "list", 1): "k_bitcol_cta<4,1,0,0> (W=2)",
    ("color", "list", 2): "k_bitcol_cta<4,1,0,0> (W=4)",
    ("color", "list", 3): "k_bitcol_cta<8,1,0,0>",
    ("color", "list", 4): "k_bitcol_cta<16,1,0,0>",
    ("color", "list", 5): "k_bitcol_cta<16,1,1,0>",
}

# DRAM bytes (read + write) per launch of the listing launches from one ncu
# capture of the same workload, keyed (k, ordering, mode, class); the source
# names the summary under profiles/.  An entry is removed when its kernel
# changes, until a new capture exists.
_DRAM = "profiles/k_bitcol_cta_rmat20.md"
TRAFFIC = {
    (5, "color", "count", 4): (30.719e6 + 0.040e6, _DRAM),
    (4, "color", "list", 4): (3.352e9 + 192.248e9, _DRAM),
    (4, "degree", "list", 4): (6.684e9 + 190.315e9, "profiles/k_sdegree_cta_rmat20.md"),
}


def class_work(entry, lo, hi, field="work_by_outdeg"):
    """Oracle work of the roots with lo <= d+ <= hi, from the power-of-two
    out-degree buckets (bucket b: 2^(b-1) < d+ <= 2^b).  Every class starts
    just above a power of two (or at k-1, below which there are no roots) and
    ends at one (or at the largest out-degree), so each bucket lies in one
    class."""
    if not entry or field not in entry:
        return None
    if lo > 1 and (lo - 1) & (lo - 2) and lo - 1 > 32:
        return None
    total = 0
    for b, w in entry[field].items():
        top = 1 << int(b)
        if top >= lo and (top >> 1) < hi:
            total += w
    return total


def _load_work():
    p = os.path.join(ROOT, "tests", "golden", "rmat20_work.json")
    if not os.path.exists(p):
        return {}
    with open(p) as f:
        return json.load(f)


# --------------------------------------------------------- oracle (CPU)
_GRAPH = None


def _oracle_task(task):
    """One call of STEP_PLAN by the oracle on a subset of the roots (the
    oracle as it stands: its own Pre-Core, Pre-List and orientation over the
    whole graph, then the roots given).  Counting calls use its count-only
    mode, listing calls enumerate and hash every clique."""
    global _GRAPH
    import numpy as np

    import oracle
    k, o, mode, roots = task
    if _GRAPH is None:
        _GRAPH = workload()
    rp, col = _GRAPH
    fn = oracle.bitcol if o == "color" else oracle.sdegree
    kw = {"L": 32} if o == "color" else {}
    t = time.perf_counter()
    r = fn(rp, col, k, roots=np.asarray(roots, np.uint32), count_only=(mode == "count"), **kw)
    return r["count"], time.perf_counter() - t


def _plan_tasks(stride, shards):
    n = 1 << SCALE
    tasks = []
    for k, o, mode in STEP_PLAN:
        roots = list(range(0, n, stride))
        tasks += [(k, o, mode, roots[i::shards]) for i in range(shards)]
    return tasks, len(range(0, n, stride))


def oracle_plan_sample(stride, pool=None, procs=1):
    """The oracle on every call of STEP_PLAN, restricted to roots 0, stride,
    2 stride, ...: sequentially in this process (pool None), or sharded over
    a spawn pool of `procs` processes.  Returns (cliques, seconds, calls)."""
    if pool is None:
        tasks, nr = _plan_tasks(stride, 1)
        t = time.perf_counter()
        found = sum(_oracle_task(tk)[0] for tk in tasks)
        return found, time.perf_counter() - t, nr
    shards = max(1, -(-procs // len(STEP_PLAN)))
    tasks, nr = _plan_tasks(stride, shards)
    t = time.perf_counter()
    found = sum(c for c, _ in pool.imap_unordered(_oracle_task, tasks))
    return found, time.perf_counter() - t, nr


def _oracle_pool(procs):
    import multiprocessing as mp
    return mp.get_context("spawn").Pool(procs)  # spawned: safe after CUDA use


CPU_STRIDE = 997


def oracle_sample():
    """cpu_baseline of the main line: the same plan as the GPU step on every
    997th root, single-threaded and on all host cores (spawned processes)."""
    procs = os.cpu_count() or 1
    one = oracle_plan_sample(CPU_STRIDE)
    with _oracle_pool(procs) as pool:
        oracle_plan_sample(CPU_STRIDE * 7, pool, procs)  # start-up (imports, graph) untimed
        allc = oracle_plan_sample(CPU_STRIDE, pool, procs)
    sample = ("the %d step calls (%s) on roots 0, %d, 2*%d, ... (%d of %d) of R-MAT scale 20; "
              "count-only mode for counting calls, every clique hashed for listing calls; "
              "each call includes the oracle's own Pre-Core/Pre-List/orientation pass"
              % (len(STEP_PLAN), ", ".join("k=%d %s %s" % p for p in STEP_PLAN), CPU_STRIDE,
                 CPU_STRIDE, one[2], 1 << SCALE))
    return {"value": allc[0] / allc[1], "unit": "k-cliques/s", "cores": procs, "kind": "oracle",
            "sample": sample, "seconds": allc[1],
            "single_thread": {"value": one[0] / one[1], "cores": 1, "seconds": one[1]},
            "nproc": procs}


def run_reference(args, rank, world):
    if rank != 0:
        return None
    procs = os.cpu_count() or 1
    vals = []
    with _oracle_pool(procs) as pool:
        for _ in range(args.warmup + args.steps):
            vals.append(oracle_plan_sample(2 * CPU_STRIDE + 1, pool, procs))
    timed = vals[args.warmup:]
    found = sum(v[0] for v in timed)
    sec = sum(v[1] for v in timed)
    value = found / sec
    sample = ("the %d step calls on roots 0, %d, ... (%d of %d) of R-MAT scale 20, sharded over %d "
              "spawned processes" % (len(STEP_PLAN), 2 * CPU_STRIDE + 1, timed[0][2], 1 << SCALE, procs))
    cb = {"value": value, "unit": "k-cliques/s", "cores": procs, "kind": "oracle", "sample": sample}
    return {"impl": "reference", "metric": METRIC, "value": value, "unit": "k-cliques/s",
            "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": sec * 1e3 / len(timed), "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "u32/u64", "data": "synthetic (seeded R-MAT generator)",
            "config": {"workload": "rmat-scale20-ef16", "sample": sample},
            "cpu_baseline": cb,
            "e2e": {"value": value, "unit": "k-cliques/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}


# ------------------------------------------------------- batched form
def run_batch(args):
    """The batched workload: graph i = kclgen.batch_graph(i) (n log-uniform in
    [50, 20000], mean degree 4-40, exponent 2.3, 0-5 planted cliques of size
    8-16, k uniform in 3..9), count + checksum per graph, both orderings as two
    sweeps.  Compares one kcl_count_batch call (per ordering: every graph in
    one disjoint union with its own k, one pass of the pipeline) with one
    library call per graph on the same resident graphs; results must be
    identical."""
    return batch_form(args.batch_graphs)


def batch_form(G, quiet=False):
    """run_batch on graphs 0..G-1."""
    import torch

    import kclgen
    import paper_2203_13512_gb300 as kcl
    t0 = time.perf_counter()
    data = [kclgen.batch_graph(i) for i in range(G)]
    gen_s = time.perf_counter() - t0
    graphs = [kcl.kcl_load_csr(rp, col) for rp, col, _ in data]
    ks = [k for _, _, k in data]
    b = kcl.kcl_batch_create()
    out = {"metric": "graphs/s, batched vs one call per graph (count + checksum)",
           "unit": "graphs/s", "higher_is_better": True, "n_gpus": 1,
           "config": {"workload": "chung-lu-batch", "graphs": G,
                      "vertices": int(sum(len(rp) - 1 for rp, _, _ in data)),
                      "undirected_edges": int(sum(len(c) // 2 for _, c, _ in data)),
                      "generation_s": round(gen_s, 1)},
           "data": "synthetic (seeded Chung-Lu generator)", "orderings": {}}
    total_per, total_bat, cliques = 0.0, 0.0, 0
    mismatches, mismatch_list = 0, []
    for o in ("color", "degree"):
        ords = [o] * G

        def per_graph():
            return [kcl.kcl_list(g, k, o, None)[:2] for g, k in zip(graphs, ks)]

        def batched():
            c, s = kcl.kcl_count_batch(b, graphs, ks, ords, checksums=True)
            return list(zip(c, s))

        ref = per_graph()  # warm-up (allocates each graph's scratch)
        if not quiet:
            print("batch %s: warm-up per-graph pass done" % o, file=sys.stderr, flush=True)
        got = batched()
        bad = [i for i, (x, y) in enumerate(zip(got, ref)) if x != y]
        mismatches += len(bad)
        for i in bad[:4]:
            mismatch_list.append({"ordering": o, "graph": i, "batched": list(got[i]),
                                  "alone": list(ref[i])})
        torch.cuda.synchronize()
        t = time.perf_counter()
        per_graph()
        torch.cuda.synchronize()
        t_per = time.perf_counter() - t
        t = time.perf_counter()
        batched()
        torch.cuda.synchronize()
        t_bat = time.perf_counter() - t
        if not quiet:
            print("batch %s: per-graph %.2f s, batched %.2f s" % (o, t_per, t_bat), file=sys.stderr,
                  flush=True)
        n_cl = sum(c for c, _ in ref)
        out["orderings"][o] = {"per_graph_s": round(t_per, 4), "batched_s": round(t_bat, 4),
                               "per_graph_graphs_per_s": G / t_per, "batched_graphs_per_s": G / t_bat,
                               "speedup": t_per / t_bat, "k_cliques": n_cl}
        total_per += t_per
        total_bat += t_bat
        cliques += n_cl
    out["value"] = 2 * G / total_bat
    out["per_graph_value"] = 2 * G / total_per
    out["speedup"] = total_per / total_bat
    out["k_cliques_per_s_batched"] = cliques / total_bat
    out["bit_exact"] = mismatches == 0
    if mismatches:
        out["mismatches"] = mismatches
        out["mismatch_examples"] = mismatch_list
    b.free()
    for g in graphs:
        g.free()
    return out


# ------------------------------------------------------- served form
def run_serve(args):
    """The served workload: 64 resident graphs -- ids 1-32 R-MAT at scale
    16 + (id mod 5) (scales 16-20, seed id), ids 33-64 graph `id` of the
    batched workload -- and a Poisson stream of (graph, k in 3..10, ordering,
    count | count + checksum) queries (numpy default_rng(1)).  Both sides run
    every pass under the same time limit (--serve-limit-ms): large k on the
    R-MAT graphs is beyond any latency budget, and such a query finishes with
    KCL_ETIMEOUT.  The server (8 slots, 100 GB scratch budget, continuous
    batching of small-graph queries) is compared with a FIFO loop that
    replays the same arrivals and runs one query per call in arrival order;
    every query that completes on both sides must have the same result."""
    return serve_form(args.serve_queries, args.serve_rates, args.serve_limit_ms)


def serve_form(Q, rates, limit, rmat_ids=range(1, 33), batch_ids=range(33, 65),
               rmat_scale=lambda i: 16 + i % 5, quiet=False):
    """run_serve over the given graph ids (R-MAT graph i at rmat_scale(i),
    seed i; batched-workload graph i)."""
    import numpy as np
    import torch

    import kclgen
    import paper_2203_13512_gb300 as kcl
    t0 = time.perf_counter()
    graphs = [kcl.kcl_load_csr(*kclgen.rmat20(seed=i, scale=rmat_scale(i))) for i in rmat_ids]
    graphs += [kcl.kcl_load_csr(*kclgen.batch_graph(i)[:2]) for i in batch_ids]
    NG = len(graphs)
    load_s = time.perf_counter() - t0
    rng = np.random.default_rng(1)
    qs = [(int(rng.integers(NG)), int(rng.integers(3, 11)),
           "color" if rng.random() < 0.5 else "degree", bool(rng.random() < 0.5)) for _ in range(Q)]
    gaps = rng.exponential(1.0, Q)
    for g in graphs:
        kcl.kcl_set_time_limit(g, limit)

    def run_one(q):
        gi, k, o, lst = q
        try:
            if lst:
                c, h, _, _ = kcl.kcl_list(graphs[gi], k, o, None)
                return c, h, 0
            return kcl.kcl_count(graphs[gi], k, o), 0, 0
        except kcl.KclError as e:
            return None, None, e.status

    for q in qs[:NG]:
        run_one(q)  # warm-up: every graph's scratch
    scales = sorted({rmat_scale(i) for i in rmat_ids})
    out = {"metric": "served queries: throughput and latency, continuous batching vs FIFO",
           "unit": "queries/s", "higher_is_better": True, "n_gpus": 1,
           "config": {"workload": "served-mixed", "graphs": NG, "rmat_graphs": len(rmat_ids),
                      "batch_graphs": len(batch_ids), "queries": Q,
                      "rmat_scales": "%d..%d" % (scales[0], scales[-1]) if scales else None,
                      "k": "3..10", "slots": 8, "scratch_budget_gb": 100,
                      "time_limit_ms": limit, "load_s": round(load_s, 1)},
           "data": "synthetic", "rates": {}}
    compared, mismatches, mismatch_list = 0, 0, []
    for rate in rates:
        arr = np.cumsum(gaps / rate)
        # FIFO: one query per call in arrival order, replayed against the clock
        fifo_res, fifo_lat = [], []
        torch.cuda.synchronize()
        base = time.perf_counter()
        for q, a in zip(qs, arr):
            now = time.perf_counter() - base
            if now < a:
                time.sleep(a - now)
            fifo_res.append(run_one(q))
            fifo_lat.append(time.perf_counter() - base - a)
        fifo_span = time.perf_counter() - base
        if not quiet:
            print("fifo at %g/s: %.1f s" % (rate, fifo_span), file=sys.stderr, flush=True)
        srv = kcl.kcl_server_create(slots=8, scratch_budget_bytes=100 << 30, small_nnz=1 << 20)
        kcl.kcl_server_set_time_limit(srv, limit)
        ids = [kcl.kcl_server_add_graph(srv, g) for g in graphs]
        for gi in range(min(8, NG)):  # warm the slots' scratch
            kcl.kcl_server_wait(srv, kcl.kcl_server_submit(srv, ids[gi], 3, "color"))
        sbase = kcl.kcl_server_clock(srv)
        tickets = []
        for (gi, k, o, lst), a in zip(qs, arr):
            while kcl.kcl_server_clock(srv) - sbase < a:
                time.sleep(0)
            tickets.append(kcl.kcl_server_submit(srv, ids[gi], k, o, lst))
        res = [kcl.kcl_server_wait(srv, t) for t in tickets]
        srv.destroy()
        if not quiet:
            print("served at %g/s" % rate, file=sys.stderr, flush=True)
        for r, (c, h, st), q in zip(res, fifo_res, qs):
            if r["status"] == 0 and st == 0:
                compared += 1
                if (r["count"], r["checksum"]) != (c, h):
                    mismatches += 1
                    if len(mismatch_list) < 8:
                        mismatch_list.append({"rate": rate, "query": list(q),
                                              "served": [r["count"], r["checksum"]],
                                              "fifo": [c, h]})
        ok_s = [r for r in res if r["status"] == 0]
        slat = [r["done_s"] - r["submit_s"] for r in ok_s]
        flat = [lt for lt, (_, _, st) in zip(fifo_lat, fifo_res) if st == 0]
        makespan = max(r["done_s"] for r in res) - sbase
        out["rates"][str(rate)] = {
            "served": {"throughput_qps": Q / makespan, "completed": len(ok_s),
                       "completed_per_s": len(ok_s) / makespan,
                       "timed_out": Q - len(ok_s),
                       "p50_ms": 1e3 * float(np.percentile(slat, 50)) if slat else None,
                       "p99_ms": 1e3 * float(np.percentile(slat, 99)) if slat else None,
                       "mean_batch": float(np.mean([r["batch"] for r in res]))},
            "fifo": {"throughput_qps": Q / fifo_span, "completed": len(flat),
                     "completed_per_s": len(flat) / fifo_span,
                     "timed_out": Q - len(flat),
                     "p50_ms": 1e3 * float(np.percentile(flat, 50)) if flat else None,
                     "p99_ms": 1e3 * float(np.percentile(flat, 99)) if flat else None}}
    last = out["rates"][str(rates[-1])]
    out["value"] = last["served"]["throughput_qps"]
    out["results_compared"] = compared
    out["results_compared_equal"] = compared - mismatches
    out["bit_exact"] = mismatches == 0
    if mismatches:
        out["mismatches"] = mismatch_list
    for g in graphs:
        g.free()
    return out


def run_c3(args):
    """The community workload at full size: Chung-Lu n = 4,000,000, 1.2e8
    drawn pairs, exponent 2.1, expected degree capped at 40,000, plus 2,000
    communities of 60-300 vertices at density 0.8 (seed 1), colour ordering
    (BitCol) with Pre-Core and Pre-List; degree ordering (SDegree) beside it.
    Every call runs under the library's time limit (--c3-limit-s, the
    paper's "exceeds the time limit" outcome otherwise): counting at
    k = 6, 8, 10, and listing k = 6 into a 4 GiB wrapping device ring."""
    import torch

    import kclgen
    import paper_2203_13512_gb300 as kcl
    t = time.perf_counter()
    rp, col = kclgen.chung_lu_communities(seed=1)
    gen_s = time.perf_counter() - t
    g = kcl.kcl_load_csr(rp, col)
    kcl.kcl_enable_timing(g, True)
    kcl.kcl_set_time_limit(g, int(args.c3_limit_s * 1000))
    ring = torch.empty(RING_BYTES // 4, dtype=torch.int32, device="cuda")
    out = {"metric": "k-cliques/s, community workload (time-limited calls)", "unit": "k-cliques/s",
           "higher_is_better": True, "n_gpus": 1,
           "config": {"workload": "chung-lu-communities-n4e6", "n": len(rp) - 1,
                      "undirected_edges": len(col) // 2, "limit_s": args.c3_limit_s,
                      "generation_s": round(gen_s, 1)},
           "data": "synthetic (seeded Chung-Lu generator, planted communities)", "calls": {}}
    plan = [(6, "color", "count"), (6, "degree", "count"), (8, "color", "count"),
            (10, "color", "count"), (6, "color", "list")]
    for k, o, m in plan:
        key = "k=%d %s %s" % (k, o, m)
        torch.cuda.synchronize()
        t = time.perf_counter()
        try:
            if m == "count":
                c, s = kcl.kcl_count(g, k, o), None
            else:
                r = ring[: ring.numel() // k * k]
                c, s, _, _ = kcl.kcl_list(g, k, o, r, wrap=True)
            ms, la, cl = kcl.kcl_last_timing(g)
            out["calls"][key] = {"count": c, "checksum": s, "ms": ms["total"],
                                 "k_cliques_per_s": c / (ms["total"] / 1e3),
                                 "stage_ms": {st: round(v, 2) for st, v in ms.items()}}
        except kcl.KclError as e:
            what = {kcl.KCL_ETIMEOUT: "exceeds the %g s limit" % args.c3_limit_s,
                    kcl.KCL_EOVERFLOW: "count exceeds 2^64 - 1"}.get(e.status, str(e))
            out["calls"][key] = {"result": what, "wall_s": round(time.perf_counter() - t, 1)}
        print("c3 %s: %s" % (key, out["calls"][key]), file=sys.stderr, flush=True)
    done = [v for v in out["calls"].values() if "count" in v]
    out["value"] = (sum(v["count"] for v in done) / (sum(v["ms"] for v in done) / 1e3)) if done else None
    g.free()
    return out


def run_ablation(args):
    """The preprocessing / pruning study, the NodeParallel / EdgeParallel study
    and the memory study on the bench graph (R-MAT scale 20): for k = 4, 5
    and both orderings, device time of one call with everything on, without
    Pre-Core, without Pre-List, (BitCol) without the colour prune, and with
    one warp per root in the CTA classes (NodeParallel: no sharing of a
    root's first-level children); and the device scratch a fresh handle holds
    after one call of each (k, ordering)."""
    import torch

    import paper_2203_13512_gb300 as kcl
    rp, col = workload()
    g = kcl.kcl_load_csr(rp, col)
    kcl.kcl_enable_timing(g, True)
    one_warp = {"sdegree_cta_warps": [1] * kcl.KCL_MAX_CLASSES,
                "bitcol_cta_warps": [1] * kcl.KCL_MAX_CLASSES}
    configs = [("all on", 0, None), ("no Pre-Core", kcl.KCL_OPT_NO_PRECORE, None),
               ("no Pre-List", kcl.KCL_OPT_NO_PRELIST, None),
               ("no colour prune", kcl.KCL_OPT_NO_COLOR_PRUNE, None),
               ("one warp per root (NodeParallel)", 0, one_warp)]
    out = {"metric": "ablation: device ms per call (R-MAT scale 20)", "unit": "ms",
           "higher_is_better": False, "n_gpus": 1,
           "config": {"workload": "rmat-scale20-ef16", "repeats": args.steps},
           "data": "synthetic", "calls": {}, "scratch_bytes": {}}
    for k in (4, 5):
        for o in ("color", "degree"):
            row = {}
            for name, flags, tune in configs:
                if o == "degree" and flags == kcl.KCL_OPT_NO_COLOR_PRUNE:
                    continue
                kcl.kcl_set_options(g, flags)
                kcl.kcl_set_tuning(g, tune or {})
                c0 = kcl.kcl_count(g, k, o)  # warm-up
                ms = []
                for _ in range(max(1, args.steps)):
                    torch.cuda.synchronize()
                    c = kcl.kcl_count(g, k, o)
                    assert c == c0
                    ms.append(kcl.kcl_last_timing(g)[0])
                row[name] = {s_: round(sum(m[s_] for m in ms) / len(ms), 3) for s_ in ms[0]}
                row[name]["count"] = c
            out["calls"]["k=%d %s" % (k, o)] = row
            v = kcl.kcl_graph_view(g)
            kcl.kcl_count(v, k, o)
            ws, ar = kcl.kcl_scratch_bytes(v)
            out["scratch_bytes"]["k=%d %s" % (k, o)] = {"workspace": ws, "arena": ar}
            v.free()
    kcl.kcl_set_options(g, 0)
    kcl.kcl_set_tuning(g, {})
    g.free()
    return out


def profile_case(spec):
    """A single library call on a smaller R-MAT graph (for ncu captures)."""
    import kclgen
    import paper_2203_13512_gb300 as kcl
    parts = spec.split(":")
    scale, k, ordering = int(parts[0]), int(parts[1]), parts[2]
    mode = parts[3] if len(parts) > 3 else "count"
    rp, col = kclgen.rmat20(seed=1, scale=scale)
    g = kcl.kcl_load_csr(rp, col)
    if mode == "count":
        print(kcl.kcl_count(g, k, ordering))
    else:  # into a wrapping device ring, as the bench's listing calls
        import torch
        ring = torch.empty(RING_BYTES // 4 // k * k, dtype=torch.int32, device="cuda")
        print(kcl.kcl_list(g, k, ordering, ring, wrap=True))
    g.free()


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-k6", action="store_true", help="skip the timed k = 6 calls")
    ap.add_argument("--no-c1", action="store_true", help="skip the small Chung-Lu line")
    ap.add_argument("--no-forms", action="store_true",
                    help="skip the bounded batched and served samples of the default line")
    ap.add_argument("--summary-batch-graphs", type=int, default=128)
    ap.add_argument("--summary-serve-queries", type=int, default=400)
    ap.add_argument("--c3-limit-s", type=float, default=60.0,
                    help="time limit of each call of the community workload (--form c3)")
    ap.add_argument("--form", default="single", choices=["single", "batch", "serve", "ablation", "c3"],
                    help="single: the R-MAT scale-20 line; batch / serve: the batched and "
                         "served workloads, each printing its own JSON line")
    ap.add_argument("--batch-graphs", type=int, default=2048)
    ap.add_argument("--serve-queries", type=int, default=5000)
    ap.add_argument("--serve-rates", type=float, nargs="+", default=[1000.0, 10000.0, 50000.0])
    ap.add_argument("--serve-limit-ms", type=int, default=50,
                    help="time limit per query of the served form: each FIFO call gets it, a "
                         "batched pass of n queries gets n times it")
    ap.add_argument("--profile-case", default=None,
                    help="SCALE:K:ORDERING[:count|list] -- one call on R-MAT at SCALE "
                         "(16 * 2^SCALE edges, seed 1), for profilers")
    args = ap.parse_args()
    if args.profile_case:
        profile_case(args.profile_case)
        return
    if args.form != "single":
        res = {"batch": run_batch, "serve": run_serve, "ablation": run_ablation,
               "c3": run_c3}[args.form](args)
        print(json.dumps(res))
        return
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    if world > 1:
        import torch
        backend = "nccl" if args.impl == "ours" else "gloo"
        if args.impl == "ours":
            torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", rank)))
        torch.distributed.init_process_group(backend)
    if args.impl == "reference":
        res = run_reference(args, rank, world)
    else:
        res = run_ours(args, rank, world)
        if rank == 0 and world == 1 and not args.no_cpu_baseline:
            res["cpu_baseline"] = oracle_sample()
    if rank == 0 and res is not None:
        print(json.dumps(res))
    if world > 1:
        import torch
        torch.distributed.barrier()
        torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
