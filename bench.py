"""Benchmark: k-cliques/s of the GB300 k-clique library on the R-MAT scale-20
workload (2^20 vertices, 16*2^20 unique undirected edges, a=0.57 b=0.19
c=0.19 d=0.05, seed 1), SDegree (degree ordering) and BitCol (colour
ordering), counting mode and listing mode (count + checksum).

One step = every (k, ordering, mode) call of STEP_PLAN on the resident
graph: Pre-Core, Pre-List, orientation and the listing kernels run inside
each call.  `value` = sum of the k-clique counts of the step / device time of
the step (CUDA events on the stream the library runs on).  `e2e` = the same
metric through the C ABI from pinned host buffers: graph copy-in (validated
on the device), the step's calls and the read-back of every count/checksum.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

--impl reference times the CPU oracle (oracle/, single thread) on a bounded
sample of the same workload: a fixed set of roots of the same DAG.
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
METRIC = "k-cliques/s (bit-exact counts; R-MAT scale 20, SDegree + BitCol)"
L2_BYTES = 129 * 2 ** 20


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
def run_ours(args, rank, world):
    import numpy as np
    import torch

    import paper_2203_13512_gb300 as kcl

    dev = rank % max(torch.cuda.device_count(), 1)
    torch.cuda.set_device(dev)
    stream = torch.cuda.current_stream()
    rp, col = workload()
    n, nnz = len(rp) - 1, len(col)
    g = kcl.kcl_load_csr(rp, col)
    kcl.kcl_enable_timing(g, True)

    flush = torch.empty(2 * L2_BYTES // 4, dtype=torch.int32, device="cuda")

    def step(graph, collect=None):
        total = 0
        for k, o, mode in STEP_PLAN:
            if mode == "count":
                c = kcl.kcl_count(graph, k, o)
            else:
                c, s, _, _ = kcl.kcl_list(graph, k, o, None)
            total += c
            if collect is not None:
                ms, la = kcl.kcl_last_timing(graph)
                collect.append((k, o, mode, c, ms, la))
        return total

    for _ in range(args.warmup):
        step(g)
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()

    clocks = ClockSampler(dev)
    clocks.start()
    per_call = []
    dev_ms = 0.0
    cliques = 0
    for _ in range(args.steps):
        flush.fill_(1)  # evict L2 between timed steps (untimed)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record(stream)
        cliques += step(g, per_call)
        e1.record(stream)
        e1.synchronize()
        dev_ms += e0.elapsed_time(e1)
    torch.cuda.synchronize()
    clk = clocks.stop()

    # e2e: pinned host CSR -> C ABI (copy, validate, all calls) -> counts back
    rp_pin = torch.from_numpy(rp.view(np.int64)).pin_memory()
    col_pin = torch.from_numpy(col.view(np.int32)).pin_memory()
    e2e_ms = 0.0
    e2e_steps = max(1, min(args.steps, 2))
    for _ in range(e2e_steps):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        g2 = kcl.kcl_load_csr(rp_pin.numpy().view(np.uint64), col_pin.numpy().view(np.uint32))
        step(g2)
        g2.free()
        torch.cuda.synchronize()
        e2e_ms += (time.perf_counter() - t0) * 1e3
    h2d = (n + 1) * 8 + nnz * 4
    d2h = 16 * len(STEP_PLAN)

    if world > 1:
        t = torch.tensor([dev_ms, e2e_ms], dtype=torch.float64, device="cuda")
        torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
        dev_ms, e2e_ms = float(t[0]), float(t[1])
    cliques_all = cliques * world
    value = cliques_all / (dev_ms / 1e3)
    e2e_value = (cliques // args.steps) * e2e_steps * world / (e2e_ms / 1e3)

    roof = roofline(per_call, args.steps)
    launches = sum(sum(la.values()) - la["total"] for (_, _, _, _, _, la) in per_call) // args.steps
    res = {
        "metric": METRIC, "value": value, "unit": "k-cliques/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": dev_ms / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u32/u64",
        "data": "synthetic (seeded R-MAT generator, no dataset)",
        "config": {"workload": "rmat-scale20-ef16", "n": n, "undirected_edges": nnz // 2,
                   "plan": ["k=%d %s %s" % p for p in STEP_PLAN],
                   "l2": "inputs (%.0f MB CSR) larger than L2; L2 also flushed between steps"
                         % ((n + 1) * 8 / 1e6 + nnz * 4 / 1e6),
                   "parallelism": "replicas" if world > 1 else "single-gpu"},
        "counts": {"k=%d %s %s" % (k, o, m): c for (k, o, m, c, _, _) in per_call[: len(STEP_PLAN)]},
        "e2e": {"value": e2e_value, "unit": "k-cliques/s", "h2d_bytes_per_step": h2d,
                "d2h_bytes_per_step": d2h},
        "gpu_launches": launches,
        "clocks": clk,
        "roofline": roof,
        "stage_ms": stage_summary(per_call, args.steps),
    }
    g.free()
    return res


def stage_summary(per_call, steps):
    out = {}
    for (k, o, m, c, ms, la) in per_call:
        key = "k=%d %s %s" % (k, o, m)
        d = out.setdefault(key, {s: 0.0 for s in ms})
        for s, v in ms.items():
            d[s] += v / steps
    return {k: {s: round(v, 3) for s, v in d.items()} for k, d in out.items()}


def roofline(per_call, steps):
    """Dominant kernel: the listing kernels of the call family with the largest
    device time.  Their bound is the integer pipe (AND + POPC per bitmap word,
    or compare per merge element); the peak is derived from the SM count and
    clock."""
    peaks, src = _peaks()
    work = _load_work()
    best = None
    for (k, o, m, c, ms, la) in per_call:
        key = "k=%d %s %s" % (k, o, m)
        best = best if best and best[1] >= ms["listing"] else (key, ms["listing"], k, o, m)
    key, _, k, o, m = best
    times = [ms["listing"] for (kk, oo, mm, _, ms, _) in per_call if (kk, oo, mm) == (k, o, m)]
    avg_ms = sum(times) / len(times)
    sm_mhz = peaks.get("sm_max_mhz", 2070.0)
    # integer pipe: 16 POPC per SM per clock on 152 SMs
    peak_gops = 152 * 16 * sm_mhz * 1e6 / 1e9
    wk = work.get("k=%d %s" % (k, o))
    achieved = (wk / (avg_ms / 1e3) / 1e9) if wk else None
    return {"kernel": "listing kernels, %s" % key, "bound": "alu", "achieved": achieved,
            "peak": peak_gops, "unit": "Gword/s" if o == "color" else "Gelem/s",
            "frac": (achieved / peak_gops) if achieved else None, "traffic": None,
            "peak_source": "derived: 152 SMs x 16 POPC/clk x %.0f MHz (%s clock)" % (sm_mhz, src),
            "avg_ms": avg_ms}


def _load_work():
    p = os.path.join(ROOT, "tests", "golden", "rmat20_work.json")
    if not os.path.exists(p):
        return {}
    with open(p) as f:
        return {k: v["work"] for k, v in json.load(f).items()}


# --------------------------------------------------------- oracle (CPU)
def oracle_sample(budget_s=15.0):
    """Time the oracle on a bounded sample of the workload: every 97th root
    of the degeneracy DAG (BitCol) and of the degree DAG (SDegree), k = 4."""
    import numpy as np

    import oracle
    rp, col = workload()
    n = len(rp) - 1
    roots = np.arange(0, n, 97, dtype=np.uint32)
    t0 = time.perf_counter()
    found = 0
    calls = 0
    for fn in (oracle.bitcol, oracle.sdegree):
        r = fn(rp, col, 4, roots=roots)
        found += r["count"]
        calls += 1
        if time.perf_counter() - t0 > budget_s:
            break
    dt = time.perf_counter() - t0
    return {"value": found / dt, "unit": "k-cliques/s", "cores": 1, "kind": "oracle",
            "sample": "k=4, roots 0,97,194,... (%d of %d) of R-MAT scale 20; %d ordering(s); "
                      "includes the oracle's full Pre-Core/Pre-List/orientation passes" %
                      (len(roots), n, calls), "seconds": dt}


def run_reference(args, rank, world):
    if rank != 0:
        return None
    vals = []
    for _ in range(args.warmup + args.steps):
        vals.append(oracle_sample(budget_s=10.0))
    timed = vals[args.warmup:]
    value = sum(v["value"] for v in timed) / len(timed)
    sec = sum(v["seconds"] for v in timed)
    cb = dict(timed[-1])
    cb["value"] = value
    return {"impl": "reference", "metric": METRIC, "value": value, "unit": "k-cliques/s",
            "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": sec * 1e3 / len(timed), "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "u32/u64", "data": "synthetic (seeded R-MAT generator)",
            "config": {"workload": "rmat-scale20-ef16", "sample": cb["sample"]},
            "cpu_baseline": cb,
            "e2e": {"value": value, "unit": "k-cliques/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    args = ap.parse_args()
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
