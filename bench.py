"""Benchmark: Boruta iterations per second on the binary N=1e5, p=1000 workload.

One step = one Boruta iteration (Alg. 1 loop body) of the whole hot path:
shadow features, bootstrap, a 500-tree depth-16 forest fit on the
shadow-augmented matrix, OOB permutation importance, Z-score hits and the
binomial test.  Steps are iterations t = 1..K of a run (no feature can be
decided before t = 17 at alpha = 0.01 with 1000 features, so every timed
iteration has the full 2000 augmented columns).

Prints one JSON line (rank 0).  --impl reference times the CPU oracle on a
bounded sample of the same workload instead.
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

WORKLOAD = dict(N=100_000, p=1000, n_trees=500, max_depth=16, n_bins=256)
# DRAM bytes (read + write) per k_items_band launch from an ncu capture of the
# same kernel (profiles/k_items_band_binary_N100000_p1000.md), scaled to 500
# trees; None until the current kernel has been captured.
ITEMS_BAND_TRAFFIC_PER_LAUNCH = None
METRIC = "Boruta iterations/sec (binary N=1e5, p=1000, 500 trees, depth 16, OOB permutation importance)"
UNIT = "iterations/s"


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            m = json.load(f)
        return float(m["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def start_clock_sampler(path):
    q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
    try:
        f = open(path, "w")
        p = subprocess.Popen(["nvidia-smi", f"--query-gpu={q}", "--format=csv,noheader,nounits", "-lms", "200"],
                             stdout=f, stderr=subprocess.DEVNULL)
        return p, f
    except Exception:
        return None, None


def stop_clock_sampler(proc, f, path, gpu_index):
    if proc is None:
        return None
    proc.terminate()
    try:
        proc.wait(timeout=5)
    except Exception:
        proc.kill()
    f.close()
    sm, mx, reasons = [], 0, set()
    names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
    for line in open(path):
        parts = [x.strip() for x in line.split(",")]
        if len(parts) < 9 or parts[0] != str(gpu_index):
            continue
        try:
            sm.append(float(parts[1]))
            mx = max(mx, float(parts[2]))
        except ValueError:
            continue
        for n, v in zip(names, parts[5:9]):
            if v.lower() == "active":
                reasons.add(n)
    if not sm:
        return None
    return {"sm_mhz": statistics.median(sm), "sm_max_mhz": mx, "reasons": sorted(reasons),
            "samples": len(sm)}


def workload(trees=None):
    from paper_2605_09950_gb300 import synth

    return synth.binary_wide(N=WORKLOAD["N"], p=WORKLOAD["p"], n_trees=trees or WORKLOAD["n_trees"],
                             max_depth=WORKLOAD["max_depth"], n_bins=WORKLOAD["n_bins"], max_iter=100)


def run_reference(args):
    """The CPU oracle (as it stands) on a bounded sample: the shadow matrix of
    iteration 1 plus `ref_trees` full trees with their OOB permutation rows;
    iterations/s = 1 / (t_shadow + 500 * t_tree)."""
    import numpy as np

    import oracle

    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    w = workload()
    P = oracle.BorutaProblem(w.X, w.y, **w.params(), N=w.N)
    live = np.arange(w.p, dtype=np.int32)
    oracle.lib()
    vals = []
    for _ in range(args.warmup + args.steps if args.steps else 1):
        t0 = time.perf_counter()
        sha = P.shadow(1, live)
        t1 = time.perf_counter()
        for tau in range(args.ref_trees):
            P.tree(1, live, sha, tau, nodes=False, permut=True)
        t2 = time.perf_counter()
        per_iter = (t1 - t0) + (t2 - t1) / args.ref_trees * w.n_trees
        vals.append(1.0 / per_iter)
    vals = vals[args.warmup:] or vals
    v = statistics.median(vals)
    sample = (f"iteration 1: full shadow matrix + {args.ref_trees} of 500 trees with their OOB permutation "
              f"rows, scaled to 500 trees; median of {len(vals)} repeats")
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1000.0 / v, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "u8+int64+f64", "data": "synthetic",
            "config": {"workload": "binary_N100000_p1000", **WORKLOAD, "importance": "permut_oob",
                       "l2": "n/a (CPU)"},
            "cpu_baseline": {"value": v, "unit": UNIT, "cores": 1, "kind": "oracle", "sample": sample},
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def cpu_baseline_sample(w, trees=1):
    import numpy as np

    import oracle

    P = oracle.BorutaProblem(w.X, w.y, **w.params(), N=w.N)
    live = np.arange(w.p, dtype=np.int32)
    t0 = time.perf_counter()
    sha = P.shadow(1, live)
    t1 = time.perf_counter()
    for tau in range(trees):
        P.tree(1, live, sha, tau, nodes=False, permut=True)
    t2 = time.perf_counter()
    per_iter = (t1 - t0) + (t2 - t1) / trees * w.n_trees
    return {"value": 1.0 / per_iter, "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": f"iteration 1: full shadow matrix + {trees} of {w.n_trees} trees (fit + OOB permutation "
                      f"row), scaled to {w.n_trees} trees; single-threaded C"}


def run_gpu(args):
    import numpy as np
    import torch

    from paper_2605_09950_gb300 import boruta, build

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    dist = None
    if world > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    build.build()
    w = workload(args.trees)
    X = torch.from_numpy(w.X).cuda()
    y = torch.from_numpy(w.y).cuda()
    params = w.params()
    nc = params.pop("n_classes")
    precision = args.precision
    S = boruta.Session(X, y, N=w.N, n_classes=nc, precision=precision, job=rank, **params)
    fresh = S.read()
    flush = torch.empty(512 << 20, dtype=torch.uint8, device="cuda")  # > L2, written between steps
    for _ in range(args.warmup):
        S.step()
    S.write(fresh)
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    clk_path = os.path.join(tempfile.gettempdir(), f"bench_clocks_{os.getpid()}.csv")
    proc, fh = start_clock_sampler(clk_path) if rank == 0 else (None, None)
    step_ms = []
    ks_tot = dict(hist_ms=0.0, hist_bytes=0.0, split_ms=0.0, split_bytes=0.0, launches=0)
    stream = torch.cuda.current_stream()
    for _ in range(args.steps):
        flush.fill_(1)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        S.step()
        e1.record(stream)
        torch.cuda.synchronize()
        step_ms.append(e0.elapsed_time(e1))
        for k, v in S.kernel_stats().items():
            ks_tot[k] += v
    levels = S.dump(boruta.DUMP_LEVELS, np.float64).reshape(-1, 3)
    total_ms = sum(step_ms)
    if dist:
        t = torch.tensor([total_ms], device="cuda")
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        total_ms = float(t.item())
        dist.barrier()
    clocks = stop_clock_sampler(proc, fh, clk_path, local) if rank == 0 else None
    value = world * args.steps / (total_ms / 1000.0)
    res = S.read()
    S.close()
    del S

    # the same iterations with FP64 per-term arithmetic (identical trees and decisions)
    other = None
    if not args.no_other:
        S2 = boruta.Session(X, y, N=w.N, n_classes=nc, precision=1 - precision, job=rank, **params)
        fresh2 = S2.read()
        S2.step()
        S2.write(fresh2)
        ms2 = []
        for _ in range(args.steps):
            flush.fill_(1)
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            S2.step()
            e1.record(stream)
            torch.cuda.synchronize()
            ms2.append(e0.elapsed_time(e1))
        res2 = S2.read()
        S2.close()
        del S2
        same = bool((res2["decision"] == res["decision"]).all() and (res2["hits"] == res["hits"]).all())
        other = {"precision": "fp64 terms" if precision else "fp32 terms",
                 "value": args.steps / (sum(ms2) / 1000.0), "unit": UNIT, "identical_hits_and_decisions": same}

    # end to end through the C ABI with host buffers (upload + K iterations + readback)
    t0 = time.perf_counter()
    boruta.boruta_fit(w.X, w.y, N=w.N, n_classes=nc, precision=precision, host_inputs=1, job=rank,
                      **{**params, "max_iter": args.steps})
    e2e_s = time.perf_counter() - t0
    h2d = int(w.X.nbytes + w.y.nbytes)
    d2h = int(w.p * (1 + 4) + 8 * args.steps * w.p + 8 * args.steps)

    if rank != 0:
        if dist:
            dist.destroy_process_group()
        return
    peak, peak_kind = peaks()
    achieved = ks_tot["hist_bytes"] / (ks_tot["hist_ms"] / 1000.0) / 1e9 if ks_tot["hist_ms"] > 0 else 0.0
    split_gbs = ks_tot["split_bytes"] / (ks_tot["split_ms"] / 1000.0) / 1e9 if ks_tot["split_ms"] > 0 else 0.0
    # per step: gather + shadow + 2 bootstrap, 12 per level, 2 permutation importance, stats + decide
    per_step_launches = 4 + 12 * w.max_depth + 2 + 2
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None,
        "dtype": "u8+int64+" + ("f32" if precision else "f64"), "data": "synthetic",
        "config": {"workload": "binary_N100000_p1000", **WORKLOAD, "n_trees": w.n_trees,
                   "importance": "permut_oob",
                   "precision": "fp32 terms, exact sums" if precision else "fp64 terms, exact sums",
                   "parallelism": "replicas" if world > 1 else "single",
                   "l2": "512 MiB buffer written between timed steps; per-step working set > 1 GB"},
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                     "frac": achieved / peak if peak else None,
                     "traffic": ITEMS_BAND_TRAFFIC_PER_LAUNCH,
                     "kernel": "k_items_band (feature histograms + exact scan of the larger nodes)",
                     "peak_kind": f"{peak_kind} hbm_gbs", "launches": int(ks_tot["launches"]),
                     "kernel_ms_per_step": ks_tot["hist_ms"] / args.steps,
                     "algorithmic_bytes_per_launch": ks_tot["hist_bytes"] / max(1, ks_tot["launches"]),
                     "algorithmic_bytes": "per node and level: rows x (mtry bins + 10 B row state)"},
        "split_stage": {"ms_per_step": ks_tot["split_ms"] / args.steps, "achieved_gbs": split_gbs,
                        "note": "all split kernels of the levels, algorithmic bytes / event time",
                        "levels": [[int(c), round(float(a), 3), round(float(h), 3)] for c, a, h in levels[:-1]],
                        "levels_note": "last timed step, per depth: nodes, split-stage ms, histogram-kernel ms"},
        "other_form": other,
        "cpu_baseline": cpu_baseline_sample(w) if (world == 1 and not args.no_cpu) else None,
        "e2e": {"value": args.steps / e2e_s, "unit": UNIT, "h2d_bytes_per_step": h2d / args.steps,
                "d2h_bytes_per_step": d2h / args.steps,
                "note": "boruta_fit with host X/y: upload, K iterations, readback; includes session setup"},
        "gpu_launches": per_step_launches * args.steps,
        "clocks": clocks,
        "iterations_checked": int(res["iterations"]),
    }
    print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gpu", choices=["gpu", "reference"])
    ap.add_argument("--precision", type=int, default=1, help="0 = FP64 terms, 1 = FP32 terms")
    ap.add_argument("--ref-trees", type=int, default=2)
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-other", action="store_true", help="skip timing the other precision form")
    ap.add_argument("--trees", type=int, default=None, help="fewer trees (profiling captures only)")
    args = ap.parse_args()
    if args.impl == "reference":
        run_reference(args)
    else:
        run_gpu(args)


if __name__ == "__main__":
    main()
