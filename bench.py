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
# same kernel (profiles/k_items_band_binary_N100000_p1000.md: all 16 launches
# at 50 trees, scaled to 500 trees); None once the kernel changes.
ITEMS_BAND_TRAFFIC_PER_LAUNCH = 10.0e9
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


# the other single-job workloads (parity cases; not the default line):
#   name -> (generator, metric, importance label)
def other_workloads():
    from paper_2605_09950_gb300 import synth

    return {
        "snp": (lambda trees: synth.snp_regression(n_trees=trees or 256),
                "Boruta iterations/sec (SNP regression N=2e4, p=2e4, 256 trees, depth 12, impurity importance)",
                "treeimp"),
        "multiclass": (lambda trees: synth.multiclass_toeplitz(n_trees=trees or 300),
                       "Boruta iterations/sec (5-class N=1e6, p=500, 300 trees, depth 20, OOB permutation "
                       "importance)", "permut_oob"),
        "small": (lambda trees: synth.binary_small(n_trees=trees or 100),
                  "Boruta iterations/sec (binary N=1000, p=50, 100 trees, depth 8, impurity importance)", "treeimp"),
    }


def combine_ranks(total_ms, units, dist=None, device="cuda"):
    """Whole-job throughput over the ranks: the slowest rank's time (max over
    ranks) and the units every rank processed.  Returns (value, max_ms)."""
    world = 1
    if dist is not None and dist.is_initialized():
        import torch

        world = dist.get_world_size()
        t = torch.tensor([float(total_ms)], dtype=torch.float64, device=device)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        total_ms = float(t.item())
        dist.barrier()
    return world * units / (total_ms / 1000.0), total_ms


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


def cpu_baseline_sample(w, trees=1, permut=True):
    import numpy as np

    import oracle

    P = oracle.BorutaProblem(w.X, w.y, **w.params(), N=w.N)
    live = np.arange(w.p, dtype=np.int32)
    t0 = time.perf_counter()
    sha = P.shadow(1, live)
    t1 = time.perf_counter()
    for tau in range(trees):
        P.tree(1, live, sha, tau, nodes=False, permut=permut)
    t2 = time.perf_counter()
    per_iter = (t1 - t0) + (t2 - t1) / trees * w.n_trees
    what = "fit + OOB permutation row" if permut else "fit + impurity row"
    return {"value": 1.0 / per_iter, "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": f"iteration 1: full shadow matrix + {trees} of {w.n_trees} trees ({what}), "
                      f"scaled to {w.n_trees} trees; single-threaded C"}


class Stepper:
    """Steps a session; a run that finished (every feature decided, or
    t = max_iter) is restarted from its initial state before the next step,
    outside any timed region (ready())."""

    def __init__(self, S, max_iter):
        self.S, self.max_iter = S, max_iter
        self.fresh = S.read()
        self.t, self.done = 0, False

    def ready(self):
        if self.done:
            self.reset()

    def reset(self):
        self.S.write(self.fresh)
        self.t, self.done = 0, False

    def step(self):
        und = self.S.step()
        self.t += 1
        self.done = und == 0 or self.t >= self.max_iter


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
    metric, importance = METRIC, "permut_oob"
    if args.workload == "binary":
        w = workload(args.trees)
    else:
        gen, metric, importance = other_workloads()[args.workload]
        w = gen(args.trees)
    X = torch.from_numpy(w.X).cuda()
    y = torch.from_numpy(w.y).cuda()
    params = w.params()
    nc = params.pop("n_classes")
    precision = args.precision
    S = boruta.Session(X, y, N=w.N, n_classes=nc, precision=precision, job=rank, **params)
    R = Stepper(S, w.max_iter)
    flush = torch.empty(512 << 20, dtype=torch.uint8, device="cuda")  # > L2, written between steps
    for _ in range(args.warmup):
        R.ready()
        R.step()
    R.reset()
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    clk_path = os.path.join(tempfile.gettempdir(), f"bench_clocks_{os.getpid()}.csv")
    proc, fh = start_clock_sampler(clk_path) if rank == 0 else (None, None)
    step_ms = []
    ks_tot = dict(hist_ms=0.0, hist_bytes=0.0, split_ms=0.0, split_bytes=0.0, launches=0)
    stream = torch.cuda.current_stream()
    for _ in range(args.steps):
        R.ready()
        flush.fill_(1)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        R.step()
        e1.record(stream)
        torch.cuda.synchronize()
        step_ms.append(e0.elapsed_time(e1))
        for k, v in S.kernel_stats().items():
            ks_tot[k] += v
    levels = S.dump(boruta.DUMP_LEVELS, np.float64).reshape(-1, 3)
    value, total_ms = combine_ranks(sum(step_ms), args.steps, dist)
    clocks = stop_clock_sampler(proc, fh, clk_path, local) if rank == 0 else None
    res = S.read()
    S.close()
    del S

    # the same iterations with FP64 per-term arithmetic (identical trees and decisions)
    other = None
    if not args.no_other:
        S2 = boruta.Session(X, y, N=w.N, n_classes=nc, precision=1 - precision, job=rank, **params)
        R2 = Stepper(S2, w.max_iter)
        R2.step()
        R2.reset()
        ms2 = []
        for _ in range(args.steps):
            R2.ready()
            flush.fill_(1)
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            R2.step()
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
    fit = boruta.boruta_fit(w.X, w.y, N=w.N, n_classes=nc, precision=precision, host_inputs=1, job=rank,
                            **{**params, "max_iter": min(args.steps, w.max_iter)})
    e2e_s = time.perf_counter() - t0
    e2e_iters = max(1, int(fit["iterations"]))  # a run may finish before max_iter
    h2d = int(w.X.nbytes + w.y.nbytes)
    d2h = int(w.p * (1 + 4) + 8 * e2e_iters * w.p + 8 * e2e_iters)

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
        "metric": metric, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None,
        "dtype": "u8+int64+" + ("f32" if precision else "f64"), "data": "synthetic",
        "config": {"workload": w.name, "N": w.N, "p": w.p, "n_trees": w.n_trees, "max_depth": w.max_depth,
                   "n_bins": w.n_bins, "importance": importance,
                   "precision": "fp32 terms, exact sums" if precision else "fp64 terms, exact sums",
                   "parallelism": "replicas" if world > 1 else "single",
                   "l2": "512 MiB buffer written between timed steps; per-step working set > 1 GB"},
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                     "frac": achieved / peak if peak else None,
                     "traffic": ITEMS_BAND_TRAFFIC_PER_LAUNCH if args.workload == "binary" and not args.trees else None,
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
        "cpu_baseline": (cpu_baseline_sample(w, permut=importance == "permut_oob")
                         if (world == 1 and not args.no_cpu) else None),
        "e2e": {"value": e2e_iters / e2e_s, "unit": UNIT, "h2d_bytes_per_step": h2d / e2e_iters,
                "d2h_bytes_per_step": d2h / e2e_iters,
                "note": "boruta_fit with host X/y: upload, K iterations, readback; includes session setup"},
        "gpu_launches": per_step_launches * args.steps,
        "clocks": clocks,
        "iterations_checked": int(res["iterations"]),
    }
    print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()


BATCH_METRIC = ("Boruta job-iterations/sec (64 independent classification jobs, N log-uniform in [500, 50000], "
                "p log-uniform in [20, 5000], 2-4 classes, 200 trees, depth 10, OOB permutation importance)")


def run_batch(args):
    """The batched-jobs workload: one step = one Boruta iteration of all 64
    jobs (boruta_batch_run, FP32 terms), against the plain form: the same
    jobs one at a time, one session each, FP64 terms."""
    # 64 job streams: more hardware work queues than the default 8 (read when
    # the CUDA context is created, so before the first CUDA call)
    os.environ.setdefault("CUDA_DEVICE_MAX_CONNECTIONS", "32")
    import numpy as np
    import torch

    from paper_2605_09950_gb300 import boruta, build, synth

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    dist = None
    if world > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    build.build()
    t0 = time.perf_counter()
    ws = synth.batch_jobs(n_jobs=args.jobs)
    gen_s = time.perf_counter() - t0
    jobs = [dict(X=torch.from_numpy(w.X).cuda(), y=torch.from_numpy(w.y).cuda(), N=w.N, **w.params()) for w in ws]
    stream = torch.cuda.current_stream()
    flush = torch.empty(512 << 20, dtype=torch.uint8, device="cuda")
    opts = dict(precision=1, job=rank * 4096, stream=stream.cuda_stream, graph=int(args.graph))

    B = boruta.Batch(jobs, **opts)  # warm-up on a throw-away batch
    B.run(args.warmup)
    B.close()
    t1 = time.perf_counter()
    B = boruta.Batch(jobs, **opts)
    setup_s = time.perf_counter() - t1
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    clk_path = os.path.join(tempfile.gettempdir(), f"bench_clocks_{os.getpid()}.csv")
    proc, fh = start_clock_sampler(clk_path) if rank == 0 else (None, None)
    # K iterations of every job, each job advancing as soon as its previous
    # iteration completes (the jobs' inputs, ~1.5 GB with shadows, exceed L2)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    flush.fill_(1)
    e0.record(stream)
    B.run(args.steps)
    e1.record(stream)
    torch.cuda.synchronize()
    value, total_ms = combine_ranks(e0.elapsed_time(e1), len(jobs) * args.steps, dist)
    clocks = stop_clock_sampler(proc, fh, clk_path, local) if rank == 0 else None
    batched = [B.read(j) for j in range(len(jobs))]
    B.close()

    # the plain form: each job alone, FP64 terms, after one untimed iteration
    plain_ms, same = 0.0, 0
    for j, jb in enumerate(jobs):
        params = ws[j].params()
        nc = params.pop("n_classes")
        S = boruta.Session(jb["X"], jb["y"], N=jb["N"], n_classes=nc, precision=0, job=rank * 4096 + j, **params)
        fresh = S.read()
        S.step()
        S.write(fresh)
        for _ in range(args.steps):
            flush.fill_(1)
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            S.step()
            e1.record(stream)
            torch.cuda.synchronize()
            plain_ms += e0.elapsed_time(e1)
        r = S.read()
        S.close()
        same += int((r["hits"] == batched[j]["hits"]).all() and (r["decision"] == batched[j]["decision"]).all())
    plain = len(jobs) * args.steps / (plain_ms / 1000.0)

    # end to end: host inputs, upload + K lockstep iterations + readback
    host_jobs = [dict(X=w.X, y=w.y, N=w.N, **{**w.params(), "max_iter": args.steps}) for w in ws]
    t2 = time.perf_counter()
    boruta.boruta_fit_batch(host_jobs, host_inputs=1, precision=1, job=rank * 4096)
    e2e_s = time.perf_counter() - t2
    h2d = sum(int(w.X.nbytes + w.y.nbytes) for w in ws)
    d2h = sum(int(w.p * 5 + 8 * args.steps * w.p + 8 * args.steps) for w in ws)
    if rank == 0:
        line = {
            "metric": BATCH_METRIC, "value": value, "unit": "job-iterations/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": total_ms / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u8+int64+f32",
            "data": "synthetic",
            "config": {"workload": "batch_64_jobs", "jobs": len(jobs), "sum_N_x_p": int(sum(w.N * w.p for w in ws)),
                       "n_trees": 200, "max_depth": 10, "n_bins": 128, "importance": "permut_oob",
                       "precision": "fp32 terms, exact sums",
                       "l2": "inputs larger than L2 (X and shadows of 64 jobs ~1.5 GB); one 512 MiB flush before",
                       "schedule": "boruta_batch_run: each job's next iteration enqueued when its last completes",
                       "graph_replay": bool(args.graph),
                       "input_generation_s": gen_s, "batch_setup_s": setup_s},
            "plain_form": {"value": plain, "unit": "job-iterations/s",
                           "form": "one job at a time, one session each, fp64 terms",
                           "jobs_with_identical_hits_and_decisions": same},
            "batched_over_plain": value / plain,
            "roofline": None, "cpu_baseline": None,
            "e2e": {"value": len(jobs) * args.steps / e2e_s, "unit": "job-iterations/s",
                    "h2d_bytes_per_step": h2d / args.steps, "d2h_bytes_per_step": d2h / args.steps,
                    "note": "boruta_fit_batch with host inputs: setup, upload, K iterations, readback"},
            "gpu_launches": len(jobs) * (8 + 11 * 10) * args.steps,
            "clocks": clocks,
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
    ap.add_argument("--ref-trees", type=int, default=1)
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-other", action="store_true", help="skip timing the other precision form")
    ap.add_argument("--trees", type=int, default=None, help="fewer trees (profiling captures only)")
    ap.add_argument("--workload", default="binary", choices=["binary", "batch", "snp", "multiclass", "small"],
                    help="binary: N=1e5 p=1000 (default); batch: 64 uneven jobs, batched vs plain form; "
                         "snp / multiclass / small: the other single-job workloads")
    ap.add_argument("--jobs", type=int, default=64, help="batch workload: number of jobs")
    ap.add_argument("--graph", action="store_true", help="batch workload: replay each job's iterations as CUDA graphs")
    args = ap.parse_args()
    if args.impl == "reference":
        run_reference(args)
    elif args.workload == "batch":
        run_batch(args)
    else:
        run_gpu(args)


if __name__ == "__main__":
    main()
