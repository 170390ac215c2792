"""Benchmark: Boruta iterations per second on one GPU, with the histogram
kernel's share of the HBM roofline.

Default workload: five-class N=1e6, p=500 (Toeplitz blocks), 300 trees,
depth 20, OOB permutation importance (Alg. 3) in the FP32-term form -- the
largest of the single-GPU workloads.  One step = one Boruta iteration (the
Alg. 1 loop body) of the whole hot path: shadow features, bootstrap, the
forest fit on the shadow-augmented matrix, the importance rows, the
Z-score hits and the binomial test.  Steps are iterations t = 1..K of a run
(a run that finishes is restarted outside the timed region).

Besides the headline it measures, in the same run: the same iterations with
FP64 terms (the plain form), the end-to-end rate through boruta_fit with
host buffers, the Alg. 3 walks (node visits/s), the 64-job batched workload
against its plain form, and the CPU oracle on every host core.

Prints one JSON line (rank 0).  --impl reference times the CPU oracle on a
bounded sample of the same workload instead.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import tempfile
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

UNIT = "iterations/s"
DEFAULT_WORKLOAD = "multiclass"

# workload name -> (generator keyword arguments, metric, importance label)
WORKLOADS = {
    "multiclass": ("multiclass_toeplitz", dict(),
                   "Boruta iterations/sec (5-class N=1e6, p=500, 300 trees, depth 20, OOB permutation importance)",
                   "permut_oob"),
    "binary": ("binary_wide", dict(),
               "Boruta iterations/sec (binary N=1e5, p=1000, 500 trees, depth 16, OOB permutation importance)",
               "permut_oob"),
    "snp": ("snp_regression", dict(),
            "Boruta iterations/sec (SNP regression N=2e4, p=2e4, 256 trees, depth 12, impurity importance)",
            "treeimp"),
    "small": ("binary_small", dict(),
              "Boruta iterations/sec (binary N=1000, p=50, 100 trees, depth 8, impurity importance)", "treeimp"),
}

# DRAM bytes (read + write) per launch of the histogram kernel, from the ncu
# capture named beside it, valid only for the kernel source it was taken on
# (sha-256 prefix of csrc/split.cu); the line reports null otherwise.
# DRAM bytes (read + write) of the histogram kernel per tree level, from one
# ncu capture of a whole iteration (the profile named), valid only while the
# kernel's and its launch code's sources hash to sources_sha16
TRAFFIC = {
    "multiclass_N1000000_p500": {"bytes_per_launch": (582.6e9 + 62.35e9) / 20, "sources_sha16": "0c5bad21bed32dbd",
                                 "profile": "profiles/k_items_band_multiclass_N1000000_p500.md"},
}


def kernel_source_sha16():
    """Hash of the histogram kernel's sources and of the host code that sets
    its launches (a recorded traffic figure holds only for these)."""
    h = hashlib.sha256()
    for name in ("split.cu", "engine.cuh", "api.cu"):
        with open(os.path.join(ROOT, "paper_2605_09950_gb300", "csrc", name), "rb") as f:
            h.update(f.read())
    return h.hexdigest()[:16]


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


def gpu_quantiser(F, n_bins):
    """The library's own quantiser (boruta_quantise) on the current GPU:
    float32 (p, N) host features -> (p, round16(N)) uint8 host bins, the
    rank rule of synth.quantise."""
    import numpy as np
    import torch

    from paper_2605_09950_gb300 import boruta

    p, N = F.shape
    out = np.zeros((p, (N + 15) // 16 * 16), dtype=np.uint8)
    step = max(1, (1 << 28) // max(1, N))  # columns per upload (~1 GiB of float32)
    for j0 in range(0, p, step):
        Fd = torch.from_numpy(np.ascontiguousarray(F[j0:j0 + step], dtype=np.float32)).cuda()
        out[j0:j0 + step] = boruta.boruta_quantise(Fd, n_bins, N=N).cpu().numpy()
        del Fd
    return out


def make_workload(name, trees=None, quantiser=None):
    from paper_2605_09950_gb300 import synth

    gen, kw, metric, importance = WORKLOADS[name]
    kw = dict(kw)
    if trees:
        kw["n_trees"] = trees
    if quantiser is not None and name == "multiclass":
        kw["quantiser"] = quantiser
    return getattr(synth, gen)(**kw), metric, importance


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


# ---------------------------------------------------------------- CPU oracle on every core

def _oracle_tree(job):
    """One tree of iteration 1 (fit plus its importance row) with the oracle,
    in a worker process; the inputs come from shared memory."""
    from multiprocessing import shared_memory

    import numpy as np

    import oracle

    names, shapes, dtypes, params, N, tau, permut = job
    blocks = [shared_memory.SharedMemory(name=n) for n in names]
    try:
        X, y, sha = (np.ndarray(s, dtype=d, buffer=b.buf) for s, d, b in zip(shapes, dtypes, blocks))
        P = oracle.BorutaProblem(X, y, **params, N=N)
        live = np.arange(X.shape[0], dtype=np.int32)
        t0 = time.perf_counter()
        P.tree(1, live, sha, tau, nodes=False, treeimp=not permut, permut=permut)
        dt = time.perf_counter() - t0
        del X, y, sha, P
    finally:
        for b in blocks:
            b.close()
    return tau, dt


class OracleSample:
    """The CPU oracle, as it stands, on a bounded sample of iteration 1 of a
    workload: the full shadow matrix (one process), then `trees` trees with
    their importance rows, one per worker process on `workers` host cores
    (spawned processes; inputs in shared memory).  Runs in a background
    thread so that GPU work can proceed meanwhile.

    iterations/s = 1 / (t_shadow + M * mean(t_tree) / workers): the M trees
    of an iteration are independent given the shadow matrix, and each
    worker fits one tree at a time (the oracle is single-threaded)."""

    def __init__(self, w, workers, trees=None):
        self.w, self.workers = w, max(1, workers)
        self.trees = self.workers if trees is None else max(1, trees)
        self.result, self.error = None, None
        self.thread = threading.Thread(target=self._run, daemon=True)

    def start(self):
        self.thread.start()
        return self

    def _run(self):
        try:
            self.result = self._sample()
        except Exception as e:  # reported in the line, never silently
            self.error = f"{type(e).__name__}: {e}"

    def _sample(self):
        import multiprocessing as mp
        from multiprocessing import shared_memory

        import numpy as np

        import oracle

        w = self.w
        permut = (w.task & 2) != 0
        P = oracle.BorutaProblem(w.X, w.y, **w.params(), N=w.N)
        live = np.arange(w.p, dtype=np.int32)
        t0 = time.perf_counter()
        sha = P.shadow(1, live)
        t_shadow = time.perf_counter() - t0
        arrays = [np.ascontiguousarray(w.X), np.ascontiguousarray(w.y), sha]
        blocks = []
        try:
            for a in arrays:
                b = shared_memory.SharedMemory(create=True, size=max(1, a.nbytes))
                np.ndarray(a.shape, dtype=a.dtype, buffer=b.buf)[...] = a
                blocks.append(b)
            jobs = [([b.name for b in blocks], [a.shape for a in arrays], [a.dtype.str for a in arrays],
                     w.params(), w.N, tau % w.n_trees, permut) for tau in range(self.trees)]
            ctx = mp.get_context("spawn")
            t1 = time.perf_counter()
            with ctx.Pool(self.workers) as pool:
                times = [dt for _, dt in pool.imap_unordered(_oracle_tree, jobs)]
            wall = time.perf_counter() - t1
        finally:
            for b in blocks:
                b.close()
                b.unlink()
        t_tree = sum(times) / len(times)
        per_iter = t_shadow + w.n_trees * t_tree / self.workers
        what = "fit + OOB permutation row" if permut else "fit + impurity row"
        return {"value": 1.0 / per_iter, "unit": UNIT, "cores": self.workers, "kind": "oracle",
                "sample": (f"iteration 1: full shadow matrix ({t_shadow:.1f} s, one process) + {len(times)} of "
                           f"{w.n_trees} trees ({what}; {t_tree:.1f} s mean per tree, {wall:.1f} s wall) on "
                           f"{self.workers} spawned processes; iteration = shadow + {w.n_trees} trees / "
                           f"{self.workers} cores; plain C oracle, single-threaded per tree"),
                "nproc": os.cpu_count(), "tree_s": sorted(times), "shadow_s": t_shadow}

    def join(self):
        self.thread.join()
        if self.error:
            return {"value": None, "unit": UNIT, "cores": self.workers, "kind": "oracle",
                    "sample": "failed: " + self.error}
        return self.result


def host_cores():
    try:
        return len(os.sched_getaffinity(0))
    except Exception:
        return os.cpu_count() or 1


def run_reference(args):
    """--impl reference: the CPU oracle, as it stands, on every host core, on
    a bounded sample of the same workload and config (OracleSample); one
    timed sample whatever --steps asks, since one sample already runs one
    tree per core."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    name = args.workload if args.workload != "batch" else DEFAULT_WORKLOAD
    w, metric, importance = make_workload(name)
    cores = host_cores()
    s = OracleSample(w, workers=cores, trees=args.ref_trees or cores).start().join()
    v = s["value"]
    line = {"impl": "reference", "metric": metric, "value": v, "unit": UNIT, "n_gpus": args.gpus,
            "steps": 1, "warmup": 0, "ms_per_step": 1000.0 / v if v else None, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "u8+int64+f64", "data": "synthetic",
            "config": {"workload": w.name, "N": w.N, "p": w.p, "n_trees": w.n_trees, "max_depth": w.max_depth,
                       "n_bins": w.n_bins, "importance": importance, "l2": "n/a (CPU)"},
            "cpu_baseline": s,
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
            "note": (f"requested --steps {args.steps} --warmup {args.warmup}: one sample of one tree per core "
                     f"is timed instead (an oracle tree of this workload takes minutes)")}
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------- GPU arm

class Stepper:
    """Steps a session; a run that finished (every feature decided, or
    t = max_iter) is restarted from its initial state before the next step,
    outside any timed region (ready())."""

    def __init__(self, S, max_iter):
        self.S, self.max_iter = S, max_iter
        self.fresh = S.read()
        self.t, self.done = 0, False
        self.launches = 0  # the library's kernels launched by this stepper's steps

    def ready(self):
        if self.done:
            self.reset()

    def reset(self):
        self.S.write(self.fresh)
        self.t, self.done = 0, False

    def step(self):
        und = self.S.step()
        self.launches += self.S.kernel_launches()
        self.t += 1
        self.done = und == 0 or self.t >= self.max_iter


def timed_steps(R, steps, stream, flush, on_step=None):
    """K steps, each bracketed by CUDA events on the launching stream, the L2
    flushed (a 512 MiB write) before each; returns per-step milliseconds."""
    import torch

    ms = []
    for _ in range(steps):
        R.ready()
        flush.fill_(1)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        R.step()
        e1.record(stream)
        torch.cuda.synchronize()
        ms.append(e0.elapsed_time(e1))
        if on_step:
            on_step()
    return ms


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
    t_gen = time.perf_counter()
    w, metric, importance = make_workload(args.workload, args.trees, quantiser=gpu_quantiser)
    gen_s = time.perf_counter() - t_gen
    cpu = None
    if world == 1 and not args.no_cpu:  # the oracle on the other host cores, meanwhile
        cpu = OracleSample(w, workers=max(1, host_cores() - 1), trees=args.cpu_trees).start()
    X = torch.from_numpy(w.X).cuda()
    y = torch.from_numpy(w.y).cuda()
    params = w.params()
    nc = params.pop("n_classes")
    precision = args.precision
    t_setup = time.perf_counter()
    S = boruta.Session(X, y, N=w.N, n_classes=nc, precision=precision, job=rank, autotune=int(args.autotune),
                       **params)
    torch.cuda.synchronize()
    setup_s = time.perf_counter() - t_setup
    R = Stepper(S, w.max_iter)
    flush = torch.empty(512 << 20, dtype=torch.uint8, device="cuda")  # > L2, written between steps
    stream = torch.cuda.current_stream()
    for _ in range(args.warmup):
        R.ready()
        R.step()
    R.reset()
    tuning = S.tuning() if args.autotune else None
    tuning_levels = S.tuning_levels() if args.autotune else None
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    clk_path = os.path.join(tempfile.gettempdir(), f"bench_clocks_{os.getpid()}.csv")
    proc, fh = start_clock_sampler(clk_path) if rank == 0 else (None, None)
    ks = dict(hist_ms=0.0, hist_bytes=0.0, split_ms=0.0, split_bytes=0.0, launches=0, imp_ms=0.0, visits=0.0)
    k_other = min(args.steps, args.other_steps)
    snap = {}

    def collect():
        for k, v in S.kernel_stats().items():
            ks[k] += v
        im = S.importance_stats()
        ks["imp_ms"] += im["ms"]
        ks["visits"] += im["node_visits"]
        if R.t == k_other and not snap:
            snap.update(S.read())
            snap["imp"] = S.dump(boruta.DUMP_IMP, np.float64)

    launches0 = R.launches
    step_ms = timed_steps(R, args.steps, stream, flush, collect)
    timed_launches = R.launches - launches0
    levels = S.dump(boruta.DUMP_LEVELS, np.float64).reshape(-1, 3)
    value, total_ms = combine_ranks(sum(step_ms), args.steps, dist)
    clocks = stop_clock_sampler(proc, fh, clk_path, local) if rank == 0 else None
    S.close()
    del S

    # the plain form: the same iterations with FP64 terms (identical trees; decisions compared)
    other = None
    if not args.no_other and k_other > 0:
        S2 = boruta.Session(X, y, N=w.N, n_classes=nc, precision=1 - precision, job=rank, **params)
        R2 = Stepper(S2, w.max_iter)
        R2.step()
        R2.reset()
        ms2 = timed_steps(R2, k_other, stream, flush)
        res2 = S2.read()
        imp2 = S2.dump(boruta.DUMP_IMP, np.float64)
        S2.close()
        del S2
        same = bool(snap) and bool((res2["decision"] == snap["decision"]).all() and
                                   (res2["hits"] == snap["hits"]).all())
        rel = None
        if snap and snap["imp"].shape == imp2.shape:  # the two forms' importance rows at iteration k
            den = np.maximum(np.abs(snap["imp"]), np.abs(imp2))
            rel = float(np.max(np.where(den > 0, np.abs(snap["imp"] - imp2) / np.where(den > 0, den, 1), 0.0)))
        other = {"precision": "fp64 terms" if precision else "fp32 terms", "steps": k_other,
                 "value": k_other / (sum(ms2) / 1000.0), "unit": UNIT,
                 "identical_hits_and_decisions_after_steps": same,
                 "max_rel_importance_difference_at_last_step": rel}

    # end to end through the C ABI with host buffers (upload + iterations + readback)
    k_e2e = max(1, min(args.steps, args.e2e_steps, w.max_iter))
    t0 = time.perf_counter()
    fit = boruta.boruta_fit(w.X, w.y, N=w.N, n_classes=nc, precision=precision, host_inputs=1, job=rank,
                            **{**params, "max_iter": k_e2e})
    e2e_s = time.perf_counter() - t0
    e2e_iters = max(1, int(fit["iterations"]))  # a run may finish before max_iter
    h2d = int(w.X.nbytes + w.y.nbytes)
    d2h = int(w.p * (1 + 4) + 8 * e2e_iters * w.p + 8 * e2e_iters)
    del X, y

    batch = None
    if not args.no_batch and world == 1:
        batch = batch_leg(args, rank, flush, stream)

    if rank != 0:
        if dist:
            dist.destroy_process_group()
        return
    peak, peak_kind = peaks()
    achieved = ks["hist_bytes"] / (ks["hist_ms"] / 1000.0) / 1e9 if ks["hist_ms"] > 0 else 0.0
    split_gbs = ks["split_bytes"] / (ks["split_ms"] / 1000.0) / 1e9 if ks["split_ms"] > 0 else 0.0
    prof = TRAFFIC.get(w.name)
    traffic = prof["bytes_per_launch"] if prof and prof["sources_sha16"] == kernel_source_sha16() \
        and not args.trees else None
    permut = importance == "permut_oob"
    walks = None
    if permut and ks["imp_ms"] > 0:
        vps = ks["visits"] / (ks["imp_ms"] / 1000.0)
        walks = {"node_visits_per_step": ks["visits"] / args.steps, "node_visits_per_s": vps,
                 "l2_gbs": vps * 17 / 1e9, "ms_per_step": ks["imp_ms"] / args.steps,
                 "l2_bytes_per_visit": "17 B: the two children's split words and child indices (16 B) "
                                       "loaded with the row's bin of the tested feature (1 B)",
                 "kernels": "k_permut_pi + k_permut + k_permut_final (CUDA events around the stage)"}
    line = {
        "metric": metric, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None,
        "dtype": "u8+int64+" + ("f32" if precision else "f64"), "data": "synthetic",
        "config": {"workload": w.name, "N": w.N, "p": w.p, "n_trees": w.n_trees, "max_depth": w.max_depth,
                   "n_bins": w.n_bins, "n_classes": nc or 1, "importance": importance,
                   "precision": "fp32 terms, exact sums" if precision else "fp64 terms, exact sums",
                   "tie_break": "lowest (feature, bin)",
                   "parallelism": "replicas" if world > 1 else "single",
                   "l2": "512 MiB buffer written before each timed step; inputs and per-step working set > L2",
                   "input_generation_s": round(gen_s, 1), "session_setup_s": round(setup_s, 2)},
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                     "frac": achieved / peak if peak else None, "traffic": traffic,
                     "traffic_source": prof["profile"] if traffic else None,
                     "kernel": "k_items_band (feature histograms + exact scan of the larger nodes)",
                     "peak_kind": f"{peak_kind} hbm_gbs (burst copy)", "launches": int(ks["launches"]),
                     "kernel_ms_per_step": ks["hist_ms"] / args.steps,
                     "algorithmic_bytes_per_launch": ks["hist_bytes"] / max(1, ks["launches"]),
                     "algorithmic_bytes": "per node and level: rows x (mtry bins + 10 B row state)"},
        "split_stage": {"ms_per_step": ks["split_ms"] / args.steps, "achieved_gbs": split_gbs,
                        "note": "all split kernels of the levels, algorithmic bytes / event time",
                        "levels": [[int(c), round(float(a), 3), round(float(h), 3)] for c, a, h in levels[:-1]],
                        "levels_note": "last timed step, per depth: nodes, split-stage ms, histogram-kernel ms"},
        "permut_walks": walks,
        "tile_autotune": ({"candidates": [{"group_work": gw, "band_mib": bb >> 20 if bb >= 0 else "per level",
                                           "launch_per_band": bl if bl >= 0 else "per level",
                                           "iteration_ms": round(ms, 2)} for gw, bb, bl, ms in tuning[0]],
                           "chosen": tuning[1],
                           "per_level": {"band_mib": [b >> 20 for b in tuning_levels[0]],
                                         "launch_per_band": tuning_levels[1],
                                         "level_ms_per_candidate": [[round(float(x), 2) for x in row]
                                                                    for row in tuning_levels[2]]}}
                          if tuning else None),
        "other_form": other,
        "batch": batch,
        "e2e": {"value": e2e_iters / e2e_s, "unit": UNIT, "h2d_bytes_per_step": h2d / e2e_iters,
                "d2h_bytes_per_step": d2h / e2e_iters, "iterations": e2e_iters,
                "note": "boruta_fit with host X/y: session setup, upload, iterations 1..k, readback"},
        "gpu_launches": timed_launches,
        "clocks": clocks,
    }
    if cpu is not None:
        line["cpu_baseline"] = cpu.join()
    else:
        line["cpu_baseline"] = None
    print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()


# ---------------------------------------------------------------- batched jobs

BATCH_METRIC = ("Boruta job-iterations/sec (64 independent classification jobs, N log-uniform in [500, 50000], "
                "p log-uniform in [20, 5000], 2-4 classes, 200 trees, depth 10, OOB permutation importance)")


def batch_jobs_on_device(n_jobs):
    import torch

    from paper_2605_09950_gb300 import synth

    ws = synth.batch_jobs(n_jobs=n_jobs, quantiser=gpu_quantiser)
    jobs = [dict(X=torch.from_numpy(w.X).cuda(), y=torch.from_numpy(w.y).cuda(), N=w.N, **w.params()) for w in ws]
    return ws, jobs


def batch_compare(ws, jobs, steps, warmup, rank, flush, stream, graph=False):
    """The batched form (boruta_batch_run over all jobs, FP32 terms) and the
    plain form (each job alone in its own session, FP64 terms) on the same
    jobs and iterations; returns (batched job-it/s, plain job-it/s, jobs
    with identical hits and decisions, batched ms, kernels the batched run
    launched)."""
    import torch

    from paper_2605_09950_gb300 import boruta

    opts = dict(precision=1, job=rank * 4096, stream=stream.cuda_stream, graph=int(graph))
    if warmup:
        B = boruta.Batch(jobs, **opts)  # warm-up on a throw-away batch
        B.run(warmup)
        B.close()
    B = boruta.Batch(jobs, **opts)
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    flush.fill_(1)
    e0.record(stream)
    B.run(steps)
    e1.record(stream)
    torch.cuda.synchronize()
    batched_ms = e0.elapsed_time(e1)
    launched = B.kernel_launches()  # a fresh batch: all of them in the timed run
    batched = [B.read(j) for j in range(len(jobs))]
    B.close()
    plain_ms, same = 0.0, 0
    for j, jb in enumerate(jobs):
        params = ws[j].params()
        nc = params.pop("n_classes")
        S = boruta.Session(jb["X"], jb["y"], N=jb["N"], n_classes=nc, precision=0, job=rank * 4096 + j, **params)
        fresh = S.read()
        S.step()
        S.write(fresh)
        R = Stepper(S, ws[j].max_iter)
        plain_ms += sum(timed_steps(R, steps, stream, flush))
        r = S.read()
        S.close()
        same += int((r["hits"] == batched[j]["hits"]).all() and (r["decision"] == batched[j]["decision"]).all())
    n = len(jobs) * steps
    return n / (batched_ms / 1000.0), n / (plain_ms / 1000.0), same, batched_ms, launched


def batch_leg(args, rank, flush, stream):
    """The 64-job workload inside the default line: batched over plain."""
    t0 = time.perf_counter()
    ws, jobs = batch_jobs_on_device(args.jobs)
    gen_s = time.perf_counter() - t0
    k = max(1, min(args.steps, args.batch_steps))
    b, p, same, _, _ = batch_compare(ws, jobs, k, 1, rank, flush, stream)
    return {"metric": BATCH_METRIC, "value": b, "unit": "job-iterations/s", "steps": k,
            "plain_form": {"value": p, "unit": "job-iterations/s",
                           "form": "one job at a time, one session each, fp64 terms"},
            "batched_over_plain": b / p, "jobs": len(jobs), "jobs_with_identical_hits_and_decisions": same,
            "input_generation_s": round(gen_s, 1)}


def run_batch(args):
    """--workload batch: one step = one Boruta iteration of all 64 jobs
    (boruta_batch_run, FP32 terms), against the plain form: the same jobs one
    at a time, one session each, FP64 terms."""
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
    t0 = time.perf_counter()
    ws, jobs = batch_jobs_on_device(args.jobs)
    gen_s = time.perf_counter() - t0
    stream = torch.cuda.current_stream()
    flush = torch.empty(512 << 20, dtype=torch.uint8, device="cuda")
    if dist:
        dist.barrier()
    clk_path = os.path.join(tempfile.gettempdir(), f"bench_clocks_{os.getpid()}.csv")
    proc, fh = start_clock_sampler(clk_path) if rank == 0 else (None, None)
    b, p, same, batched_ms, launched = batch_compare(ws, jobs, args.steps, args.warmup, rank, flush, stream,
                                                     args.graph)
    value, total_ms = combine_ranks(batched_ms, len(jobs) * args.steps, dist)
    clocks = stop_clock_sampler(proc, fh, clk_path, local) if rank == 0 else None

    # end to end: host inputs, upload + K iterations + readback
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
                       "graph_replay": bool(args.graph), "input_generation_s": gen_s},
            "plain_form": {"value": p, "unit": "job-iterations/s",
                           "form": "one job at a time, one session each, fp64 terms",
                           "jobs_with_identical_hits_and_decisions": same},
            "batched_over_plain": b / p,
            "roofline": None, "cpu_baseline": None,
            "e2e": {"value": len(jobs) * args.steps / e2e_s, "unit": "job-iterations/s",
                    "h2d_bytes_per_step": h2d / args.steps, "d2h_bytes_per_step": d2h / args.steps,
                    "note": "boruta_fit_batch with host inputs: setup, upload, K iterations, readback"},
            "gpu_launches": launched,
            "clocks": clocks,
        }
        print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gpu", choices=["gpu", "reference"])
    ap.add_argument("--precision", type=int, default=1, help="0 = FP64 terms, 1 = FP32 terms")
    ap.add_argument("--workload", default=DEFAULT_WORKLOAD, choices=list(WORKLOADS) + ["batch"],
                    help="multiclass: N=1e6 p=500 (default); binary: N=1e5 p=1000; snp: N=2e4 p=2e4; "
                         "small: N=1000 p=50; batch: 64 uneven jobs, batched vs plain form")
    ap.add_argument("--ref-trees", type=int, default=0, help="reference arm: trees timed (0 = one per core)")
    ap.add_argument("--cpu-trees", type=int, default=None, help="cpu_baseline: trees timed (default one per worker)")
    ap.add_argument("--no-cpu", action="store_true", help="skip the CPU oracle baseline")
    ap.add_argument("--no-other", action="store_true", help="skip timing the other precision form")
    ap.add_argument("--no-batch", action="store_true", help="skip the 64-job batched leg")
    ap.add_argument("--other-steps", type=int, default=5, help="iterations timed in the other precision form")
    ap.add_argument("--e2e-steps", type=int, default=5, help="iterations of the end-to-end boruta_fit")
    ap.add_argument("--batch-steps", type=int, default=3, help="iterations of the batched leg")
    ap.add_argument("--trees", type=int, default=None, help="fewer trees (profiling captures only)")
    ap.add_argument("--autotune", action="store_true", help="time the histogram tile shapes on the first step")
    ap.add_argument("--jobs", type=int, default=64, help="batch workload: number of jobs")
    ap.add_argument("--graph", action="store_true", help="batch workload: replay each job's iterations as CUDA graphs")
    args = ap.parse_args()
    # up to 64 job streams in the batched legs: more hardware work queues
    # than the default 8 (read when the CUDA context is created)
    os.environ.setdefault("CUDA_DEVICE_MAX_CONNECTIONS", "32")
    if args.impl == "reference":
        run_reference(args)
    elif args.workload == "batch":
        run_batch(args)
    else:
        run_gpu(args)


if __name__ == "__main__":
    main()
