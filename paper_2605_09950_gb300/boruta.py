"""Thin Python binding of the C ABI in include/boruta.h (ctypes).

Argument marshalling only: every step of the Boruta iteration runs in the
CUDA kernels of libboruta_gb300.so.  PyTorch supplies device memory and the
current stream.  There is no CPU fallback: if the library is missing this
module raises.
"""
from __future__ import annotations

import ctypes as ct
import os

import numpy as np

_LIB_PATH = os.path.join(os.path.dirname(os.path.abspath(__file__)), "_build", "libboruta_gb300.so")
_lib = None

CLASSIFICATION, REGRESSION = 0, 1
TREEIMP, PERMUT = 0, 2
DUMP_SHADOW, DUMP_BOOT, DUMP_IMP, DUMP_STAT, DUMP_NODES, DUMP_TREE_PTR, DUMP_LIVE, DUMP_LEVELS = range(1, 9)
STATUS = {0: "BORUTA_OK", -1: "BORUTA_EINVAL", -2: "BORUTA_EOVERFLOW", -3: "BORUTA_ETIMEOUT",
          -4: "BORUTA_ECUDA", -5: "BORUTA_ENOMEM"}

# the exported symbols of include/boruta.h
EXPORTS = [
    "boruta_default_opts", "boruta_fit", "boruta_fit_batch", "boruta_batch_create", "boruta_batch_step",
    "boruta_batch_run",
    "boruta_batch_read", "boruta_batch_destroy", "boruta_session_create", "boruta_session_step",
    "boruta_session_read", "boruta_session_write", "boruta_session_dump",
    "boruta_session_kernel_stats", "boruta_session_importance_stats", "boruta_session_tuning",
    "boruta_session_tuning_levels", "boruta_session_kernel_launches", "boruta_batch_kernel_launches",
    "boruta_session_destroy",
    "boruta_philox", "boruta_perm",
    "boruta_u256_to_double", "boruta_binom_tails", "boruta_binom_tails_noalloc", "boruta_quantise",
    "boruta_last_error", "boruta_rank", "boruta_select_median", "boruta_fit_seeds",
]


class BorutaError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"{STATUS.get(code, code)}: {msg}")
        self.code = code


class Opts(ct.Structure):
    _fields_ = [("stat", ct.c_int), ("precision", ct.c_int), ("tie_break", ct.c_int),
                ("n_classes", ct.c_int), ("kl_eps", ct.c_double), ("stream", ct.c_void_p),
                ("job", ct.c_uint32), ("host_inputs", ct.c_int), ("graph", ct.c_int), ("split_path", ct.c_int),
                ("chunk_nodes", ct.c_int), ("permut_form", ct.c_int), ("forest_rows", ct.c_int),
                ("autotune", ct.c_int), ("band_launch", ct.c_int)]


class Job(ct.Structure):
    _fields_ = [("X", ct.c_void_p), ("ld", ct.c_int64), ("y", ct.c_void_p), ("N", ct.c_int64), ("p", ct.c_int64),
                ("task", ct.c_int), ("n_trees", ct.c_int), ("max_depth", ct.c_int), ("mtry", ct.c_int),
                ("n_bins", ct.c_int), ("max_iter", ct.c_int), ("alpha", ct.c_double), ("seed", ct.c_uint64),
                ("n_classes", ct.c_int)]


class Result(ct.Structure):
    _fields_ = [("decision", ct.c_void_p), ("hits", ct.c_void_p), ("imp_history", ct.c_void_p),
                ("shadow_max", ct.c_void_p), ("iterations", ct.c_int32)]


NODE_DTYPE = np.dtype([
    ("heap", "<u8"), ("depth", "<i4"), ("feature", "<i4"), ("bin", "<i4"), ("n_rows", "<u4"),
    ("n", "<u8"), ("stat", "<i8", (8,)), ("delta", "<f8"),
])


def library_path() -> str:
    return _LIB_PATH


def lib():
    """Loads libboruta_gb300.so; raises if it has not been built."""
    global _lib
    if _lib is None:
        if not os.path.exists(_LIB_PATH):
            raise RuntimeError(f"{_LIB_PATH} is missing: build it with paper_2605_09950_gb300.build.build()")
        L = ct.CDLL(_LIB_PATH)
        vp, i64, i32 = ct.c_void_p, ct.c_int64, ct.c_int
        fit_args = [vp, i64, vp, i64, i64, i32, i32, i32, i32, i32, i32, ct.c_double, ct.c_uint64,
                    ct.POINTER(Opts)]
        L.boruta_default_opts.argtypes = [ct.POINTER(Opts)]
        L.boruta_default_opts.restype = None
        L.boruta_fit.argtypes = fit_args + [ct.POINTER(Result)]
        L.boruta_fit_batch.argtypes = [i32, ct.POINTER(Job), ct.POINTER(Opts), ct.POINTER(Result)]
        L.boruta_session_create.argtypes = fit_args + [ct.POINTER(vp)]
        L.boruta_session_step.argtypes = [vp, ct.POINTER(ct.c_int32)]
        L.boruta_session_read.argtypes = [vp, vp, vp, vp, vp, ct.POINTER(ct.c_int32)]
        L.boruta_session_write.argtypes = [vp, vp, vp, vp, vp, ct.c_int32]
        L.boruta_session_dump.argtypes = [vp, i32, vp, i64, ct.POINTER(i64)]
        L.boruta_session_kernel_stats.argtypes = [vp, ct.POINTER(ct.c_double), ct.POINTER(ct.c_int32),
                                                  ct.POINTER(ct.c_double), ct.POINTER(ct.c_double),
                                                  ct.POINTER(ct.c_double)]
        L.boruta_session_importance_stats.argtypes = [vp, ct.POINTER(ct.c_double), ct.POINTER(ct.c_double)]
        L.boruta_session_tuning.argtypes = [vp, ct.c_int32, ct.POINTER(ct.c_int32), vp, vp, vp, vp,
                                            ct.POINTER(ct.c_int32)]
        L.boruta_session_tuning_levels.argtypes = [vp, ct.c_int32, ct.POINTER(ct.c_int32), vp, vp, vp]
        L.boruta_session_kernel_launches.argtypes = [vp, ct.POINTER(ct.c_int64)]
        L.boruta_batch_kernel_launches.argtypes = [vp, ct.POINTER(ct.c_int64)]
        L.boruta_session_destroy.argtypes = [vp]
        L.boruta_session_destroy.restype = None
        L.boruta_batch_create.argtypes = [ct.c_int, vp, vp, ct.POINTER(ct.c_void_p)]
        L.boruta_batch_step.argtypes = [vp, ct.POINTER(ct.c_int32)]
        L.boruta_batch_run.argtypes = [vp, ct.c_int, ct.POINTER(ct.c_int32)]
        L.boruta_batch_read.argtypes = [vp, ct.c_int, vp, vp, vp, vp, ct.POINTER(ct.c_int32)]
        L.boruta_batch_destroy.argtypes = [vp]
        L.boruta_batch_destroy.restype = None
        L.boruta_philox.argtypes = [vp, vp, vp, i64, vp]
        L.boruta_perm.argtypes = [ct.c_uint64, ct.c_uint64, ct.c_uint32, ct.c_uint32, ct.c_uint32, vp, vp,
                                  i64, vp]
        L.boruta_u256_to_double.argtypes = [vp, vp, i64, vp]
        L.boruta_binom_tails.argtypes = [vp, vp, vp, vp, i64, vp]
        L.boruta_binom_tails_noalloc.argtypes = [vp, vp, vp, vp, i64, vp]
        L.boruta_quantise.argtypes = [vp, i64, i64, i64, ct.c_int, vp, i64, vp]
        L.boruta_last_error.restype = ct.c_char_p
        L.boruta_rank.argtypes = [vp, vp, i64, ct.c_int32, vp]
        L.boruta_select_median.argtypes = [i32, i64, ct.c_int32, vp, vp, vp, vp, ct.POINTER(ct.c_double), vp]
        L.boruta_fit_seeds.argtypes = [vp, i64, vp, i64, i64, i32, i32, i32, i32, i32, i32, ct.c_double, i32, vp,
                                       ct.POINTER(Opts), vp, vp, ct.POINTER(ct.c_double), vp]
        for name in EXPORTS:
            if name not in ("boruta_default_opts", "boruta_session_destroy", "boruta_batch_destroy",
                            "boruta_last_error"):
                getattr(L, name).restype = ct.c_int
        _lib = L
    return _lib


def _check(rc):
    if rc != 0:
        raise BorutaError(rc, lib().boruta_last_error().decode())


def _stream():
    import torch
    return ct.c_void_p(torch.cuda.current_stream().cuda_stream)


def make_opts(stat=0, precision=0, tie_break=0, n_classes=0, kl_eps=1e-7, job=0, host_inputs=0,
              graph=0, split_path=0, chunk_nodes=0, permut_form=0, forest_rows=0, autotune=0,
              band_launch=0, stream=None) -> Opts:
    o = Opts()
    lib().boruta_default_opts(ct.byref(o))
    o.stat, o.precision, o.tie_break, o.n_classes = stat, precision, tie_break, n_classes
    o.kl_eps, o.job, o.host_inputs, o.graph, o.split_path = kl_eps, job, host_inputs, graph, split_path
    o.chunk_nodes, o.permut_form, o.forest_rows, o.autotune = chunk_nodes, permut_form, forest_rows, autotune
    o.band_launch = band_launch
    o.stream = stream if stream is not None else (None if host_inputs else _stream())
    return o


def _xy(X, y, N, host_inputs):
    """(pointer, ld, N, p) for X given as a (p, ld) uint8 tensor / array."""
    if host_inputs:
        Xa = np.ascontiguousarray(X, dtype=np.uint8)
        ya = np.ascontiguousarray(y)
        return Xa.ctypes.data, Xa.shape[1], (Xa.shape[1] if N is None else N), Xa.shape[0], ya.ctypes.data, (Xa, ya)
    import torch
    assert X.is_cuda and X.dtype == torch.uint8 and X.is_contiguous() and X.dim() == 2
    assert y.is_cuda and y.is_contiguous()
    return X.data_ptr(), X.shape[1], (X.shape[1] if N is None else N), X.shape[0], y.data_ptr(), (X, y)


def boruta_fit(X, y, task, n_trees, max_depth, mtry, n_bins, max_iter, alpha, seed, N=None, **opts):
    """Alg. 1 on one problem.  X: (p, ld) uint8 (CUDA tensor, or numpy with
    host_inputs=1), column j = X[j, :N]; y: uint8 labels or int64 fixed point."""
    host = opts.get("host_inputs", 0)
    xp, ld, N, p, yp, keep = _xy(X, y, N, host)
    o = make_opts(**opts)
    dec = np.zeros(p, np.int8)
    hits = np.zeros(p, np.int32)
    hist = np.zeros((max_iter, p))
    smax = np.zeros(max_iter)
    res = Result(dec.ctypes.data, hits.ctypes.data, hist.ctypes.data, smax.ctypes.data, 0)
    _check(lib().boruta_fit(xp, ld, yp, N, p, task, n_trees, max_depth, mtry, n_bins, max_iter, alpha,
                            seed, ct.byref(o), ct.byref(res)))
    del keep
    return dict(decision=dec, hits=hits, imp_history=hist, shadow_max=smax, iterations=res.iterations)


def boruta_fit_batch(jobs, **opts):
    """Many independent problems at once.  jobs: list of dicts with X, y and
    the boruta_fit parameters (task, n_trees, max_depth, mtry, n_bins,
    max_iter, alpha, seed, n_classes, N); X/y as for boruta_fit."""
    host = opts.get("host_inputs", 0)
    o = make_opts(**opts)
    arr = (Job * max(1, len(jobs)))()
    res = (Result * max(1, len(jobs)))()
    keep, outs = [], []
    for j, jb in enumerate(jobs):
        xp, ld, N, p, yp, k = _xy(jb["X"], jb["y"], jb.get("N"), host)
        keep.append(k)
        arr[j] = Job(xp, ld, yp, N, p, jb["task"], jb["n_trees"], jb["max_depth"], jb.get("mtry", 0), jb["n_bins"],
                     jb["max_iter"], jb.get("alpha", 0.01), jb.get("seed", 0), jb.get("n_classes", 0))
        out = dict(decision=np.zeros(p, np.int8), hits=np.zeros(p, np.int32),
                   imp_history=np.zeros((jb["max_iter"], p)), shadow_max=np.zeros(jb["max_iter"]))
        outs.append(out)
        res[j] = Result(out["decision"].ctypes.data, out["hits"].ctypes.data, out["imp_history"].ctypes.data,
                        out["shadow_max"].ctypes.data, 0)
    _check(lib().boruta_fit_batch(len(jobs), arr, ct.byref(o), res))
    for j, out in enumerate(outs):
        out["iterations"] = res[j].iterations
    del keep
    return outs


def _jobs_struct(jobs, host):
    arr = (Job * max(1, len(jobs)))()
    keep = []
    for j, jb in enumerate(jobs):
        xp, ld, N, p, yp, k = _xy(jb["X"], jb["y"], jb.get("N"), host)
        keep.append(k)
        arr[j] = Job(xp, ld, yp, N, p, jb["task"], jb["n_trees"], jb["max_depth"], jb.get("mtry", 0), jb["n_bins"],
                     jb["max_iter"], jb.get("alpha", 0.01), jb.get("seed", 0), jb.get("n_classes", 0))
    return arr, keep


class Batch:
    """Step-wise batch (boruta_batch_*): one lockstep iteration of every
    unfinished job per step().  jobs as for boruta_fit_batch (device X/y)."""

    def __init__(self, jobs, **opts):
        self._arr, self._keep = _jobs_struct(jobs, 0)
        self._opts = make_opts(**opts)
        self._shapes = [(int(self._arr[j].p), int(jb["max_iter"])) for j, jb in enumerate(jobs)]
        h = ct.c_void_p()
        _check(lib().boruta_batch_create(len(jobs), self._arr, ct.byref(self._opts), ct.byref(h)))
        self._h = h

    def step(self) -> int:
        running = ct.c_int32()
        _check(lib().boruta_batch_step(self._h, ct.byref(running)))
        return running.value

    def run(self, iterations) -> int:
        """Up to `iterations` more iterations per job, jobs advancing independently."""
        running = ct.c_int32()
        _check(lib().boruta_batch_run(self._h, iterations, ct.byref(running)))
        return running.value

    def kernel_launches(self) -> int:
        """Kernels all jobs have launched since the batch was created."""
        n = ct.c_int64()
        _check(lib().boruta_batch_kernel_launches(self._h, ct.byref(n)))
        return n.value

    def read(self, j):
        p, max_iter = self._shapes[j]
        out = dict(decision=np.zeros(p, np.int8), hits=np.zeros(p, np.int32),
                   imp_history=np.zeros((max_iter, p)), shadow_max=np.zeros(max_iter))
        t = ct.c_int32()
        _check(lib().boruta_batch_read(self._h, j, out["decision"].ctypes.data, out["hits"].ctypes.data,
                                       out["imp_history"].ctypes.data, out["shadow_max"].ctypes.data,
                                       ct.byref(t)))
        out["iterations"] = t.value
        return out

    def close(self):
        if getattr(self, "_h", None):
            lib().boruta_batch_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Session:
    """Step-wise Boruta (boruta_session_*): one iteration per step()."""

    def __init__(self, X, y, task, n_trees, max_depth, mtry, n_bins, max_iter, alpha, seed, N=None, **opts):
        host = opts.get("host_inputs", 0)
        xp, ld, N, p, yp, self._keep = _xy(X, y, N, host)
        self.p, self.N, self.max_iter, self.n_trees = p, N, max_iter, n_trees
        self._opts = make_opts(**opts)
        h = ct.c_void_p()
        _check(lib().boruta_session_create(xp, ld, yp, N, p, task, n_trees, max_depth, mtry, n_bins,
                                           max_iter, alpha, seed, ct.byref(self._opts), ct.byref(h)))
        self._h = h

    def step(self) -> int:
        und = ct.c_int32()
        _check(lib().boruta_session_step(self._h, ct.byref(und)))
        return und.value

    def read(self):
        dec = np.zeros(self.p, np.int8)
        hits = np.zeros(self.p, np.int32)
        hist = np.zeros((self.max_iter, self.p))
        smax = np.zeros(self.max_iter)
        t = ct.c_int32()
        _check(lib().boruta_session_read(self._h, dec.ctypes.data, hits.ctypes.data, hist.ctypes.data,
                                         smax.ctypes.data, ct.byref(t)))
        return dict(decision=dec, hits=hits, imp_history=hist, shadow_max=smax, iterations=t.value)

    def write(self, state):
        dec = np.ascontiguousarray(state["decision"], np.int8)
        hits = np.ascontiguousarray(state["hits"], np.int32)
        hist = np.ascontiguousarray(state["imp_history"], np.float64)
        smax = np.ascontiguousarray(state["shadow_max"], np.float64)
        _check(lib().boruta_session_write(self._h, dec.ctypes.data, hits.ctypes.data, hist.ctypes.data,
                                          smax.ctypes.data, int(state["iterations"])))

    def dump(self, what, dtype):
        need = ct.c_int64()
        _check(lib().boruta_session_dump(self._h, what, None, 0, ct.byref(need)))
        buf = np.zeros(need.value, dtype=np.uint8)
        _check(lib().boruta_session_dump(self._h, what, buf.ctypes.data, buf.size, ct.byref(need)))
        return buf.view(dtype)

    def kernel_stats(self):
        hms, n, hb, sms, sb = ct.c_double(), ct.c_int32(), ct.c_double(), ct.c_double(), ct.c_double()
        _check(lib().boruta_session_kernel_stats(self._h, ct.byref(hms), ct.byref(n), ct.byref(hb), ct.byref(sms),
                                                 ct.byref(sb)))
        return dict(hist_ms=hms.value, launches=n.value, hist_bytes=hb.value, split_ms=sms.value,
                    split_bytes=sb.value)

    def tuning(self):
        """The autotuner's candidates: list of (group work, band bytes, per-band launch, ms)
        and the index kept; band bytes and launch are -1 for the per-level combination."""
        n, ch = ct.c_int32(), ct.c_int32()
        cap = 32
        gw = np.zeros(cap, np.uint32)
        bb = np.zeros(cap, np.int64)
        bl = np.zeros(cap, np.int32)
        ms = np.zeros(cap)
        _check(lib().boruta_session_tuning(self._h, cap, ct.byref(n), gw.ctypes.data, bb.ctypes.data, bl.ctypes.data,
                                           ms.ctypes.data, ct.byref(ch)))
        k = min(n.value, cap)
        return [(int(gw[i]), int(bb[i]), int(bl[i]), float(ms[i])) for i in range(k)], ch.value

    def tuning_levels(self):
        """Per tree level: the band bytes and launch mode in use, and the
        autotuner's split-stage ms of that level in each candidate run
        (array [candidates, levels])."""
        n_tried = len(self.tuning()[0])
        cap = 64
        nl = ct.c_int32()
        bb = np.zeros(cap, np.int64)
        bl = np.zeros(cap, np.int32)
        lm = np.zeros((max(n_tried, 1), cap))
        _check(lib().boruta_session_tuning_levels(self._h, cap, ct.byref(nl), bb.ctypes.data, bl.ctypes.data,
                                                  lm.ctypes.data))
        k = min(nl.value, cap)
        return bb[:k].tolist(), bl[:k].tolist(), lm[:n_tried, :k]

    def kernel_launches(self) -> int:
        """Kernels the last step launched."""
        n = ct.c_int64()
        _check(lib().boruta_session_kernel_launches(self._h, ct.byref(n)))
        return n.value

    def importance_stats(self):
        ms, visits = ct.c_double(), ct.c_double()
        _check(lib().boruta_session_importance_stats(self._h, ct.byref(ms), ct.byref(visits)))
        return dict(ms=ms.value, node_visits=visits.value)

    def close(self):
        if getattr(self, "_h", None):
            lib().boruta_session_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# ---------------- device primitives (torch CUDA tensors) ----------------

def boruta_philox(ctr, key):
    import torch
    out = torch.empty_like(ctr)
    _check(lib().boruta_philox(ctr.data_ptr(), key.data_ptr(), out.data_ptr(), ctr.numel() // 4, _stream()))
    return out


def boruta_perm(n, seed, w1, w2, w3, idx):
    import torch
    out = torch.empty_like(idx)
    _check(lib().boruta_perm(n, seed, w1, w2, w3, idx.data_ptr(), out.data_ptr(), idx.numel(), _stream()))
    return out


def boruta_u256_to_double(v):
    import torch
    out = torch.empty(v.numel() // 4, dtype=torch.float64, device=v.device)
    _check(lib().boruta_u256_to_double(v.data_ptr(), out.data_ptr(), out.numel(), _stream()))
    return out


def boruta_binom_tails(t, h):
    import torch
    pa = torch.empty(t.numel(), dtype=torch.float64, device=t.device)
    pr = torch.empty_like(pa)
    _check(lib().boruta_binom_tails(t.data_ptr(), h.data_ptr(), pa.data_ptr(), pr.data_ptr(), t.numel(),
                                    _stream()))
    return pa, pr


def boruta_binom_tails_noalloc(t, h, p_acc, p_rej):
    """Same as boruta_binom_tails, writing into caller-provided tensors and
    allocating nothing on the device (fixed table inside the library)."""
    _check(lib().boruta_binom_tails_noalloc(t.data_ptr(), h.data_ptr(), p_acc.data_ptr(), p_rej.data_ptr(),
                                            t.numel(), _stream()))
    return p_acc, p_rej


def boruta_quantise(F, n_bins, N=None):
    """Quantile bins of float features on the GPU.  F: (p, ld) float32 CUDA
    tensor, column j = F[j, :N].  Returns a (p, round16(N)) uint8 tensor,
    zero past N (the layout boruta_fit takes)."""
    import torch

    if not (F.is_cuda and F.dtype == torch.float32 and F.dim() == 2 and F.stride(1) == 1):
        raise ValueError("F must be a row-contiguous (p, ld) float32 CUDA tensor")
    p, ld = F.shape
    N = ld if N is None else N
    out = torch.zeros((p, (N + 15) // 16 * 16), dtype=torch.uint8, device=F.device)
    _check(lib().boruta_quantise(F.data_ptr(), F.stride(0), N, p, n_bins, out.data_ptr(), out.stride(0),
                                 _stream()))
    return out



def boruta_rank(decision, imp_history, iterations):
    """Alg. 1's final ranking of a finished run (host arrays)."""
    dec = np.ascontiguousarray(decision, dtype=np.int8)
    hist = np.ascontiguousarray(imp_history, dtype=np.float64)
    out = np.zeros(dec.size, np.int32)
    _check(lib().boruta_rank(dec.ctypes.data, hist.ctypes.data, dec.size, iterations, out.ctypes.data))
    return out


def boruta_select_median(runs):
    """Median selection over runs with different seeds.  runs: list of run
    dicts (imp_history [max_iter, p], shadow_max, iterations), as
    boruta_fit returns them.  Returns (median importance, median shadow,
    selected)."""
    hist = np.ascontiguousarray(np.stack([r["imp_history"] for r in runs]), dtype=np.float64)
    smax = np.ascontiguousarray(np.stack([r["shadow_max"] for r in runs]), dtype=np.float64)
    its = np.array([r["iterations"] for r in runs], dtype=np.int32)
    n, T, p = hist.shape
    med = np.zeros(p)
    sel = np.zeros(p, np.int8)
    ms = ct.c_double()
    _check(lib().boruta_select_median(n, p, T, its.ctypes.data, hist.ctypes.data, smax.ctypes.data, med.ctypes.data,
                                      ct.byref(ms), sel.ctypes.data))
    return med, ms.value, sel


def boruta_fit_seeds(X, y, task, n_trees, max_depth, mtry, n_bins, max_iter, alpha, seeds, N=None, **opts):
    """boruta_fit for each seed as jobs of one batch, then the median
    selection.  Returns (runs, median importance, median shadow, selected)."""
    host = opts.get("host_inputs", 0)
    xp, ld, N, p, yp, keep = _xy(X, y, N, host)
    o = make_opts(**opts)
    sd = np.ascontiguousarray(seeds, dtype=np.uint64)
    res = (Result * len(sd))()
    runs = []
    for r in range(len(sd)):
        run = dict(decision=np.zeros(p, np.int8), hits=np.zeros(p, np.int32),
                   imp_history=np.zeros((max_iter, p)), shadow_max=np.zeros(max_iter))
        res[r] = Result(run["decision"].ctypes.data, run["hits"].ctypes.data, run["imp_history"].ctypes.data,
                        run["shadow_max"].ctypes.data, 0)
        runs.append(run)
    med = np.zeros(p)
    sel = np.zeros(p, np.int8)
    ms = ct.c_double()
    _check(lib().boruta_fit_seeds(xp, ld, yp, N, p, task, n_trees, max_depth, mtry, n_bins, max_iter, alpha, len(sd),
                                  sd.ctypes.data, ct.byref(o), res, med.ctypes.data, ct.byref(ms), sel.ctypes.data))
    for r, run in enumerate(runs):
        run["iterations"] = res[r].iterations
    del keep
    return runs, med, ms.value, sel
