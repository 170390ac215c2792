"""CPU oracle for GPU Boruta -- TEST INFRASTRUCTURE ONLY.

Plain C (``oracle/*.c``) loaded through ctypes.  Only the test suite, the
smoke check and the benchmark's ``cpu_baseline`` leg may import this
package; the product path (``paper_2605_09950_gb300``) never does, and the
two share no code.  The C sources cite the paper's algorithms they follow
(Alg. 1 Boruta loop, Alg. 2 impurity importance, Alg. 3 permutation
importance).
"""
from __future__ import annotations

import ctypes as ct
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = ["rng.c", "exact.c", "forest.c", "boruta.c"]
_LIB_PATH = os.path.join(_HERE, "_build", "liboracle.so")
_lock = threading.Lock()
_lib = None

MAX_CLASSES = 8
CLASSIFICATION, REGRESSION = 0, 1
TREEIMP, PERMUT = 0, 2


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (no FMA contraction, no fast-math)."""
    srcs = [os.path.join(_HERE, s) for s in _SRC] + [os.path.join(_HERE, h) for h in ("oracle.h", "exact.h")]
    newest = max(os.path.getmtime(s) for s in srcs)
    if not force and os.path.exists(_LIB_PATH) and os.path.getmtime(_LIB_PATH) >= newest:
        return _LIB_PATH
    os.makedirs(os.path.dirname(_LIB_PATH), exist_ok=True)
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=gnu11", "-fPIC", "-shared", "-ffp-contract=off", "-fno-fast-math",
           "-Wall", "-o", tmp] + [os.path.join(_HERE, s) for s in _SRC] + ["-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


class Problem(ct.Structure):
    _fields_ = [
        ("X", ct.c_void_p), ("ld", ct.c_int64), ("ycls", ct.c_void_p), ("yreg", ct.c_void_p),
        ("N", ct.c_int64), ("p", ct.c_int64), ("task", ct.c_int), ("n_classes", ct.c_int),
        ("n_trees", ct.c_int), ("max_depth", ct.c_int), ("mtry", ct.c_int), ("n_bins", ct.c_int),
        ("max_iter", ct.c_int), ("alpha", ct.c_double), ("seed", ct.c_uint64), ("job", ct.c_uint32),
        ("stat", ct.c_int), ("kl_eps", ct.c_double), ("tie_break", ct.c_int), ("permut_form", ct.c_int),
    ]


NODE_DTYPE = np.dtype([
    ("heap", "<u8"), ("depth", "<i4"), ("feature", "<i4"), ("bin", "<i4"), ("n_rows", "<u4"),
    ("n", "<u8"), ("stat", "<i8", (MAX_CLASSES,)), ("delta", "<f8"),
])


def lib():
    global _lib
    with _lock:
        if _lib is None:
            path = build()
            L = ct.CDLL(path)
            P = ct.POINTER
            vp = ct.c_void_p
            L.orc_philox4x32_10.argtypes = [vp, vp, vp]
            L.orc_fmix32.argtypes = [ct.c_uint32]
            L.orc_fmix32.restype = ct.c_uint32
            L.orc_perm.argtypes = [ct.c_uint64, ct.c_uint64, ct.c_uint32, ct.c_uint32, ct.c_uint32,
                                   vp, vp, ct.c_int64]
            L.orc_bootstrap.argtypes = [ct.c_uint64, ct.c_uint32, ct.c_int, ct.c_int, ct.c_int64, vp]
            L.orc_mtry.argtypes = [ct.c_uint64, ct.c_uint32, ct.c_int, ct.c_int, ct.c_uint32,
                                   ct.c_int64, ct.c_int, vp]
            L.orc_default_mtry.argtypes = [ct.c_int, ct.c_int64]
            L.orc_default_mtry.restype = ct.c_int64
            L.orc_shadow_count.argtypes = [ct.c_int64]
            L.orc_shadow_count.restype = ct.c_int64
            L.orc_shadow.argtypes = [P(Problem), ct.c_int, vp, ct.c_int64, vp]
            L.orc_permut_table.argtypes = [P(Problem), ct.c_int, vp]
            L.orc_cmp_products.argtypes = [vp, vp, vp, vp]
            L.orc_cmp_products.restype = ct.c_int
            L.orc_u256_to_double.argtypes = [vp]
            L.orc_u256_to_double.restype = ct.c_double
            L.orc_exact_sum.argtypes = [vp, ct.c_int64]
            L.orc_exact_sum.restype = ct.c_double
            L.orc_binom_tails.argtypes = [ct.c_int, ct.c_int, P(ct.c_double), P(ct.c_double), vp, vp]
            L.orc_node_split.argtypes = [ct.c_int, ct.c_int, ct.c_int, ct.c_int64, ct.c_int64, vp, vp,
                                         vp, vp, vp, ct.c_int, P(ct.c_int32), P(ct.c_int32),
                                         P(ct.c_double)]
            L.orc_node_split.restype = ct.c_int
            L.orc_tree.argtypes = [P(Problem), ct.c_int, vp, ct.c_int64, vp, ct.c_int, vp, ct.c_int64,
                                   P(ct.c_int64), vp, vp]
            L.orc_tree.restype = ct.c_int
            L.orc_forest_permut.argtypes = [P(Problem), ct.c_int, vp, ct.c_int64, vp, vp]
            L.orc_forest_permut.restype = ct.c_int
            L.orc_rank.argtypes = [ct.c_int64, ct.c_int32, vp, vp, vp]
            L.orc_select_median.argtypes = [ct.c_int, ct.c_int64, ct.c_int32, vp, vp, vp, vp, P(ct.c_double), vp]
            L.orc_decide.argtypes = [ct.c_int, ct.c_double, ct.c_int64, vp, vp]
            L.orc_iteration.argtypes = [P(Problem), ct.c_int, vp, vp, vp, P(ct.c_double), vp, vp,
                                        P(ct.c_int64)]
            L.orc_iteration.restype = ct.c_int
            L.orc_boruta.argtypes = [P(Problem), vp, vp, vp, vp, P(ct.c_int32)]
            L.orc_boruta.restype = ct.c_int
            _lib = L
    return _lib


def _ptr(a):
    return None if a is None else a.ctypes.data


# ---------------- random streams ----------------

def philox(ctr, key):
    c = np.asarray(ctr, dtype=np.uint32)
    k = np.asarray(key, dtype=np.uint32)
    out = np.zeros(4, dtype=np.uint32)
    lib().orc_philox4x32_10(_ptr(c), _ptr(k), _ptr(out))
    return out


def fmix32(x: int) -> int:
    return int(lib().orc_fmix32(x))


def perm(n, seed, w1, w2, w3, idx):
    idx = np.ascontiguousarray(idx, dtype=np.uint64)
    out = np.zeros_like(idx)
    lib().orc_perm(n, seed, w1, w2, w3, _ptr(idx), _ptr(out), idx.size)
    return out


def bootstrap(seed, job, t, tree, N):
    out = np.zeros(N, dtype=np.uint32)
    lib().orc_bootstrap(seed, job, t, tree, N, _ptr(out))
    return out


def mtry_features(seed, job, t, tree, heap, p_aug, mtry):
    out = np.zeros(mtry, dtype=np.uint32)
    lib().orc_mtry(seed, job, t, tree, heap, p_aug, mtry, _ptr(out))
    return out


def default_mtry(task, p_aug):
    return int(lib().orc_default_mtry(task, p_aug))


def shadow_count(p_live):
    return int(lib().orc_shadow_count(p_live))


# ---------------- exact arithmetic ----------------

def _limbs(v: int, n=4):
    return np.array([(v >> (64 * i)) & 0xFFFFFFFFFFFFFFFF for i in range(n)], dtype=np.uint64)


def cmp_products(a1: int, b1: int, a2: int, b2: int) -> int:
    arrs = [_limbs(v) for v in (a1, b1, a2, b2)]  # keep the buffers alive across the call
    return int(lib().orc_cmp_products(*[_ptr(a) for a in arrs]))


def u256_to_double(v: int) -> float:
    a = _limbs(v)
    return float(lib().orc_u256_to_double(_ptr(a)))


def exact_sum(x) -> float:
    x = np.ascontiguousarray(x, dtype=np.float64)
    return float(lib().orc_exact_sum(_ptr(x), x.size))


def binom_tails(t: int, h: int):
    pa, pr = ct.c_double(), ct.c_double()
    up = np.zeros(2, np.uint64)
    lo = np.zeros(2, np.uint64)
    lib().orc_binom_tails(t, h, ct.byref(pa), ct.byref(pr), _ptr(up), _ptr(lo))
    return pa.value, pr.value, int(up[0]) | (int(up[1]) << 64), int(lo[0]) | (int(lo[1]) << 64)


def decide(t: int, alpha: float, hits, state):
    """Alg. 1's test after iteration t: returns the updated state."""
    hits = np.ascontiguousarray(hits, dtype=np.int32)
    st = np.array(state, dtype=np.int8)
    lib().orc_decide(t, alpha, st.size, _ptr(hits), _ptr(st))
    return st


def rank(decision, imp_history, iterations):
    """Alg. 1's final ranking of a finished run (see oracle.h)."""
    dec = np.ascontiguousarray(decision, dtype=np.int8)
    hist = np.ascontiguousarray(imp_history, dtype=np.float64)
    out = np.zeros(dec.size, np.int32)
    lib().orc_rank(dec.size, iterations, _ptr(dec), _ptr(hist), _ptr(out))
    return out


def select_median(runs):
    """Median selection over runs with different seeds (see oracle.h).
    runs: list of run dicts (imp_history [max_iter, p], shadow_max,
    iterations).  Returns (median importance [p], median shadow, selected)."""
    hist = np.ascontiguousarray(np.stack([r["imp_history"] for r in runs]), dtype=np.float64)
    smax = np.ascontiguousarray(np.stack([r["shadow_max"] for r in runs]), dtype=np.float64)
    its = np.array([r["iterations"] for r in runs], dtype=np.int32)
    n, T, p = hist.shape
    med = np.zeros(p)
    sel = np.zeros(p, np.int8)
    ms = ct.c_double()
    lib().orc_select_median(n, p, T, _ptr(its), _ptr(hist), _ptr(smax), _ptr(med), ct.byref(ms), _ptr(sel))
    return med, ms.value, sel


def node_split(task, n_classes, n_bins, bins, w, y, feats):
    """Best split of an explicit node.  bins: (nrows, nf) uint8."""
    bins = np.ascontiguousarray(bins, dtype=np.uint8)
    w = np.ascontiguousarray(w, dtype=np.uint32)
    feats = np.ascontiguousarray(feats, dtype=np.int32)
    ycls = np.ascontiguousarray(y, dtype=np.uint8) if (task & 1) == 0 else None
    yreg = np.ascontiguousarray(y, dtype=np.int64) if (task & 1) == 1 else None
    f, b, d = ct.c_int32(-1), ct.c_int32(-1), ct.c_double(0.0)
    rc = lib().orc_node_split(task, n_classes, n_bins, bins.shape[0], bins.shape[1], _ptr(bins),
                              _ptr(w), _ptr(ycls), _ptr(yreg), _ptr(feats), feats.size,
                              ct.byref(f), ct.byref(b), ct.byref(d))
    if rc < 0:
        raise OverflowError("oracle: 256-bit bound exceeded")
    return (f.value, b.value, d.value) if rc == 1 else None


# ---------------- Boruta ----------------

class BorutaProblem:
    """Holds the arrays of one problem and its C description.

    X: (p, ld) uint8 array, column j = X[j, :N] (column-major bins).
    y: uint8 labels (classification) or int64 fixed point at 2^-20 (regression).
    """

    def __init__(self, X, y, task, n_trees, max_depth, n_bins, max_iter, alpha=0.01, seed=0,
                 mtry=0, n_classes=0, job=0, stat=0, kl_eps=1e-7, tie_break=0, permut_form=0, N=None):
        self.X = np.ascontiguousarray(X, dtype=np.uint8)
        self.N = int(N if N is not None else self.X.shape[1])
        self.p = int(self.X.shape[0])
        self.task = int(task)
        if (task & 1) == CLASSIFICATION:
            self.y = np.ascontiguousarray(y, dtype=np.uint8)
            if n_classes == 0:
                n_classes = int(self.y[: self.N].max()) + 1
        else:
            self.y = np.ascontiguousarray(y, dtype=np.int64)
            n_classes = 1
        self.n_classes = int(n_classes)
        self.c = Problem(
            X=self.X.ctypes.data, ld=self.X.shape[1],
            ycls=self.y.ctypes.data if (task & 1) == 0 else None,
            yreg=self.y.ctypes.data if (task & 1) == 1 else None,
            N=self.N, p=self.p, task=self.task, n_classes=self.n_classes, n_trees=n_trees,
            max_depth=max_depth, mtry=mtry, n_bins=n_bins, max_iter=max_iter, alpha=alpha,
            seed=seed, job=job, stat=stat, kl_eps=kl_eps, tie_break=tie_break, permut_form=permut_form)

    @property
    def n_trees(self):
        return self.c.n_trees

    def live(self, state):
        return np.flatnonzero(np.asarray(state) >= 0).astype(np.int32)

    def shadow(self, t, live):
        live = np.ascontiguousarray(live, dtype=np.int32)
        n_sha = shadow_count(live.size)
        out = np.zeros((n_sha, self.N), dtype=np.uint8)
        lib().orc_shadow(ct.byref(self.c), t, _ptr(live), live.size, _ptr(out))
        return out

    def permut_table(self, t):
        out = np.zeros(self.N, dtype=np.uint64)
        lib().orc_permut_table(ct.byref(self.c), t, _ptr(out))
        return out

    def tree(self, t, live, Xsha, tree, nodes=True, treeimp=False, permut=False):
        live = np.ascontiguousarray(live, dtype=np.int32)
        Xsha = np.ascontiguousarray(Xsha, dtype=np.uint8)
        p_aug = live.size + Xsha.shape[0]
        cap = 2 * self.N + 1
        nd = np.zeros(cap, dtype=NODE_DTYPE) if nodes else None
        ti = np.zeros(p_aug) if treeimp else None
        pm = np.zeros(p_aug) if permut else None
        nn = ct.c_int64(0)
        rc = lib().orc_tree(ct.byref(self.c), t, _ptr(live), live.size, _ptr(Xsha), tree, _ptr(nd),
                            cap, ct.byref(nn), _ptr(ti), _ptr(pm))
        if rc:
            raise RuntimeError(f"oracle tree failed ({rc})")
        return (nd[: nn.value] if nodes else None), ti, pm

    def forest_permut(self, t, live, Xsha):
        """Alg. 3 as printed (every row, the forest's prediction): one
        importance per augmented column."""
        live = np.ascontiguousarray(live, dtype=np.int32)
        Xsha = np.ascontiguousarray(Xsha, dtype=np.uint8)
        imp = np.zeros(live.size + Xsha.shape[0])
        rc = lib().orc_forest_permut(ct.byref(self.c), t, _ptr(live), live.size, _ptr(Xsha), _ptr(imp))
        if rc:
            raise RuntimeError(f"oracle forest failed ({rc})")
        return imp

    def iteration(self, t, state, hits):
        """One Alg. 1 loop body; returns dict with the updated state and dumps."""
        state = np.array(state, dtype=np.int8)
        hits = np.array(hits, dtype=np.int32)
        p_live = int((state >= 0).sum())
        p_aug = p_live + shadow_count(p_live)
        hist = np.zeros(self.p)
        smax = ct.c_double()
        rows = 1 if (self.task & PERMUT and self.c.permut_form == 1) else self.n_trees
        imp = np.zeros((self.n_trees, p_aug))
        s = np.zeros(p_aug)
        pa = ct.c_int64()
        rc = lib().orc_iteration(ct.byref(self.c), t, _ptr(state), _ptr(hits), _ptr(hist),
                                 ct.byref(smax), _ptr(imp), _ptr(s), ct.byref(pa))
        if rc:
            raise RuntimeError(f"oracle iteration failed ({rc})")
        return dict(state=state, hits=hits, hist=hist, shadow_max=smax.value, imp=imp[:rows], s=s)

    def run(self):
        p, T = self.p, self.c.max_iter
        dec = np.zeros(p, np.int8)
        hits = np.zeros(p, np.int32)
        hist = np.zeros((T, p))
        smax = np.zeros(T)
        it = ct.c_int32()
        rc = lib().orc_boruta(ct.byref(self.c), _ptr(dec), _ptr(hits), _ptr(hist), _ptr(smax),
                              ct.byref(it))
        if rc:
            raise ValueError(f"oracle rejected the problem ({rc})")
        return dict(decision=dec, hits=hits, imp_history=hist, shadow_max=smax, iterations=it.value)
