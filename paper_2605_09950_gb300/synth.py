"""Seeded synthetic workloads shaped like the paper's feature-selection data.

This module only *generates inputs*: it holds none of the Boruta / forest
arithmetic, and both the CUDA path and the CPU oracle consume its output.
The paper's public datasets (CT, NEWS, ENERGY, MADELON; Sec. 3.2) are not
available here, so these generators stand in for them; the first config
mirrors the planted-informative-feature design of the paper's synthetic
study (Sec. 3.1), the others scale it to the sizes the method targets.

Every workload returns the quantised matrix in the layout the library
expects: ``X`` of shape (p, ld) uint8, column j = ``X[j, :N]`` (column-major
bins, column stride ``ld`` = N rounded up to 16 bytes, padding zero).
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

CLASSIFICATION, REGRESSION = 0, 1
TREEIMP, PERMUT = 0, 2


@dataclasses.dataclass
class Workload:
    name: str
    X: np.ndarray            # (p, ld) uint8 bins
    y: np.ndarray            # uint8 labels or int64 fixed point (2^-20)
    N: int
    p: int
    task: int                # kind | importance
    n_classes: int
    n_bins: int
    n_trees: int
    max_depth: int
    max_iter: int
    alpha: float = 0.01
    seed: int = 0
    mtry: int = 0            # 0 = default, recomputed each iteration
    informative: np.ndarray | None = None

    @property
    def ld(self) -> int:
        return int(self.X.shape[1])

    def params(self) -> dict:
        return dict(task=self.task, n_trees=self.n_trees, max_depth=self.max_depth, mtry=self.mtry,
                    n_bins=self.n_bins, max_iter=self.max_iter, alpha=self.alpha, seed=self.seed,
                    n_classes=self.n_classes if (self.task & 1) == CLASSIFICATION else 0)


def pad16(n: int) -> int:
    return (n + 15) // 16 * 16


def quantise(F: np.ndarray, n_bins: int) -> np.ndarray:
    """float (p, N) -> uint8 (p, ld): bin = min(B-1, floor(B * rank / N)),
    rank = number of strictly smaller values in the column (ties share a bin)."""
    p, N = F.shape
    out = np.zeros((p, pad16(N)), dtype=np.uint8)
    idx = np.arange(N)
    for j in range(p):
        col = F[j]
        order = np.argsort(col, kind="stable")
        s = col[order]
        start = np.empty(N, dtype=bool)  # first position of each run of equal values
        start[0] = True
        np.not_equal(s[1:], s[:-1], out=start[1:])
        rank = np.empty(N, dtype=np.int64)
        rank[order] = np.maximum.accumulate(np.where(start, idx, 0))
        out[j, :N] = np.minimum(n_bins - 1, (n_bins * rank) // N).astype(np.uint8)
    return out


def _classif_gaussian(rng, N, p, n_inf, shift, n_lin=0, lin_sd=0.1):
    y = rng.integers(0, 2, size=N).astype(np.uint8)
    F = rng.standard_normal((p, N))
    pos = np.sort(rng.choice(p, size=n_inf + n_lin, replace=False))
    inf = pos[:n_inf] if n_lin == 0 else rng.permutation(pos)[:n_inf]
    inf = np.sort(inf)
    for j in inf:
        F[j] += shift * y
    if n_lin:
        lin = np.setdiff1d(pos, inf)
        weights = np.array([0.1, 0.2, 0.3, 0.4])
        for j in lin:
            src = rng.choice(inf, size=4, replace=False)
            F[j] = weights @ F[src] + rng.normal(0.0, lin_sd, size=N)
    return F, y, inf


def binary_small(N=1000, p=50, n_inf=10, seed=0, n_trees=100, max_depth=8, max_iter=20,
                 n_bins=64, importance=TREEIMP) -> Workload:
    """Binary classification, N=1000, p=50: 10 informative columns drawn
    from class-conditional Gaussians (mean shift 1.0), 40 N(0,1) noise,
    64 quantile bins; 100 trees, depth 8, Gini, TreeImp, 20 iterations."""
    rng = np.random.default_rng(np.random.PCG64(seed))
    F, y, inf = _classif_gaussian(rng, N, p, n_inf, 1.0)
    return Workload(f"binary_N{N}_p{p}", quantise(F, n_bins), y, N, p, CLASSIFICATION | importance, 2,
                    n_bins, n_trees, max_depth, max_iter, seed=seed, informative=inf)


def binary_wide(N=100_000, p=1000, n_inf=20, n_lin=40, seed=1, n_trees=500, max_depth=16,
                max_iter=100, n_bins=256, importance=PERMUT) -> Workload:
    """Binary classification, N=1e5, p=1000: 20 informative (shift 1.0),
    40 linear combinations of 4 informative columns with weights
    0.1/0.2/0.3/0.4 plus N(0, 0.1^2) (the multicollinearity pattern of the
    paper's Sec. 3.1.3), 940 noise; 256 bins; 500 trees, depth 16."""
    rng = np.random.default_rng(np.random.PCG64(seed))
    F, y, inf = _classif_gaussian(rng, N, p, n_inf, 1.0, n_lin=n_lin)
    return Workload(f"binary_N{N}_p{p}", quantise(F, n_bins), y, N, p, CLASSIFICATION | importance, 2,
                    n_bins, n_trees, max_depth, max_iter, seed=seed, informative=inf)


def snp_regression(N=20_000, p=20_000, n_add=30, n_pairs=10, seed=2, n_trees=256, max_depth=12,
                   max_iter=100, n_bins=256, importance=TREEIMP) -> Workload:
    """High-dimensional regression on SNP-like genotypes g ~ Bin(2, f_j),
    f_j ~ U(0.05, 0.5); y = additive effects + pairwise interactions +
    N(0,1), stored as int64 fixed point at 2^-20; bins are the genotypes."""
    rng = np.random.default_rng(np.random.PCG64(seed))
    f = rng.uniform(0.05, 0.5, size=p)
    G = (rng.random((p, N)) < f[:, None]).astype(np.uint8) + (rng.random((p, N)) < f[:, None]).astype(np.uint8)
    causal = rng.choice(p, size=n_add + 2 * n_pairs, replace=False)
    add, pair = causal[:n_add], causal[n_add:].reshape(n_pairs, 2)
    beta = rng.standard_normal(n_add)
    gamma = rng.standard_normal(n_pairs)
    yv = beta @ G[add].astype(np.float64)
    for (a, b), g in zip(pair, gamma):
        yv += g * G[a].astype(np.float64) * G[b]
    yv += rng.standard_normal(N)
    y_fx = np.rint(yv * 2.0**20).astype(np.int64)  # round half to even
    X = np.zeros((p, pad16(N)), dtype=np.uint8)
    X[:, :N] = G
    return Workload(f"snp_N{N}_p{p}", X, y_fx, N, p, REGRESSION | importance, 1, n_bins, n_trees,
                    max_depth, max_iter, seed=seed, informative=np.sort(causal))


def multiclass_toeplitz(N=1_000_000, p=500, block=10, n_inf=25, n_classes=5, seed=5, n_trees=300,
                        max_depth=20, max_iter=60, n_bins=256, importance=PERMUT, quantiser=None) -> Workload:
    """Large-N multiclass: p float32 columns in blocks of 10 with AR(1)
    correlation 0.8 inside each block (Toeplitz 0.8^|i-j|), 5 classes drawn
    from a softmax over the first column of the first 25 blocks.
    quantiser(F, n_bins) bins the float32 (p, N) features (default: the
    numpy statement of the rank rule, `quantise`)."""
    rng = np.random.default_rng(np.random.PCG64(seed))
    inf = np.arange(n_inf) * block
    W = rng.normal(0.0, 1.0 / math.sqrt(n_inf), size=(n_classes, n_inf))
    F = np.empty((p, N), dtype=np.float32)
    logits = np.zeros((n_classes, N))
    col = None
    for j in range(p):  # column by column: AR(1) inside each block
        z = rng.standard_normal(N)
        col = z if j % block == 0 else 0.8 * col + 0.6 * z
        if j % block == 0 and j // block < n_inf:
            logits += np.outer(W[:, j // block], col)
        F[j] = col
    X = (quantiser or quantise)(F, n_bins)
    del F
    logits -= logits.max(axis=0)
    P = np.exp(logits)
    P /= P.sum(axis=0)
    u = rng.random(N)
    y = (u[None, :] > np.cumsum(P, axis=0)).sum(axis=0).clip(0, n_classes - 1).astype(np.uint8)
    return Workload(f"multiclass_N{N}_p{p}", X, y, N, p, CLASSIFICATION | importance, n_classes, n_bins,
                    n_trees, max_depth, max_iter, seed=seed, informative=inf)


# the paper's synthetic regression study (Sec. 3.1): 1-based column names of
# the ten variables its target uses, and the five collinear columns of the
# multicollinearity variant with the four variables each one combines
PAPER_INFORMATIVE = (14, 18, 20, 26, 27, 31, 33, 40, 46, 49)
PAPER_COLLINEAR = {13: ((14, 0.1), (40, 0.2), (7, 0.3), (42, 0.4)),
                   5: ((31, 0.4), (46, 0.2), (47, 0.3), (48, 0.1)),
                   38: ((18, 0.1), (49, 0.3), (16, 0.2), (10, 0.4)),
                   9: ((27, 0.4), (26, 0.3), (17, 0.2), (25, 0.1)),
                   4: ((33, 0.2), (20, 0.4), (35, 0.1), (32, 0.3))}


def paper_regression(variant="direct", N=10_000, seed=0, n_trees=100, max_depth=16, max_iter=100, n_bins=128,
                     importance=PERMUT, mtry=1 << 20) -> Workload:
    """The paper's synthetic regression data (Sec. 3.1): X_1..X_50 ~ U(0, 1)
    and y = 5 X27^3 + 4 X49^2 + 5 X31 X46 + 2 X14 - 2.5 X40 + 3.5 X18^(1/3)
    + exp(X20) + 2 sin(3.14 X26) + 5 cos(3.14 X33) + eps1, eps1 ~ N(0, 1e-5)
    (read as the variance); 10,000 rows; the other 40 columns are noise.
    variant "biased" (Sec. 3.1.2): 99% of the rows, drawn at random, have
    X20 = -1.0 before the target is formed; "collinear" (Sec. 3.1.3): X13,
    X5, X38, X9 and X4 are replaced by the paper's linear combinations of
    four other columns plus eps2 ~ N(0, 0.01) (variance).  Targets are int64
    fixed point at 2^-20; features are quantile bins.  The forest defaults
    are those of the regression forest the paper used (cuML's
    RandomForestRegressor: 100 trees, depth 16, 128 bins, every column tried
    at each split -- mtry clamps to the augmented width).  `informative`
    holds the 0-based columns of the ten target variables."""
    rng = np.random.default_rng(np.random.PCG64(seed))
    p = 50
    F = rng.uniform(0.0, 1.0, size=(p, N))
    x = lambda i: F[i - 1]  # 1-based names of the paper
    if variant == "biased":
        rows = rng.choice(N, size=int(round(0.99 * N)), replace=False)
        F[19, rows] = -1.0
    elif variant == "collinear":
        for dst, terms in PAPER_COLLINEAR.items():
            F[dst - 1] = sum(w * x(src) for src, w in terms) + rng.normal(0.0, math.sqrt(0.01), size=N)
    elif variant != "direct":
        raise ValueError(f"unknown variant {variant!r}")
    yv = (5 * x(27) ** 3 + 4 * x(49) ** 2 + 5 * x(31) * x(46) + 2 * x(14) - 2.5 * x(40) + 3.5 * np.cbrt(x(18))
          + np.exp(x(20)) + 2 * np.sin(3.14 * x(26)) + 5 * np.cos(3.14 * x(33)))
    yv = yv + rng.normal(0.0, math.sqrt(1e-5), size=N)
    y_fx = np.rint(yv * 2.0**20).astype(np.int64)
    inf = np.array([i - 1 for i in PAPER_INFORMATIVE])
    return Workload(f"paper_{variant}_N{N}", quantise(F, n_bins), y_fx, N, p, REGRESSION | importance, 1, n_bins,
                    n_trees, max_depth, max_iter, seed=seed, mtry=mtry, informative=inf)


def batch_jobs(n_jobs=64, seed=4, n_trees=200, max_depth=10, max_iter=50, n_bins=128,
               N_range=(500, 50_000), p_range=(20, 5000), quantiser=None) -> list[Workload]:
    """Independent classification problems of uneven size: N and p
    log-uniform, 2-4 classes, 10% informative float32 columns with per-class
    mean shifts 0.8 * Bernoulli(1/2) (class 0 at 0).  quantiser as for
    multiclass_toeplitz."""
    rng = np.random.default_rng(np.random.PCG64(seed))
    jobs = []
    for j in range(n_jobs):
        N = int(round(math.exp(rng.uniform(math.log(N_range[0]), math.log(N_range[1])))))
        p = int(round(math.exp(rng.uniform(math.log(p_range[0]), math.log(p_range[1])))))
        C = int(rng.integers(2, 5))
        y = rng.integers(0, C, size=N).astype(np.uint8)
        F = rng.standard_normal((p, N))
        inf = np.sort(rng.choice(p, size=math.ceil(0.1 * p), replace=False))
        for col in inf:
            mu = 0.8 * (rng.random(C) < 0.5)
            mu[0] = 0.0
            F[col] += mu[y]
        jobs.append(Workload(f"job{j}_N{N}_p{p}_C{C}", (quantiser or quantise)(F.astype(np.float32), n_bins), y, N, p,
                             CLASSIFICATION | PERMUT, C, n_bins, n_trees, max_depth, max_iter,
                             seed=seed * 1000 + j, informative=inf))
    return jobs
