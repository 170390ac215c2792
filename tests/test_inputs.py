"""The input side: the quantiser that defines the bins (and is the reference
of the GPU quantiser) against the rank definition written out by brute
force, and the generators' shapes and planted structure."""
import numpy as np
import pytest

from paper_2605_09950_gb300 import synth


def _brute_bins(col, B):
    N = len(col)
    return np.array([min(B - 1, (B * sum(1 for v in col if v < x)) // N) for x in col], dtype=np.uint8)


@pytest.mark.parametrize("N,B", [(1, 2), (7, 2), (50, 4), (97, 64), (300, 256)])
def test_quantise_is_the_rank_definition(N, B):
    rng = np.random.default_rng(N + B)
    F = np.round(rng.standard_normal((3, N)) * 2) / 2  # ties
    F[1] = rng.standard_normal(N)
    F[2, : N // 2] = -0.0  # -0 equals +0
    F[2, N // 2 :] = 0.0
    got = synth.quantise(F, B)
    assert got.shape == (3, (N + 15) // 16 * 16)
    assert not got[:, N:].any()
    for j in range(3):
        np.testing.assert_array_equal(got[j, :N], _brute_bins(F[j].tolist(), B))


def test_quantile_bins_are_balanced_without_ties():
    F = np.random.default_rng(0).standard_normal((1, 1024))
    counts = np.bincount(synth.quantise(F, 64)[0, :1024], minlength=64)
    assert (counts == 16).all()


def test_generators_shapes_and_planted_columns():
    w = synth.binary_small()
    assert (w.N, w.p, w.n_bins, w.n_trees, w.max_depth, w.max_iter) == (1000, 50, 64, 100, 8, 20)
    assert len(w.informative) == 10 and w.X.dtype == np.uint8 and w.X.shape == (50, 1008)
    # informative columns separate the classes, noise columns do not
    diff = [abs(w.X[j, : w.N][w.y == 1].mean() - w.X[j, : w.N][w.y == 0].mean()) for j in range(w.p)]
    noise = np.setdiff1d(np.arange(w.p), w.informative)
    assert min(diff[j] for j in w.informative) > max(diff[j] for j in noise)
    s = synth.snp_regression(N=500, p=40, n_add=3, n_pairs=1)
    assert s.X[:, : s.N].max() <= 2 and s.y.dtype == np.int64
    m = synth.multiclass_toeplitz(N=2000, p=20, block=10, n_inf=2, n_classes=5)
    assert m.y.max() < 5 and m.X.shape == (20, 2000)
    jobs = synth.batch_jobs(n_jobs=3, N_range=(100, 300), p_range=(5, 20))
    assert len(jobs) == 3 and all(2 <= j.n_classes <= 4 for j in jobs)


def test_paper_regression_workload():
    """The paper's synthetic regression data (Sec. 3.1): 50 uniform columns,
    the target built from the ten named ones (checked on raw rows against
    the printed equation term by term), and the two variants: X20 set to
    -1.0 in 99% of the rows before the target is formed; X13, X5, X38, X9,
    X4 replaced by the printed linear combinations (their correlation with
    the combination is close to 1)."""
    import math

    from paper_2605_09950_gb300 import synth

    w = synth.paper_regression("direct", N=2000, seed=3)
    assert w.X.shape == (50, 2000) and w.y.dtype == np.int64 and w.task == 1 | 2
    assert sorted(w.informative.tolist()) == [13, 17, 19, 25, 26, 30, 32, 39, 45, 48]
    assert w.X[:, :w.N].max() == 127 and (w.X[:, :w.N].min(axis=1) == 0).all()
    rng = np.random.default_rng(np.random.PCG64(3))
    F = rng.uniform(0.0, 1.0, size=(50, 2000))
    y = np.rint((5 * F[26] ** 3 + 4 * F[48] ** 2 + 5 * F[30] * F[45] + 2 * F[13]
                - 2.5 * F[39] + 3.5 * np.cbrt(F[17]) + np.exp(F[19]) + 2 * np.sin(3.14 * F[25])
                + 5 * np.cos(3.14 * F[32]) + rng.normal(0.0, math.sqrt(1e-5), size=2000)) * 2.0**20)
    np.testing.assert_array_equal(w.y, y.astype(np.int64))
    b = synth.paper_regression("biased", N=2000, seed=3)
    assert (b.X[19, :b.N] == 0).sum() >= 0.99 * 2000  # -1.0 is the smallest value: bin 0
    c = synth.paper_regression("collinear", N=2000, seed=3)
    for dst in (13, 5, 38, 9, 4):
        assert not np.array_equal(c.X[dst - 1], w.X[dst - 1])
    keep = [j for j in range(50) if j + 1 not in (13, 5, 38, 9, 4)]
    np.testing.assert_array_equal(c.X[keep], w.X[keep])
