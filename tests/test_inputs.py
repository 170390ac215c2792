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
