"""CUDA path against the CPU oracle, element by element on the same seeded
inputs (through the C ABI).

Bar: trees, bootstrap counts, shadow columns, hits and decisions bit-exact;
FP64 TreeImp and regression Permut importances bit-exact (both sides sum
exactly and round once); classification Permut importances within 1e-12
relative (the KL loss calls log, whose last bit may differ between CUDA and
the C library); the FP32 form within 1e-5 relative of the FP64 oracle.
"""
import numpy as np
import pytest

import oracle
from paper_2605_09950_gb300 import synth

pytestmark = pytest.mark.gpu

REL64 = 1e-12
REL32 = 1e-5


@pytest.fixture(scope="module", autouse=True)
def built():
    import torch

    import __graft_entry__

    __graft_entry__.build()
    assert torch.cuda.is_available()


def session(w, **opts):
    import torch

    from paper_2605_09950_gb300 import boruta

    X = torch.from_numpy(w.X).cuda()
    y = torch.from_numpy(w.y).cuda()
    params = w.params()
    n_classes = params.pop("n_classes")
    return boruta.Session(X, y, N=w.N, n_classes=n_classes, **params, **opts)


def oracle_problem(w, **kw):
    return oracle.BorutaProblem(w.X, w.y, **w.params(), N=w.N, **kw)


def close(a, b, rel):
    a, b = np.asarray(a, float), np.asarray(b, float)
    assert a.shape == b.shape
    both_nan = np.isnan(a) & np.isnan(b)
    ok = both_nan | (a == b) | (np.abs(a - b) <= rel * np.maximum(np.abs(a), np.abs(b)))
    assert ok.all(), (a[~ok][:5], b[~ok][:5])


def compare_nodes(g, o, exact_delta=True, rel=REL32):
    assert len(g) == len(o), (len(g), len(o))
    for k in ("heap", "depth", "feature", "bin", "n_rows", "n"):
        np.testing.assert_array_equal(g[k], o[k], err_msg=k)
    np.testing.assert_array_equal(g["stat"], o["stat"])
    if exact_delta:
        np.testing.assert_array_equal(g["delta"], o["delta"])
    else:
        close(g["delta"], o["delta"], rel)


def check_iteration(w, trees=None, precision=0, state=None, t=1, tie_break=0, **opts):
    """Runs iteration t on the GPU and checks every dump against the oracle."""
    from paper_2605_09950_gb300 import boruta

    S = session(w, precision=precision, tie_break=tie_break, **opts)
    p = w.p
    if state is None:
        state = dict(decision=np.zeros(p, np.int8), hits=np.zeros(p, np.int32),
                     imp_history=np.full((w.max_iter, p), np.nan), shadow_max=np.full(w.max_iter, np.nan),
                     iterations=t - 1)
    S.write(state)
    S.step()
    P = oracle_problem(w, tie_break=tie_break)
    live = P.live(state["decision"])
    np.testing.assert_array_equal(S.dump(boruta.DUMP_LIVE, np.int32), live)
    sha_o = P.shadow(t, live)
    sha_g = S.dump(boruta.DUMP_SHADOW, np.uint8).reshape(sha_o.shape)
    np.testing.assert_array_equal(sha_g, sha_o)
    boot = S.dump(boruta.DUMP_BOOT, np.uint32).reshape(w.n_trees, w.N)
    nodes = S.dump(boruta.DUMP_NODES, boruta.NODE_DTYPE)
    ptr = S.dump(boruta.DUMP_TREE_PTR, np.int64)
    imp = S.dump(boruta.DUMP_IMP, np.float64).reshape(w.n_trees, -1)
    permut = (w.task & 2) != 0
    reg = (w.task & 1) == 1
    for tau in (trees if trees is not None else range(w.n_trees)):
        np.testing.assert_array_equal(boot[tau], oracle.bootstrap(w.seed, 0, t, tau, w.N))
        nd, ti, pm = P.tree(t, live, sha_o, tau, treeimp=not permut, permut=permut)
        compare_nodes(nodes[ptr[tau]:ptr[tau + 1]], nd, exact_delta=precision == 0)
        want = pm if permut else ti
        if precision == 1:
            close(imp[tau], want, REL32)
        elif permut and not reg:
            close(imp[tau], want, REL64)
        else:
            np.testing.assert_array_equal(imp[tau], want)
    return S, P, state, imp


# ---------------------------------------------------------------- single iterations

@pytest.mark.parametrize("importance", [0, 2])
def test_binary_iteration(importance):
    w = synth.binary_small(N=500, p=20, n_inf=4, n_trees=16, max_depth=7, max_iter=5, importance=importance)
    S, P, st, imp = check_iteration(w)
    o = P.iteration(1, st["decision"], st["hits"])
    from paper_2605_09950_gb300 import boruta

    s = S.dump(boruta.DUMP_STAT, np.float64)
    if importance == 0:
        np.testing.assert_array_equal(s, o["s"])
    else:
        close(s, o["s"], 1e-9)
    g = S.read()
    np.testing.assert_array_equal(g["hits"], o["hits"])
    np.testing.assert_array_equal(g["decision"], o["state"])


@pytest.mark.parametrize("importance", [0, 2])
def test_multiclass_iteration(importance):
    w = synth.multiclass_toeplitz(N=3000, p=30, block=10, n_inf=3, n_classes=5, n_trees=10, max_depth=9,
                                  max_iter=3, importance=importance)
    check_iteration(w)


@pytest.mark.parametrize("importance", [0, 2])
def test_regression_iteration(importance):
    w = synth.snp_regression(N=900, p=40, n_add=5, n_pairs=2, n_trees=10, max_depth=7, max_iter=3,
                             importance=importance)
    check_iteration(w)


@pytest.mark.parametrize("importance", [0, 2])
def test_fp32_form_iteration(importance):
    w = synth.binary_small(N=700, p=25, n_inf=5, n_trees=12, max_depth=8, max_iter=3, importance=importance)
    check_iteration(w, precision=1)
    w = synth.snp_regression(N=600, p=30, n_add=4, n_pairs=2, n_trees=6, max_depth=6, max_iter=3,
                             importance=importance)
    check_iteration(w, precision=1)


@pytest.mark.parametrize("importance", [0, 2])
def test_draw_order_tie_break(importance):
    """tie_break = 1: equal scores go to the feature drawn first at the node
    (the default, 0, takes the lowest feature index and runs in every other
    test)."""
    w = synth.binary_small(N=300, p=10, n_inf=2, n_trees=8, max_depth=8, max_iter=3, importance=importance)
    check_iteration(w, tie_break=1)
    w = synth.snp_regression(N=500, p=20, n_add=4, n_pairs=2, n_trees=6, max_depth=7, max_iter=3,
                             importance=importance)
    check_iteration(w, tie_break=1)


def test_later_iteration_with_rejected_columns():
    """t = 9 with some columns rejected and some accepted: the live list,
    shadow doubling (p_live < 5) and hit bookkeeping follow the state."""
    w = synth.binary_small(N=400, p=7, n_inf=2, n_trees=8, max_depth=6, max_iter=12)
    dec = np.array([1, -1, 0, -1, -1, 0, -1], np.int8)
    hits = np.array([8, 0, 4, 1, 0, 2, 0], np.int32)
    hist = np.full((12, 7), np.nan)
    smax = np.full(12, np.nan)
    st = dict(decision=dec, hits=hits, imp_history=hist, shadow_max=smax, iterations=8)
    S, P, _, _ = check_iteration(w, state=st, t=9)
    o = P.iteration(9, dec, hits)
    g = S.read()
    np.testing.assert_array_equal(g["hits"], o["hits"])
    np.testing.assert_array_equal(g["decision"], o["state"])
    np.testing.assert_array_equal(g["imp_history"][8], o["hist"])
    assert g["shadow_max"][8] == o["shadow_max"]


# ---------------------------------------------------------------- edge cases

@pytest.mark.parametrize("case", ["ragged", "tiny", "one_row", "depth0", "two_bins", "full_mtry",
                                  "constant", "deep_small"])
def test_edge_cases(case):
    if case == "ragged":      # N not a multiple of 16, dense and sparse node paths
        w = synth.binary_small(N=37, p=3, n_inf=1, n_trees=6, max_depth=5, max_iter=2, n_bins=5)
    elif case == "tiny":      # every node on the one-row-per-lane path
        w = synth.binary_small(N=20, p=4, n_inf=1, n_trees=5, max_depth=10, max_iter=2, n_bins=8)
    elif case == "one_row":
        w = synth.binary_small(N=1, p=2, n_inf=1, n_trees=3, max_depth=4, max_iter=2, n_bins=4)
        w.y[:] = 0
    elif case == "depth0":    # stumps that never split: all importances 0
        w = synth.binary_small(N=200, p=6, n_inf=2, n_trees=4, max_depth=0, max_iter=2)
    elif case == "two_bins":
        w = synth.binary_small(N=300, p=6, n_inf=2, n_trees=5, max_depth=6, max_iter=2, n_bins=2)
    elif case == "full_mtry":
        w = synth.binary_small(N=300, p=6, n_inf=2, n_trees=5, max_depth=6, max_iter=2)
        w.mtry = 1000         # clamps to p_aug
    elif case == "constant":
        w = synth.binary_small(N=300, p=6, n_inf=2, n_trees=5, max_depth=6, max_iter=2, importance=2)
        w.X[3, :] = 2
    else:
        w = synth.multiclass_toeplitz(N=2000, p=10, block=5, n_inf=2, n_classes=3, n_trees=4, max_depth=14,
                                      max_iter=2, n_bins=256, importance=2)
    check_iteration(w)


# ---------------------------------------------------------------- whole runs

@pytest.mark.parametrize("importance", [0, 2])
def test_full_run_small(importance):
    w = synth.binary_small(N=400, p=12, n_inf=3, n_trees=20, max_depth=6, max_iter=16, importance=importance)
    from paper_2605_09950_gb300 import boruta
    import torch

    params = w.params()
    nc = params.pop("n_classes")
    g = boruta.boruta_fit(torch.from_numpy(w.X).cuda(), torch.from_numpy(w.y).cuda(), N=w.N, n_classes=nc,
                          **params)
    o = oracle_problem(w).run()
    assert g["iterations"] == o["iterations"]
    np.testing.assert_array_equal(g["decision"], o["decision"])
    np.testing.assert_array_equal(g["hits"], o["hits"])
    if importance == 0:
        np.testing.assert_array_equal(g["imp_history"], o["imp_history"])
        np.testing.assert_array_equal(g["shadow_max"], o["shadow_max"])
    else:
        close(g["imp_history"], o["imp_history"], 1e-9)
        close(g["shadow_max"], o["shadow_max"], 1e-9)


@pytest.mark.parametrize("tie_break", [0, 1])
def test_binary_n1000_p50_full_run(tie_break):
    """The small workload: binary N=1000, p=50, 100 trees, depth 8, TreeImp,
    20 iterations -- bit-exact against the oracle under either tie rule; the
    planted set is accepted (exactly it when ties go to the feature drawn
    first; with ties to the lowest index real columns also win the ties of
    tiny nodes against the higher-indexed shadows, so noise columns can be
    accepted too)."""
    import torch

    from paper_2605_09950_gb300 import boruta

    w = synth.binary_small()
    params = w.params()
    nc = params.pop("n_classes")
    g = boruta.boruta_fit(torch.from_numpy(w.X).cuda(), torch.from_numpy(w.y).cuda(), N=w.N, n_classes=nc,
                          tie_break=tie_break, **params)
    o = oracle_problem(w, tie_break=tie_break).run()
    assert g["iterations"] == o["iterations"]
    np.testing.assert_array_equal(g["decision"], o["decision"])
    np.testing.assert_array_equal(g["hits"], o["hits"])
    np.testing.assert_array_equal(g["imp_history"], o["imp_history"])
    accepted = set(np.flatnonzero(g["decision"] == 1))
    assert set(w.informative.tolist()) <= accepted
    if tie_break == 1:
        assert accepted == set(w.informative.tolist())


@pytest.mark.parametrize("importance", [synth.TREEIMP, synth.PERMUT])
def test_graph_replay_matches_stream_launches(importance):
    """opts.graph = 1 (each iteration captured, the executable graph updated
    in place and replayed) gives the same run, bit for bit, as plain launches
    -- including iterations after columns are rejected."""
    import torch

    from paper_2605_09950_gb300 import boruta

    w = synth.binary_small(N=600, p=20, n_inf=4, n_trees=24, max_depth=7, max_iter=30, importance=importance)
    params = w.params()
    nc = params.pop("n_classes")
    X, y = torch.from_numpy(w.X).cuda(), torch.from_numpy(w.y).cuda()
    a = boruta.boruta_fit(X, y, N=w.N, n_classes=nc, precision=1, **params)
    b = boruta.boruta_fit(X, y, N=w.N, n_classes=nc, precision=1, graph=1, **params)
    assert a["iterations"] == b["iterations"] and (a["decision"] != 0).any()
    for key in ("decision", "hits", "imp_history", "shadow_max"):
        np.testing.assert_array_equal(a[key], b[key], err_msg=key)


@pytest.mark.parametrize("importance", [synth.TREEIMP, synth.PERMUT])
def test_autotuned_tiles_give_the_same_run(importance):
    """opts.autotune = 1: the first step times fourteen histogram tile shapes
    (band bytes x launch per chunk or per band, a single band, then the
    per-level combination at three group works) on iteration 1, restoring
    the state after each, and keeps the fastest; the run is the same, bit for
    bit, as with the default shape, and the batched form with autotune equals
    it too."""
    import torch

    from paper_2605_09950_gb300 import boruta

    w = synth.binary_small(N=900, p=20, n_inf=4, n_trees=16, max_depth=8, max_iter=6, importance=importance)
    A = session(w)
    B = session(w, autotune=1)
    for _ in range(w.max_iter):
        ua, ub = A.step(), B.step()
        assert ua == ub
        if ua == 0:
            break
    ra, rb = A.read(), B.read()
    for key in ("decision", "hits", "imp_history", "shadow_max", "iterations"):
        np.testing.assert_array_equal(ra[key], rb[key], err_msg=key)
    tried, chosen = B.tuning()
    assert len(tried) == 14 and 0 <= chosen < 14 and all(ms > 0 for _, _, _, ms in tried)
    assert {gw for gw, _, _, _ in tried} == {4096, 8192, 16384} and {bl for _, _, bl, _ in tried} == {-1, 0, 1}
    assert [bb for _, bb, _, _ in tried[11:]] == [-1, -1, -1]
    bb, bl, lm = B.tuning_levels()
    assert len(bb) == w.max_depth and lm.shape == (14, w.max_depth)
    uniform = [b for _, b, _, _ in tried[:11]]
    assert all(b in uniform for b in bb) and all(x in (0, 1) for x in bl)
    assert A.tuning() == ([], -1)
    params = w.params()
    job = dict(X=torch.from_numpy(w.X).cuda(), y=torch.from_numpy(w.y).cuda(), N=w.N, **params)
    outs = boruta.boruta_fit_batch([job, job], autotune=1)
    plain = boruta.boruta_fit_batch([job, job])
    for a, b in zip(outs, plain):
        for key in ("decision", "hits", "imp_history", "shadow_max"):
            np.testing.assert_array_equal(a[key], b[key], err_msg=key)


def test_checkpoint_resume_is_exact():
    """Counter-based randomness: resuming from a state read at t = 4
    reproduces the uninterrupted run bit for bit."""
    w = synth.binary_small(N=400, p=12, n_inf=3, n_trees=12, max_depth=6, max_iter=14)
    A = session(w)
    while True:
        if A.step() == 0 or A.read()["iterations"] == w.max_iter:
            break
    full = A.read()
    B = session(w)
    for _ in range(4):
        B.step()
    ck = B.read()
    B.close()
    C = session(w)
    C.write(ck)
    while C.read()["iterations"] < full["iterations"]:
        C.step()
    res = C.read()
    for k in ("decision", "hits", "imp_history", "shadow_max"):
        np.testing.assert_array_equal(res[k], full[k])


# ---------------------------------------------------------------- full size, sampled

def _oracle_trees(P, t, live, sha, taus, **what):
    """Oracle trees on host threads (the oracle's C releases the GIL and
    keeps no global state)."""
    from concurrent.futures import ThreadPoolExecutor

    with ThreadPoolExecutor(max_workers=len(taus)) as ex:
        return list(ex.map(lambda tau: P.tree(t, live, sha, tau, **what), taus))


@pytest.mark.parametrize("precision", [0, 1])
def test_binary_n100000_p1000_sampled(precision):
    """Binary N=1e5, p=1000, 500 trees, depth 16, in both precision forms
    (one iteration, in the launch configuration the benchmark times): trees
    0 and 499 node by node and their Permut rows against the oracle (FP64
    terms within 1e-12, FP32 terms within 1e-5); properties of every tree."""
    from paper_2605_09950_gb300 import boruta

    w = synth.binary_wide(max_iter=3)
    S = session(w, precision=precision)
    S.step()
    P = oracle_problem(w)
    live = np.arange(w.p, dtype=np.int32)
    sha = P.shadow(1, live)
    np.testing.assert_array_equal(S.dump(boruta.DUMP_SHADOW, np.uint8).reshape(sha.shape), sha)
    nodes = S.dump(boruta.DUMP_NODES, boruta.NODE_DTYPE)
    ptr = S.dump(boruta.DUMP_TREE_PTR, np.int64)
    imp = S.dump(boruta.DUMP_IMP, np.float64).reshape(w.n_trees, -1)
    boot = S.dump(boruta.DUMP_BOOT, np.uint32).reshape(w.n_trees, w.N)
    taus = [0, w.n_trees - 1]
    for tau, (nd, _, pm) in zip(taus, _oracle_trees(P, 1, live, sha, taus, permut=True)):
        np.testing.assert_array_equal(boot[tau], oracle.bootstrap(w.seed, 0, 1, tau, w.N))
        compare_nodes(nodes[ptr[tau]:ptr[tau + 1]], nd, exact_delta=precision == 0)
        close(imp[tau], pm, REL64 if precision == 0 else REL32)
    assert (boot.sum(axis=1) == w.N).all()
    assert np.isfinite(imp).all() and (imp >= -1e-15).all()


# ---------------------------------------------------------------- larger-node paths

@pytest.mark.parametrize("case", ["binary", "multiclass", "regression"])
def test_grouped_item_path(case):
    """The grouped path for larger nodes (used when a level has more items
    than the band plan holds) gives the same trees and importances."""
    if case == "binary":
        w = synth.binary_small(N=800, p=20, n_inf=4, n_trees=8, max_depth=9, max_iter=3)
    elif case == "multiclass":
        w = synth.multiclass_toeplitz(N=3000, p=20, block=5, n_inf=3, n_classes=6, n_trees=6, max_depth=8,
                                      max_iter=3, importance=2)
    else:
        w = synth.snp_regression(N=900, p=40, n_add=5, n_pairs=2, n_trees=6, max_depth=7, max_iter=3)
    check_iteration(w, split_path=1)


@pytest.mark.parametrize("case", ["binary", "multiclass", "regression"])
def test_band_path_in_many_chunks(case):
    """The band path runs a level's larger nodes in chunks that fit its plan
    buffers (at full size: SNP regression from about depth 6, multiclass
    N=1e6 at depths 17-19).  opts.chunk_nodes = 3 forces several chunks per
    level on small problems: trees and importances against the oracle, and
    the same dumps as the one-chunk run."""
    from paper_2605_09950_gb300 import boruta

    if case == "binary":
        w = synth.binary_small(N=900, p=20, n_inf=4, n_trees=8, max_depth=9, max_iter=3, importance=2)
    elif case == "multiclass":
        w = synth.multiclass_toeplitz(N=3000, p=20, block=5, n_inf=3, n_classes=4, n_trees=6, max_depth=8,
                                      max_iter=3, importance=2)
    else:
        w = synth.snp_regression(N=900, p=40, n_add=5, n_pairs=2, n_trees=6, max_depth=7, max_iter=3)
    S, _, _, imp = check_iteration(w, chunk_nodes=3)
    ref = session(w)
    ref.step()
    per_band = session(w, chunk_nodes=3, band_launch=1)  # one histogram launch per band
    per_band.step()
    per_chunk = session(w, chunk_nodes=3, band_launch=2)  # one per chunk at every level
    per_chunk.step()
    for what, dt in ((boruta.DUMP_NODES, boruta.NODE_DTYPE), (boruta.DUMP_IMP, np.float64),
                     (boruta.DUMP_STAT, np.float64)):
        np.testing.assert_array_equal(S.dump(what, dt), ref.dump(what, dt))
        np.testing.assert_array_equal(per_band.dump(what, dt), ref.dump(what, dt))
        np.testing.assert_array_equal(per_chunk.dump(what, dt), ref.dump(what, dt))
    assert set(per_band.tuning_levels()[1]) == {1} and set(per_chunk.tuning_levels()[1]) == {0}
    levels = S.dump(boruta.DUMP_LEVELS, np.float64).reshape(-1, 3)
    assert levels[:, 0].max() > 3 * 3  # some level held more than three chunks of nodes


# ---------------------------------------------------------------- Alg. 3 as printed

@pytest.mark.parametrize("case,rows", [("binary", 0), ("binary", 37), ("multiclass", 0), ("multiclass", 100),
                                       ("regression", 0), ("regression", 64)])
def test_forest_permut_form_iteration(case, rows):
    """opts.permut_form = 1 (every row against the forest's prediction, one
    importance row for the forest, which is the hit statistic), with the
    default row blocks and with several blocks (forest_rows): trees node by
    node, the importance row (regression bit-exact, KL within 1e-12), the
    statistic, hits and decisions against the oracle."""
    from paper_2605_09950_gb300 import boruta

    if case == "binary":
        w = synth.binary_small(N=500, p=12, n_inf=3, n_trees=12, max_depth=7, max_iter=5, importance=2)
    elif case == "multiclass":
        w = synth.multiclass_toeplitz(N=1500, p=16, block=4, n_inf=3, n_classes=4, n_trees=8, max_depth=8,
                                      max_iter=3, importance=2)
    else:
        w = synth.snp_regression(N=700, p=20, n_add=4, n_pairs=2, n_trees=8, max_depth=7, max_iter=3,
                                 importance=2)
    S = session(w, permut_form=1, forest_rows=rows)
    S.step()
    P = oracle_problem(w, permut_form=1)
    live = np.arange(w.p, dtype=np.int32)
    sha = P.shadow(1, live)
    nodes = S.dump(boruta.DUMP_NODES, boruta.NODE_DTYPE)
    ptr = S.dump(boruta.DUMP_TREE_PTR, np.int64)
    for tau in range(w.n_trees):
        nd, _, _ = P.tree(1, live, sha, tau)
        compare_nodes(nodes[ptr[tau]:ptr[tau + 1]], nd)
    imp = S.dump(boruta.DUMP_IMP, np.float64)
    want = P.forest_permut(1, live, sha)
    if case == "regression":
        np.testing.assert_array_equal(imp, want)
    else:
        close(imp, want, REL64)
    assert (imp > 0).any()
    np.testing.assert_array_equal(S.dump(boruta.DUMP_STAT, np.float64), imp)
    o = P.iteration(1, np.zeros(w.p, np.int8), np.zeros(w.p, np.int32))
    g = S.read()
    np.testing.assert_array_equal(g["hits"], o["hits"])
    np.testing.assert_array_equal(g["decision"], o["state"])


def test_forest_permut_form_full_run():
    """A whole Boruta run with Alg. 3 as printed, through boruta_fit:
    iterations, decisions and hits equal the oracle's run; the history of
    the statistic within 1e-12."""
    import torch

    from paper_2605_09950_gb300 import boruta

    w = synth.binary_small(N=400, p=10, n_inf=3, n_trees=16, max_depth=6, max_iter=18, importance=2)
    params = w.params()
    nc = params.pop("n_classes")
    g = boruta.boruta_fit(torch.from_numpy(w.X).cuda(), torch.from_numpy(w.y).cuda(), N=w.N, n_classes=nc,
                          permut_form=1, **params)
    o = oracle_problem(w, permut_form=1).run()
    assert g["iterations"] == o["iterations"]
    np.testing.assert_array_equal(g["decision"], o["decision"])
    np.testing.assert_array_equal(g["hits"], o["hits"])
    close(g["imp_history"], o["imp_history"], REL64)
    assert (g["decision"] != 0).any()


# ---------------------------------------------------------------- full-size workloads, sampled

def _importance_properties(S, nodes, ptr, n_trees, permut):
    from paper_2605_09950_gb300 import boruta

    imp = S.dump(boruta.DUMP_IMP, np.float64).reshape(n_trees, -1)
    assert np.isfinite(imp).all()
    for tau in range(n_trees):
        used = np.unique(nodes["feature"][ptr[tau]:ptr[tau + 1]])
        used = used[used >= 0]
        unused = np.setdiff1d(np.arange(imp.shape[1]), used)
        assert (imp[tau, unused] == 0.0).all()  # never split on: exactly 0 (Alg. 2 and Alg. 3)
        if not permut and used.size:
            assert imp[tau].sum() == pytest.approx(1.0, abs=1e-12)


def test_snp_regression_n20000_p20000_whole_trees():
    """SNP regression N=2e4, p=2e4 (40,000 augmented columns, mtry 13,333),
    256 trees, depth 12, TreeImp (its levels run the band path in several
    chunks from about depth 6): every shadow column, two bootstrap rows, and
    two whole trees node by node with their TreeImp rows (bit-exact) against
    the oracle; importance properties of every tree."""
    from paper_2605_09950_gb300 import boruta

    w = synth.snp_regression(max_iter=3)
    S = session(w)
    S.step()
    P = oracle_problem(w)
    live = np.arange(w.p, dtype=np.int32)
    sha = P.shadow(1, live)
    np.testing.assert_array_equal(S.dump(boruta.DUMP_SHADOW, np.uint8).reshape(sha.shape), sha)
    boot = S.dump(boruta.DUMP_BOOT, np.uint32).reshape(w.n_trees, w.N)
    nodes = S.dump(boruta.DUMP_NODES, boruta.NODE_DTYPE)
    ptr = S.dump(boruta.DUMP_TREE_PTR, np.int64)
    imp = S.dump(boruta.DUMP_IMP, np.float64).reshape(w.n_trees, -1)
    taus = [0, w.n_trees - 1]
    for tau, (nd, ti, _) in zip(taus, _oracle_trees(P, 1, live, sha, taus, treeimp=True)):
        np.testing.assert_array_equal(boot[tau], oracle.bootstrap(w.seed, 0, 1, tau, w.N))
        compare_nodes(nodes[ptr[tau]:ptr[tau + 1]], nd)
        np.testing.assert_array_equal(imp[tau], ti)
    _importance_properties(S, nodes, ptr, w.n_trees, permut=False)


def test_multiclass_n1000000_p500_whole_trees():
    """Five classes, N=1e6, p=500 (Toeplitz blocks), 300 trees, depth 20,
    Permut in the FP32-term form the benchmark times (its deepest levels run
    the band path in several chunks): shadows, two bootstrap rows and two
    whole trees node by node against the oracle (split deltas within 1e-5);
    importance properties of every tree.  (An oracle Permut row of this size
    takes minutes; the rows' arithmetic is checked on the smaller cases.)"""
    from paper_2605_09950_gb300 import boruta

    w = synth.multiclass_toeplitz(max_iter=3)
    S = session(w, precision=1)
    S.step()
    P = oracle_problem(w)
    live = np.arange(w.p, dtype=np.int32)
    sha = P.shadow(1, live)
    np.testing.assert_array_equal(S.dump(boruta.DUMP_SHADOW, np.uint8).reshape(sha.shape), sha)
    boot = S.dump(boruta.DUMP_BOOT, np.uint32).reshape(w.n_trees, w.N)
    nodes = S.dump(boruta.DUMP_NODES, boruta.NODE_DTYPE)
    ptr = S.dump(boruta.DUMP_TREE_PTR, np.int64)
    taus = [0, w.n_trees - 1]
    for tau, (nd, _, _) in zip(taus, _oracle_trees(P, 1, live, sha, taus)):
        np.testing.assert_array_equal(boot[tau], oracle.bootstrap(w.seed, 0, 1, tau, w.N))
        compare_nodes(nodes[ptr[tau]:ptr[tau + 1]], nd, exact_delta=False)
    _importance_properties(S, nodes, ptr, w.n_trees, permut=True)
