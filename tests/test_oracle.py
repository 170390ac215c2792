"""Pins of the CPU oracle against facts other than itself (no GPU needed).

Each test names what fixes the expected value: published known answers,
Python's exact integer / rational arithmetic, math.fsum (a correctly rounded
sum), brute-force enumeration, hand-worked examples, closed forms and
invariants of the method (Alg. 1-3 of the paper).
"""
import math
import os
from fractions import Fraction

import numpy as np
import pytest

import oracle
from paper_2605_09950_gb300 import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# ---------------------------------------------------------------- Philox

def test_philox_known_answers():
    """Philox4x32-10 against the generator's published known answers."""
    n = 0
    for line in open(os.path.join(GOLDEN, "philox4x32_10_kat.txt")):
        if line.startswith("#") or not line.strip():
            continue
        lhs, rhs = line.split("->")
        words = [int(x, 16) for x in lhs.split()]
        expect = [int(x, 16) for x in rhs.split()]
        got = oracle.philox(words[:4], words[4:6])
        assert [int(v) for v in got] == expect
        n += 1
    assert n == 3


def test_fmix32_is_a_bijection_and_avalanches():
    """MurmurHash3's finaliser is invertible (no collisions on a large sample)
    and flips about half of the output bits per input bit."""
    rng = np.random.default_rng(7)
    xs = np.unique(rng.integers(0, 2**32, size=200_000, dtype=np.uint64))
    ys = {oracle.fmix32(int(x)) for x in xs[:20000]}
    assert len(ys) == min(20000, xs.size)
    flips = []
    for x in xs[:500]:
        h = oracle.fmix32(int(x))
        for b in range(32):
            flips.append(bin(h ^ oracle.fmix32(int(x) ^ (1 << b))).count("1"))
    assert abs(np.mean(flips) - 16.0) < 0.5
    assert oracle.fmix32(0) == 0


# ---------------------------------------------------------------- permutations

@pytest.mark.parametrize("n", [1, 2, 3, 4, 5, 7, 16, 17, 63, 64, 65, 1000, 4097])
def test_feistel_is_a_permutation(n):
    """Cycle-walked Feistel network: a bijection of [0, n) for every n."""
    out = oracle.perm(n, 12345, 1, 2, 3, np.arange(n))
    assert sorted(out.tolist()) == list(range(n))


def test_feistel_positions_are_uniform():
    """Across many keys, sigma(i) is uniform over [0, n) (chi-square)."""
    n, keys = 37, 4000
    counts = np.zeros((n, n))
    for k in range(keys):
        s = oracle.perm(n, 99, k, 5, 6, np.arange(n))
        counts[np.arange(n), s] += 1
    exp = keys / n
    chi2 = ((counts - exp) ** 2 / exp).sum()
    dof = (n - 1) * (n - 1)
    assert abs(chi2 - dof) < 6 * math.sqrt(2 * dof)


def test_shadow_columns_are_row_permutations():
    """Alg. 1: each shadow column holds the values of its source column,
    shuffled; columns are doubled until there are at least five."""
    w = synth.binary_small(N=300, p=3, n_inf=1)
    P = oracle.BorutaProblem(w.X, w.y, **w.params(), N=w.N)
    live = np.array([0, 2], dtype=np.int32)
    sha = P.shadow(1, live)
    assert sha.shape == (oracle.shadow_count(2), 300) == (8, 300)
    for c in range(sha.shape[0]):
        src = w.X[live[c % 2], :300]
        assert np.array_equal(np.sort(sha[c]), np.sort(src))
        assert not np.array_equal(sha[c], src)
    assert not np.array_equal(sha[0], sha[2])  # copies get different shuffles
    assert [oracle.shadow_count(k) for k in (1, 2, 3, 4, 5, 6)] == [8, 8, 6, 8, 5, 6]


def test_permut_table_is_a_permutation():
    w = synth.binary_small(N=777, p=2, n_inf=1)
    P = oracle.BorutaProblem(w.X, w.y, **w.params(), N=w.N)
    pi = P.permut_table(3)
    assert sorted(pi.tolist()) == list(range(777))


# ---------------------------------------------------------------- bootstrap, mtry

def test_bootstrap_counts_are_multinomial():
    """N draws with replacement: counts sum to N, out-of-bag fraction near
    (1-1/N)^N, count histogram near Poisson(1)."""
    N = 20000
    c = oracle.bootstrap(0, 0, 1, 3, N)
    assert c.sum() == N
    assert abs((c == 0).mean() - (1 - 1 / N) ** N) < 0.01
    for k in range(4):
        pk = math.exp(-1) / math.factorial(k)
        assert abs((c == k).mean() - pk) < 0.01
    assert not np.array_equal(c, oracle.bootstrap(0, 0, 1, 4, N))


def test_mtry_sample_is_distinct_and_uniform():
    p_aug, mtry = 40, 6
    freq = np.zeros(p_aug)
    for v in range(3000):
        f = oracle.mtry_features(5, 0, 2, 1, v, p_aug, mtry)
        assert len(set(f.tolist())) == mtry and f.max() < p_aug
        freq[f] += 1
    exp = 3000 * mtry / p_aug
    assert np.all(np.abs(freq - exp) < 5 * math.sqrt(exp))


def test_default_mtry():
    assert oracle.default_mtry(0, 100) == 10
    assert oracle.default_mtry(0, 2000) == 44
    assert oracle.default_mtry(1, 40000) == 13333
    assert oracle.default_mtry(0, 1000) == 31
    assert oracle.default_mtry(1, 2) == 1


# ---------------------------------------------------------------- exact arithmetic

def test_cmp_products_matches_python_integers():
    rng = np.random.default_rng(1)
    for _ in range(3000):
        bits = rng.integers(1, 128)
        a1, b1, a2, b2 = (int(rng.integers(0, 2**63)) << int(rng.integers(0, bits)) for _ in range(4))
        want = (a1 * b1 > a2 * b2) - (a1 * b1 < a2 * b2)
        if max(a1 * b1, a2 * b2) >= 2**256:
            want = 2
        assert oracle.cmp_products(a1, b1, a2, b2) == want
    assert oracle.cmp_products(2**200, 2**56, 1, 1) == 2  # 2^256 overflows


def test_u256_to_double_is_correctly_rounded():
    """Against Python's int -> float (round half to even)."""
    cases = [0, 1, 2**53 - 1, 2**53, 2**53 + 1, 2**53 + 2, 2**53 + 3, 2**54 + 2, 2**54 + 6,
             2**64 - 1, 2**127, 2**127 + 2**74, 2**127 + 2**74 + 1, 2**255 + 1, 2**256 - 1,
             (2**53 - 1) << 100, ((2**53 - 1) << 100) + (1 << 99)]
    rng = np.random.default_rng(2)
    for _ in range(2000):
        v = int(rng.integers(1, 2**63)) << int(rng.integers(0, 190))
        v += int(rng.integers(0, 2**63))
        cases.append(v)
    for v in cases:
        assert oracle.u256_to_double(v) == float(v), hex(v)


def test_exact_sum_matches_fsum():
    """math.fsum is a correctly rounded sum of doubles."""
    rng = np.random.default_rng(3)
    for trial in range(300):
        n = int(rng.integers(1, 400))
        x = rng.standard_normal(n) * np.exp2(rng.integers(-60, 60, size=n))
        if trial % 3 == 0:  # heavy cancellation
            x = np.concatenate([x, -x[::-1] * (1 + 2**-40)])
        assert oracle.exact_sum(x) == math.fsum(x)
    assert oracle.exact_sum([1e300, 1.0, -1e300]) == 1.0
    assert oracle.exact_sum([2**-1074, 2**-1074]) == math.fsum([2**-1074, 2**-1074])
    assert oracle.exact_sum([]) == 0.0


@pytest.mark.parametrize("t", [1, 2, 7, 20, 63, 64, 100, 126])
def test_binomial_tails(t):
    """Exact tails against math.comb; closed forms and symmetry."""
    for h in range(0, t + 1):
        pa, pr, up, lo = oracle.binom_tails(t, h)
        assert up == sum(math.comb(t, k) for k in range(h, t + 1))
        assert lo == sum(math.comb(t, k) for k in range(0, h + 1))
        assert pa == float(Fraction(up, 2**t))  # one correct rounding
        assert pr == float(Fraction(lo, 2**t))
        assert oracle.binom_tails(t, t - h)[3] == up  # U(t,h) = L(t,t-h)
    assert oracle.binom_tails(t, 0)[0] == 1.0
    assert oracle.binom_tails(t, t)[0] == 2.0**-t
    assert oracle.binom_tails(t, 0)[1] == 2.0**-t


# ---------------------------------------------------------------- split search

def _golden_examples():
    for line in open(os.path.join(GOLDEN, "gini_worked_examples.txt")):
        if line.startswith("#") or not line.strip():
            continue
        kind, C, y, x, w, f, b, d = line.strip().split("|")
        num, den = d.split("/")
        yield (kind, int(C), [int(v) for v in y.split(",")], [int(v) for v in x.split(",")],
               [int(v) for v in w.split(",")], int(f), int(b), Fraction(int(num), int(den)))


@pytest.mark.parametrize("ex", list(_golden_examples()))
def test_hand_worked_gains(ex):
    kind, C, y, x, w, f, b, delta = ex
    task = 0 if kind == "cls" else 1
    bins = np.array(x, dtype=np.uint8)[:, None]
    got = oracle.node_split(task, C, 8, bins, w, y, [0])
    assert got is not None
    assert got[0] == f and got[1] == b
    assert got[2] == pytest.approx(float(delta), rel=1e-15)


def _impurity(task, C, ys, ws):
    """n * impurity from its definition: Gini n(1 - sum p_k^2) or n * Var."""
    n = sum(ws)
    if task == 0:
        return n * (1 - sum(Fraction(sum(w for yy, w in zip(ys, ws) if yy == k), n) ** 2
                            for k in range(C)))
    mean = Fraction(sum(w * yy for yy, w in zip(ys, ws)), n)
    return sum(w * (yy - mean) ** 2 for yy, w in zip(ys, ws))


def _brute_force(task, C, B, bins, w, y, feats):
    bins = np.asarray(bins).tolist()  # exact Python integers from here on
    w = [int(v) for v in w]
    y = [int(v) for v in y]
    feats = [int(f) for f in feats]
    rows = range(len(bins))
    n_par = _impurity(task, C, list(y), list(w))
    best = None
    for f in feats:
        for b in range(B - 1):
            L = [r for r in rows if bins[r][f] <= b]
            R = [r for r in rows if bins[r][f] > b]
            if sum(w[r] for r in L) == 0 or sum(w[r] for r in R) == 0:
                continue
            d = (n_par - _impurity(task, C, [y[r] for r in L], [w[r] for r in L])
                 - _impurity(task, C, [y[r] for r in R], [w[r] for r in R]))
            if best is None or d > best[2]:
                best = (f, b, d)
    if best is None or best[2] <= 0:
        return None
    return best


@pytest.mark.parametrize("task", [0, 1])
def test_split_search_matches_brute_force(task):
    """Exhaustive enumeration with exact fractions of the impurity-decrease
    definition (a different formula from the oracle's integer form)."""
    rng = np.random.default_rng(11 + task)
    for _ in range(250):
        nrows = int(rng.integers(1, 13))
        nf = int(rng.integers(1, 5))
        B = int(rng.integers(2, 9))
        C = int(rng.integers(2, 5)) if task == 0 else 1
        bins = rng.integers(0, B, size=(nrows, nf)).astype(np.uint8)
        w = rng.integers(1, 4, size=nrows)
        y = rng.integers(0, C, size=nrows) if task == 0 else rng.integers(-50, 50, size=nrows)
        feats = rng.permutation(nf)[: int(rng.integers(1, nf + 1))]
        want = _brute_force(task, C, B, bins, w, y, feats)
        got = oracle.node_split(task, C, B, bins, w, y, feats)
        if want is None:
            assert got is None
        else:
            assert got is not None and got[:2] == want[:2]
            assert got[2] == pytest.approx(float(want[2]), rel=1e-15)


# ---------------------------------------------------------------- trees

def _small(importance=0, **kw):
    args = dict(N=400, p=12, n_inf=3, n_trees=5, max_depth=6, max_iter=3)
    args.update(kw)
    w = synth.binary_small(importance=importance, **args)
    return w, oracle.BorutaProblem(w.X, w.y, **w.params(), N=w.N)


def _naive_tree(P, t, live, Xsha, tree, w):
    """Second, naive recursive tree builder: bootstrap and feature sample from
    the (separately pinned) streams, splits from exact-fraction brute force."""
    N = P.N
    cols = np.concatenate([P.X[live, :N], Xsha], axis=0)
    p_aug = cols.shape[0]
    cnt = oracle.bootstrap(P.c.seed, 0, t, tree, N)
    mtry = oracle.default_mtry(0, p_aug)
    out = []

    def grow(rows, heap, depth):
        ws = cnt[rows]
        ys = P.y[rows]
        node = dict(heap=heap, depth=depth, feature=-1, bin=0, n_rows=len(rows), n=int(ws.sum()))
        out.append(node)
        if depth >= P.c.max_depth:
            return
        feats = oracle.mtry_features(P.c.seed, 0, t, tree, heap, p_aug, mtry)
        if P.c.tie_break == 0:  # equal scores: lowest feature index first
            feats = np.sort(feats)
        best = _brute_force(0, P.n_classes, P.c.n_bins, cols[:, rows].T, ws, ys, feats)
        if best is None:
            return
        f, b, _ = best
        node["feature"], node["bin"] = int(f), int(b)
        grow(rows[cols[f, rows] <= b], 2 * heap + 1, depth + 1)
        grow(rows[cols[f, rows] > b], 2 * heap + 2, depth + 1)

    grow(np.flatnonzero(cnt > 0), 0, 0)
    return sorted(out, key=lambda d: (d["depth"], d["heap"]))


@pytest.mark.parametrize("tie_break", [0, 1])
def test_tree_rebuilds_from_naive_builder(tie_break):
    w, P = _small(N=120, p=5, max_depth=4)
    P.c.tie_break = tie_break
    live = np.arange(5, dtype=np.int32)
    sha = P.shadow(1, live)
    for tree in range(2):
        nodes, _, _ = P.tree(1, live, sha, tree)
        naive = _naive_tree(P, 1, live, sha, tree, w)
        assert len(nodes) == len(naive)
        for a, b in zip(nodes, naive):
            for k in ("heap", "depth", "feature", "bin", "n_rows", "n"):
                assert int(a[k]) == b[k], (k, a, b)


def test_tree_structure_invariants():
    w, P = _small(N=600, p=20, max_depth=7)
    live = np.arange(20, dtype=np.int32)
    sha = P.shadow(2, live)
    nodes, _, _ = P.tree(2, live, sha, 0)
    by_heap = {int(n["heap"]): n for n in nodes}
    for n in nodes:
        assert n["depth"] <= 7
        assert n["stat"][:2].sum() == n["n"]
        if n["feature"] >= 0:
            L, R = by_heap[2 * int(n["heap"]) + 1], by_heap[2 * int(n["heap"]) + 2]
            assert L["n"] + R["n"] == n["n"] and L["n_rows"] + R["n_rows"] == n["n_rows"]
            assert np.array_equal(L["stat"] + R["stat"], n["stat"])
            assert n["delta"] > 0
        else:
            assert 2 * int(n["heap"]) + 1 not in by_heap
    root = by_heap[0]
    assert root["n"] == 600  # N bootstrap draws


def test_treeimp_invariants():
    """Alg. 2: per-tree rows sum to 1 (or are all 0); features never split
    on get exactly 0; a depth-1 tree puts everything on its root feature."""
    w, P = _small(N=500, p=15, max_depth=5)
    live = np.arange(15, dtype=np.int32)
    sha = P.shadow(1, live)
    for tree in range(3):
        nodes, ti, _ = P.tree(1, live, sha, tree, treeimp=True)
        assert ti.sum() == pytest.approx(1.0, abs=1e-14)
        used = set(int(f) for f in nodes["feature"] if f >= 0)
        for j in range(ti.size):
            if j not in used:
                assert ti[j] == 0.0
            else:
                assert ti[j] > 0.0
    w1, P1 = _small(N=500, p=15, max_depth=1)
    nodes, ti, _ = P1.tree(1, live, P1.shadow(1, live), 0, treeimp=True)
    assert ti[nodes["feature"][0]] == 1.0 and ti.sum() == 1.0


def test_treeimp_matches_alg2_recursion():
    """Alg. 2 literally: CalcNodeImp recursion in float, normalised by the
    per-tree total -- equal to the oracle's exact sums up to rounding."""
    w, P = _small(N=500, p=15, max_depth=6)
    live = np.arange(15, dtype=np.int32)
    sha = P.shadow(1, live)
    nodes, ti, _ = P.tree(1, live, sha, 1, treeimp=True)
    by_heap = {int(n["heap"]): n for n in nodes}
    gains = np.zeros(ti.size)

    def calc(v):
        n = by_heap[v]
        if n["feature"] < 0:
            return
        gains[n["feature"]] += n["delta"]
        calc(2 * v + 1)
        calc(2 * v + 2)

    calc(0)
    np.testing.assert_allclose(ti, gains / gains.sum(), rtol=1e-13, atol=1e-16)


def test_permut_invariants_and_stump_closed_form():
    """Alg. 3 on out-of-bag rows: exactly 0 for features not on any path; for a
    stump, the importance of the root feature is the mean over OOB rows of
    the loss between the two leaves, counted over rows whose permuted value
    crosses the threshold -- computed here from the raw data."""
    w, P = _small(importance=2, N=500, p=15, max_depth=4)
    live = np.arange(15, dtype=np.int32)
    sha = P.shadow(1, live)
    nodes, _, pm = P.tree(1, live, sha, 0, permut=True)
    used = set(int(f) for f in nodes["feature"] if f >= 0)
    for j in range(pm.size):
        if j not in used:
            assert pm[j] == 0.0
    assert all(pm[j] >= 0 for j in used)

    w1, P1 = _small(importance=2, N=500, p=15, max_depth=1)
    sha = P1.shadow(1, live)
    nodes, _, pm = P1.tree(1, live, sha, 2, permut=True)
    root, L, R = nodes[0], nodes[1], nodes[2]
    f, b = int(root["feature"]), int(root["bin"])
    col = np.concatenate([w1.X[live, :500], sha])[f]
    pi = P1.permut_table(1)
    oob = np.flatnonzero(oracle.bootstrap(0, 0, 1, 2, 500) == 0)
    eps = 1e-7

    def probs(n):
        return (n["stat"][:2] / n["n"] + eps) / (1 + 2 * eps)

    def kl(a, c):
        pa, pc = probs(a), probs(c)
        return float(np.sum(pa * np.log(pa / pc)))

    total = 0.0
    for i in oob:
        q = L if col[i] <= b else R
        q2 = L if col[pi[i]] <= b else R
        if q is not q2:
            total += kl(q, q2)
    assert pm[f] == pytest.approx(total / oob.size, rel=1e-12)
    assert np.count_nonzero(pm) <= 1


def test_permut_constant_column_is_zero():
    """Swapping in values of a constant column changes no prediction."""
    w, P = _small(importance=2, N=300, p=6, max_depth=5)
    X = w.X.copy()
    X[2, :] = 7
    P2 = oracle.BorutaProblem(X, w.y, **w.params(), N=w.N)
    live = np.arange(6, dtype=np.int32)
    sha = P2.shadow(1, live)
    _, _, pm = P2.tree(1, live, sha, 0, permut=True)
    assert pm[2] == 0.0


def _stump(task, C, N=600, p=6, B=8, seed=11, tree=1):
    """A depth-1 forest on raw seeded data (no generator): bins uniform in
    [0, B); labels uniform in [0, C) with column 0 shifting them, or targets
    at 2^-20 fixed point that depend on column 0."""
    rng = np.random.default_rng(seed)
    X = np.zeros((p, synth.pad16(N)), np.uint8)
    X[:, :N] = rng.integers(0, B, size=(p, N))
    if task & 1:
        y = (rng.standard_normal(N) * 2**20 + X[0, :N].astype(np.int64) * 2**19).astype(np.int64)
    else:
        y = ((rng.integers(0, C, size=N) + (X[0, :N] >= B // 2)) % C).astype(np.uint8)
    P = oracle.BorutaProblem(X, y, task | 2, n_trees=1, max_depth=1, n_bins=B, max_iter=1, seed=seed,
                             n_classes=C if task == 0 else 0, N=N)
    live = np.arange(p, dtype=np.int32)
    sha = P.shadow(1, live)
    nodes, _, pm = P.tree(1, live, sha, tree, permut=True)
    assert len(nodes) == 3 and nodes[0]["feature"] >= 0
    cols = np.concatenate([X[:, :N], sha])
    oob = np.flatnonzero(oracle.bootstrap(seed, 0, 1, tree, N) == 0)
    cnt = oracle.bootstrap(seed, 0, 1, tree, N)
    return nodes, pm, cols[int(nodes[0]["feature"])], P.permut_table(1), oob, y[:N], cnt


def test_permut_regression_stump_exact():
    """Alg. 3 with the squared-error loss of the paper's regression case, on a
    stump: the root feature's importance is (1/|OOB|) times the sum, over the
    OOB rows whose permuted value crosses the threshold, of the squared
    difference of the two leaf means in real units, ((S_L/n_L - S_R/n_R) *
    2^-20)^2 -- here in exact rationals from the raw targets, not from the
    oracle's node records.  Every other feature gets exactly 0.  (Checked to
    fail when the oracle's 2^-20 scale is dropped or its leaf mean is taken
    as an integer quotient.)"""
    nodes, pm, col, pi, oob, y, cnt = _stump(1, 1)
    b = int(nodes[0]["bin"])
    f = int(nodes[0]["feature"])
    N = col.size
    left = col <= b
    SL = sum(int(cnt[i]) * int(y[i]) for i in range(N) if left[i])
    nL = int(cnt[left].sum())
    SR = sum(int(cnt[i]) * int(y[i]) for i in range(N) if not left[i])
    nR = int(cnt[~left].sum())
    diff = (Fraction(SL, nL) - Fraction(SR, nR)) * Fraction(1, 2**20)
    crossing = sum(1 for i in oob if left[i] != left[pi[i]])
    want = diff * diff * crossing / len(oob)
    assert crossing > 0
    assert pm[f] == pytest.approx(float(want), rel=1e-13)
    assert np.count_nonzero(pm) == 1


@pytest.mark.parametrize("C", [3, 5])
def test_permut_multiclass_stump_kl(C):
    """Alg. 3 with the KL loss for C > 2 classes on a stump: for each OOB row
    whose permuted value crosses the threshold, KL(P~_q || P~_q') with
    P~_k = (c_k/n + eps) / (1 + C eps), q the row's own leaf -- computed
    here from the raw labels in exact rationals and 50-digit logarithms
    (decimal), so the normalisation 1 + C*eps, the direction of the
    divergence and the C library's log are all checked.  (Checked to fail
    when the oracle normalises with 1 + 2 eps, or swaps the two leaves.)"""
    import decimal

    nodes, pm, col, pi, oob, y, cnt = _stump(0, C)
    f, b = int(nodes[0]["feature"]), int(nodes[0]["bin"])
    N = col.size
    left = col <= b
    eps = Fraction(1e-7)

    def probs(side):
        c = [sum(int(cnt[i]) for i in range(N) if left[i] == side and y[i] == k) for k in range(C)]
        n = sum(c)
        return [(Fraction(ck, n) + eps) / (1 + C * eps) for ck in c]

    ctx = decimal.Context(prec=50)

    def dec(q):
        return ctx.divide(decimal.Decimal(q.numerator), decimal.Decimal(q.denominator))

    def kl(P, Q):
        return sum(ctx.multiply(dec(a), ctx.ln(dec(a / c))) for a, c in zip(P, Q))

    PL, PR = probs(True), probs(False)
    total = decimal.Decimal(0)
    for i in oob:
        if left[i] != left[pi[i]]:
            total += kl(PL, PR) if left[i] else kl(PR, PL)
    want = float(total / len(oob))
    assert want > 0
    assert pm[f] == pytest.approx(want, rel=1e-12)
    assert kl(PL, PR) != kl(PR, PL)  # the direction matters on this data
    assert np.count_nonzero(pm) == 1


# ---------------------------------------------------------------- Alg. 3 as printed

def _stump_forest(task, C, M=2, N=500, p=5, B=8, seed=21):
    """M depth-1 trees on raw seeded data (as _stump); returns the problem,
    its augmented columns, live set, shadow matrix, the trees' (feature, bin)
    and bootstrap counts, flush_index and the raw targets."""
    rng = np.random.default_rng(seed)
    X = np.zeros((p, synth.pad16(N)), np.uint8)
    X[:, :N] = rng.integers(0, B, size=(p, N))
    if task & 1:
        y = (rng.standard_normal(N) * 2**20 + X[0, :N].astype(np.int64) * 2**19
             - X[1, :N].astype(np.int64) * 2**18).astype(np.int64)
    else:
        y = ((rng.integers(0, C, size=N) + (X[0, :N] >= B // 2) + (X[1, :N] >= B // 2)) % C).astype(np.uint8)
    P = oracle.BorutaProblem(X, y, task | 2, n_trees=M, max_depth=1, n_bins=B, max_iter=1, seed=seed,
                             n_classes=C if task == 0 else 0, permut_form=1, N=N)
    live = np.arange(p, dtype=np.int32)
    sha = P.shadow(1, live)
    cols = np.concatenate([X[:, :N], sha])
    splits, cnts = [], []
    for tau in range(M):
        nodes, _, _ = P.tree(1, live, sha, tau)
        assert nodes[0]["feature"] >= 0
        splits.append((int(nodes[0]["feature"]), int(nodes[0]["bin"])))
        cnts.append(oracle.bootstrap(seed, 0, 1, tau, N))
    return P, cols, live, sha, splits, cnts, P.permut_table(1), y[:N]


def _forest_pred(cols, splits, leafval, i, f=None, pi_i=None):
    """Mean over trees of the leaf value reached by row i (column f read at
    row pi_i), in exact rationals."""
    total = Fraction(0)
    for tau, (g, b) in enumerate(splits):
        v = cols[g][pi_i] if g == f else cols[g][i]
        total += leafval[tau][bool(v <= b)]
    return total / len(splits)


def test_forest_permut_regression_two_stumps_exact():
    """Alg. 3 as printed, regression: the model is the forest (the mean of
    the trees' leaf means), the rows are all N rows, and imp[f] is the mean
    squared difference between the forest's prediction and its prediction
    with column f read at flush_index -- recomputed here in exact rationals
    from the raw targets for a forest of two stumps.  Columns that no tree
    splits on get exactly 0.  (Checked to fail when the forest mean drops
    its 1/M, when the mean runs over OOB rows only, or when the loss is
    taken against the true targets.)"""
    P, cols, live, sha, splits, cnts, pi, y = _stump_forest(1, 1)
    N = cols.shape[1]
    leafval = []
    for (g, b), cnt in zip(splits, cnts):
        left = cols[g] <= b
        vals = {}
        for side in (True, False):
            m = left == side
            vals[side] = Fraction(int((cnt[m].astype(object) * y[m].astype(object)).sum()), int(cnt[m].sum()))
        leafval.append(vals)
    imp = P.forest_permut(1, live, sha)
    used = {g for g, _ in splits}
    for f in range(cols.shape[0]):
        if f not in used:
            assert imp[f] == 0.0
            continue
        tot = Fraction(0)
        for i in range(N):
            d = (_forest_pred(cols, splits, leafval, i) - _forest_pred(cols, splits, leafval, i, f, pi[i]))
            tot += (d * Fraction(1, 2**20)) ** 2
        assert imp[f] == pytest.approx(float(tot / N), rel=1e-12)
        assert imp[f] > 0


@pytest.mark.parametrize("C", [2, 3])
def test_forest_permut_classification_two_stumps_kl(C):
    """Alg. 3 as printed, classification: the forest's predicted class
    probabilities are the mean over trees of the leaves' class fractions;
    imp[f] is the mean over all rows of KL(P~_base || P~_perm) with
    P~_k = (P_k + eps) / (1 + C eps) -- recomputed from the raw labels in
    exact rationals and 50-digit logarithms for a forest of two stumps."""
    import decimal

    P, cols, live, sha, splits, cnts, pi, y = _stump_forest(0, C)
    N = cols.shape[1]
    eps = Fraction(1e-7)
    ctx = decimal.Context(prec=50)

    def dec(q):
        return ctx.divide(decimal.Decimal(q.numerator), decimal.Decimal(q.denominator))

    leafvals = []  # per class: per tree: {side: fraction}
    for k in range(C):
        per_tree = []
        for (g, b), cnt in zip(splits, cnts):
            left = cols[g] <= b
            per_tree.append({side: Fraction(int(cnt[(left == side) & (y == k)].sum()), int(cnt[left == side].sum()))
                             for side in (True, False)})
        leafvals.append(per_tree)
    imp = P.forest_permut(1, live, sha)
    used = {g for g, _ in splits}
    for f in range(cols.shape[0]):
        if f not in used:
            assert imp[f] == 0.0
            continue
        tot = decimal.Decimal(0)
        for i in range(N):
            kl = decimal.Decimal(0)
            for k in range(C):
                a = (_forest_pred(cols, splits, leafvals[k], i) + eps) / (1 + C * eps)
                c = (_forest_pred(cols, splits, leafvals[k], i, f, pi[i]) + eps) / (1 + C * eps)
                if a != c:
                    kl += ctx.multiply(dec(a), ctx.ln(dec(a / c)))
            tot += kl
        assert imp[f] == pytest.approx(float(tot / N), rel=1e-11)
        assert imp[f] > 0


def test_forest_permut_invariants_and_iteration():
    """Alg. 3 as printed on a deeper forest: importances are >= 0, exactly 0
    for columns no tree splits on and for a constant column; with
    permut_form = 1 the iteration's hit statistic is that single row."""
    w, _ = _small(importance=2, N=300, p=8, n_trees=6, max_depth=5)
    X = w.X.copy()
    X[2, :] = 3
    P = oracle.BorutaProblem(X, w.y, **w.params(), N=w.N, permut_form=1)
    live = np.arange(8, dtype=np.int32)
    sha = P.shadow(1, live)
    imp = P.forest_permut(1, live, sha)
    used = set()
    for tau in range(6):
        nodes, _, _ = P.tree(1, live, sha, tau)
        used |= {int(f) for f in nodes["feature"] if f >= 0}
    assert (imp >= 0).all() and imp[2] == 0.0
    for j in range(imp.size):
        if j not in used:
            assert imp[j] == 0.0
    out = P.iteration(1, np.zeros(8, np.int8), np.zeros(8, np.int32))
    np.testing.assert_array_equal(out["s"], imp)
    np.testing.assert_array_equal(out["imp"], imp[None, :])
    smax = imp[8:].max()
    np.testing.assert_array_equal(out["hits"], (imp[:8] > smax).astype(np.int32))


# ---------------------------------------------------------------- statistics

def test_zscore_closed_forms():
    """One tree: sd = 0, so Z is 0 for zero mean and +inf otherwise; with the
    mean statistic, s is the single tree's importance row."""
    w, P = _small(N=300, p=8, n_trees=1, max_iter=1)
    out = P.iteration(1, np.zeros(8, np.int8), np.zeros(8, np.int32))
    imp = out["imp"][0]
    assert np.all(out["s"][imp == 0] == 0.0) and np.all(np.isinf(out["s"][imp > 0]))
    w2, P2 = _small(N=300, p=8, n_trees=1, max_iter=1, )
    P2.c.stat = 1
    out2 = P2.iteration(1, np.zeros(8, np.int8), np.zeros(8, np.int32))
    np.testing.assert_array_equal(out2["s"], out2["imp"][0])


def test_iteration_statistics_from_importance_rows():
    """Mean, sd (M-1), Z, shadow max and hits recomputed from the dumped
    importance matrix with exactly rounded sums (math.fsum)."""
    w, P = _small(N=400, p=10, n_trees=7, max_iter=1)
    state = np.zeros(10, np.int8)
    state[3] = -1
    state[5] = 1
    out = P.iteration(1, state, np.zeros(10, np.int32))
    imp, s = out["imp"], out["s"]
    M = imp.shape[0]
    live = np.flatnonzero(state >= 0)
    for j in range(imp.shape[1]):
        mean = math.fsum(imp[:, j]) / M
        sd = math.sqrt(math.fsum([(v - mean) * (v - mean) for v in imp[:, j]]) / (M - 1))
        z = (0.0 if mean == 0 else math.inf) if sd == 0 else mean / (sd / math.sqrt(M))
        assert s[j] == z
    smax = s[live.size:].max()
    assert out["shadow_max"] == smax
    for a, j in enumerate(live):
        assert out["hits"][j] == int(s[a] > smax)
        assert out["hist"][j] == s[a]
    assert np.isnan(out["hist"][3])
    assert out["state"][3] == -1 and out["state"][5] == 1


def test_decision_thresholds():
    """Earliest possible decision: accept needs 2^-t < alpha/m, so with
    alpha = 0.01 and m = 50 undecided features the first accept can come at
    t = ceil(log2(m/alpha)) = 13 and never before."""
    m, alpha = 50, 0.01
    t_min = math.ceil(math.log2(m / alpha))
    assert t_min == 13
    assert oracle.binom_tails(t_min, t_min)[0] < alpha / m
    assert not oracle.binom_tails(t_min - 1, t_min - 1)[0] < alpha / m


def _alg1_test(t, alpha, hits, state):
    """Alg. 1's test() restated with exact rationals: m = features undecided
    before the test (fixed for the whole test); for each undecided j,
    P_acc = P(Bin(t, 1/2) >= h_j) and P_rej = P(Bin(t, 1/2) <= h_j) from
    math.comb; accept if P_acc < alpha/m, else reject if P_rej < alpha/m."""
    m = sum(1 for s in state if s == 0)
    out = list(state)
    if m == 0:
        return out
    thr = Fraction(alpha) / m
    for j, s in enumerate(state):
        if s != 0:
            continue
        h = int(hits[j])
        up = Fraction(sum(math.comb(t, k) for k in range(h, t + 1)), 2**t)
        lo = Fraction(sum(math.comb(t, k) for k in range(0, h + 1)), 2**t)
        if up < thr:
            out[j] = 1
        elif lo < thr:
            out[j] = -1
    return out


def test_decision_step_cases():
    """Hand-built cases of Alg. 1's test, each fixing one rule:
    (a) strict <: alpha/m = 2^-t exactly; h = t gives P_acc = alpha/m and
        h = 0 gives P_rej = alpha/m, so nothing is decided (fails if the
        oracle compares with <=);
    (b) Bonferroni m = undecided features, not p: with 6 of 10 columns
        decided, alpha = 2^-7 accepts at t = 10 with m = 4 but would not
        with m = 10 (fails if the oracle counts every column);
    (c) m is fixed before the test: the feature accepted first does not
        lower m for the next one (fails if m is decremented as features
        are decided);
    (d) accept is tried before reject: with alpha/m = 0.9 both tails of
        h = 2 at t = 4 (11/16 each) are below it (fails if reject is
        tried first)."""
    # (a)
    st = oracle.decide(10, 2.0**-8, [10, 0, 10, 3, 3, 0], [0, -1, 0, 1, 0, 0])
    assert st.tolist() == _alg1_test(10, 2.0**-8, [10, 0, 10, 3, 3, 0], [0, -1, 0, 1, 0, 0])
    assert st.tolist() == [0, -1, 0, 1, 0, 0]  # P_rej of h = 0 is also exactly alpha/m
    # (b)
    state = [1, 1, 1, -1, -1, -1, 0, 0, 0, 0]
    hits = [10, 10, 10, 0, 0, 0, 10, 10, 5, 10]
    st = oracle.decide(10, 2.0**-7, hits, state)
    assert st.tolist() == _alg1_test(10, 2.0**-7, hits, state) == [1, 1, 1, -1, -1, -1, 1, 1, 0, 1]
    assert _alg1_test(10, 2.0**-7, hits, [0] * 10)[6] == 0
    # (c)
    st = oracle.decide(10, 2.0**-6, [10, 9], [0, 0])
    assert st.tolist() == _alg1_test(10, 2.0**-6, [10, 9], [0, 0]) == [1, 0]
    # (d)
    st = oracle.decide(4, 0.9, [2], [0])
    assert st.tolist() == _alg1_test(4, 0.9, [2], [0]) == [1]


def test_decision_step_random_runs():
    """Random hit sequences over many iterations, with m shrinking as
    features are decided: the oracle's test equals the exact restatement
    after every iteration."""
    rng = np.random.default_rng(3)
    checked = 0
    for run in range(40):
        p = int(rng.integers(1, 40))
        alpha = float(rng.choice([0.01, 0.05, 0.2, 0.9]))
        rate = rng.uniform(0, 1, size=p)
        state = np.zeros(p, np.int8)
        hits = np.zeros(p, np.int32)
        for t in range(1, 60):
            hits += (rng.random(p) < rate) & (state >= 0)
            want = _alg1_test(t, alpha, hits, state.tolist())
            state = oracle.decide(t, alpha, hits, state)
            assert state.tolist() == want, (run, t)
            checked += 1
            if not (state == 0).any():
                break
    assert checked > 500


# ---------------------------------------------------------------- after the run

def test_final_ranking_hand_worked():
    """Alg. 1's final ranking (reading of its garbled rankdata line):
    accepted 1, tentative 2, rejected 3, 4, ... by descending median of the
    feature's history over the iterations it was in play (NaN skipped, even
    counts take the mean of the two middle values), equal medians to the
    lower index.  Worked by hand: medians of the rejected columns 2, 3, 4, 6
    are 0.5, 0.7, 0.5 and (0.1 + 0.3) / 2 = 0.2, so column 3 ranks 3, then
    2 (lower index of the tie), 4, 6.  (Fails when the order is ascending,
    the tie goes to the higher index, or the even median takes one value.)"""
    nan = float("nan")
    decision = np.array([1, 0, -1, -1, -1, 1, -1], np.int8)
    hist = np.array([[0.9, 0.1, 0.5, 0.7, 0.6, 0.8, 0.1],
                     [0.8, 0.2, 0.4, 0.9, 0.5, 0.9, 0.3],
                     [0.9, 0.3, 0.6, 0.2, 0.4, 0.7, nan],
                     [nan, nan, nan, nan, nan, nan, nan]])
    got = oracle.rank(decision, hist, 3)
    assert got.tolist() == [1, 2, 4, 3, 5, 1, 6]


def test_median_selection_matches_numpy():
    """Multi-seed selection (reading of the paper's 20-seed median rule):
    per run the median of each feature's history and of the shadow maxima,
    then the median over runs; a feature is selected when its median beats
    the shadows' -- against numpy's nanmedian/median on random histories
    with NaN gaps and runs of different lengths."""
    rng = np.random.default_rng(5)
    for n_runs in (1, 2, 5, 20):
        T, p = 12, 9
        runs = []
        for r in range(n_runs):
            it = int(rng.integers(1, T + 1))
            h = np.full((T, p), np.nan)
            h[:it] = rng.random((it, p))
            h[:it][rng.random((it, p)) < 0.2] = np.nan
            h[0] = rng.random(p)  # every feature in play at t = 1
            sm = np.full(T, np.nan)
            sm[:it] = rng.random(it)
            runs.append(dict(imp_history=h, shadow_max=sm, iterations=it))
        med, ms, sel = oracle.select_median(runs)
        want = np.median(np.stack([np.nanmedian(r["imp_history"][:r["iterations"]], axis=0) for r in runs]), axis=0)
        want_s = np.median([np.nanmedian(r["shadow_max"][:r["iterations"]]) for r in runs])
        np.testing.assert_array_equal(med, want)
        assert ms == want_s
        np.testing.assert_array_equal(sel, (want > want_s).astype(np.int8))
    # strict: a feature whose median equals the shadows' is not selected
    h = np.array([[0.5, 0.6], [0.3, 0.6], [0.4, 0.6]])
    med, ms, sel = oracle.select_median([dict(imp_history=h, shadow_max=np.array([0.2, 0.4, 0.9]), iterations=3)])
    assert med.tolist() == [0.4, 0.6] and ms == 0.4 and sel.tolist() == [0, 1]


# ---------------------------------------------------------------- end to end

@pytest.mark.slow
@pytest.mark.parametrize("tie_break", [0, 1])
def test_planted_informative_set_is_found(tie_break):
    """Binary N=1000, p=50: all 10 planted class-conditional columns are
    accepted within 20 iterations under either tie rule, and no decision
    comes before t = 13.  With ties to the feature drawn first (tie_break
    = 1) no noise column is accepted and at least 36 are rejected; with
    ties to the lowest index (the default) real columns win the many ties
    of tiny nodes against the shadows, whose indices are all higher, so
    some noise columns can be accepted too."""
    w = synth.binary_small()
    P = oracle.BorutaProblem(w.X, w.y, **w.params(), N=w.N, tie_break=tie_break)
    r = P.run()
    acc = set(np.flatnonzero(r["decision"] == 1).tolist())
    assert set(w.informative.tolist()) <= acc
    if tie_break == 1:
        assert acc == set(w.informative.tolist())
        assert (r["decision"] == -1).sum() >= 36
    assert r["iterations"] <= 20
    first = np.isnan(r["imp_history"]).any(axis=1).argmax()
    assert first == 0 or first >= 13
