"""Pins of the CPU oracle against what the paper and mathematics fix.

Every test here checks the oracle against something other than itself:
published known-answer vectors, exact rational arithmetic, a library routine
(scipy chi^2 quantiles, numpy binary search and sorting), the distribution the
paper's lemmas state, exact invariants of the paper's definitions, or brute
force on tiny inputs.
"""
from fractions import Fraction

import numpy as np
import pytest
import scipy.stats as st

import oracle
import workloads
from tests.golden.kat import philox_kat


# ---------------------------------------------------------------- Philox --
def test_philox_known_answers():
    for ctr, key, want in philox_kat():
        got = oracle.philox4x32_10(ctr, key)
        assert [int(v) for v in got] == want


# ------------------------------------------------------ Eq. 1 projection --
def test_projection_matrix_is_standard_normal():
    A = oracle.projection_matrix(64, 1000, 7)
    assert A.dtype == np.float32
    # Eq. 1: entries i.i.d. N(0,1); both Box-Muller outputs separately.
    assert st.kstest(A[:, 0::2].ravel(), "norm").pvalue > 1e-4
    assert st.kstest(A[:, 1::2].ravel(), "norm").pvalue > 1e-4
    # pairs from one Philox block are uncorrelated
    assert abs(np.corrcoef(A[:, 0::2].ravel(), A[:, 1::2].ravel())[0, 1]) < 0.02
    # deterministic in the seed, different across seeds
    assert np.array_equal(A, oracle.projection_matrix(64, 1000, 7))
    assert not np.array_equal(A, oracle.projection_matrix(64, 1000, 8))


def _rn32_exact(fr):
    """FP32 nearest to an exact rational, ties to even (independent of the oracle)."""
    if fr == 0:
        return np.float32(0.0)
    f = np.float32(float(fr))
    if np.isinf(f):
        return f
    cands = [np.nextafter(f, np.float32(-np.inf)), f, np.nextafter(f, np.float32(np.inf))]

    def key(c):
        return (abs(Fraction(float(c)) - fr), int(np.array(c, np.float32).view(np.uint32)) & 1)
    return min(cands, key=key)


def _exact_dot(a, x):
    return sum((Fraction(float(u)) * Fraction(float(v)) for u, v in zip(a, x)), Fraction(0))


@pytest.mark.parametrize("d", [1, 2, 7, 128, 960])
def test_dot_rn32_equals_exact_rational(d):
    g = np.random.default_rng(d)
    for trial in range(30):
        a = g.normal(size=d).astype(np.float32)
        x = (g.normal(size=d) * 2.0 ** g.integers(-40, 40, size=d)).astype(np.float32)
        if trial % 3 == 0:  # heavy cancellation
            x[: d // 2] = (g.normal(size=d // 2) * 1e6).astype(np.float32)
        want = _rn32_exact(_exact_dot(a, x))
        got = oracle.dot_rn32(a, x)
        assert np.array(got).view(np.uint32) == np.array(want).view(np.uint32), (d, trial)


def test_dot_rn32_special_cases():
    f32 = np.float32
    cases = [
        ([2.0 ** 24, 1.0], [1.0, 1.0]),          # 2^24+1: tie -> even (2^24)
        ([2.0 ** 24, 3.0], [1.0, 1.0]),          # 2^24+3: tie -> even (2^24+4)
        ([1e20, 1.0, -1e20], [1.0, 1.0, 1.0]),   # exact cancellation -> 1
        ([1e-20, 3e-21], [1e-20, 7e-21]),        # subnormal result
        ([1e-30], [1e-30]),                      # underflows to 0
        ([3e38, 3e38], [1.0, 1.0]),              # overflows to +inf
        ([-3e38, -3e38], [1.0, 1.0]),            # overflows to -inf
        ([2.0 ** -149, 2.0 ** -149], [0.5, 0.5]),  # exactly 2^-149
        ([2.0 ** -149], [0.5]),                  # tie at 2^-150 -> even (0)
        ([2.0 ** -149], [0.75]),                 # above the tie -> 2^-149
    ]
    for a, x in cases:
        a, x = np.array(a, f32), np.array(x, f32)
        want = _rn32_exact(_exact_dot(a, x))
        got = oracle.dot_rn32(a, x)
        assert np.array(got).view(np.uint32) == np.array(want).view(np.uint32), (a, x, got, want)
    # exact zero, from either sign, is +0
    z = oracle.dot_rn32(np.array([-1.0], f32), np.array([0.0], f32))
    assert np.array(z).view(np.uint32) == 0


def test_project_matches_integer_matmul():
    # Integer inputs: the exact product is an integer the FP32 grid holds,
    # so the projection equals int64 matmul (pins row/column indexing).
    g = np.random.default_rng(3)
    X = g.integers(-100, 101, (37, 19)).astype(np.float32)
    A = g.integers(-10, 11, (12, 19)).astype(np.float32)
    P = oracle.project(X, A)
    want = (X.astype(np.int64) @ A.astype(np.int64).T).astype(np.float32)
    assert np.array_equal(P, want)


def _random_pair_ratio(K, d, seeds):
    g = np.random.default_rng(11)
    x = g.normal(size=(2, d)).astype(np.float32)
    s2 = float(np.sum((x[0].astype(np.float64) - x[1]) ** 2))
    out = []
    for s in seeds:
        A = oracle.projection_matrix(K, d, s)
        P = oracle.project(x, A).astype(np.float64)
        out.append(np.sum((P[0] - P[1]) ** 2) / s2)
    return np.array(out)


def test_lemma1_projected_distance_is_chi2():
    # Lemma 1: s'^2 / s^2 ~ chi^2(K) over the draw of the projection.
    K = 16
    r = _random_pair_ratio(K, 24, range(1500))
    assert st.kstest(r, st.chi2(K).cdf).pvalue > 1e-4


def test_lemma3_eps_probability():
    # Lemma 2 with alpha1: Pr[s' > eps s] = alpha1 = exp(-1/L).
    K, L = 16, 4
    e2 = oracle.eps2(K, L)
    r = _random_pair_ratio(K, 24, range(2000, 4000))
    frac = np.mean(r > e2)
    a1 = np.exp(-1.0 / L)
    assert abs(frac - a1) < 4.5 * np.sqrt(a1 * (1 - a1) / r.size)


# ------------------------------------------------------- Eq. 2 / Lemma 3 --
@pytest.mark.parametrize("K", [1, 2, 3, 4, 5, 8, 15, 16, 17])
def test_chi2_tail_matches_scipy(K):
    for x in [0.01, 0.5, 1.0, 3.7, 10.0, 25.0, 60.0]:
        assert oracle.chi2_sf(x, K) == pytest.approx(st.chi2.sf(x, K), rel=1e-9, abs=1e-300)


@pytest.mark.parametrize("K,L", [(16, 4), (4, 16), (8, 2), (12, 6), (3, 5), (16, 1)])
def test_eps2_is_upper_quantile(K, L):
    # Eq. 2: eps^2 = chi^2_{alpha1}(K) with L = -1/ln(alpha1).
    want = st.chi2.isf(np.exp(-1.0 / L), K)
    assert oracle.eps2(K, L) == pytest.approx(want, rel=1e-9)


def test_eps2_paper_defaults():
    # K=16, L=4 (Sec. V-B1): alpha1 = e^{-1/4}; eps^2 = 11.4820... and the
    # guarantee constant 1/2 - 1/e of Theorems 1-3.
    assert oracle.eps2(16, 4) == pytest.approx(11.482032, rel=1e-6)
    T = oracle.level_table(oracle.eps2(16, 4), 1.5)
    j = np.arange(oracle.NLEV) + oracle.JMIN
    assert T[-1] == np.inf
    assert np.all(T[1:] >= T[:-1])
    assert T[127] == np.float32(oracle.eps2(16, 4))  # j = 0, r = 1
    np.testing.assert_allclose(T[100:150], (11.482031866 * 1.5 ** (2.0 * j[100:150])).astype(np.float32),
                               rtol=1e-6)


# -------------------------------------------------- sampling / encoding --
def test_sample_is_bernoulli_fraction():
    n = 100_000
    ids = oracle.sample(n, 5, 0.1, 256)
    assert np.all(np.diff(ids) > 0)
    assert abs(ids.size - 0.1 * n) < 5 * np.sqrt(n * 0.1 * 0.9)
    assert np.array_equal(ids, oracle.sample(n, 5, 0.1, 256))
    # too small a sample: every point is used
    assert np.array_equal(oracle.sample(1000, 5, 0.1, 256), np.arange(1000))
    assert np.array_equal(oracle.sample(5000, 5, 1.0, 256), np.arange(5000))


@pytest.fixture(scope="module")
def small_proj():
    X, _, _ = workloads.workload("c1", n=20_000, m=1)
    X = X[:, :24].copy()
    A = oracle.projection_matrix(8, X.shape[1], 3)
    P = oracle.project(X, A)
    s = oracle.sample(X.shape[0], 3, 0.1, 16)
    return X, P, s


@pytest.mark.parametrize("N_r", [2, 16, 256])
def test_breakpoints_equal_frequency(small_proj, N_r):
    # Dynamic encoding (Sec. III-A): the interior breakpoints cut the sorted
    # sample into equal-count regions.  With distinct values every region but
    # the last holds exactly floor(m/N_r) sample points.
    X, P, s = small_proj
    B = oracle.breakpoints(P, s, N_r)
    codes = oracle.encode(P, B)
    m = s.size
    q = m // N_r
    for t in range(P.shape[1]):
        assert np.unique(P[s, t]).size == m
        cnt = np.bincount(codes[s, t], minlength=N_r)
        assert np.all(cnt[: N_r - 1] == q), cnt
        assert cnt[N_r - 1] == m - (N_r - 1) * q
        assert B[t, 0] == P[:, t].min() and B[t, N_r] == P[:, t].max()
        assert np.all(np.diff(B[t]) >= 0)
        # whole data: about n/N_r per region (binomial spread)
        full = np.bincount(codes[:, t], minlength=N_r)
        p = 1.0 / N_r
        n = P.shape[0]
        tol = 6 * n * np.sqrt(p * (1 - p) / m) + 6 * np.sqrt(n * p)
        assert np.all(np.abs(full[: N_r - 1] - n * p) < tol)


def test_encode_is_binary_search(small_proj):
    # Alg. 1: the code is the region found by BinarySearch; first region on ties.
    X, P, s = small_proj
    N_r = 16
    B = oracle.breakpoints(P, s, N_r)
    codes = oracle.encode(P, B)
    for t in range(P.shape[1]):
        want = np.searchsorted(B[t, 1:N_r], P[:, t], side="left")
        assert np.array_equal(codes[:, t], want)
    # a value exactly on a breakpoint takes the lower region
    Pt = B[:, 5][None, :].copy()
    assert np.all(oracle.encode(Pt, B)[0] <= 4)


# --------------------------------------------------------------- DE-Tree --
def _small_index(n=6000, d=32, L=2, K=8, N_r=16, M=16, box_mode=0, insertion_order=0, seed=1):
    X, Q, _ = workloads.workload("c1", n=n, m=8)
    X, Q = X[:, :d].copy(), Q[:, :d].copy()
    ix = oracle.Index(X, L=L, K=K, N_r=N_r, seed=seed, frac=0.1, M=M, box_mode=box_mode,
                      insertion_order=insertion_order)
    return ix, X, Q


def _first_key(codes_t, K, bbits):
    key = np.zeros(codes_t.shape[0], np.int64)
    for j in range(K):
        key |= ((codes_t[:, j] >> (bbits - 1)) & 1).astype(np.int64) << (K - 1 - j)
    return key


@pytest.mark.parametrize("box_mode", [0, 1])
def test_tree_invariants(box_mode):
    ix, X, _ = _small_index(box_mode=box_mode)
    arr = ix.arrays()
    K, L, N_r, M, bb = ix.K, ix.L, ix.N_r, ix.M, 4
    for t in range(L):
        tr = ix.tree(t)
        codes = arr["codes"][:, t * K:(t + 1) * K]
        perm, begin = tr["perm"], tr["begin"]
        nl = begin.size - 1
        assert np.array_equal(np.sort(perm), np.arange(ix.n))  # each point in exactly one leaf
        sizes = np.diff(begin)
        assert np.all(sizes > 0)
        fk = _first_key(codes, K, bb)
        prev_key = -1
        for lf in range(nl):
            mem = perm[begin[lf]:begin[lf + 1]]
            assert np.all(np.diff(mem) > 0)  # ascending ids
            assert np.all(tr["leaf_of"][mem] == lf)
            nb = tr["nb"][lf].astype(np.int64)
            # members share the leaf's iSAX prefix
            pref = codes[mem] >> (bb - nb)
            assert np.all(pref == pref[0])
            plo = (pref[0] << (bb - nb)).astype(np.uint8)
            phi = (plo.astype(np.int64) + (1 << (bb - nb)) - 1).astype(np.uint8)
            if box_mode == 0:
                assert np.array_equal(tr["lo"][lf], plo) and np.array_equal(tr["hi"][lf], phi)
            else:
                assert np.array_equal(tr["lo"][lf], codes[mem].min(0))
                assert np.array_equal(tr["hi"][lf], codes[mem].max(0))
            # Alg. 2: leaves hold at most max_size unless nothing is left to split
            assert mem.size <= M or np.all(nb == bb)
            # canonical order: first-layer key ascending
            assert fk[mem[0]] >= prev_key
            prev_key = fk[mem[0]]


def test_tree_first_split_is_most_even():
    # Sec. III-B: a node splits on the dimension that most evenly partitions
    # its points (ties: smallest dimension), children in bit order.
    ix, X, _ = _small_index(n=8000, M=16)
    arr = ix.arrays()
    K, bb = ix.K, 4
    for t in range(ix.L):
        tr = ix.tree(t)
        codes = arr["codes"][:, t * K:(t + 1) * K]
        fk = _first_key(codes, K, bb)
        for key in np.unique(fk):
            mem = np.nonzero(fk == key)[0]
            leaves = np.unique(tr["leaf_of"][mem])
            if mem.size <= ix.M:
                assert leaves.size == 1 and np.all(tr["nb"][leaves[0]] == 1)
                continue
            bits = (codes[mem] >> (bb - 2)) & 1            # next bit, every dim
            n1 = bits.astype(np.int64).sum(0)
            jstar = int(np.argmin(np.abs(mem.size - 2 * n1)))
            assert np.all(tr["nb"][leaves][:, jstar] >= 2)
            # child 0 (bit 0) precedes child 1
            order = tr["leaf_of"][mem]
            b = bits[:, jstar]
            if b.min() == 0 and b.max() == 1:
                assert order[b == 0].max() < order[b == 1].min()


def test_bulk_equals_insertion_when_no_split():
    ix_b, _, _ = _small_index(n=3000, M=10 ** 9)
    ix_i, _, _ = _small_index(n=3000, M=10 ** 9, insertion_order=1)
    for t in range(ix_b.L):
        a, b = ix_b.tree(t), ix_i.tree(t)
        for key in ("perm", "begin", "lo", "hi", "nb", "leaf_of"):
            assert np.array_equal(a[key], b[key]), key


def test_insertion_order_leaves_respect_max_size():
    ix, _, _ = _small_index(n=6000, M=16, insertion_order=1)
    for t in range(ix.L):
        tr = ix.tree(t)
        sizes = np.diff(tr["begin"])
        full = np.all(tr["nb"] == 4, axis=1)
        assert np.all((sizes <= 16) | full)


# ---------------------------------------------------------- lower bound --
@pytest.mark.parametrize("box_mode", [0, 1])
def test_lower_bound_is_sound(box_mode):
    # Sec. IV-C: the node lower bound never exceeds the projected distance of
    # any point in the node (same FP32 operation order on both sides).
    ix, X, Q = _small_index(box_mode=box_mode)
    arr = ix.arrays()
    K = ix.K
    for t in range(ix.L):
        tr = ix.tree(t)
        for q in Q[:4]:
            lb2 = ix.leaf_lb2(t, q)
            qp = oracle.project(q[None, :], arr["A"][t * K:(t + 1) * K])[0]
            Pt = arr["P"][:, t * K:(t + 1) * K]
            d2 = np.zeros(ix.n, np.float32)
            for j in range(K):
                diff = (Pt[:, j] - qp[j]).astype(np.float32)
                d2 = (d2 + diff * diff).astype(np.float32)
            assert np.all(lb2[tr["leaf_of"]] <= d2)
            assert lb2.min() >= 0


# --------------------------------------------------------------- queries --
def _numpy_knn(X, q, k):
    d = np.sqrt(((X.astype(np.float64) - q.astype(np.float64)) ** 2).sum(1))
    order = np.lexsort((np.arange(X.shape[0]), d))[:k]
    return order, d[order]


def test_bruteforce_knn_matches_numpy():
    X, Q, _ = workloads.workload("c1", n=3000, m=5)
    ids, dists = oracle.bruteforce_knn(X, Q, 17)
    for i in range(5):
        wi, wd = _numpy_knn(X, Q[i], 17)
        assert np.array_equal(ids[i], wi)
        np.testing.assert_allclose(dists[i], wd, rtol=1e-12)


def test_query_with_unreachable_budget_is_exact_knn():
    ix, X, Q = _small_index(n=2000)
    for q in Q[:3]:
        r = ix.query(q, 10, beta=2.0)  # beta*n + k > n
        wi, wd = _numpy_knn(X, q, 10)
        assert np.array_equal(r["ids"], wi)
        np.testing.assert_allclose(r["dists"], wd, rtol=1e-12)
        assert r["S_size"] == ix.n


def _expected_S(ix, q, k, beta, c, jstar):
    """Alg. 5 at r_min, recomputed from the exported leaves with numpy."""
    T = ix.level_table(c)
    tau = int(np.ceil(beta * ix.n)) + k
    thr = T[jstar - oracle.JMIN]
    inS = np.zeros(ix.n, bool)
    for t in range(ix.L):
        tr = ix.tree(t)
        lb2 = ix.leaf_lb2(t, q)
        hit = np.nonzero(lb2 <= thr)[0]
        hit = hit[np.lexsort((hit, lb2[hit]))]
        for lf in hit:
            inS[tr["perm"][tr["begin"][lf]:tr["begin"][lf + 1]]] = True
            if inS.sum() >= tau:
                return inS, t
    return inS, ix.L - 1


@pytest.mark.parametrize("box_mode", [0, 1])
@pytest.mark.parametrize("beta,k", [(0.1, 10), (0.02, 5), (0.3, 50)])
def test_query_magic_rmin_and_candidates(box_mode, beta, k):
    ix, X, Q = _small_index(box_mode=box_mode, n=6000)
    c = 1.5
    T = ix.level_table(c)
    tau = int(np.ceil(beta * ix.n)) + k
    trees = [ix.tree(t) for t in range(ix.L)]
    for q in Q[:4]:
        r = ix.query(q, k, beta=beta, c=c)
        js = r["jstar"]
        lbp = [ix.leaf_lb2(t, q)[trees[t]["leaf_of"]] for t in range(ix.L)]

        def N(j):
            return int(np.any([lbp[t] <= T[j - oracle.JMIN] for t in range(ix.L)], axis=0).sum())
        # magic r_min (Sec. V-B1): |S(r_min)| >= tau and |S(r_min / c)| < tau
        assert N(js) >= tau
        if js > oracle.JMIN:
            assert N(js - 1) < tau
        inS, ist = _expected_S(ix, q, k, beta, c, js)
        assert ist == r["istar"]
        S = r["S"]
        assert np.unique(S).size == S.size == r["S_size"]
        assert np.array_equal(np.sort(S), np.nonzero(inS)[0])
        maxleaf = max(np.diff(tr["begin"]).max() for tr in trees)
        assert tau <= S.size < tau + maxleaf
        # verification (Alg. 5): exact top-k of S, ties by id
        wi, wd = _numpy_knn(X[S], q, k)
        assert np.array_equal(r["ids"], S[wi])
        np.testing.assert_allclose(r["dists"], wd, rtol=1e-12)


def test_guarantee_c2_k_ann():
    # Theorem 2: every returned o_i is within c^2 of the i-th true neighbour
    # with probability >= 1/2 - 1/e when beta >= the theoretical beta.
    c, k, beta = 1.5, 10, 0.1
    ok = []
    for seed in range(6):
        X, Q, _ = workloads.workload("c1", n=3000, m=10)
        X = X[:, :32] + np.float32(seed)
        Q = Q[:, :32] + np.float32(seed)
        ix = oracle.Index(X, L=4, K=16, N_r=256, seed=seed, frac=0.1, M=64)
        ids, dists = oracle.bruteforce_knn(X, Q, k)
        for i in range(Q.shape[0]):
            r = ix.query(Q[i], k, beta=beta, c=c, want_S=False)
            ok.append(bool(np.all(r["dists"] <= c * c * dists[i] + 1e-9)))
    assert np.mean(ok) >= 0.5 - 1.0 / np.e


# ------------------------------------- Alg. 3 as printed, Alg. 4 (r,c)-ANN --
def _proj_dist2(ix, arr, t, q):
    """FP32 squared projected distances of every point in tree t (numpy)."""
    K = ix.K
    qp = oracle.project(q[None, :], arr["A"][t * K:(t + 1) * K])[0]
    Pt = arr["P"][:, t * K:(t + 1) * K]
    d2 = np.zeros(ix.n, np.float32)
    for j in range(K):
        diff = (Pt[:, j] - qp[j]).astype(np.float32)
        d2 = (d2 + diff * diff).astype(np.float32)
    return d2


@pytest.mark.parametrize("box_mode", [0, 1])
def test_upper_bound_is_sound(box_mode):
    # Sec. IV-C / Fig. 6: the node upper bound is never below the projected
    # distance of a point in the node, and never below the lower bound.
    ix, X, Q = _small_index(box_mode=box_mode)
    arr = ix.arrays()
    for t in range(ix.L):
        tr = ix.tree(t)
        for q in Q[:4]:
            ub2 = ix.leaf_ub2(t, q)
            lb2 = ix.leaf_lb2(t, q)
            d2 = _proj_dist2(ix, arr, t, q)
            assert np.all(ub2[tr["leaf_of"]] >= d2)
            assert np.all(ub2 >= lb2)


@pytest.mark.parametrize("box_mode", [0, 1])
def test_range_query_exact_is_projected_ball(box_mode):
    # Alg. 3 (pruning by lower bound, whole leaves by upper bound, otherwise a
    # per-point test) returns exactly the points whose projection lies within
    # r' = eps*r of q' -- brute force over every point.
    ix, X, Q = _small_index(box_mode=box_mode)
    arr = ix.arrays()
    e2 = oracle.eps2(ix.K, ix.L)
    for t in range(ix.L):
        for q in Q[:3]:
            d2 = _proj_dist2(ix, arr, t, q)
            for frac in (0.001, 0.01, 0.1):
                # radius at which about frac*n points fall inside
                r = float(np.sqrt(np.quantile(d2.astype(np.float64), frac) / e2))
                got = np.sort(ix.range_exact(t, q, r))
                R2 = np.float32(e2 * r * r)
                assert np.array_equal(got, np.nonzero(d2 <= R2)[0])
                assert got.size > 0


def test_rc_ann_follows_alg4():
    # Alg. 4 recomputed with numpy: S grows tree by tree; once |S| >= beta*n+1
    # the closest point of S is returned; after all trees, the closest point
    # of S only when it lies within c*r, else nothing.
    ix, X, Q = _small_index(n=4000)
    arr = ix.arrays()
    e2 = oracle.eps2(ix.K, ix.L)
    c = 1.5
    seen_stop = seen_cond2 = seen_none = False
    for q in Q[:6]:
        d2s = [_proj_dist2(ix, arr, t, q) for t in range(ix.L)]
        dist = np.sqrt(((X.astype(np.float64) - q.astype(np.float64)) ** 2).sum(1))
        for beta in (0.005, 0.05):
            for frac in (0.0005, 0.003, 0.02):
                r = float(np.sqrt(np.quantile(d2s[0].astype(np.float64), frac) / e2))
                R2 = np.float32(e2 * r * r)
                need = int(np.ceil(beta * ix.n)) + 1
                inS = np.zeros(ix.n, bool)
                stop = -1
                for t in range(ix.L):
                    inS |= d2s[t] <= R2
                    if inS.sum() >= need:
                        stop = t
                        break
                got = ix.rc_ann(q, r, beta=beta, c=c)
                assert got["tree_stop"] == stop
                assert np.array_equal(np.sort(got["S"]), np.nonzero(inS)[0])
                S = np.nonzero(inS)[0]
                want = -1
                if S.size:
                    o = S[np.lexsort((S, dist[S]))[0]]
                    if stop >= 0 or dist[o] <= c * r:
                        want = o
                assert got["id"] == want
                if want >= 0:
                    assert got["dist"] == pytest.approx(dist[want], rel=1e-12)
                seen_stop |= stop >= 0
                seen_cond2 |= stop < 0 and want >= 0
                seen_none |= want < 0
    assert seen_stop and seen_cond2 and seen_none


def test_theorem1_rc_ann_guarantee():
    # Theorem 1: when some point lies within r of q, Alg. 4 returns a point
    # within c*r with probability >= 1/2 - 1/e (beta at its default 0.1).
    c, beta = 1.5, 0.1
    ok = []
    for seed in range(4):
        X, Q, _ = workloads.workload("c1", n=3000, m=10)
        X = X[:, :32] + np.float32(seed)
        Q = Q[:, :32] + np.float32(seed)
        ix = oracle.Index(X, L=4, K=16, N_r=256, seed=seed, frac=0.1, M=64)
        _, nn = oracle.bruteforce_knn(X, Q, 1)
        for i in range(Q.shape[0]):
            r = float(nn[i, 0]) if nn[i, 0] > 0 else 1e-3
            got = ix.rc_ann(Q[i], r, beta=beta, c=c, want_S=False)
            ok.append(got["id"] >= 0 and got["dist"] <= c * r + 1e-9)
    assert np.mean(ok) >= 0.5 - 1.0 / np.e


# ------------------------------- Alg. 5 from a fixed r_min, condition 2 --
def _fixed_grid(ix, r_min, c, i):
    if i == oracle.NLEV - 1:
        return np.float32(np.inf)
    return np.float32(oracle.eps2(ix.K, ix.L) * r_min * r_min * c ** (2.0 * i))


def _exact_within(q, x, R):
    """||q - x|| <= R in exact rational arithmetic."""
    d2 = sum((Fraction(float(a)) - Fraction(float(b))) ** 2 for a, b in zip(q, x))
    return d2 <= Fraction(R) ** 2


def _within_count(X, q, ids, dist, R):
    """Points of ids within R of q, exactly: FP64 decides where it is clear
    by a wide margin, exact rationals decide the rest."""
    n = 0
    for p in ids:
        if abs(dist[p] - R) > 1e-9 * R:
            n += int(dist[p] < R)
        else:
            n += int(_exact_within(q, X[p], R))
    return n


@pytest.mark.parametrize("d", [1, 3, 16, 128])
def test_dist2_le_equals_exact_rational(d):
    g = np.random.default_rng(d)
    for trial in range(60):
        scale = 2.0 ** g.integers(-30, 30)
        q = (g.normal(size=d) * scale).astype(np.float32)
        x = (q + g.normal(size=d) * scale * 10.0 ** g.integers(-7, 1)).astype(np.float32)
        d2 = sum((Fraction(float(a)) - Fraction(float(b))) ** 2 for a, b in zip(q, x))
        r = float(np.sqrt(float(d2)))
        for R in (r, np.nextafter(r, 0.0), np.nextafter(r, np.inf), r * (1 + 1e-12), 0.0):
            if 0.0 < R < 1e-30:
                continue  # below what FP32 pieces can hold (the function says -1)
            assert oracle.dist_le(q, x, R) == int(_exact_within(q, x, R)), (d, trial, R)


def test_dist2_le_special_cases():
    q, x = np.zeros(2, np.float32), np.array([3.0, 4.0], np.float32)
    assert oracle.dist_le(q, x, 5.0) == 1                      # on the sphere: within
    assert oracle.dist_le(q, x, np.nextafter(5.0, 0.0)) == 0   # one ulp inside: beyond
    assert oracle.dist_le(q, q, 0.0) == 1                      # zero distance, zero radius
    assert oracle.dist_le(q, x, float("inf")) == 1
    assert oracle.dist_le(q, x, -1.0) == -1
    assert oracle.dist_le(q, x, 1e300) == 1                    # beyond FP32: within
    # a radius whose square needs the low pieces: 1 + 2^-40 against a point at 1
    one = np.array([1.0], np.float32)
    assert oracle.dist_le(np.zeros(1, np.float32), one, 1.0 + 2.0 ** -40) == 1
    assert oracle.dist_le(np.zeros(1, np.float32), one, 1.0 - 2.0 ** -40) == 0
    # subnormal coordinates against FP32 radii (a single piece each)
    tiny = np.array([1e-45, 3e-45], np.float32)
    d2 = sum(Fraction(float(v)) ** 2 for v in tiny)
    r = np.float32(np.sqrt(float(d2)))
    for R in (r, np.nextafter(r, np.float32(0)), np.nextafter(r, np.float32(1))):
        assert oracle.dist_le(np.zeros(2, np.float32), tiny, float(R)) == int(d2 <= Fraction(float(R)) ** 2)
    # a double radius with bits below FP32's subnormal spacing cannot be cut
    assert oracle.dist_le(np.zeros(2, np.float32), tiny, 3.133398622996355e-45) == -1


def test_query_fixed_rmin_follows_alg5():
    # Alg. 5 literally, from a given r_min: the loop recomputed from the
    # exported leaves (their lower bounds and members) with numpy, and the
    # two stopping conditions checked as invariants at the stopping radius
    # and the one before it.
    ix, X, Q = _small_index(n=4000)
    c, k = 1.5, 10
    trees = [ix.tree(t) for t in range(ix.L)]
    seen = set()
    for q in Q[:5]:
        dist = np.sqrt(((X.astype(np.float64) - q.astype(np.float64)) ** 2).sum(1))
        lbs = [ix.leaf_lb2(t, q) for t in range(ix.L)]
        for r_min in (0.3, 3.0, 30.0):
            for beta in (0.002, 0.05):
                tau = int(np.ceil(beta * ix.n)) + k
                got = ix.query_fixed(q, k, r_min, beta=beta, c=c)
                inS = np.zeros(ix.n, bool)
                js = ist = None
                for i in range(oracle.NLEV):
                    T = _fixed_grid(ix, r_min, c, i)
                    for t in range(ix.L):
                        hit = np.nonzero(lbs[t] <= T)[0]
                        hit = hit[np.lexsort((hit, lbs[t][hit]))]
                        for lf in hit:
                            inS[trees[t]["perm"][trees[t]["begin"][lf]:trees[t]["begin"][lf + 1]]] = True
                            if inS.sum() >= tau:
                                js, ist = i, t
                                break
                        if js is not None:
                            break
                    if js is not None:
                        break
                    if _within_count(X, q, np.nonzero(inS)[0], dist, c * (r_min * c ** i)) >= k:
                        js, ist = i, -1
                        break
                assert (got["jstop"], got["istop"]) == (js, ist)
                S = got["S"]
                assert np.array_equal(np.sort(S), np.nonzero(inS)[0])
                order = np.lexsort((S, dist[S]))[:k]
                assert np.array_equal(got["ids"], S[order])
                if ist == -1:  # condition 2 holds here and neither held one radius before
                    assert _within_count(X, q, S, dist, c * (r_min * c ** js)) >= k
                    assert S.size < tau
                seen.add(ist == -1)
    assert seen == {True, False}


# ------------------------------------------------ static encoding scheme --
@pytest.mark.parametrize("N_r", [2, 16, 256])
def test_static_breakpoints_are_normal_quantiles(N_r):
    # Sec. III-A, static scheme: b_z = Phi^-1(z/N_r), b_0 = -inf, b_{N_r} = +inf
    B = oracle.static_breakpoints(3, N_r)
    want = st.norm.ppf(np.arange(1, N_r) / N_r).astype(np.float32)
    for t in range(3):
        assert np.array_equal(B[t, 1:N_r], want)
        assert B[t, 0] == -np.inf and B[t, N_r] == np.inf


def test_static_encoding_has_equal_mass_on_normal_data():
    # each region holds probability 1/N_r under N(0,1): a chi-square test of
    # the codes of N(0,1) samples, and the index built with the static
    # scheme encodes its projections with those breakpoints
    N_r = 16
    B = oracle.static_breakpoints(1, N_r)
    x = np.random.default_rng(3).normal(size=(200000, 1)).astype(np.float32)
    codes = oracle.encode(x, B)[:, 0]
    cnt = np.bincount(codes, minlength=N_r)
    assert st.chisquare(cnt).pvalue > 1e-4
    X, _, _ = workloads.workload("c4", n=3000, m=1)
    ix = oracle.Index(X, L=2, K=8, N_r=N_r, seed=2, M=16, encoding=1)
    arr = ix.arrays()
    assert np.array_equal(arr["B"], oracle.static_breakpoints(16, N_r))
    assert np.array_equal(arr["codes"], oracle.encode(arr["P"], arr["B"]))


# ------------------------------------------- Alg. 5 at the continuous r_min --
def test_query_magic_min_is_smallest_radius():
    # the smallest continuous r_min: |S(v*)| >= beta*n + k and every smaller
    # lower-bound value leaves fewer points; S and i* recomputed from the
    # exported leaves; the result equals the grid query whenever v* falls on
    # the same leaves (a radius grid that is fine enough)
    ix, X, Q = _small_index(n=5000)
    trees = [ix.tree(t) for t in range(ix.L)]
    for q in Q[:5]:
        lbs = [ix.leaf_lb2(t, q) for t in range(ix.L)]
        mo = np.min([lbs[t][trees[t]["leaf_of"]] for t in range(ix.L)], axis=0)
        for beta, k in ((0.01, 10), (0.1, 5)):
            tau = int(np.ceil(beta * ix.n)) + k
            got = ix.query_magic_min(q, k, beta=beta)
            v = np.float32(got["vstar"])
            assert (mo <= v).sum() >= tau
            assert (mo < v).sum() < tau  # no smaller lower-bound value reaches tau
            inS = np.zeros(ix.n, bool)
            ist = -1
            for t in range(ix.L):
                hit = np.nonzero(lbs[t] <= v)[0]
                hit = hit[np.lexsort((hit, lbs[t][hit]))]
                for lf in hit:
                    inS[trees[t]["perm"][trees[t]["begin"][lf]:trees[t]["begin"][lf + 1]]] = True
                    if inS.sum() >= tau:
                        ist = t
                        break
                if ist >= 0:
                    break
            assert got["istar"] == ist
            assert np.array_equal(np.sort(got["S"]), np.nonzero(inS)[0])
            wi, wd = _numpy_knn(X[got["S"]], q, k)
            assert np.array_equal(got["ids"], got["S"][wi])


def test_rc_ann_optimised_takes_whole_leaves():
    # optimisation (1) of Sec. VI-B2 inside Alg. 4: a tree returns every point
    # of every leaf whose lower bound is within r' (numpy from the exported
    # leaves), a superset of Alg. 3 as printed at the same radius
    ix, X, Q = _small_index(n=4000)
    arr = ix.arrays()
    e2 = oracle.eps2(ix.K, ix.L)
    trees = [ix.tree(t) for t in range(ix.L)]
    for q in Q[:4]:
        dist = np.sqrt(((X.astype(np.float64) - q.astype(np.float64)) ** 2).sum(1))
        d2 = _proj_dist2(ix, arr, 0, q)
        for frac in (0.001, 0.01):
            r = float(np.sqrt(np.quantile(d2.astype(np.float64), frac) / e2))
            R2 = np.float32(e2 * r * r)
            for beta in (0.005, 0.05):
                need = int(np.ceil(beta * ix.n)) + 1
                inS = np.zeros(ix.n, bool)
                stop = -1
                for t in range(ix.L):
                    inS |= ix.leaf_lb2(t, q)[trees[t]["leaf_of"]] <= R2
                    if inS.sum() >= need:
                        stop = t
                        break
                got = ix.rc_ann(q, r, beta=beta, optimised=True)
                assert got["tree_stop"] == stop
                assert np.array_equal(np.sort(got["S"]), np.nonzero(inS)[0])
                exact = ix.rc_ann(q, r, beta=beta)
                if exact["tree_stop"] < 0 and stop < 0:
                    assert set(exact["S"].tolist()) <= set(got["S"].tolist())
                S = got["S"]
                if S.size and (stop >= 0 or dist[S].min() <= 1.5 * r):
                    assert got["id"] == S[np.lexsort((S, dist[S]))[0]]


def test_query_per_tree_check_takes_whole_trees():
    # Alg. 5 without the priority queue: S is the union of whole range
    # queries, trees in order, up to the first tree where |S| >= beta*n + k;
    # it contains the per-leaf S and shares j* and i*
    ix, X, Q = _small_index(n=5000)
    trees = [ix.tree(t) for t in range(ix.L)]
    c = 1.5
    T = ix.level_table(c)
    for q in Q[:5]:
        for beta, k in ((0.01, 10), (0.1, 5)):
            tau = int(np.ceil(beta * ix.n)) + k
            leafwise = ix.query(q, k, beta=beta, c=c)
            got = ix.query(q, k, beta=beta, c=c, per_tree=True)
            assert got["jstar"] == leafwise["jstar"] and got["istar"] == leafwise["istar"]
            thr = T[got["jstar"] - oracle.JMIN]
            inS = np.zeros(ix.n, bool)
            for t in range(got["istar"] + 1):
                inS |= ix.leaf_lb2(t, q)[trees[t]["leaf_of"]] <= thr
            assert np.array_equal(np.sort(got["S"]), np.nonzero(inS)[0])
            assert set(leafwise["S"].tolist()) <= set(got["S"].tolist())
            assert got["S"].size >= tau
