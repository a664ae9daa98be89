"""CUDA path vs the CPU oracle, element by element, through the C-ABI.

Bit-exact: projection matrix, sample, projections (the exact dot product
rounded once to FP32), breakpoints, codes, every DE-Tree array, the radius
grid, and per-query candidate sets with j* and i*.  Floating-point results:
distances within 1e-5 relative of the oracle's FP64 distances, and the ids a
valid top-k of the (identical) candidate set under that tolerance.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle  # noqa: E402
import workloads  # noqa: E402
from paper_2603_24920_gb300 import detlsh as D  # noqa: E402

pytestmark = pytest.mark.gpu

RTOL = 1e-5


def _gauss(n, d, seed=0):
    X, _, _ = workloads.workload("c1", n=max(n, 1), m=1)
    g = np.random.default_rng(seed)
    return np.ascontiguousarray(X[:n, :d] if d <= 128 else g.normal(size=(n, d)), np.float32)


def _queries(d, m=12, seed=1):
    _, Q, _ = workloads.workload("c1", n=1, m=m)
    return np.ascontiguousarray(Q[:, :d], np.float32)


def _build_pair(X, L, K, N_r, M, box, seed=3, frac=0.1):
    h = D.detlsh_build(X, L=L, K=K, N_r=N_r, seed=seed, max_size=M, box_mode=box,
                       sample_frac=frac, keep_projections=1)
    ox = oracle.Index(X, L=L, K=K, N_r=N_r, seed=seed, frac=frac, M=M, box_mode=box)
    return h, ox


def _bits(a):
    return np.ascontiguousarray(a).view(np.uint32)


CASES = [
    # name, n, d, L, K, N_r, M, box
    ("default", 6000, 32, 4, 16, 256, 64, 0),
    ("tight", 6000, 32, 4, 16, 256, 64, 1),
    ("nr16", 5000, 24, 2, 8, 16, 16, 0),
    ("ragged", 3001, 7, 3, 5, 32, 5, 0),
    ("k1_nr2", 777, 3, 1, 1, 2, 1, 0),
    ("single_point", 1, 4, 2, 3, 8, 4, 0),
    ("n_below_nr", 100, 9, 2, 4, 256, 8, 0),
    ("wide_lk", 2000, 40, 8, 16, 64, 32, 0),
]


@pytest.fixture(scope="module", params=CASES, ids=[c[0] for c in CASES])
def pair(request):
    name, n, d, L, K, N_r, M, box = request.param
    X = _gauss(n, d)
    h, ox = _build_pair(X, L, K, N_r, M, box)
    yield dict(h=h, ox=ox, X=X, L=L, K=K, N_r=N_r, M=M, box=box, n=n, d=d)
    D.detlsh_free(h)


def test_build_arrays_bit_exact(pair):
    h, ox = pair["h"], pair["ox"]
    ref = ox.arrays()
    assert np.array_equal(_bits(D.detlsh_get_projection_matrix(h)), _bits(ref["A"]))
    assert np.array_equal(D.detlsh_get_sample(h), ref["sample"])
    assert np.array_equal(_bits(D.detlsh_get_projections(h)), _bits(ref["P"]))
    assert np.array_equal(_bits(D.detlsh_get_breakpoints(h)), _bits(ref["B"]))
    assert np.array_equal(D.detlsh_get_codes(h), ref["codes"])
    info = D.detlsh_get_info(h)
    assert info.sample_size == ref["sample"].size
    assert info.eps2 == pytest.approx(oracle.eps2(pair["K"], pair["L"]), rel=1e-12)


def test_trees_bit_exact(pair):
    h, ox = pair["h"], pair["ox"]
    info = D.detlsh_get_info(h)
    for t in range(pair["L"]):
        g, r = D.detlsh_get_tree(h, t), ox.tree(t)
        assert info.num_leaves[t] == ox.num_leaves(t)
        for key in ("perm", "begin", "lo", "hi", "nb", "leaf_of"):
            assert np.array_equal(g[key], r[key]), (t, key)
    assert info.max_leaf_size == max(np.diff(ox.tree(t)["begin"]).max() for t in range(pair["L"]))


def test_level_table_bit_exact(pair):
    for c in (1.1, 1.5, 2.0, 3.7):
        assert np.array_equal(_bits(D.detlsh_get_level_table(pair["h"], c)),
                              _bits(pair["ox"].level_table(c)))


def _check_topk(ids_g, d_g, S, X, q, k):
    """ids_g/d_g: a valid top-k of candidate set S (tolerance RTOL)."""
    S = np.asarray(S)
    dd = np.sqrt(((X[S].astype(np.float64) - q.astype(np.float64)) ** 2).sum(1))
    order = np.lexsort((S, dd))
    kth = dd[order[k - 1]]
    assert len(set(ids_g.tolist())) == k
    pos = {int(p): i for i, p in enumerate(S)}
    assert all(int(p) in pos for p in ids_g)
    dg = dd[[pos[int(p)] for p in ids_g]]
    np.testing.assert_allclose(d_g.astype(np.float64), dg, rtol=RTOL, atol=1e-6)
    assert np.all(np.diff(d_g) >= 0)
    assert np.all(dg <= kth * (1 + RTOL) + 1e-6)
    must = S[dd < kth * (1 - RTOL) - 1e-6]
    assert set(must.tolist()) <= set(ids_g.tolist())


@pytest.mark.parametrize("beta,k", [(0.1, 10), (0.01, 1), (0.3, 50), (2.0, 5)])
def test_query_candidates_and_results(pair, beta, k):
    h, ox, X = pair["h"], pair["ox"], pair["X"]
    n = pair["n"]
    k = min(k, n)
    Q = _queries(pair["d"])
    c = 1.5
    S_g, js, ist = D.detlsh_query_candidates(h, Q, k, beta=beta, c=c)
    ids, dists = D.detlsh_query_ex(h, Q, k, beta=beta, c=c)
    for i in range(Q.shape[0]):
        r = ox.query(Q[i], k, beta=beta, c=c)
        assert np.array_equal(np.sort(S_g[i]), np.sort(r["S"])), i
        assert js[i] == r["jstar"] and ist[i] == r["istar"], (i, js[i], r["jstar"], ist[i], r["istar"])
        _check_topk(ids[i], dists[i], r["S"], X, Q[i], k)
        # the oracle's own answer is the same up to near-ties
        np.testing.assert_allclose(dists[i], r["dists"], rtol=RTOL, atol=1e-6)


def test_query_device_pointers_and_mixed_k(pair):
    h, ox, X = pair["h"], pair["ox"], pair["X"]
    n = pair["n"]
    Q = _queries(pair["d"])
    kmax = min(20, n)
    kq = np.array([1 + (i * 7) % kmax for i in range(Q.shape[0])], np.int32)
    ids, dists = D.detlsh_query_ex(h, torch.from_numpy(Q).cuda(), kmax, beta=0.05,
                                   k_per_query=kq)
    ids, dists = ids.cpu().numpy(), dists.cpu().numpy()
    for i in range(Q.shape[0]):
        k = int(kq[i])
        r = ox.query(Q[i], k, beta=0.05, c=1.5)
        _check_topk(ids[i, :k], dists[i, :k], r["S"], X, Q[i], k)
        assert np.all(ids[i, k:] == -1) and np.all(np.isinf(dists[i, k:]))


def test_bf16_refine_path(pair):
    h, ox, X = pair["h"], pair["ox"], pair["X"]
    if pair["d"] % 8:
        with pytest.raises(D.DetlshError):
            D.detlsh_query_ex(h, _queries(pair["d"]), 1, precision=D.PREC_BF16_REFINE)
        return
    Q = _queries(pair["d"])
    k = min(10, pair["n"])
    i32, d32 = D.detlsh_query_ex(h, Q, k, beta=0.1)
    # certified pool (default): the FP32 path's answer, bit for bit
    ib, db = D.detlsh_query_ex(h, Q, k, beta=0.1, precision=D.PREC_BF16_REFINE)
    assert np.array_equal(ib, i32) and np.array_equal(db.view(np.uint32), d32.view(np.uint32))
    # fixed pool of the 4k best scores: exact FP32 distances of the returned ids
    ib, db = D.detlsh_query_ex(h, Q, k, beta=0.1, precision=D.PREC_BF16_REFINE, rerank_mult=4)
    for i in range(Q.shape[0]):
        dd = np.sqrt(((X[ib[i]].astype(np.float64) - Q[i]) ** 2).sum(1))
        np.testing.assert_allclose(db[i], dd, rtol=RTOL, atol=1e-6)
        assert len(set(ib[i].tolist()) & set(i32[i].tolist())) >= k - 1


# ---------------------------------------------------------- projections --
@pytest.mark.parametrize("d", [1, 5, 32, 128, 960])
def test_projection_kernel_exact_on_hard_inputs(d):
    g = np.random.default_rng(d)
    X = _gauss(300, min(d, 128))
    if d > 128:
        X = g.normal(size=(300, d)).astype(np.float32)
    h = D.detlsh_build(X, L=2, K=8, N_r=16, seed=5)
    try:
        A = D.detlsh_get_projection_matrix(h)
        rows = [
            (g.normal(size=(64, d)) * 2.0 ** g.integers(-30, 30, (64, d))).astype(np.float32),
            g.integers(-3, 4, (64, d)).astype(np.float32),          # exact ties, zeros
            np.zeros((8, d), np.float32),                           # exact zero -> +0
            (g.normal(size=(16, d)) * 1e-20).astype(np.float32),     # subnormal products
            np.repeat(g.normal(size=(1, d)).astype(np.float32), 70, 0),
        ]
        for R in rows:
            got = D.detlsh_project(h, R)
            want = oracle.project(R, A)
            assert np.array_equal(_bits(got), _bits(want))
            got_dev = D.detlsh_project(h, torch.from_numpy(R).cuda()).cpu().numpy()
            assert np.array_equal(_bits(got_dev), _bits(want))
    finally:
        D.detlsh_free(h)


# ------------------------------------------------------------ edge cases --
def test_duplicates_and_constant_columns():
    g = np.random.default_rng(9)
    base = g.normal(size=(50, 16)).astype(np.float32)
    X = np.repeat(base, 40, axis=0)            # 40 copies of every point
    X[:, 3] = 7.0                              # a constant column
    h, ox = _build_pair(X, 3, 6, 32, 8, 0)
    try:
        for t in range(3):
            g_, r = D.detlsh_get_tree(h, t), ox.tree(t)
            for key in ("perm", "begin", "lo", "hi", "nb", "leaf_of"):
                assert np.array_equal(g_[key], r[key]), (t, key)
        Q = base[:6] + np.float32(0.01)
        S_g, js, ist = D.detlsh_query_candidates(h, Q, 5, beta=0.05)
        ids, dists = D.detlsh_query_ex(h, Q, 5, beta=0.05)
        for i in range(6):
            r = ox.query(Q[i], 5, beta=0.05)
            assert np.array_equal(np.sort(S_g[i]), np.sort(r["S"]))
            assert np.array_equal(ids[i], r["ids"])  # exact ties broken by smaller id
    finally:
        D.detlsh_free(h)


def test_all_identical_points():
    X = np.ones((300, 8), np.float32)
    h, ox = _build_pair(X, 2, 4, 16, 4, 0)
    try:
        g_, r = D.detlsh_get_tree(h, 0), ox.tree(0)
        assert np.array_equal(g_["begin"], r["begin"]) and np.array_equal(g_["nb"], r["nb"])
        ids, dists = D.detlsh_query_ex(h, np.zeros((2, 8), np.float32), 7, beta=0.1)
        assert np.array_equal(ids[0], np.arange(7)) and np.allclose(dists, np.sqrt(8.0))
    finally:
        D.detlsh_free(h)


def test_nonfinite_inputs_rejected():
    X = _gauss(500, 8)
    X[17, 3] = np.nan
    with pytest.raises(D.DetlshError) as e:
        D.detlsh_build(X, L=2, K=4, N_r=16)
    assert e.value.status == -2
    X[17, 3] = 0.0
    h = D.detlsh_build(X, L=2, K=4, N_r=16)
    try:
        Q = _queries(8, m=3)
        Q[1, 0] = np.inf
        with pytest.raises(D.DetlshError) as e:
            D.detlsh_query_ex(h, Q, 3)
        assert e.value.status == -2
        # the index is still valid after a rejected call
        ids, _ = D.detlsh_query_ex(h, _queries(8, m=3), 3)
        assert ids.shape == (3, 3)
    finally:
        D.detlsh_free(h)


def test_query_argument_errors():
    X = _gauss(200, 8)
    h = D.detlsh_build(X, L=2, K=4, N_r=16)
    try:
        Q = _queries(8, m=2)
        for kw in (dict(k=0), dict(k=201), dict(k=2000), dict(k=3, c=1.0), dict(k=3, beta=-1.0)):
            k = kw.pop("k")
            with pytest.raises(D.DetlshError) as e:
                D.detlsh_query_ex(h, Q, k, **kw)
            assert e.value.status == -1
        ids, dists = D.detlsh_query_ex(h, Q[:0], 3)
        assert ids.shape == (0, 3)
    finally:
        D.detlsh_free(h)


@pytest.mark.parametrize("beta,k", [(0.01, 10), (0.1, 5)])
def test_query_per_tree_check(pair, beta, k):
    # Alg. 5 as printed (whole trees, budget checked after each tree)
    h, ox, X = pair["h"], pair["ox"], pair["X"]
    k = min(k, pair["n"])
    Q = _queries(pair["d"])
    S_g, js, ist = D.detlsh_query_candidates(h, Q, k, beta=beta, per_tree=True)
    ids, dists = D.detlsh_query_ex(h, Q, k, beta=beta, per_tree=True)
    for i in range(Q.shape[0]):
        r = ox.query(Q[i], k, beta=beta, per_tree=True)
        assert np.array_equal(np.sort(S_g[i]), np.sort(r["S"])), i
        assert js[i] == r["jstar"] and ist[i] == r["istar"]
        _check_topk(ids[i], dists[i], r["S"], X, Q[i], k)


@pytest.mark.parametrize("L,groups", [(4, (1, 2, 3)), (3, (2,)), (5, (4,))])
def test_tree_group_independent(L, groups):
    """Trees built G at a time (the group size only changes how many trees a
    launch covers) equal the trees built all at once, array by array, and
    give the same candidate sets, j* and i*."""
    X = _gauss(6000, 24, seed=5)
    Q = _queries(24, m=8)
    h0 = D.detlsh_build(X, L=L, K=8, N_r=64, seed=3, max_size=16, tree_group=L)
    try:
        ref = [D.detlsh_get_tree(h0, t) for t in range(L)]
        S0, j0, i0 = D.detlsh_query_candidates(h0, Q, 5, beta=0.05)
        for g in groups:
            h = D.detlsh_build(X, L=L, K=8, N_r=64, seed=3, max_size=16, tree_group=g)
            try:
                for t in range(L):
                    got = D.detlsh_get_tree(h, t)
                    for key, v in ref[t].items():
                        np.testing.assert_array_equal(got[key], v, err_msg=f"group {g} tree {t} {key}")
                S, js, ist = D.detlsh_query_candidates(h, Q, 5, beta=0.05)
                np.testing.assert_array_equal(js, j0)
                np.testing.assert_array_equal(ist, i0)
                for a, b in zip(S, S0):
                    np.testing.assert_array_equal(np.sort(a), np.sort(b))
            finally:
                D.detlsh_free(h)
    finally:
        D.detlsh_free(h0)
