"""The BF16+refine path with its certified re-rank pool.

Each candidate's BF16 tensor-core score gives an interval that holds the FP32
path's key (its error bound covers the BF16 rounding of both rows, the FP32
sums and the score's cancellation); every candidate whose interval can reach
the k best is re-ranked in FP32.  So the answer is the FP32 path's answer bit
for bit, and it equals the oracle's exact top k whenever the oracle's k-th and
(k+1)-th distances are apart by more than the FP32 tolerance."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle  # noqa: E402
import workloads  # noqa: E402
from paper_2603_24920_gb300 import detlsh as D  # noqa: E402

pytestmark = pytest.mark.gpu

RTOL = 1e-5


def _rows(kind, n, d, seed):
    g = np.random.default_rng(seed)
    if kind == "sift":       # integers 0-255: exact in BF16
        X, Q, _ = workloads.workload("c2", n=n, m=24)
        return X[:, :d].copy(), Q[:, :d].copy()
    if kind == "gauss":      # BF16 rounds every coordinate
        X, Q, _ = workloads.workload("c1", n=n, m=24)
        return X[:, :d].copy(), Q[:, :d].copy()
    if kind == "sphere":     # unit vectors, the c4 recipe
        X, Q, _ = workloads.workload("c4", n=n, m=24)
        return X[:, :d].copy(), Q[:, :d].copy()
    if kind == "wide":       # rows scaled over 2^-40 .. 2^40
        X = g.normal(size=(n, d)) * 2.0 ** g.integers(-40, 40, (n, 1))
        Q = X[g.integers(0, n, 24)] * (1 + 1e-3 * g.normal(size=(24, d)))
        return X.astype(np.float32), Q.astype(np.float32)
    raise ValueError(kind)


CASES = [("sift", 6000, 128), ("gauss", 6000, 64), ("sphere", 5000, 96), ("wide", 3000, 32)]


@pytest.fixture(scope="module", params=CASES, ids=[c[0] for c in CASES])
def idx(request):
    kind, n, d = request.param
    X, Q = _rows(kind, n, d, 5)
    h = D.detlsh_build(X, L=4, K=16, N_r=256, seed=2, max_size=32)
    yield dict(h=h, X=X, Q=Q, n=n, kind=kind)
    D.detlsh_free(h)


@pytest.mark.parametrize("beta,k", [(0.01, 10), (0.05, 50), (1.5, 5)])
def test_certified_equals_fp32(idx, beta, k):
    h, Q = idx["h"], idx["Q"]
    i32, d32 = D.detlsh_query_ex(h, Q, k, beta=beta)
    ib, db = D.detlsh_query_ex(h, Q, k, beta=beta, precision=D.PREC_BF16_REFINE)
    assert np.array_equal(ib, i32)
    assert np.array_equal(db.view(np.uint32), d32.view(np.uint32))
    t = D.detlsh_get_timings(h)
    assert k * Q.shape[0] <= t.query_reranked


def test_certified_equals_the_oracle_without_near_ties(idx):
    h, X, Q = idx["h"], idx["X"], idx["Q"]
    ox = oracle.Index(X, L=4, K=16, N_r=256, seed=2, frac=0.1, M=32)
    k, beta = 10, 0.05
    ib, db = D.detlsh_query_ex(h, Q, k, beta=beta, precision=D.PREC_BF16_REFINE)
    checked = 0
    for i in range(Q.shape[0]):
        r = ox.query(Q[i], k, beta=beta, c=1.5)
        S = np.asarray(r["S"])
        dd = np.sort(np.sqrt(((X[S].astype(np.float64) - Q[i].astype(np.float64)) ** 2).sum(1)))
        top = dd[:k + 1]
        if np.any(np.diff(top) <= 2 * RTOL * top[1:]):
            continue  # a near-tie in the top k (or at its edge): either order is valid
        assert np.array_equal(ib[i], r["ids"]), i
        np.testing.assert_allclose(db[i], r["dists"], rtol=RTOL, atol=1e-6)
        checked += 1
    assert checked >= Q.shape[0] // 2


def test_pool_beyond_the_rerank_buffers():
    # 5,000 copies of one point: every candidate ties, the pool holds them all
    g = np.random.default_rng(3)
    X = np.concatenate([np.repeat(g.normal(size=(1, 32)), 5000, 0),
                        g.normal(size=(1000, 32))]).astype(np.float32)
    Q = (X[:4] + 0.01).astype(np.float32)
    h = D.detlsh_build(X, L=2, K=8, N_r=16, seed=1, max_size=64)
    try:
        i32, d32 = D.detlsh_query_ex(h, Q, 7, beta=2.0)
        ib, db = D.detlsh_query_ex(h, Q, 7, beta=2.0, precision=D.PREC_BF16_REFINE)
        assert np.array_equal(ib, i32) and np.array_equal(db.view(np.uint32), d32.view(np.uint32))
        assert np.all(ib == np.arange(7))  # ties by smaller id
    finally:
        D.detlsh_free(h)


def test_rerank_mult_is_validated(idx):
    with pytest.raises(D.DetlshError):
        D.detlsh_query_ex(idx["h"], idx["Q"], 5, precision=D.PREC_BF16_REFINE, rerank_mult=-1)
