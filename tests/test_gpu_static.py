"""Static (Gaussian) encoding scheme of Sec. III-A: CUDA path vs the oracle.

Bit-exact: breakpoints (N(0,1) quantiles, infinite ends), codes, every
DE-Tree array, candidate sets with j* and i*; distances within 1e-5 relative
and a valid top-k.  Two data sets: unit vectors (projections are N(0,1), the
static scheme's assumption) and unnormalised data (most coordinates fall in
the outer regions, so leaves cannot be split and grow large).
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle  # noqa: E402
import workloads  # noqa: E402
from paper_2603_24920_gb300 import detlsh as D  # noqa: E402
from tests.test_gpu_parity import _bits, _check_topk  # noqa: E402

pytestmark = pytest.mark.gpu

CASES = [
    # name, workload, n, d, L, K, N_r, M
    ("sphere", "c4", 5000, 96, 4, 16, 256, 32),
    ("unnormalised", "c1", 3000, 24, 2, 8, 16, 16),
]


@pytest.fixture(scope="module", params=CASES, ids=[c[0] for c in CASES])
def pair(request):
    name, wl, n, d, L, K, N_r, M = request.param
    X, Q, _ = workloads.workload(wl, n=n, m=8)
    X = np.ascontiguousarray(X[:, :d])
    Q = np.ascontiguousarray(Q[:, :d])
    h = D.detlsh_build(X, L=L, K=K, N_r=N_r, seed=11, max_size=M, encoding=D.ENC_STATIC,
                       keep_projections=1)
    ox = oracle.Index(X, L=L, K=K, N_r=N_r, seed=11, frac=0.1, M=M, encoding=1)
    yield dict(h=h, ox=ox, X=X, Q=Q, n=n, L=L, K=K, N_r=N_r)
    D.detlsh_free(h)


def test_static_build_bit_exact(pair):
    h, ox = pair["h"], pair["ox"]
    ref = ox.arrays()
    B = D.detlsh_get_breakpoints(h)
    assert np.array_equal(_bits(B), _bits(ref["B"]))
    assert np.all(np.isneginf(B[:, 0])) and np.all(np.isposinf(B[:, -1]))
    assert np.array_equal(_bits(D.detlsh_get_projections(h)), _bits(ref["P"]))
    assert np.array_equal(D.detlsh_get_codes(h), ref["codes"])
    info = D.detlsh_get_info(h)
    assert info.encoding == D.ENC_STATIC and info.sample_size == 0
    for t in range(pair["L"]):
        g, r = D.detlsh_get_tree(h, t), ox.tree(t)
        for key in ("perm", "begin", "lo", "hi", "nb", "leaf_of"):
            assert np.array_equal(g[key], r[key]), (t, key)


@pytest.mark.parametrize("beta,k", [(0.01, 10), (0.1, 5)])
def test_static_queries_match_oracle(pair, beta, k):
    h, ox, X, Q = pair["h"], pair["ox"], pair["X"], pair["Q"]
    S_g, js, ist = D.detlsh_query_candidates(h, Q, k, beta=beta, c=1.5)
    ids, dists = D.detlsh_query_ex(h, Q, k, beta=beta, c=1.5)
    for i in range(Q.shape[0]):
        r = ox.query(Q[i], k, beta=beta, c=1.5)
        assert np.array_equal(np.sort(S_g[i]), np.sort(r["S"])), i
        assert js[i] == r["jstar"] and ist[i] == r["istar"]
        _check_topk(ids[i], dists[i], r["S"], X, Q[i], k)


def test_encoding_argument_checked():
    X, _, _ = workloads.workload("c1", n=300, m=1)
    with pytest.raises(D.DetlshError):
        D.detlsh_build(np.ascontiguousarray(X[:, :8]), L=1, K=4, N_r=16, encoding=2)
