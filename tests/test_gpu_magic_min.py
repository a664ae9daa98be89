"""Alg. 5 at the smallest continuous r_min (DETLSH_RMIN_CONTINUOUS): CUDA path
vs the oracle.  Bit-exact: S and i*; results a valid top-k of S within 1e-5."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle  # noqa: E402
import workloads  # noqa: E402
from paper_2603_24920_gb300 import detlsh as D  # noqa: E402
from tests.test_gpu_parity import _check_topk  # noqa: E402

pytestmark = pytest.mark.gpu

CASES = [
    # name, n, d, L, K, N_r, M, box
    ("default", 6000, 32, 4, 16, 256, 64, 0),
    ("tight", 6000, 32, 4, 16, 256, 64, 1),
    ("nr16", 5000, 24, 2, 8, 16, 16, 0),
    ("ragged", 3001, 7, 3, 5, 32, 5, 0),
]


@pytest.fixture(scope="module", params=CASES, ids=[c[0] for c in CASES])
def pair(request):
    name, n, d, L, K, N_r, M, box = request.param
    X, Q, _ = workloads.workload("c1", n=n, m=10)
    X = np.ascontiguousarray(X[:, :d])
    Q = np.ascontiguousarray(Q[:, :d])
    h = D.detlsh_build(X, L=L, K=K, N_r=N_r, seed=9, max_size=M, box_mode=box)
    ox = oracle.Index(X, L=L, K=K, N_r=N_r, seed=9, frac=0.1, M=M, box_mode=box)
    yield dict(h=h, ox=ox, X=X, Q=Q, n=n)
    D.detlsh_free(h)


@pytest.mark.parametrize("beta,k", [(0.01, 10), (0.1, 5), (0.3, 50), (2.0, 3)])
@pytest.mark.parametrize("precision", [D.PREC_FP32, D.PREC_BF16_REFINE])
def test_magic_min_matches_oracle(pair, beta, k, precision):
    h, ox, X, Q = pair["h"], pair["ox"], pair["X"], pair["Q"]
    if precision == D.PREC_BF16_REFINE and X.shape[1] % 8:
        pytest.skip("the BF16 path needs d % 8 == 0")
    k = min(k, pair["n"])
    pol = D.RMIN_CONTINUOUS
    S_g, js, ist = D.detlsh_query_candidates(h, Q, k, beta=beta, rmin_policy=pol)
    ids, dists = D.detlsh_query_ex(h, Q, k, beta=beta, rmin_policy=pol, precision=precision)
    for i in range(Q.shape[0]):
        r = ox.query_magic_min(Q[i], k, beta=beta)
        assert np.array_equal(np.sort(S_g[i]), np.sort(r["S"])), i
        assert ist[i] == r["istar"]
        if precision == D.PREC_FP32:
            _check_topk(ids[i], dists[i], r["S"], X, Q[i], k)
        else:
            assert set(ids[i].tolist()) <= set(r["S"].tolist())
