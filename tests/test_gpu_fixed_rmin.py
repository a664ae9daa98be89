"""Alg. 5 from a fixed r_min with condition 2: CUDA path vs the CPU oracle.

The oracle runs the radius loop literally (radii r_min c^i; trees in order,
leaves by (LB^2, id) with the budget check after each leaf; then condition 2
with each distance compared with c*r exactly).  Bit-exact on the GPU: the
stopping radius, the stopping tree (-1 = condition 2) and S, also for points
placed within a few ulps of the spheres c*r_i (the GPU's certified FP32 test
hands those to its exact test).  Results: a valid top-k of S within 1e-5.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle  # noqa: E402
import workloads  # noqa: E402
from paper_2603_24920_gb300 import detlsh as D  # noqa: E402
from tests.test_gpu_parity import _check_topk  # noqa: E402

pytestmark = pytest.mark.gpu

RTOL = 1e-5

CASES = [
    # name, n, d, L, K, N_r, M, box
    ("default", 6000, 32, 4, 16, 256, 64, 0),
    ("nr16", 5000, 24, 2, 8, 16, 16, 0),
    ("ragged", 3001, 7, 3, 5, 32, 5, 0),
]


@pytest.fixture(scope="module", params=CASES, ids=[c[0] for c in CASES])
def pair(request):
    name, n, d, L, K, N_r, M, box = request.param
    X, Q, _ = workloads.workload("c1", n=n, m=8)
    X = np.ascontiguousarray(X[:, :d])
    Q = np.ascontiguousarray(Q[:, :d])
    h = D.detlsh_build(X, L=L, K=K, N_r=N_r, seed=7, max_size=M, box_mode=box)
    ox = oracle.Index(X, L=L, K=K, N_r=N_r, seed=7, frac=0.1, M=M, box_mode=box)
    yield dict(h=h, ox=ox, X=X, Q=Q, n=n)
    D.detlsh_free(h)


_SEEN = set()  # stopping conditions met across the parity cases


@pytest.mark.parametrize("beta,k", [(0.002, 10), (0.05, 5), (2.0, 3)])
def test_fixed_rmin_matches_oracle(pair, beta, k):
    h, ox, X, Q = pair["h"], pair["ox"], pair["X"], pair["Q"]
    c = 1.5
    seen = set()
    for r_min in (0.2, 2.0, 20.0):
        S_g, js, ist = D.detlsh_query_candidates(h, Q, k, beta=beta, c=c, r_min=r_min)
        ids, dists = D.detlsh_query_ex(h, Q, k, beta=beta, c=c, r_min=r_min)
        for i in range(Q.shape[0]):
            want = ox.query_fixed(Q[i], k, r_min, beta=beta, c=c)
            assert (js[i], ist[i]) == (want["jstop"], want["istop"]), (r_min, i)
            assert np.array_equal(np.sort(S_g[i]), np.sort(want["S"])), (r_min, i)
            _check_topk(ids[i], dists[i], want["S"], X, Q[i], k)
            seen.add(int(ist[i]) >= 0)
    _SEEN.update(seen)


def test_fixed_rmin_near_the_spheres():
    # points within a few ulps of the spheres c*r_i around each query: the
    # GPU's certified FP32 test cannot place them and its exact test decides,
    # as the oracle's exact comparison does
    g = np.random.default_rng(11)
    d, c, r_min, k = 16, 1.5, 2.0, 12
    Q = (g.normal(size=(6, d)) * 3).astype(np.float32)
    parts = [(g.normal(size=(2000, d)) * 6).astype(np.float32)]
    for q in Q:
        for i in range(4):
            cr = c * (r_min * c ** i)
            u = g.normal(size=(60, d))
            u /= np.linalg.norm(u, axis=1, keepdims=True)
            pts = (q.astype(np.float64) + u * cr * (1 + g.integers(-4, 5, (60, 1)) * 2.0 ** -24))
            parts.append(pts.astype(np.float32))
    X = np.concatenate(parts)
    h = D.detlsh_build(X, L=3, K=8, N_r=32, seed=5, max_size=16)
    ox = oracle.Index(X, L=3, K=8, N_r=32, seed=5, frac=0.1, M=16)
    try:
        stops = set()
        for beta in (0.01, 0.3):
            S_g, js, ist = D.detlsh_query_candidates(h, Q, k, beta=beta, c=c, r_min=r_min)
            for i in range(Q.shape[0]):
                want = ox.query_fixed(Q[i], k, r_min, beta=beta, c=c)
                assert (js[i], ist[i]) == (want["jstop"], want["istop"]), (beta, i)
                assert np.array_equal(np.sort(S_g[i]), np.sort(want["S"])), (beta, i)
                stops.add(int(ist[i]))
        assert -1 in stops  # condition 2 decided some of them
    finally:
        D.detlsh_free(h)


def test_fixed_rmin_argument_errors(pair):
    h, Q = pair["h"], pair["Q"]
    # (1e-30: c * r_min below 2^-60, radii the exact test cannot hold)
    for bad in (0.0, -1.0, float("inf"), float("nan"), 1e-30):
        with pytest.raises(D.DetlshError):
            D.detlsh_query_ex(h, Q, 3, r_min=bad)
    with pytest.raises(D.DetlshError):  # the fixed radius loop runs on the FP32 path only
        D.detlsh_query_ex(h, Q, 3, r_min=1.0, precision=D.PREC_BF16_REFINE)


def test_fixed_rmin_both_conditions_seen():
    # the parity cases above reached both stopping conditions of Alg. 5
    assert _SEEN == {True, False}
