"""Parity at the benchmark's full size: the SIFT-like workload (n = 1,000,000,
d = 128, L = 4, K = 16, N_r = 256, max_size = 64), built and queried in the
launch configuration bench.py times (device-resident data, all 10,000
queries in one call at beta = 0.0015, k = 50, BF16+refine and FP32).

The oracle builds the same index on the host (OpenMP, ~15 s on 16 cores) and
everything the build produces is compared bit for bit; the queries are
compared on a sample of 40 of the 10,000 answers (candidate sets, j*, i*,
top-k within 1e-5 relative), which the oracle computes one by one.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle  # noqa: E402
import workloads  # noqa: E402
from paper_2603_24920_gb300 import detlsh as D  # noqa: E402
from tests.test_gpu_parity import _bits, _check_topk  # noqa: E402

pytestmark = pytest.mark.gpu

BETA, C, K_NN = 0.0015, 1.5, 50
SAMPLE = np.linspace(0, 9999, 40).astype(np.int64)


@pytest.fixture(scope="module")
def full():
    X, Q, k = workloads.workload("c2")
    Xd = torch.from_numpy(X).cuda()
    Qd = torch.from_numpy(Q).cuda()
    h = D.detlsh_build(Xd, L=4, K=16, N_r=256, seed=0, max_size=64)
    ox = oracle.Index(X, L=4, K=16, N_r=256, seed=0, frac=0.1, M=64)
    yield dict(h=h, ox=ox, X=X, Q=Q, Qd=Qd)
    D.detlsh_free(h)


def test_fullsize_build_bit_exact(full):
    h, ox = full["h"], full["ox"]
    ref = ox.arrays()
    assert np.array_equal(_bits(D.detlsh_get_projection_matrix(h)), _bits(ref["A"]))
    assert np.array_equal(D.detlsh_get_sample(h), ref["sample"])
    assert np.array_equal(_bits(D.detlsh_get_breakpoints(h)), _bits(ref["B"]))
    assert np.array_equal(D.detlsh_get_codes(h), ref["codes"])
    info = D.detlsh_get_info(h)
    for t in range(4):
        g, r = D.detlsh_get_tree(h, t), ox.tree(t)
        assert info.num_leaves[t] == ox.num_leaves(t)
        for key in ("perm", "begin", "lo", "hi", "nb", "leaf_of"):
            assert np.array_equal(g[key], r[key]), (t, key)


@pytest.mark.parametrize("precision", [D.PREC_FP32, D.PREC_BF16_REFINE])
def test_fullsize_queries_sampled(full, precision):
    h, ox, X, Q, Qd = full["h"], full["ox"], full["X"], full["Q"], full["Qd"]
    ids, dists = D.detlsh_query_ex(h, Qd, K_NN, beta=BETA, c=C, precision=precision)
    ids, dists = ids.cpu().numpy(), dists.cpu().numpy()
    S_g, js, ist = D.detlsh_query_candidates(h, Q[SAMPLE], K_NN, beta=BETA, c=C)
    for j, i in enumerate(SAMPLE):
        r = ox.query(Q[i], K_NN, beta=BETA, c=C)
        assert np.array_equal(np.sort(S_g[j]), np.sort(r["S"])), i
        assert js[j] == r["jstar"] and ist[j] == r["istar"]
        if precision == D.PREC_FP32:
            _check_topk(ids[i], dists[i], r["S"], X, Q[i], K_NN)
        else:
            # BF16 scores pick the re-rank pool; the answer is exact FP32 over it
            S = np.asarray(r["S"])
            assert set(ids[i].tolist()) <= set(S.tolist())
            dd = np.sqrt(((X[ids[i]].astype(np.float64) - Q[i].astype(np.float64)) ** 2).sum(1))
            np.testing.assert_allclose(dists[i], dd, rtol=1e-5, atol=1e-6)
            assert np.all(np.diff(dists[i]) >= 0)
