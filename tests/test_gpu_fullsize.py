"""Parity at the benchmark's full size: the SIFT-like workload (n = 1,000,000,
d = 128, L = 4, K = 16, N_r = 256, max_size = 64), built and queried in the
launch configuration bench.py times (device-resident data, all 10,000
queries in one call at beta = 0.0015, k = 50, BF16+refine and FP32).

The oracle builds the same index on the host (OpenMP, ~15 s on 16 cores) and
everything the build produces is compared bit for bit; the queries are
compared on a sample of 40 of the 10,000 answers (candidate sets, j*, i*,
top-k within 1e-5 relative), which the oracle computes one by one.  The
BF16+refine answers equal the FP32 answers bit for bit, and recall@10 at the
operating point is at least 0.9 on 200 queries.
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


@pytest.fixture(scope="module")
def answers(full):
    h, Qd = full["h"], full["Qd"]
    out = {}
    for prec in (D.PREC_FP32, D.PREC_BF16_REFINE):
        ids, dists = D.detlsh_query_ex(h, Qd, K_NN, beta=BETA, c=C, precision=prec)
        out[prec] = (ids.cpu().numpy(), dists.cpu().numpy(), D.detlsh_get_timings(h))
    return out


def test_fullsize_queries_sampled(full, answers):
    h, ox, X, Q = full["h"], full["ox"], full["X"], full["Q"]
    ids, dists, _ = answers[D.PREC_FP32]
    S_g, js, ist = D.detlsh_query_candidates(h, Q[SAMPLE], K_NN, beta=BETA, c=C)
    for j, i in enumerate(SAMPLE):
        r = ox.query(Q[i], K_NN, beta=BETA, c=C)
        assert np.array_equal(np.sort(S_g[j]), np.sort(r["S"])), i
        assert js[j] == r["jstar"] and ist[j] == r["istar"]
        _check_topk(ids[i], dists[i], r["S"], X, Q[i], K_NN)


def test_fullsize_bf16_refine_equals_fp32(answers):
    # the certified re-rank pool holds the FP32 path's top k: same bits
    i32, d32, _ = answers[D.PREC_FP32]
    ib, db, tb = answers[D.PREC_BF16_REFINE]
    assert np.array_equal(ib, i32)
    assert np.array_equal(db.view(np.uint32), d32.view(np.uint32))
    # and it re-ranks fewer rows than the 4k of a fixed pool
    assert tb.query_reranked < 4 * K_NN * tb.query_count


def test_fullsize_recall_at_the_operating_point(full, answers):
    # recall@10 >= 0.9 at beta = 0.0015 on 200 queries, exact FP64 ground truth
    X, Q = full["X"], full["Q"]
    Xd = torch.from_numpy(X).cuda().double()
    gt = []
    for i in range(0, 200, 25):
        q = torch.from_numpy(Q[i:i + 25]).cuda().double()
        dd = torch.cdist(q, Xd, compute_mode="donot_use_mm_for_euclid_dist")
        gt.append(torch.topk(dd, 10, largest=False).indices.cpu().numpy())
    gt = np.concatenate(gt)
    for prec in (D.PREC_FP32, D.PREC_BF16_REFINE):
        ids = answers[prec][0][:200, :10]
        rec = np.mean([len(set(ids[i]) & set(gt[i])) / 10 for i in range(200)])
        assert rec >= 0.9, (prec, rec)
