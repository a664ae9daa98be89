"""detlsh_query_async captured in a CUDA graph and replayed with new queries:
the results equal detlsh_query_ex's bit for bit, device-side errors reach the
status word, and host-side argument errors are returned."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import workloads  # noqa: E402
from paper_2603_24920_gb300 import detlsh as D  # noqa: E402

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def index():
    X, Q, _ = workloads.workload("c1", n=8000, m=96)
    X = np.ascontiguousarray(X[:, :32])
    Q = np.ascontiguousarray(Q[:, :32])
    h = D.detlsh_build(X, L=4, K=16, N_r=256, seed=3, max_size=32)
    yield h, Q
    D.detlsh_free(h)


def _bits(t):
    return t.cpu().numpy().view(np.uint32)


@pytest.mark.parametrize("precision,r_min", [(D.PREC_FP32, None), (D.PREC_BF16_REFINE, None),
                                             (D.PREC_FP32, 3.0)])
def test_graph_replay_matches_sync(index, precision, r_min):
    h, Q = index
    m, k = 32, 10
    D.detlsh_query_reserve(h, m, k, beta=0.02, precision=precision, r_min=r_min)
    q_buf = torch.zeros((m, Q.shape[1]), dtype=torch.float32, device="cuda")
    ids = torch.empty((m, k), dtype=torch.int64, device="cuda")
    dists = torch.empty((m, k), dtype=torch.float32, device="cuda")
    status = torch.zeros(1, dtype=torch.int32, device="cuda")
    q_buf.copy_(torch.from_numpy(Q[:m]))
    # one plain asynchronous call first (warms up; also checked)
    D.detlsh_query_async(h, q_buf, k, ids, dists, status, stream=torch.cuda.current_stream())
    torch.cuda.synchronize()
    want_i, want_d = D.detlsh_query_ex(h, q_buf, k, beta=0.02, precision=precision, r_min=r_min)
    assert int(status.item()) == 0
    assert torch.equal(ids, want_i) and np.array_equal(_bits(dists), _bits(want_d))
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        D.detlsh_query_async(h, q_buf, k, ids, dists, status,
                             stream=torch.cuda.current_stream())
    for rep in range(3):
        lo = m * (rep % 3)
        q_buf.copy_(torch.from_numpy(Q[lo:lo + m]))
        ids.fill_(-7)
        g.replay()
        torch.cuda.synchronize()
        assert int(status.item()) == 0
        want_i, want_d = D.detlsh_query_ex(h, q_buf, k, beta=0.02, precision=precision,
                                           r_min=r_min)
        assert torch.equal(ids, want_i), rep
        assert np.array_equal(_bits(dists), _bits(want_d)), rep


def test_async_mixed_k_and_errors(index):
    h, Q = index
    m, k = 24, 16
    D.detlsh_query_reserve(h, m, k, beta=0.05)
    q = torch.from_numpy(Q[:m]).cuda()
    kq = torch.from_numpy(np.resize(np.array([1, 5, 16], np.int32), m)).cuda()
    ids = torch.empty((m, k), dtype=torch.int64, device="cuda")
    dists = torch.empty((m, k), dtype=torch.float32, device="cuda")
    status = torch.zeros(1, dtype=torch.int32, device="cuda")
    D.detlsh_query_async(h, q, k, ids, dists, status, k_per_query=kq)
    torch.cuda.synchronize()
    want_i, want_d = D.detlsh_query_ex(h, q, k, beta=0.05, k_per_query=kq.cpu().numpy())
    assert int(status.item()) == 0 and torch.equal(ids, want_i)
    # device-side errors: a NaN query, a per-query k beyond k_max
    qn = q.clone()
    qn[3, 0] = float("nan")
    D.detlsh_query_async(h, qn, k, ids, dists, status)
    torch.cuda.synchronize()
    assert int(status.item()) == -2  # DETLSH_ERR_NONFINITE_INPUT
    bad = kq.clone()
    bad[0] = k + 1
    D.detlsh_query_async(h, q, k, ids, dists, status, k_per_query=bad)
    torch.cuda.synchronize()
    assert int(status.item()) == -1  # DETLSH_ERR_INVALID_ARG
    # host-side errors: too many queries, k above the reservation, host memory
    with pytest.raises(D.DetlshError):
        D.detlsh_query_async(h, torch.from_numpy(Q[:m + 1]).cuda(), k, ids, dists, status)
    with pytest.raises(D.DetlshError):
        D.detlsh_query_async(h, q, k + 1, ids, dists, status)
    with pytest.raises(D.DetlshError):
        D.detlsh_query_async(h, torch.from_numpy(Q[:m]), k, ids, dists, status)
