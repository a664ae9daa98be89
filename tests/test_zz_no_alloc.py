"""detlsh_query_noalloc answers queries from the library's fixed 32 MiB scratch
array instead of allocated device memory.  It exists for callers that cannot
allocate while serving: a framework that has already claimed nearly all device
memory for its own pool, a latency-critical path where cudaMalloc/cudaFree
would stall the device, or a deployment that forbids allocation after
start-up.  Its answers must equal those of detlsh_query_ex, call after call
(the scratch keeps the previous call's bytes, so each call must start clean).

This file is collected last on purpose: a failure here leaves every other
test already run.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import workloads  # noqa: E402
from paper_2603_24920_gb300 import detlsh as D  # noqa: E402

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def index():
    X, Q, _ = workloads.workload("c1", n=20_000, m=64)
    X, Q = X[:, :64].copy(), Q[:, :64].copy()
    h = D.detlsh_build(torch.from_numpy(X).cuda(), L=4, K=16, N_r=256, seed=0)
    yield h, torch.from_numpy(Q).cuda()
    D.detlsh_free(h)


@pytest.mark.parametrize("per_tree", [False, True])
@pytest.mark.parametrize("precision", [D.PREC_FP32, D.PREC_BF16_REFINE])
def test_noalloc_matches_query_ex_on_two_calls_in_a_row(index, precision, per_tree):
    h, Qd = index
    ref_ids, ref_d = D.detlsh_query_ex(h, Qd, 10, beta=0.05, precision=precision,
                                       per_tree=per_tree)
    for _ in range(2):
        ids, dists = D.detlsh_query_noalloc(h, Qd, 10, beta=0.05, precision=precision,
                                            per_tree=per_tree)
        torch.cuda.synchronize()
        assert torch.equal(ids.cpu(), ref_ids.cpu())
        np.testing.assert_allclose(dists.cpu().numpy(), ref_d.cpu().numpy(), rtol=1e-5, atol=1e-6)


def test_noalloc_rejects_oversized_batches_and_host_buffers(index):
    h, Qd = index
    big = torch.zeros((200_000, Qd.shape[1]), dtype=torch.float32, device="cuda")
    with pytest.raises(D.DetlshError) as e:
        D.detlsh_query_noalloc(h, big, 10, beta=0.05)
    assert e.value.status == -7
    with pytest.raises(D.DetlshError) as e:
        D.detlsh_query_noalloc(h, Qd.cpu().numpy(), 10, ids=np.zeros((Qd.shape[0], 10), np.int64),
                               dists=np.zeros((Qd.shape[0], 10), np.float32))
    assert e.value.status == -1
    # a fitting call afterwards still matches
    ref_ids, _ = D.detlsh_query_ex(h, Qd, 10, beta=0.05)
    ids, _ = D.detlsh_query_noalloc(h, Qd, 10, beta=0.05)
    assert torch.equal(ids.cpu(), ref_ids.cpu())


def test_noalloc_rejects_misaligned_buffers_before_any_launch(index):
    # The caller's buffers reach the kernels without a staging copy, so a
    # query block that starts 4 bytes past a 16-byte boundary (d = 64, read
    # as float4) and ids off an 8-byte boundary are refused on the host.
    h, Qd = index
    m, d = Qd.shape
    buf = torch.zeros(m * d + 4, dtype=torch.float32, device="cuda")
    shifted = buf[1:1 + m * d].view(m, d)
    shifted.copy_(Qd)
    assert shifted.data_ptr() % 16 == 4
    with pytest.raises(D.DetlshError) as e:
        D.detlsh_query_noalloc(h, shifted, 10, beta=0.05)
    assert e.value.status == -1
    raw = torch.zeros(m * 10 * 8 + 8, dtype=torch.uint8, device="cuda")
    ids_bad = raw[4:4 + m * 10 * 8]
    dists = torch.zeros((m, 10), dtype=torch.float32, device="cuda")
    assert ids_bad.data_ptr() % 8 == 4
    with pytest.raises(D.DetlshError) as e:
        D.detlsh_query_noalloc(h, Qd, 10, beta=0.05, ids=ids_bad, dists=dists)
    assert e.value.status == -1


def test_noalloc_stops_on_a_nonfinite_query(index):
    h, Qd = index
    bad = Qd.clone()
    bad[3, 5] = float("nan")
    with pytest.raises(D.DetlshError) as e:
        D.detlsh_query_noalloc(h, bad, 10, beta=0.05)
    assert e.value.status == -2
    ref_ids, _ = D.detlsh_query_ex(h, Qd, 10, beta=0.05)
    ids, _ = D.detlsh_query_noalloc(h, Qd, 10, beta=0.05)
    assert torch.equal(ids.cpu(), ref_ids.cpu())
