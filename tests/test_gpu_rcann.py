"""(r,c)-ANN (Alg. 4) over the range query of Alg. 3 as printed, and with
optimisation (1) of Sec. VI-B2 (whole leaves): CUDA path vs the CPU oracle
through the C-ABI.

Bit-exact: the candidate set S (union of the per-tree exact range queries up
to the stopping tree) and the stopping tree.  The returned point: the same id
unless the oracle's FP64 distances of the two ids agree within 1e-5 relative
(near tie), its distance within 1e-5 relative, and "nothing" exactly when the
oracle returns nothing, unless the nearest distance of S is within 1e-5
relative of c*r (FP32 against FP64 decision at the boundary).
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle  # noqa: E402
import workloads  # noqa: E402
from paper_2603_24920_gb300 import detlsh as D  # noqa: E402

pytestmark = pytest.mark.gpu

RTOL = 1e-5

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
    h = D.detlsh_build(X, L=L, K=K, N_r=N_r, seed=5, max_size=M, box_mode=box,
                       keep_projections=1)
    ox = oracle.Index(X, L=L, K=K, N_r=N_r, seed=5, frac=0.1, M=M, box_mode=box)
    yield dict(h=h, ox=ox, X=X, Q=Q, n=n, K=K, L=L)
    D.detlsh_free(h)


def _radii(ox, q, K, L):
    """Radii at which about 0.05%, 0.3% and 2% of the points fall in tree 0's ball."""
    arr = ox.arrays()
    qp = oracle.project(q[None, :], arr["A"][:K])[0]
    d2 = ((arr["P"][:, :K].astype(np.float64) - qp.astype(np.float64)) ** 2).sum(1)
    e2 = oracle.eps2(K, L)
    return [float(np.sqrt(np.quantile(d2, f) / e2)) for f in (0.0005, 0.003, 0.02)]


@pytest.mark.parametrize("optimised", [False, True])
@pytest.mark.parametrize("beta", [0.005, 0.05])
def test_rc_ann_matches_oracle(pair, beta, optimised):
    h, ox, X, Q, n = pair["h"], pair["ox"], pair["X"], pair["Q"], pair["n"]
    c = 1.5
    outcomes = set()
    for i in range(Q.shape[0]):
        q = Q[i]
        dist = np.sqrt(((X.astype(np.float64) - q.astype(np.float64)) ** 2).sum(1))
        for r in _radii(ox, q, pair["K"], pair["L"]):
            want = ox.rc_ann(q, r, beta=beta, c=c, optimised=optimised)
            ids, dists, stop, ssz, S = D.detlsh_rc_ann(h, Q[i:i + 1], r, beta=beta, c=c, S_cap=n,
                                                       optimised=optimised)
            assert stop[0] == want["tree_stop"], (i, r)
            assert ssz[0] == want["S_size"]
            assert np.array_equal(np.sort(S[0]), np.sort(want["S"]))
            g, w = int(ids[0]), int(want["id"])
            if w >= 0 and g >= 0:
                assert g == w or abs(dist[g] - dist[w]) <= RTOL * dist[w] + 1e-6
                assert abs(float(dists[0]) - dist[g]) <= RTOL * dist[g] + 1e-6
            elif w != g:
                # only a boundary case may differ: nearest distance ~ c*r
                S_all = want["S"]
                nearest = dist[S_all].min()
                assert want["tree_stop"] < 0 and abs(nearest - c * r) <= RTOL * c * r
            else:
                assert np.isinf(dists[0])
            outcomes.add("stop" if want["tree_stop"] >= 0 else ("cr" if w >= 0 else "none"))
    assert "stop" in outcomes


def test_rc_ann_device_pointers_and_batch(pair):
    # a batch from device memory gives the same answers as one query at a time
    h, Q = pair["h"], pair["Q"]
    ox = pair["ox"]
    r = _radii(ox, Q[0], pair["K"], pair["L"])[1]
    ids1, d1, s1, z1, _ = D.detlsh_rc_ann(h, Q, r, beta=0.01)
    Qd = torch.from_numpy(Q).cuda()
    ids2, d2, s2, z2, _ = D.detlsh_rc_ann(h, Qd, r, beta=0.01)
    assert np.array_equal(ids1, ids2) and np.array_equal(s1, s2) and np.array_equal(z1, z2)
    assert np.array_equal(d1.view(np.uint32), d2.view(np.uint32))
    for i in range(Q.shape[0]):
        one = D.detlsh_rc_ann(h, Q[i:i + 1], r, beta=0.01)
        assert one[0][0] == ids1[i] and one[2][0] == s1[i] and one[3][0] == z1[i]


def test_rc_ann_argument_errors():
    X, Q, _ = workloads.workload("c1", n=500, m=2)
    h = D.detlsh_build(np.ascontiguousarray(X[:, :16]), L=2, K=4, N_r=16, seed=1)  # no projections
    q = np.ascontiguousarray(Q[:, :16])
    with pytest.raises(D.DetlshError):
        D.detlsh_rc_ann(h, q, 1.0)
    D.detlsh_rc_ann(h, q, 1.0, optimised=True)  # whole leaves need no projections
    D.detlsh_free(h)
    h = D.detlsh_build(np.ascontiguousarray(X[:, :16]), L=2, K=4, N_r=16, seed=1,
                       keep_projections=1)
    for bad in (dict(r=0.0), dict(r=-1.0), dict(r=float("nan")), dict(r=1.0, c=1.0),
                dict(r=1.0, beta=-0.1)):
        with pytest.raises(D.DetlshError):
            D.detlsh_rc_ann(h, q, **bad)
    qn = q.copy()
    qn[0, 0] = np.nan
    with pytest.raises(D.DetlshError):
        D.detlsh_rc_ann(h, qn, 1.0)
    ids, dists, stop, ssz, _ = D.detlsh_rc_ann(h, q, 1e30, beta=0.1)  # every point in range
    assert np.all(stop == 0) and np.all(ssz == 500) and np.all(ids >= 0)
    D.detlsh_free(h)
