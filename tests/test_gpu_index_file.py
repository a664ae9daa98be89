"""Index files (detlsh_save / detlsh_load) round-trip on the GPU: the loaded
index holds the same arrays as the saved one, answers the same queries with
the same candidate sets, and those sets still equal the oracle's; damaged
files are refused."""
import os

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle  # noqa: E402
import workloads  # noqa: E402
from paper_2603_24920_gb300 import detlsh as D  # noqa: E402

pytestmark = pytest.mark.gpu

CASES = [
    # name, n, d, L, K, N_r, M, box, encoding
    ("dynamic", 5000, 32, 4, 16, 256, 16, D.BOX_PREFIX, D.ENC_DYNAMIC),
    ("tight_static", 3001, 24, 3, 8, 64, 8, D.BOX_TIGHT, D.ENC_STATIC),
]


def _data(n, d):
    X, Q, _ = workloads.workload("c1", n=n, m=16)
    return np.ascontiguousarray(X[:, :d]), np.ascontiguousarray(Q[:, :d])


@pytest.fixture(scope="module", params=CASES, ids=[c[0] for c in CASES])
def saved(request, tmp_path_factory):
    name, n, d, L, K, N_r, M, box, enc = request.param
    X, Q = _data(n, d)
    h = D.detlsh_build(torch.from_numpy(X).cuda(), L=L, K=K, N_r=N_r, seed=11, max_size=M,
                       box_mode=box, encoding=enc, keep_projections=1)
    path = tmp_path_factory.mktemp("ix") / ("%s.detlsh" % name)
    D.detlsh_save(h, path)
    g = D.detlsh_load(path)
    yield dict(h=h, g=g, X=X, Q=Q, L=L, K=K, N_r=N_r, M=M, box=box, enc=enc, path=path)
    D.detlsh_free(g)
    D.detlsh_free(h)


def test_loaded_arrays_identical(saved):
    h, g = saved["h"], saved["g"]
    a, b = D.detlsh_get_info(h), D.detlsh_get_info(g)
    for f in ("n", "d", "L", "K", "N_r", "max_size", "box_mode", "has_bf16", "sample_size",
              "max_leaf_size", "eps2", "projection_fallbacks", "encoding"):
        assert getattr(a, f) == getattr(b, f), f
    assert list(a.num_leaves) == list(b.num_leaves)
    for get in (D.detlsh_get_projection_matrix, D.detlsh_get_sample, D.detlsh_get_breakpoints,
                D.detlsh_get_codes, D.detlsh_get_projections):
        x, y = get(h), get(g)
        assert x.dtype == y.dtype and np.array_equal(x.view(np.uint8), y.view(np.uint8)), get
    for t in range(saved["L"]):
        x, y = D.detlsh_get_tree(h, t), D.detlsh_get_tree(g, t)
        for key in x:
            assert np.array_equal(x[key], y[key]), (t, key)
    for c in (1.1, 1.5, 3.0):
        assert np.array_equal(D.detlsh_get_level_table(h, c).view(np.uint32),
                              D.detlsh_get_level_table(g, c).view(np.uint32))


@pytest.mark.parametrize("beta,k", [(0.05, 10), (0.3, 3)])
def test_loaded_index_answers_the_same(saved, beta, k):
    h, g, Q = saved["h"], saved["g"], saved["Q"]
    for prec in (D.PREC_FP32, D.PREC_BF16_REFINE):
        ih, dh = D.detlsh_query_ex(h, Q, k, beta=beta, precision=prec)
        ig, dg = D.detlsh_query_ex(g, Q, k, beta=beta, precision=prec)
        assert np.array_equal(ih, ig) and np.array_equal(dh.view(np.uint32), dg.view(np.uint32))
    Sh, jh, ih_ = D.detlsh_query_candidates(h, Q, k, beta=beta)
    Sg, jg, ig_ = D.detlsh_query_candidates(g, Q, k, beta=beta)
    assert np.array_equal(jh, jg) and np.array_equal(ih_, ig_)
    for i in range(Q.shape[0]):
        assert np.array_equal(np.sort(Sh[i]), np.sort(Sg[i]))


def test_loaded_index_matches_the_oracle(saved):
    g, X, Q = saved["g"], saved["X"], saved["Q"]
    ox = oracle.Index(X, L=saved["L"], K=saved["K"], N_r=saved["N_r"], seed=11, frac=0.1,
                      M=saved["M"], box_mode=saved["box"], encoding=saved["enc"])
    k, beta = 5, 0.05
    S, js, ist = D.detlsh_query_candidates(g, Q, k, beta=beta)
    for i in range(Q.shape[0]):
        r = ox.query(Q[i], k, beta=beta, c=1.5)
        assert np.array_equal(np.sort(S[i]), np.sort(r["S"])), i
        assert (js[i], ist[i]) == (r["jstar"], r["istar"])


def _refused(path, status):
    with pytest.raises(D.DetlshError) as e:
        D.detlsh_load(path)
    assert e.value.status == status


def test_damaged_files_are_refused(saved, tmp_path):
    raw = open(saved["path"], "rb").read()
    cases = {
        "flip": raw[:len(raw) // 2] + bytes([raw[len(raw) // 2] ^ 1]) + raw[len(raw) // 2 + 1:],
        "short": raw[:-9],
        "trailing": raw + b"\0",
        "header_only": raw[:672],
        "version": raw[:8] + (2).to_bytes(4, "little") + raw[12:],
    }
    for name, blob in cases.items():
        p = tmp_path / name
        p.write_bytes(blob)
        _refused(p, -10)
    _refused(tmp_path / "missing.detlsh", -9)
    # the loads above left nothing behind: a good file still loads
    g = D.detlsh_load(saved["path"])
    D.detlsh_free(g)


def test_save_errors(saved, tmp_path):
    with pytest.raises(D.DetlshError) as e:
        D.detlsh_save(saved["h"], tmp_path / "no_such_dir" / "x.detlsh")
    assert e.value.status == -9
    assert not os.path.exists(tmp_path / "no_such_dir")
