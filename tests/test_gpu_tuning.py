"""Tuning knobs and the autotuner: every tuning gives the same answers (the
knobs only schedule the work of Alg. 3 and Alg. 5, including the top-hull
level of the pruned scan that large trees use), out-of-range knobs are
refused, and the autotuner picks a valid tuning, stores it in the index and
in its cache file, and takes it from the file the second time."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import workloads  # noqa: E402
from paper_2603_24920_gb300 import detlsh as D  # noqa: E402

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ix():
    X, Q, _ = workloads.workload("c2", n=60_000, m=300)
    h = D.detlsh_build(torch.from_numpy(X).cuda(), L=4, K=16, N_r=256, seed=0, max_size=64)
    yield dict(h=h, Q=Q)
    D.detlsh_free(h)


# (0, 4, 512, 1) and (4, 3, 192, 2) force the top-hull level of the pruned
# scan (normally used only for trees of over a million leaves) on this small
# index; hash_kb > 0 gives the leaf-level hash a larger shared region (and
# fewer resident CTAs), so more queries keep their levels on chip
TUNINGS = [(0, 4, 512, 1024, 0), (1, 1, 64, 1024, 0), (3, 8, 128, 1024, 0), (5, 2, 256, 1024, 0),
           (2, 6, 448, 1024, 0), (0, 4, 512, 1, 0), (4, 3, 192, 2, 0), (0, 4, 512, 1024, 40),
           (0, 2, 256, 1024, 160), (5, 4, 512, 2, 80), (0, 4, 512, 1024, 1), (0, 4, 512, 1024, 0, 1),
           (0, 4, 512, 1024, 40, 3)]


@pytest.mark.parametrize("prec", [D.PREC_FP32, D.PREC_BF16_REFINE])
def test_every_tuning_gives_the_same_answers(ix, prec):
    h, Q = ix["h"], ix["Q"]
    want = None
    for t in TUNINGS:
        D.detlsh_set_tuning(h, *t)
        got = D.detlsh_query_ex(h, Q, 20, beta=0.003, precision=prec)
        S = D.detlsh_query_candidates(h, Q[:40], 20, beta=0.003)
        if want is None:
            want = (got, S)
            continue
        assert np.array_equal(got[0], want[0][0]), t
        assert np.array_equal(got[1].view(np.uint32), want[0][1].view(np.uint32)), t
        for i in range(40):
            assert np.array_equal(np.sort(S[0][i]), np.sort(want[1][0][i])), (t, i)
        assert np.array_equal(S[1], want[1][1]) and np.array_equal(S[2], want[1][2])
    D.detlsh_set_tuning(h)


@pytest.mark.parametrize("bad", [(-1, 4, 512, 1024), (6, 4, 512, 1024), (0, 0, 512, 1024),
                                 (0, 9, 512, 1024), (0, 4, 32, 1024), (0, 4, 1024, 1024),
                                 (0, 4, 100, 1024), (0, 4, 512, 0), (0, 4, 512, 1024, -1),
                                 (0, 4, 512, 1024, 161), (0, 4, 512, 1024, 0, -1)])
def test_bad_tunings_are_refused(ix, bad):
    with pytest.raises(D.DetlshError):
        D.detlsh_set_tuning(ix["h"], *bad)
    t = D.detlsh_get_tuning(ix["h"])
    assert (t.query_ctas_per_sm, t.expand_runs, t.visit_chunk, t.top_hull_min, t.hash_kb,
            t.query_scratch_mb) == (0, 4, 512, 1024, 0, 0)


def test_autotune_and_its_cache(ix, tmp_path):
    h, Q = ix["h"], ix["Q"]
    path = tmp_path / "tuning.txt"
    t, cached = D.detlsh_autotune(h, Q, 20, beta=0.003, precision=D.PREC_BF16_REFINE,
                                  cache_path=path)
    assert not cached
    assert 0 <= t.query_ctas_per_sm <= 5 and 1 <= t.expand_runs <= 8
    assert t.visit_chunk in (128, 256, 512)
    assert t.hash_kb in (0, 20, 40, 80)
    assert D.detlsh_get_tuning(h).as_dict() == t.as_dict()
    lines = path.read_text().splitlines()
    assert len(lines) == 1 and "|d128|L4|K16|Nr256|" in lines[0]
    assert len(lines[0].split()) == 6 and lines[0].split()[0].endswith("|v2")
    D.detlsh_set_tuning(h)
    t2, cached2 = D.detlsh_autotune(h, Q, 20, beta=0.003, precision=D.PREC_BF16_REFINE,
                                    cache_path=path)
    assert cached2 and t2.as_dict() == t.as_dict()
    assert len(path.read_text().splitlines()) == 1
    # another shape (k) is another key: a second search and line
    _, cached3 = D.detlsh_autotune(h, Q, 5, beta=0.003, cache_path=path)
    assert not cached3 and len(path.read_text().splitlines()) == 2
    D.detlsh_set_tuning(h)


def test_bound_guess_carried_across_launches(ix):
    # each CTA starts its first tree from the bound its slot kept from the
    # previous launch; a guess from another radius grid (c) or another
    # budget (beta) must not change any answer
    h, Q = ix["h"], ix["Q"]
    ref = D.detlsh_query_ex(h, Q, 10, beta=0.003, c=1.5)
    S_ref = D.detlsh_query_candidates(h, Q[:40], 10, beta=0.003, c=1.5)
    for beta, c in ((0.2, 3.0), (0.0005, 1.1), (0.003, 16.0), (0.05, 1.5)):
        D.detlsh_query_ex(h, Q, 10, beta=beta, c=c)  # leaves its bounds in the slots
        got = D.detlsh_query_ex(h, Q, 10, beta=0.003, c=1.5)
        assert np.array_equal(got[0], ref[0]) and np.array_equal(got[1].view(np.uint32), ref[1].view(np.uint32))
        S = D.detlsh_query_candidates(h, Q[:40], 10, beta=0.003, c=1.5)
        assert np.array_equal(S[1], S_ref[1]) and np.array_equal(S[2], S_ref[2])
        for i in range(40):
            assert np.array_equal(np.sort(S[0][i]), np.sort(S_ref[0][i]))


def _kept_leaves_bounds(h, Q, js, tau, c=1.5):
    """Per query, bounds on the number of leaves whose levels the query keeps
    (the leaves at or below its final expansion bound J, with j* <= J <= the
    first level at which one tree alone holds tau points), from the exported
    boxes: each leaf's lower bound (Sec. IV-C: the gap to the box per
    projected dimension, squared and summed), here in float64 with a small
    margin either way.  Returns (lower, upper)."""
    info = D.detlsh_get_info(h)
    B = D.detlsh_get_breakpoints(h).astype(np.float64)
    P = D.detlsh_project(h, np.ascontiguousarray(Q)).astype(np.float64)
    T = D.detlsh_get_level_table(h, c).astype(np.float64)  # j = -127..127 at j + 127
    K = info.K
    lb2, size = [], []
    for t in range(info.L):
        tr = D.detlsh_get_tree(h, t)
        cols = np.arange(t * K, (t + 1) * K)[None, :]
        blo = B[cols, tr["lo"].astype(np.int64)]
        bhi = B[cols, tr["hi"].astype(np.int64) + 1]
        per = []
        for i in range(len(Q)):
            q = P[i, t * K:(t + 1) * K]
            gap = np.maximum(0.0, np.maximum(blo - q, q - bhi))
            per.append((gap * gap).sum(1))
        lb2.append(np.array(per))
        size.append(np.diff(tr["begin"]))
    lower = np.zeros(len(Q), np.int64)
    upper = np.zeros(len(Q), np.int64)
    for i in range(len(Q)):
        lower[i] = sum(np.count_nonzero(lb2[t][i] <= T[js[i] + 127] * (1.0 - 1e-6))
                       for t in range(info.L))
        jt = []
        for t in range(info.L):
            o = np.argsort(lb2[t][i], kind="stable")
            cum = np.cumsum(size[t][o])
            p = int(np.searchsorted(cum, tau))  # first leaf prefix holding tau points
            jt.append(int(np.searchsorted(T, lb2[t][i][o[p]] * (1.0 + 1e-6))))
        upper[i] = sum(np.count_nonzero(lb2[t][i] <= T[min(jt)] * (1.0 + 1e-6))
                       for t in range(info.L))
    return lower, upper


@pytest.mark.parametrize("prec", [D.PREC_FP32, D.PREC_BF16_REFINE])
def test_level_hash_and_slot_levels_agree(ix, prec):
    # Queries that keep the levels of more leaves (at or below their final
    # expansion bound, bounded from both sides below from the exported
    # boxes) than the default shared hash holds (1,024 at load 1/2) read them
    # in the union counts, the cut and the collection from the slot's
    # epoch-tagged array in device memory; a 160 KiB region (16,384) keeps
    # them on chip.  The answers and S must not depend on where the levels
    # come from.
    h, Q = ix["h"], ix["Q"]
    beta, k = 0.05, 20
    S0 = D.detlsh_query_candidates(h, Q[:64], k, beta=beta)
    tau = int(np.ceil(beta * D.detlsh_get_info(h).n)) + k
    lower, upper = _kept_leaves_bounds(h, Q[:64], S0[1], tau)
    pick = np.flatnonzero((lower > 1024) & (upper <= 16384))
    assert len(pick) >= 8, (lower, upper)
    Qs = np.ascontiguousarray(Q[:64][pick])
    want = None
    for hk in (0, 160, 20):
        D.detlsh_set_tuning(h, hash_kb=hk)
        got = D.detlsh_query_ex(h, Qs, k, beta=beta, precision=prec)
        S = D.detlsh_query_candidates(h, Qs, k, beta=beta)
        if want is None:
            want = (got, S)
            continue
        assert np.array_equal(got[0], want[0][0]), hk
        assert np.array_equal(got[1].view(np.uint32), want[0][1].view(np.uint32)), hk
        for i in range(len(pick)):
            assert np.array_equal(np.sort(S[0][i]), np.sort(want[1][0][i])), (hk, i)
        assert np.array_equal(S[1], want[1][1]) and np.array_equal(S[2], want[1][2])
    D.detlsh_set_tuning(h)
