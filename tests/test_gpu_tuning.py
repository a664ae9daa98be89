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
