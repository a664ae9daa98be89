"""The union counts of the magic r_min (Sec. V-B1) from per-tree difference
arrays.  With lv_t(p) the level at which tree t's range query first takes
point p (absent: above every level), the query kernel counts, for each tree
t, +1 at lv_t and -1 at f_t = min over earlier trees of lv_u, when f_t > lv_t.
Summed over trees and levels up to j this must be the size of the union of
the range queries at level j, N(j) = #{p : min_t lv_t(p) <= j}, and the
running sum of tree t's array the points new in tree t (Alg. 5's count)."""
import numpy as np
import pytest

ABSENT = 255


def difference_arrays(lv, jhi):
    n, L = lv.shape
    D = np.zeros((L, 256), np.int64)
    for t in range(L):
        f = lv[:, :t].min(axis=1) if t else np.full(n, ABSENT)
        listed = lv[:, t] <= jhi
        new = listed & (f > lv[:, t])
        np.add.at(D[t], lv[new, t], 1)
        close = new & (f <= jhi)
        np.add.at(D[t], f[close], -1)
    return D


@pytest.mark.parametrize("seed,L,jhi", [(0, 4, 40), (1, 2, 10), (2, 8, 63), (3, 1, 5), (4, 4, 0)])
def test_union_counts_from_difference_arrays(seed, L, jhi):
    g = np.random.default_rng(seed)
    n = 3000
    lv = g.integers(0, 64, (n, L))
    lv[g.random((n, L)) < 0.3] = ABSENT  # points outside a tree's listed leaves
    lv[lv > jhi] = ABSENT                # only levels within the bound are listed
    D = difference_arrays(lv, jhi)
    N = np.array([(lv.min(axis=1) <= j).sum() for j in range(jhi + 1)])
    np.testing.assert_array_equal(np.cumsum(D.sum(axis=0))[:jhi + 1], N)
    # per tree: points taken by tree t at level j and by no earlier tree
    for t in range(L):
        earlier = lv[:, :t].min(axis=1) if t else np.full(n, ABSENT)
        newt = np.array([((lv[:, t] <= j) & (earlier > j)).sum() for j in range(jhi + 1)])
        np.testing.assert_array_equal(np.cumsum(D[t])[:jhi + 1], newt)
