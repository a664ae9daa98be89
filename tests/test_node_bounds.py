"""Two-sided pins of the oracle's node lower and upper bounds (Sec. IV-C).

Soundness alone (LB <= every member's projected distance, UB >= it) would
also accept a looser bound, such as a gap measured to one edge of the box
only or to a box edge one region off.  These tests pin the bounds from the
other side as well:

  * a hand-worked two-dimensional box with literal expected values, one query
    inside, on the edge, beside, above and diagonal to it;
  * tightness over the real index: LB^2 is the minimum of |y - q'|^2 over the
    leaf's box, found by scipy's bounded least squares, and UB^2 is the
    maximum, found by enumerating the box's 2^K corners (a convex function
    on a box peaks at a vertex), for every leaf of a small index, both box
    modes.
"""
import itertools

import numpy as np
import pytest
from scipy.optimize import lsq_linear

import oracle
import workloads

# Two dimensions, N_r = 4: dimension 0 has breakpoints 0 1 2 4 8,
# dimension 1 has -3 -1 0 1 5.  The box takes regions 1..2 of dimension 0,
# i.e. [B(1), B(3)] = [1, 4], and regions 0..1 of dimension 1, [-3, 0].
_B2 = np.array([[0.0, 1.0, 2.0, 4.0, 8.0], [-3.0, -1.0, 0.0, 1.0, 5.0]], np.float32)
_LO2 = np.array([1, 0], np.uint8)
_HI2 = np.array([2, 1], np.uint8)

# (query, LB^2, UB^2), worked by hand:
#   LB: per dimension the distance to the interval (0 inside), squared, summed
#   UB: per dimension the distance to the farther end, squared, summed
_CASES2 = [
    ((2.0, -1.0), 0.0, 2.0 ** 2 + 2.0 ** 2),                  # inside: far ends 4 and -3
    ((4.0, 0.0), 0.0, 3.0 ** 2 + 3.0 ** 2),                  # on the corner (4, 0)
    ((0.0, -2.0), 1.0, 4.0 ** 2 + 2.0 ** 2),                  # left of the box
    ((6.0, -1.0), 4.0, 5.0 ** 2 + 2.0 ** 2),                  # right of the box
    ((3.0, 2.5), 6.25, 2.0 ** 2 + 5.5 ** 2),                  # above the box
    ((-1.0, 2.0), 8.0, 5.0 ** 2 + 5.0 ** 2),                  # diagonal, upper left
    ((5.0, -5.0), 5.0, 4.0 ** 2 + 5.0 ** 2),                  # diagonal, lower right
]


@pytest.mark.parametrize("q,lb2,ub2", _CASES2)
def test_hand_worked_two_dimensional_box(q, lb2, ub2):
    got_lb, got_ub = oracle.box_bounds(_B2, np.array(q, np.float32), _LO2, _HI2)
    assert got_lb == lb2
    assert got_ub == ub2


def test_one_region_box_edges():
    # A box of one region per dimension spans [B(z), B(z + 1)]: region 3 of
    # dimension 0 is [4, 8] and region 2 of dimension 1 is [0, 1].
    lo = np.array([3, 2], np.uint8)
    lb, ub = oracle.box_bounds(_B2, np.array([3.0, 1.5], np.float32), lo, lo)
    assert lb == 1.0 + 0.25
    assert ub == 25.0 + 2.25


def _small(box_mode):
    X, Q, _ = workloads.workload("c1", n=3000, m=4)
    X, Q = X[:, :24].copy(), Q[:, :24].copy()
    ix = oracle.Index(X, L=2, K=6, N_r=16, seed=3, frac=0.2, M=8, box_mode=box_mode)
    return ix, Q


def _box_min_dist2(q, e_lo, e_hi):
    # min |y - q|^2 over e_lo <= y <= e_hi by bounded least squares; a
    # dimension whose interval is a single value is fixed there
    fixed = e_lo >= e_hi
    out = float(np.sum((q[fixed] - e_lo[fixed]) ** 2))
    free = ~fixed
    if free.any():
        r = lsq_linear(np.eye(int(free.sum())), q[free], bounds=(e_lo[free], e_hi[free]),
                       method="bvls", tol=1e-15)
        out += float(np.sum((r.x - q[free]) ** 2))
    return out


def _box_max_dist2(q, e_lo, e_hi):
    K = q.shape[0]
    best = 0.0
    for corner in itertools.product((0, 1), repeat=K):
        y = np.where(np.array(corner, bool), e_hi, e_lo)
        best = max(best, float(np.sum((y - q) ** 2)))
    return best


@pytest.mark.parametrize("box_mode", [0, 1])
def test_bounds_are_the_box_extremes_of_every_leaf(box_mode):
    ix, Q = _small(box_mode)
    arr = ix.arrays()
    K = ix.K
    checked = 0
    for t in range(ix.L):
        tr = ix.tree(t)
        Bt = arr["B"][t * K:(t + 1) * K].astype(np.float64)
        for q in Q[:2]:
            qp = oracle.project(q[None, :], arr["A"][t * K:(t + 1) * K])[0].astype(np.float64)
            lb2 = ix.leaf_lb2(t, q)
            ub2 = ix.leaf_ub2(t, q)
            for leaf in range(tr["lo"].shape[0]):
                lo = tr["lo"][leaf].astype(np.int64)
                hi = tr["hi"][leaf].astype(np.int64)
                e_lo = Bt[np.arange(K), lo]
                e_hi = Bt[np.arange(K), hi + 1]
                mn = _box_min_dist2(qp, e_lo, e_hi)
                mx = _box_max_dist2(qp, e_lo, e_hi)
                scale = float(np.sum(qp ** 2) + np.sum(np.maximum(e_lo ** 2, e_hi ** 2))) + 1.0
                # the oracle sums K FP32 squares: relative error below 1e-5
                assert abs(lb2[leaf] - mn) <= 1e-5 * mn + 1e-9 * scale, (t, leaf, lb2[leaf], mn)
                assert abs(ub2[leaf] - mx) <= 1e-5 * mx + 1e-9 * scale, (t, leaf, ub2[leaf], mx)
                checked += 1
    assert checked > 500
