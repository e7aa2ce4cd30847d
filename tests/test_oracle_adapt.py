"""Pins for the oracle's refinement indicator and adaptation step (reading
R16): the indicator's closed form on a linear density, 2:1 balance and the
refine/coarsen rules after an adaptation, conservation of the totals through
the state transfer, and refine-everything-then-coarsen-everything giving the
original forest and state back."""
import numpy as np
import pytest

import workloads as W
from oracle import adapt as A
from oracle import dg
from oracle import forest as FO


def _linear_density(slope):
    def fun(x):
        x = np.asarray(x, float)
        d = x.shape[-1]
        rho = 1.0 + np.tensordot(x, slope, axes=([-1], [0]))
        return W.prim_to_cons(rho, np.zeros(x.shape[:-1] + (d,)), np.ones(x.shape[:-1]))
    return fun


@pytest.mark.parametrize("p", [1, 2])
def test_indicator_closed_form_on_a_linear_density(p):
    """rho = 1 + s.x on affine cube cells of edge h: g = h |s| / rho(centre)."""
    w = W.lattice_forest(3, 2, 1.0, 2, rotate_roots=True, seed=3, periodic=False)
    w["refine"] = [[(0, 1, (0, 0, 0))]]
    S = dg.Solver(FO.build(w), p)
    s = np.array([0.3, -0.2, 0.5])
    U = S.project(_linear_density(s))
    g = A.indicator(S, U)
    xq = S.quad_points()
    for li, key in enumerate(S.leaves):
        h = 1.0 / 2 / 2 ** (key[1] - 1) / 2          # root edge 1/2, n = 2
        centres = xq[li].mean(axis=1)                 # Gauss points are symmetric
        want = np.max(h * np.linalg.norm(s) / (1.0 + centres @ s))
        assert abs(g[li] - want) < 1e-12 * want


def test_indicator_is_zero_for_p0():
    S = dg.Solver(FO.build(W.rotated_pair_2d(n_seg=2)), 0)
    U = W.random_modal_state(len(S.leaves), 2, 2, 0, seed=1)
    assert np.all(A.indicator(S, U) == 0.0)


def _blast_solver(p=1):
    w = W.lattice_forest(3, 2, 1.0, 2, seed=1)
    S = dg.Solver(FO.build(w), p)
    U = S.project(lambda x: W.blast(x, (0.3, 0.3, 0.3), r0=0.15, width=0.08))
    return S, U


def test_adapt_rules_balance_and_conservation():
    S, U = _blast_solver()
    g = A.indicator(S, U)
    thr = float(np.median(g))
    S1, U1, nr, nc = A.adapt(S, U, thr, 0.0, max_level=3)
    assert nr == int(np.sum(g > thr)) and nc == 0
    assert not S1.F._violations()
    for i, k in enumerate(S.leaves):
        assert (not S1.F.is_leaf(k)) == (g[i] > thr) or (S1.F.tree.get(k) is False)
    T0, T1 = S.totals(U), S1.totals(U1)
    assert np.max(np.abs(T1 - T0)) < 1e-13 * np.max(np.abs(T0))
    # coarsen where the new leaves are smooth: every coarsened parent's
    # children were leaves below the threshold, balance holds
    g1 = A.indicator(S1, U1)
    groups = {}
    for i, k in enumerate(S1.leaves):
        if k[1] == 2:
            parent = (k[0], 1, tuple(x >> 1 for x in k[2]))
            groups[parent] = max(groups.get(parent, 0.0), g1[i])
    cthr = float(np.median(sorted(groups.values()))) * (1 + 1e-9)  # about half the groups qualify
    S2, U2, nr2, nc2 = A.adapt(S1, U1, np.inf, cthr, max_level=3)
    assert nr2 == 0 and nc2 > 0 and not S2.F._violations()
    low = {k for i, k in enumerate(S1.leaves) if g1[i] < cthr}
    for k in set(S2.leaves) - set(S1.leaves):
        kids = [kk for kk in S1.leaves if kk[0] == k[0] and kk[1] == k[1] + 1
                and all((kk[2][a] >> 1) == k[2][a] for a in range(3))]
        assert len(kids) == 8 and all(kk in low for kk in kids)
    T2 = S2.totals(U2)
    assert np.max(np.abs(T2 - T0)) < 1e-13 * np.max(np.abs(T0))


def test_adapt_refine_all_then_coarsen_all_is_identity():
    S, U = _blast_solver(p=2)
    S1, U1, nr, _ = A.adapt(S, U, -1.0, 0.0, max_level=2)
    assert nr == len(S.leaves) and len(S1.leaves) == 8 * len(S.leaves)
    S2, U2, nr2, nc2 = A.adapt(S1, U1, np.inf, np.inf, max_level=2)
    assert nr2 == 0 and nc2 == len(S.leaves)
    assert S2.leaves == S.leaves
    assert np.max(np.abs(U2 - U)) < 1e-12


def test_adapt_with_nothing_flagged_is_identity():
    S, U = _blast_solver()
    S1, U1, nr, nc = A.adapt(S, U, np.inf, 0.0, max_level=4)
    assert (nr, nc) == (0, 0) and S1.leaves == S.leaves and np.array_equal(U1, U)


def test_coarsening_that_would_break_balance_is_skipped():
    """2x2 periodic roots; root 0 refined once, root 1 twice at its corner
    next to root 0 (the 2:1 closure also refines root 3).  With every block
    below the threshold, one pass in canonical order: root 0's group stays
    (a level-1 root 0 would touch root 1's level-3 blocks), root 1's level-3
    group and root 3's group coarsen; root 1's level-2 group is not visited
    (its first child was not a leaf when the pass began)."""
    w = W.lattice_forest(2, 2, 1.0, 2, seed=0)
    w["refine"] = [[(0, 1, (0, 0)), (1, 1, (0, 0))], [(1, 2, (0, 0))]]
    S = dg.Solver(FO.build(w), 1)
    assert (3, 2, (0, 0)) in S.leaves  # closure
    U = W.random_modal_state(len(S.leaves), 2, 2, 1, seed=2, amp=0.0)  # g = 0 everywhere
    S1, U1, nr, nc = A.adapt(S, U, np.inf, 1.0, max_level=4)
    want = [(0, 2, (0, 0)), (0, 2, (1, 0)), (0, 2, (0, 1)), (0, 2, (1, 1)),
            (1, 2, (0, 0)), (1, 2, (1, 0)), (1, 2, (0, 1)), (1, 2, (1, 1)),
            (2, 1, (0, 0)), (3, 1, (0, 0))]
    assert (nr, nc) == (0, 2) and S1.leaves == want and not S1.F._violations()
