"""Pins for the oracle's forest topology (hand-derived tables, invariants)."""
import os

import numpy as np
import pytest

import workloads as W
from oracle import forest as FO

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def _read_table(name):
    rows = []
    for line in open(os.path.join(GOLD, name)):
        if line.startswith("#") or not line.strip():
            continue
        parts = [p.split() for p in line.split("|")]
        rows.append([list(map(int, p)) for p in parts])
    return rows


def test_rotated_pair_root_relations():
    w = W.rotated_pair_2d(refine_root0=False)
    F = FO.build(w)
    rf = F.root_face
    assert [rf[(0, f)][0] for f in range(4)] == [1, 1, 0, 0]
    assert [FO.orient_code(*rf[(0, f)][2]) for f in range(4)] == [5, 5, 0, 0]
    assert [rf[(1, f)][0] for f in range(4)] == [1, 1, 0, 0]
    assert [FO.orient_code(*rf[(1, f)][2]) for f in range(4)] == [0, 0, 6, 6]


def test_rotated_pair_leaf_table_golden():
    F = FO.build(W.rotated_pair_2d())
    T = F.leaf_table()
    rows = _read_table("forest_2d_rotated_pair.txt")
    assert len(rows) == len(F.leaves())
    for i, (a, kind, nb0, nb1, orient) in enumerate(rows):
        assert a[0] == i
        assert T["root"][i] == a[1] and T["level"][i] == a[2]
        assert list(T["pos"][i]) == a[3:5]
        assert list(T["kind"][i]) == kind
        assert list(T["nbr"][i, :, 0]) == nb0
        assert list(T["nbr"][i, :, 1]) == nb1
        assert list(T["orient"][i]) == orient


def _inverse(code, d):
    pi, sigma = FO.orient_decode(code, d)
    ipi = [0] * d
    isg = [0] * d
    for a in range(d):
        ipi[pi[a]] = a
        isg[pi[a]] = sigma[a]
    return FO.orient_code(ipi, isg)


@pytest.mark.parametrize("seed", [0, 1, 2, "strip3", "single"])
def test_same_level_relations_are_mutual(seed):
    if seed == "strip3":
        w = W.three_root_strip_2d(n_seg=2)
    elif seed == "single":
        w = W.single_root_2d(n_seg=2)
    else:
        w = W.jitter3d_forest(seed=seed, n_seg=2)
    F = FO.build(w)
    T = F.leaf_table()
    d = w["dim"]
    for i in range(len(F.leaves())):
        for f in range(2 * d):
            if T["kind"][i, f] != FO.SAME:
                continue
            j = T["nbr"][i, f, 0]
            pi, sigma = FO.orient_decode(int(T["orient"][i, f]), d)
            a, s = divmod(f, 2)
            b2 = pi[a]
            s2 = (1 - s) if sigma[a] > 0 else s
            f2 = 2 * b2 + s2
            assert T["kind"][j, f2] == FO.SAME and T["nbr"][j, f2, 0] == i
            assert T["orient"][j, f2] == _inverse(int(T["orient"][i, f]), d)


def test_jitter_forest_counts_and_balance():
    F = FO.build(W.jitter3d_forest(seed=0))
    assert len(F.leaves()) == 71
    T = F.leaf_table()
    lv = T["level"]
    for i in range(len(lv)):
        for f in range(6):
            for j in T["nbr"][i, f]:
                if j >= 0:
                    assert abs(int(lv[j]) - int(lv[i])) <= 1


def test_refine_closure_and_coarsen_refusal():
    # 2D 1x1 periodic root; refine twice into one corner -> 2:1 closure
    w = W.lattice_forest(2, 1, 1.0, 2)
    F = FO.build(w)
    F.refine([(0, 1, (0, 0))])
    F.refine([(0, 2, (0, 0))])
    assert len(F.leaves()) == 7
    F.refine([(0, 3, (0, 0))])
    # (0,3,(0,0)) touches level-2 blocks (1,0) and (0,1) directly and, through
    # the periodic faces, (1,0)/(0,1) again -> those are refined by closure
    keys = set(F.leaves())
    assert (0, 2, (1, 0)) not in keys and (0, 2, (0, 1)) not in keys
    T = F.leaf_table()
    for i in range(len(keys)):
        for f in range(4):
            for j in T["nbr"][i, f]:
                if j >= 0:
                    assert abs(int(T["level"][j]) - int(T["level"][i])) <= 1
    before = list(F.leaves())
    with pytest.raises(FO.BalanceError):
        F.coarsen([(0, 2, (1, 0))])  # its fine neighbours would be 2 levels finer
    assert F.leaves() == before


def test_leaf_order_depth_first():
    w = W.lattice_forest(2, 2, 1.0, 2)
    F = FO.build(w)
    F.refine([(1, 1, (0, 0))])
    assert F.leaves() == [(0, 1, (0, 0)), (1, 2, (0, 0)), (1, 2, (1, 0)), (1, 2, (0, 1)),
                          (1, 2, (1, 1)), (2, 1, (0, 0)), (3, 1, (0, 0))]


def test_child_nodes_bisect_parent_cells():
    w = W.jitter3d_forest(seed=3, n_seg=2)
    F = FO.build(w)
    # every leaf cell's corners are the trilinear images of its parent cell
    from oracle.dg import map_points
    for key in F.leaves():
        r, lev, pos = key
        if lev == 1:
            continue
        parent = (r, lev - 1, tuple(p >> 1 for p in pos))
        PC = F.cell_corners(parent)
        C = F.cell_corners(key)
        n = F.n
        cb = [p & 1 for p in pos]
        for c in range(n ** 3):
            I = [(c // n ** a) % n for a in range(3)]
            for k in range(8):
                bits = [(k >> a) & 1 for a in range(3)]
                H = [cb[a] * n + I[a] + bits[a] for a in range(3)]
                Pc = [min(h // 2, n - 1) for h in H]
                xi = np.array([[H[a] - 2 * Pc[a] - 1.0 for a in range(3)]])
                x = map_points(PC[[sum(Pc[a] * n ** a for a in range(3))]], xi)[0, 0]
                assert np.allclose(C[c, k], x, atol=1e-15)
