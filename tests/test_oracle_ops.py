"""Pins for the oracle's split S, combine C and rotation R^n (Secs. 3.4-3.5)."""
import os

import numpy as np
import pytest

import workloads as W
from oracle import basis as B
from oracle import dg
from oracle import forest as FO

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def _unit_cell(d, jitter=0.0, seed=0):
    rng = np.random.default_rng(seed)
    C = np.array([[float(b[a]) for a in range(d)] for b in B.all_corner_bits(d)])
    return C + jitter * rng.uniform(-1, 1, C.shape)


def test_split_matches_hand_computed_p2():
    ops = dg.Ops(2, 2)
    S = {"minus": [], "plus": []}
    for line in open(os.path.join(GOLD, "split_1d_p2.txt")):
        if line.startswith("#") or not line.strip():
            continue
        side, *vals = line.split()
        S[side].append([float(v) for v in vals])
    C = _unit_cell(2)
    for side, e in (("minus", (0, 0)), ("plus", (1, 0))):
        for k in range(3):
            K = np.zeros(9)
            K[k] = 1.0  # parent mode (k, 0)
            Kc = dg._split(ops, K, C, e)
            want = np.zeros(9)
            want[0:3] = [S[side][l][k] for l in range(3)]
            assert np.allclose(Kc, want, atol=1e-14)


@pytest.mark.parametrize("d,p,jit", [(2, 1, 0.0), (2, 3, 0.15), (3, 2, 0.1), (3, 1, 0.0)])
def test_split_is_exact_restriction(d, p, jit):
    ops = dg.Ops(d, p)
    C = _unit_cell(d, jit, seed=p)
    rng = np.random.default_rng(d + p)
    K = rng.standard_normal(ops.M)
    for e in B.all_corner_bits(d):
        Kc = dg._split(ops, K, C, e)
        xi = rng.uniform(-1, 1, (7, d))
        xP = (xi + (2 * np.asarray(e) - 1.0)) / 2
        assert np.allclose(B.eval_basis(xi, ops.N) @ Kc, B.eval_basis(xP, ops.N) @ K, atol=1e-12)


@pytest.mark.parametrize("d,p,jit", [(2, 2, 0.0), (2, 2, 0.2), (3, 1, 0.1), (3, 3, 0.0)])
def test_combine_after_split_is_identity(d, p, jit):
    """restriction(prolongation(u)) = u (Eqs. (11)-(14), reading R6)."""
    ops = dg.Ops(d, p)
    C = _unit_cell(d, jit, seed=11)
    rng = np.random.default_rng(5)
    K = rng.standard_normal((3, ops.M))
    kids, corners = [], []
    for e in B.all_corner_bits(d):
        kids.append(dg._split(ops, K, C, e))
        xi = np.array([[2.0 * b - 1.0 for b in bits] for bits in B.all_corner_bits(d)])
        xP = (xi + (2 * np.asarray(e) - 1.0)) / 2
        corners.append(dg.map_points(C[None], xP)[0])
    KP = dg._combine(ops, np.array(kids), np.array(corners))
    assert np.allclose(KP, K, atol=1e-12)


def test_combine_conserves_weighted_integral():
    """C keeps int u dV over the union of the children (phi_0 = 1 row)."""
    d, p = 3, 2
    ops = dg.Ops(d, p)
    C = _unit_cell(d, 0.12, seed=3)
    rng = np.random.default_rng(9)
    kids, corners, total = [], [], 0.0
    for e in B.all_corner_bits(d):
        Kc = rng.standard_normal(ops.M)
        xi = np.array([[2.0 * b - 1.0 for b in bits] for bits in B.all_corner_bits(d)])
        xP = (xi + (2 * np.asarray(e) - 1.0)) / 2
        cc = dg.map_points(C[None], xP)[0]
        _, J, _ = dg.jacobian(cc[None], ops.xq)
        total += np.sum(ops.wq * J[0] * (ops.Phi @ Kc))
        kids.append(Kc)
        corners.append(cc)
    KP = dg._combine(ops, np.array(kids), np.array(corners))
    # same integral evaluated with the children's rules on the parent polynomial
    tp = 0.0
    for e, cc in zip(B.all_corner_bits(d), corners):
        xP = (ops.xq + (2 * np.asarray(e) - 1.0)) / 2
        _, J, _ = dg.jacobian(cc[None], ops.xq)
        tp += np.sum(ops.wq * J[0] * (B.eval_basis(xP, ops.N) @ KP))
    assert abs(tp - total) < 1e-12 * max(1.0, abs(total))


@pytest.mark.parametrize("d", [2, 3])
def test_rotation_inverse_and_pointwise(d):
    p = 3 if d == 2 else 2
    ops = dg.Ops(d, p)
    rng = np.random.default_rng(2)
    K = rng.standard_normal(ops.M)
    for code in range(len(FO.perm_list(d)) * (1 << d)):
        pi, sigma = FO.orient_decode(code, d)
        Kr = dg._rotate(ops, K, pi, sigma)
        xi = rng.uniform(-1, 1, (5, d))
        xs = np.zeros_like(xi)
        for a in range(d):
            xs[:, pi[a]] = sigma[a] * xi[:, a]
        assert np.allclose(B.eval_basis(xi, ops.N) @ Kr, B.eval_basis(xs, ops.N) @ K, atol=1e-12)
        ipi = [0] * d
        isg = [0] * d
        for a in range(d):
            ipi[pi[a]] = a
            isg[pi[a]] = sigma[a]
        assert np.allclose(dg._rotate(ops, Kr, ipi, isg), K, atol=1e-12)


def test_geometry_tiles_the_domain():
    """Jittered, refined cells tile the unit cube: total volume 1, and the
    p+1 point Gauss rule integrates J exactly (J has degree <= 2 per axis)."""
    F = FO.build(W.jitter3d_forest(seed=1, n_seg=2))
    vol = 0.0
    for key in F.leaves():
        C = F.cell_corners(key)
        x3, w3 = B.tensor_points(3, 3)
        x6, w6 = B.tensor_points(3, 6)
        _, J3, _ = dg.jacobian(C, x3)
        _, J6, _ = dg.jacobian(C, x6)
        v3 = J3 @ w3
        assert np.allclose(v3, J6 @ w6, rtol=1e-13)
        assert np.all(v3 > 0)
        vol += v3.sum()
    assert abs(vol - 1.0) < 1e-13
