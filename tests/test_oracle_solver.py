"""Pins for the oracle's residual and time march against what the method
fixes: an independent textbook 1D DG, free-stream preservation, conservation,
the SSP-RK3 stability polynomial, design order on the isentropic vortex, and
restriction(prolongation(u)) = u through a regrid."""
import copy

import numpy as np
import pytest

import workloads as W
from oracle import dg
from oracle import euler as E
from oracle import forest as FO

GAM = 1.4


# ------------------------------------------------------------ textbook 1D DG
def _leg(k, x):
    return np.polynomial.legendre.legval(x, [0] * k + [1])


def _leg_d(k, x):
    return np.polynomial.legendre.legval(x, np.polynomial.legendre.legder([0] * k + [1]))


def _flux1d(u):
    rho, m, En = u[..., 0], u[..., 1], u[..., 2]
    vel = m / rho
    p = (GAM - 1) * (En - 0.5 * rho * vel ** 2)
    return np.stack([m, m * vel + p, vel * (En + p)], -1), vel, np.sqrt(GAM * p / rho)


def dg1d_residual(U, h, p):
    """Modal DG on a periodic 1D grid: U[cell, var, k]; returns dU/dt."""
    N = p + 1
    x, w = np.polynomial.legendre.leggauss(N)
    V = np.array([[_leg(k, xq) for k in range(N)] for xq in x])
    dV = np.array([[_leg_d(k, xq) for k in range(N)] for xq in x])
    uq = np.einsum("qk,cvk->cqv", V, U)
    F, _, _ = _flux1d(uq)
    r = np.einsum("q,cqv,qk->cvk", w, F, dV)
    plus = np.array([1.0] * N)
    minus = np.array([(-1.0) ** k for k in range(N)])
    uR = U @ plus          # trace at xi=+1 of each cell
    uL = U @ minus         # trace at xi=-1
    a, b = uR, np.roll(uL, -1, axis=0)   # face c+1/2: left state a, right b
    Fa, va, ca = _flux1d(a)
    Fb, vb, cb = _flux1d(b)
    alpha = np.maximum(np.abs(va) + ca, np.abs(vb) + cb)
    Fh = 0.5 * (Fa + Fb + alpha[:, None] * (a - b))
    r -= Fh[:, :, None] * plus[None, None, :]
    r += np.roll(Fh, 1, axis=0)[:, :, None] * minus[None, None, :]
    mass = (h / 2) * np.array([2.0 / (2 * k + 1) for k in range(N)])
    return r / mass


def _dg1d_setup(K, h, p, fun):
    N = p + 1
    x, w = np.polynomial.legendre.leggauss(N)
    Vinv = np.array([[(2 * k + 1) / 2 * w[q] * _leg(k, x[q]) for q in range(N)] for k in range(N)])
    U = np.zeros((K, 3, N))
    for c in range(K):
        xp = (c + 0.5 * (x + 1)) * h
        vals = fun(np.stack([xp, np.zeros_like(xp)], -1))   # 2D state, v = 0
        v3 = vals[:, [0, 1, 3]]
        U[c] = (Vinv @ v3).T
    return U


def _eval1d(U, h, x, p):
    c = np.floor(x / h).astype(int) % U.shape[0]
    xi = 2 * (x - c * h) / h - 1
    P = np.stack([_leg(k, xi) for k in range(p + 1)], -1)
    return np.einsum("pk,pvk->pv", P, U[c])


def _compare_1d(p):
    """Max deviation between the oracle on the rotated root pair (state
    constant along global y) and the textbook 1D DG on the same x cells."""
    n = 4
    w = W.rotated_pair_2d(n_seg=n, refine_root0=False)
    S = dg.Solver(FO.build(w), p)
    U = S.project(W.smooth_x_state)
    L = S.residual(U)
    K = 8
    h = 2.0 / K
    U1 = _dg1d_setup(K, h, p, W.smooth_x_state)
    L1 = dg1d_residual(U1, h, p)
    xq = S.quad_points()
    errs = []
    for li in range(len(S.leaves)):
        Lq = np.einsum("qm,vmc->cqv", S.ops.Phi, L[li])
        ref = _eval1d(L1, h, xq[li][..., 0].ravel(), p).reshape(Lq.shape[0], Lq.shape[1], 3)
        errs.append(np.max(np.abs(Lq[..., [0, 1, 3]] - ref)))
        errs.append(np.max(np.abs(Lq[..., 2])))
    return max(errs)


@pytest.mark.parametrize("p", [0, 1, 2, 3])
def test_reduces_to_textbook_1d_dg_through_rotated_roots(p):
    assert _compare_1d(p) < 1e-11


def test_planted_lf_sign_flip_is_caught(monkeypatch):
    """Planting the printed sign of Eq. (5) (anti-dissipative for an outward
    normal) in the oracle must break the 1D reduction pin."""
    orig = E.lax_friedrichs

    def flipped(UL, UR, n, gamma=GAM):
        FLR = orig(UL, UR, n, gamma)
        Fc = orig(UL, UL, n, gamma) * 0.5 + orig(UR, UR, n, gamma) * 0.5
        return 2 * Fc - FLR
    monkeypatch.setattr(dg, "lax_friedrichs", flipped)
    assert _compare_1d(2) > 1e-3


def test_planted_rotation_drop_is_caught(monkeypatch):
    monkeypatch.setattr(dg, "_rotate", lambda ops, K, pi, sigma: K)
    assert _compare_1d(2) > 1e-3


# ------------------------------------------------------- invariants
@pytest.mark.parametrize("p,seed", [(1, 0), (2, 1), (3, 2)])
def test_free_stream_preserved_on_jittered_rotated_multilevel(p, seed):
    S = dg.Solver(FO.build(W.jitter3d_forest(seed=seed, n_seg=2)), p)
    U = S.project(W.free_stream)
    L = S.residual(U)
    assert np.max(np.abs(L)) < 1e-10


@pytest.mark.parametrize("case", ["single_root", "strip3"])
@pytest.mark.parametrize("p", [1, 3])
def test_free_stream_preserved_on_paper_2d_root_sets(case, p):
    """The self-glued single root and the three rotated rectangular roots of
    the 2D convection test (Sec. 5), each with a level jump."""
    w = W.single_root_2d(n_seg=4) if case == "single_root" else W.three_root_strip_2d(n_seg=4)
    S = dg.Solver(FO.build(w), p)
    L = S.residual(S.project(W.free_stream))
    assert np.max(np.abs(L)) < 1e-10


def test_free_stream_preserved_with_outflow_boundaries():
    w = W.lattice_forest(2, 2, 1.0, 2, periodic=False, jitter=0.1, seed=4)
    w["refine"] = [[(0, 1, (0, 0))]]
    S = dg.Solver(FO.build(w), 2)
    L = S.residual(S.project(W.free_stream))
    assert np.max(np.abs(L)) < 1e-11


def _conservation(w, p, steps=2, seed=0):
    S = dg.Solver(FO.build(w), p, cfl=0.1)
    U = W.random_modal_state(len(S.leaves), S.d, S.n, p, seed=seed)
    T0 = S.totals(U)
    U, _ = S.run(U, steps)
    return np.max(np.abs(S.totals(U) - T0)) / np.max(np.abs(T0))


def test_conservation_single_level_periodic():
    assert _conservation(W.rotated_pair_2d(n_seg=2, refine_root0=False), 2) < 1e-14
    w = W.jitter3d_forest(seed=2, n_seg=2)
    w["refine"] = []
    assert _conservation(w, 1) < 1e-14


def test_multilevel_guard_fill_is_not_conservative():
    """Sec. 3.5's guard-cell scheme evaluates the coarse and fine side fluxes
    from different data, so the totals drift on multilevel forests."""
    assert _conservation(W.rotated_pair_2d(n_seg=2), 2) > 1e-10


def test_ssp_rk3_stability_polynomial():
    class Lin(dg.Solver):
        def __init__(self, lam):
            self.lam = lam

        def residual(self, U):
            return self.lam * U
    for z in (-0.3, -1.0, 0.5, -2.2):
        out = Lin(z).ssp_rk3_step(np.array([1.0]), 1.0)[0]
        assert abs(out - (1 + z + z * z / 2 + z ** 3 / 6)) < 1e-15


def test_regrid_restriction_of_prolongation_is_identity():
    w = W.jitter3d_forest(seed=5, n_seg=2)
    w["refine"] = [w["refine"][0]]
    F = FO.build(w)
    S0 = dg.Solver(F, 2)
    U0 = W.random_modal_state(len(S0.leaves), 3, 2, 2, seed=3)
    F1 = copy.deepcopy(F)
    F1.refine([S0.leaves[5], S0.leaves[40]])
    S1 = dg.Solver(F1, 2)
    U1 = S1.regrid_state(S0, U0)
    F2 = copy.deepcopy(F1)
    parents = sorted({(k[0], k[1] - 1, tuple(x >> 1 for x in k[2]))
                      for k in set(S1.leaves) - set(S0.leaves)})
    F2.coarsen(parents)
    S2 = dg.Solver(F2, 2)
    assert S2.leaves == S0.leaves
    U2 = S2.regrid_state(S1, U1)
    assert np.max(np.abs(U2 - U0)) < 1e-12


# ------------------------------------------------------- design order
@pytest.mark.parametrize("p", [1, 2])
def test_vortex_design_order(p):
    errs = []
    for n in (4, 8):
        w = W.lattice_forest(2, 2, 10.0, n)
        S = dg.Solver(FO.build(w), p, cfl=0.1)
        U = S.project(W.isentropic_vortex)
        U, t = S.run(U, 100000, t_end=0.5)
        errs.append(S.l2_error(U, lambda x: W.vortex_exact(x, t)))
    order = np.log2(errs[0] / errs[1])
    assert order > p + 0.6, (errs, order)


def test_prescribed_state_boundaries():
    """A free stream stays exact when the tagged boundary faces prescribe that
    same state (jittered, refined, non-periodic forest); a different
    prescribed state changes only the cells next to tagged faces, and
    tagging no face equals the outflow default."""
    w = W.lattice_forest(2, 2, 1.0, 2, periodic=False, jitter=0.1, seed=4)
    w["refine"] = [[(0, 1, (0, 0))]]
    F = FO.build(w)
    R = len(w["root_corners"])
    fs = (1.0, 0.3, -0.2, 1.0)
    state = W.free_stream(np.zeros((1, 2)), state=fs)[0]
    tags = [[1, 1, 1, 1] for _ in range(R)]
    S = dg.Solver(F, 2, boundary=(tags, state))
    L = S.residual(S.project(lambda x: W.free_stream(x, state=fs)))
    assert np.max(np.abs(L)) < 1e-11
    U = W.random_modal_state(len(S.leaves), 2, 2, 2, seed=5)
    S0 = dg.Solver(FO.build(w), 2)
    Sn = dg.Solver(FO.build(w), 2, boundary=([[0] * 4 for _ in range(R)], state))
    assert np.array_equal(S0.residual(U), Sn.residual(U))
    tags1 = [[1, 0, 0, 0] for _ in range(R)]  # x- faces only
    S1 = dg.Solver(FO.build(w), 2, boundary=(tags1, 2.0 * state))
    D = np.abs(S1.residual(U) - S0.residual(U)).max(axis=(1, 2))  # per (leaf, cell)
    T = FO.build(w).leaf_table()
    cells_x0 = np.array([c % 2 == 0 for c in range(4)])  # the cells next to x-
    for li in range(len(S1.leaves)):
        on_xminus = T["kind"][li][0] == 3
        assert np.all(D[li][~cells_x0] == 0)
        assert np.any(D[li][cells_x0] > 0) == on_xminus
