"""Pins for the oracle's mortar treatment of level jumps (reading R15): the
totals are conserved to round-off on multilevel forests, a free stream stays
exact, a state whose flux is a polynomial gets the exact residual (so the
coarse-side quadrature points and weights are right, through rotated roots),
and nothing changes on single-level forests."""
import numpy as np
import pytest

import workloads as W
from oracle import dg
from oracle import forest as FO


def _conservation(w, p, mode, steps=2, seed=0):
    S = dg.Solver(FO.build(w), p, cfl=0.1, nonconforming=mode)
    U = W.random_modal_state(len(S.leaves), S.d, S.n, p, seed=seed)
    T0 = S.totals(U)
    U, _ = S.run(U, steps)
    return np.max(np.abs(S.totals(U) - T0)) / np.max(np.abs(T0))


@pytest.mark.parametrize("case,p", [("pair_2d", 2), ("pair_2d", 0), ("jitter_3d", 1), ("jitter_3d", 2)])
def test_mortar_conserves_totals_across_level_jumps(case, p):
    w = W.rotated_pair_2d(n_seg=2) if case == "pair_2d" else W.jitter3d_forest(seed=3, n_seg=2)
    assert _conservation(w, p, "mortar") < 1e-14
    if p > 0:
        assert _conservation(w, p, "paper") > 1e-10  # the paper's scheme drifts


@pytest.mark.parametrize("p,seed", [(1, 0), (2, 1), (3, 2)])
def test_mortar_free_stream(p, seed):
    S = dg.Solver(FO.build(W.jitter3d_forest(seed=seed, n_seg=2)), p, nonconforming="mortar")
    assert np.max(np.abs(S.residual(S.project(W.free_stream)))) < 1e-10


def test_mortar_equals_paper_on_single_level_forests():
    w = W.jitter3d_forest(seed=2, n_seg=2)
    w["refine"] = []
    U = W.random_modal_state(8, 3, 2, 2, seed=4)
    La = dg.Solver(FO.build(w), 2).residual(U)
    Lb = dg.Solver(FO.build(w), 2, nonconforming="mortar").residual(U)
    assert np.array_equal(La, Lb)


def _affine_multilevel_3d():
    # 2x2x2 rotated affine roots, outflow boundaries, two refinement levels
    w = W.lattice_forest(3, 2, 1.0, 2, periodic=False, rotate_roots=True, seed=7)
    w["refine"] = [[(0, 1, (0, 0, 0)), (5, 1, (0, 0, 0))], [(0, 2, (1, 1, 1))]]
    return w


def _grad_rho(x, p):
    X, Y, Z = x[..., 0], x[..., 1], x[..., 2]
    g = [np.full_like(X, 0.1), np.full_like(X, 0.2), np.full_like(X, -0.15)]
    if p >= 2:
        g = [g[0] + 0.05 * Y, g[1] + 0.05 * X - 0.08 * Y, g[2]]
    if p >= 3:
        g = [g[0] + 0.06 * X * X - 0.03 * Y * Z, g[1] - 0.03 * X * Z, g[2] - 0.03 * X * Y]
    return np.stack(g, -1)


@pytest.mark.parametrize("mode", ["mortar", "paper"])
@pytest.mark.parametrize("p", [1, 2, 3])
def test_exact_residual_for_polynomial_flux(mode, p):
    """u, pressure constant and rho a degree-p polynomial: the flux is a
    degree-p polynomial, the traces are continuous (no LF dissipation) and
    every integral is exact at the (p+1)-point rule on affine cells, so
    L(U) = -div F(U) = -(u.grad rho)(1, u, |u|^2/2) at every Gauss point."""
    S = dg.Solver(FO.build(_affine_multilevel_3d()), p, nonconforming=mode)
    assert any(k == dg.FINER for kk in S.kinds for k in kk)
    U = S.project(lambda x: W.advected_polynomial(x, p))
    L = S.residual(U)
    xq = S.quad_points()
    u = np.array(W.ADVECT_VEL)
    adv = -np.einsum("lcqa,a->lcq", _grad_rho(xq, p), u)
    want = adv[..., None] * np.concatenate([[1.0], u, [0.5 * u @ u]])
    got = np.einsum("qm,lvmc->lcqv", S.ops.Phi, L)
    # round-off of O(1) fluxes through 2/h_min = 32 and the degree-p lift
    assert np.max(np.abs(got - want)) < 1e-12 * (p + 1) ** 2 / 4


def test_planted_mortar_orientation_slip_is_caught(monkeypatch):
    """Reversing the tangential axes in the coarse-side point map (a wrong
    axis flip) breaks the exact-residual pin."""
    real = dg.Solver._coarse_points

    def flip(xc):
        out = xc.copy()
        tang = ~np.all(np.abs(xc) == 1.0, axis=0)
        out[:, tang] *= -1.0
        return out

    def slipped(self, li, f):
        ci, pts = real(self, li, f)
        return ci, [(h, flip(xc)) for h, xc in pts]
    monkeypatch.setattr(dg.Solver, "_coarse_points", slipped)
    S = dg.Solver(FO.build(_affine_multilevel_3d()), 2, nonconforming="mortar")
    U = S.project(lambda x: W.advected_polynomial(x, 2))
    L = S.residual(U)
    xq = S.quad_points()
    u = np.array(W.ADVECT_VEL)
    adv = -np.einsum("lcqa,a->lcq", _grad_rho(xq, 2), u)
    want = adv[..., None] * np.concatenate([[1.0], u, [0.5 * u @ u]])
    got = np.einsum("qm,lvmc->lcqv", S.ops.Phi, L)
    assert np.max(np.abs(got - want)) > 1e-4
