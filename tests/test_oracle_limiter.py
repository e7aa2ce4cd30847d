"""Pins for the oracle's positivity limiter (reading R17, the scaling limiter
of Zhang & Shu): admissible cells are untouched; limited cells keep their
J-weighted mean, are a single scaling of the polynomial about that mean,
reach the bound with equality (the scaling is the largest admissible) and
have rho, p >= eps at every volume and face Gauss point; a blast that breaks
down without the limiter runs with it and conserves its totals."""
import numpy as np
import pytest

import workloads as W
from oracle import dg
from oracle import forest as FO
from oracle import limiter as LIM
from oracle.euler import primitives

EPS = 1e-6


def _check_points(S, K):
    Pchk = np.concatenate([S.ops.Phi] + [S.ops.faces[f][2] for f in range(2 * S.d)], axis=0)
    return Pchk @ K.T


def _stressed_state(S, seed):
    """A random admissible state with a few cells pushed to negative density
    or pressure at some points (large higher modes)."""
    rng = np.random.default_rng(seed)
    U = W.random_modal_state(len(S.leaves), S.d, S.n, S.p, seed=seed)
    for li in range(len(S.leaves)):
        for c in rng.choice(U.shape[3], size=2, replace=False):
            U[li, :, 1:, c] *= 25.0  # oscillations larger than the mean
    return U


@pytest.mark.parametrize("case,p", [("jitter_3d", 1), ("jitter_3d", 2), ("pair_2d", 3)])
def test_limited_cells_are_admissible_mean_preserving_scalings(case, p):
    w = W.jitter3d_forest(seed=1, n_seg=2) if case == "jitter_3d" else W.rotated_pair_2d(n_seg=2)
    S = dg.Solver(FO.build(w), p)
    U = _stressed_state(S, seed=p)
    V, changed, bad = LIM.positivity_limit(S, U, EPS)
    assert changed > 0 and bad == 0
    ops = S.ops
    n_active = 0
    for li in range(len(S.leaves)):
        J, _ = S.geo_vol[li]
        for c in range(U.shape[3]):
            K, L = U[li, :, :, c], V[li, :, :, c]
            wj = ops.wq * J[c]
            ubar = wj @ (ops.Phi @ K.T) / wj.sum()
            vbar = wj @ (ops.Phi @ L.T) / wj.sum()
            assert np.max(np.abs(vbar - ubar)) < 1e-13 * np.max(np.abs(ubar))
            rb, _, pb = primitives(ubar[None])
            vals = _check_points(S, L)
            r, _, pr = primitives(vals)
            # the bounds hold up to the round-off of evaluating O(1) terms
            assert r.min() >= (EPS - 1e-13) * rb[0] and pr.min() >= (EPS - 1e-13) * pb[0]
            if np.array_equal(K, L):
                continue
            # a single scaling about the mean
            D0, D1 = K.copy(), L.copy()
            D0[:, 0] -= ubar
            D1[:, 0] -= ubar
            theta = float(np.sum(D1 * D0) / np.sum(D0 * D0))
            assert 0 <= theta < 1 and np.max(np.abs(D1 - theta * D0)) < 1e-12 * np.max(np.abs(D0))
            # the largest admissible scaling: one bound is met
            slack = min(r.min() / (EPS * rb[0]), pr.min() / (EPS * pb[0]))
            assert abs(slack - 1.0) < 1e-6
            n_active += 1
    assert n_active == changed


def test_admissible_state_is_untouched():
    S = dg.Solver(FO.build(W.jitter3d_forest(seed=2, n_seg=2)), 2)
    U = W.random_modal_state(len(S.leaves), 3, 2, 2, seed=3)
    V, changed, bad = LIM.positivity_limit(S, U, EPS)
    assert changed == 0 and bad == 0 and np.array_equal(U, V)


def test_pressure_root_closed_form():
    """Zero momentum: p is linear in t, p(t) = p_bar + t (p~ - p_bar)."""
    g = 1.4
    ubar = np.array([1.0, 0.0, 0.0, 2.0 / (g - 1)])    # rho 1, p 2
    du = np.array([0.0, 0.0, 0.0, -3.0 / (g - 1)])     # p~ = -1
    t = LIM._pressure_root(ubar, du, 0.5, g)
    assert abs(t - 0.5) < 1e-15  # 2 - 3t = 0.5


def test_blast_runs_with_the_limiter_and_conserves():
    w = W.lattice_forest(3, 2, 1.0, 2, rotate_roots=True, seed=1)
    ic = lambda x: W.blast(x, (0.3, 0.3, 0.3), r0=0.15, width=0.08)
    S0 = dg.Solver(FO.build(w), 1)
    U0 = S0.project(ic)
    with np.errstate(all="ignore"):
        bad = ~np.isfinite(S0.ssp_rk3_step(U0, S0.dt(U0)))
    assert bad.any()  # breaks down without the limiter
    S = dg.Solver(FO.build(w), 1, limiter=EPS)
    U = LIM.positivity_limit(S, U0, EPS)[0]  # the initial data too
    T0 = S.totals(U)
    for _ in range(6):
        U = S.ssp_rk3_step(U, S.dt(U))
    assert np.all(np.isfinite(U))
    r, _, pr = primitives(np.einsum("qm,lvmc->lcqv", S.ops.Phi, U))
    assert r.min() > 0 and pr.min() > 0
    # periodic forest: the scheme and the limiter (which keeps every cell
    # mean) conserve the totals
    assert np.max(np.abs(S.totals(U) - T0)) < 1e-12 * np.max(np.abs(T0))
