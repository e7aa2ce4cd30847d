"""Pins for the oracle's residual and time march against what the method
fixes: an independent textbook 1D DG, free-stream preservation, conservation,
the SSP-RK3 stability polynomial, design order on the isentropic vortex, and
restriction(prolongation(u)) = u through a regrid."""
import copy
import itertools
import math

import numpy as np
import pytest

import workloads as W
from oracle import basis as B
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


# ------------------------------------------------------- time increment (reading R5)
def _one_cell_3d(moved_corner_offset, n_seg=1, corner=7):
    """One root on the unit cube (outflow faces) whose corner `corner` (bit a
    of the index = side along axis a) is moved by the given offset; its
    n_seg^3 cells are trilinear in the root's corners."""
    nodes = np.array([[(k >> a) & 1 for a in range(3)] for k in range(8)], float)
    nodes[corner] += np.asarray(moved_corner_offset, float)
    return dict(dim=3, n_seg=n_seg, nodes=nodes, root_corners=np.arange(8, dtype=np.int64)[None],
                root_cell_nodes=None, periodic=[], refine=[])


def _lam(prim):
    """sum_i (|u_i| + c) of one primitive state (rho, u, v, w, p)."""
    rho, u, pr = prim[0], np.asarray(prim[1:4]), prim[4]
    return float(np.sum(np.abs(u)) + 3.0 * math.sqrt(1.4 * pr / rho))


@pytest.mark.parametrize("p", [0, 1, 2])
def test_dt_closed_form_uniform_state_affine_cube(p):
    """Affine periodic cube of 2^3 roots with 2^3 cells each (edge h = 1/4):
    dt = CFL h / sum_i(|u_i| + c) for a uniform state."""
    prim = (1.3, 0.4, -0.7, 0.2, 0.8)
    S = dg.Solver(FO.build(W.periodic_cube_forest(2, n_seg=2)), p, cfl=0.3)
    U = S.project(lambda x: W.free_stream(x, state=prim))
    assert abs(S.dt(U) - 0.3 * 0.25 / _lam(prim)) < 1e-14


@pytest.mark.parametrize("delta", [(0.1, -0.05, 0.08), (-0.2, -0.1, -0.15)])
def test_dt_closed_form_jittered_single_cell(delta):
    """One trilinear cell, the unit cube with corner (1,1,1) moved by delta:
    J = 1 + delta . grad(s0 s1 s2), so the volume is 1 + (d0 + d1 + d2)/4
    and h = volume^(1/3)."""
    prim = (0.9, -0.3, 0.5, 0.1, 1.2)
    S = dg.Solver(FO.build(_one_cell_3d(delta)), 1, cfl=0.25)
    U = S.project(lambda x: W.free_stream(x, state=prim))
    h = (1.0 + sum(delta) / 4.0) ** (1.0 / 3.0)
    assert abs(S.dt(U) - 0.25 * h / _lam(prim)) < 1e-14


def test_dt_is_the_minimum_over_cells():
    """Root of 2^3 cells of edge 1/2 whose centre node is moved by delta:
    the cell with that node as its corner k has volume
    h^3 (1 + sum_a s_a delta_a / (4 h)), s_a = +1 if the node is on the
    cell's upper side along axis a; the smallest volume sets dt."""
    delta = np.array([0.06, -0.04, 0.05])
    w = _one_cell_3d((0, 0, 0), n_seg=2)
    cn = np.array([[i, j, k] for k in range(3) for j in range(3) for i in range(3)], float) / 2.0
    cn[13] += delta  # the centre node (1, 1, 1) of the 3^3 cell-node lattice
    w["root_cell_nodes"] = cn[None]
    prim = (1.0, 0.2, 0.3, -0.4, 1.0)
    S = dg.Solver(FO.build(w), 1, cfl=0.2)
    U = S.project(lambda x: W.free_stream(x, state=prim))
    vols = []
    for bits in itertools.product((0, 1), repeat=3):  # cell at the lower (0) or upper (1) half
        s = np.array([1.0 if b == 0 else -1.0 for b in bits])  # the centre is the cell's upper corner when b = 0
        vols.append(0.125 * (1.0 + float(s @ delta) / (4 * 0.5)))
    assert abs(S.dt(U) - 0.2 * min(vols) ** (1 / 3) / _lam(prim)) < 1e-14


def test_dt_is_the_minimum_over_gauss_points():
    """Unit cube cell, p = 1, rho u = a + b P_1(xi_x) with the other
    conserved variables constant: velocity and sound speed differ at the two
    Gauss points xi_x = -+1/sqrt(3); dt takes the larger sum_i(|u_i| + c)."""
    S = dg.Solver(FO.build(_one_cell_3d((0, 0, 0))), 1, cfl=0.4)
    U = np.zeros(S.shape())
    rho, a, b, E = 1.1, 0.3, 0.5, 2.5
    U[0, 0, 0, 0] = rho
    U[0, 1, 0, 0] = a
    U[0, 1, 1, 0] = b  # mode k = (1, 0, 0)
    U[0, 4, 0, 0] = E
    lam = []
    for xi in (-1 / math.sqrt(3), 1 / math.sqrt(3)):
        u = (a + b * xi) / rho
        pr = 0.4 * (E - 0.5 * rho * u * u)
        lam.append(abs(u) + 3.0 * math.sqrt(1.4 * pr / rho))
    assert abs(S.dt(U) - 0.4 * 1.0 / max(lam)) < 1e-14


def test_run_clips_the_last_increment_to_t_end():
    """The last increment is shortened so the march ends at t_end exactly."""
    S = dg.Solver(FO.build(W.periodic_cube_forest(1, n_seg=2)), 1, cfl=0.3)
    U = S.project(lambda x: W.free_stream(x, state=(1.0, 0.5, 0.0, 0.0, 1.0)))
    dt = S.dt(U)
    t_end = 2.5 * dt
    _, t = S.run(U, 100, t_end=t_end)
    assert t == pytest.approx(t_end, rel=0, abs=1e-15)
    _, t2 = S.run(U, 2, t_end=t_end)
    assert t2 == pytest.approx(2 * dt, rel=1e-15)


# ------------------------------------------------------- design order, p = 1..3
def _entropy_wave(x, t=0.0, d=2):
    """rho = 1 + 0.2 sin(2 pi (sum_a x_a - d t)), unit velocity along every
    axis, unit pressure: an exact Euler solution (the density is carried by
    the flow), periodic on the unit square/cube."""
    x = np.asarray(x, float)
    s = 2 * math.pi * (np.sum(x, axis=-1) - x.shape[-1] * t)
    vel = np.ones(x.shape[:-1] + (x.shape[-1],))
    return W.prim_to_cons(1.0 + 0.2 * np.sin(s), vel, np.ones(x.shape[:-1]))


def _l2_error_overintegrated(S, U, fun, extra=3):
    """Relative L2 error against fun with a Gauss rule of p + 1 + extra points
    per axis (the error between the Gauss points counts too)."""
    xq, wq = B.tensor_points(S.d, S.ops.N + extra)
    Phi = B.eval_basis(xq, S.ops.N)
    num = den = 0.0
    for li, C in enumerate(S.corners):
        ex = fun(dg.map_points(C, xq))
        uq = np.einsum("qm,vmc->cqv", Phi, U[li])
        _, J, _ = dg.jacobian(C, xq)
        num += float(np.einsum("q,cq,cqv->", wq, J, (uq - ex) ** 2))
        den += float(np.einsum("q,cq,cqv->", wq, J, ex ** 2))
    return math.sqrt(num / den)


def _wave_error(w, p, t_end, dt):
    S = dg.Solver(FO.build(w), p, cfl=1.0)
    U = S.project(_entropy_wave)
    t = 0.0
    while t < t_end - 1e-14:
        h = min(dt, t_end - t)
        U = S.ssp_rk3_step(U, h)
        t += h
    return _l2_error_overintegrated(S, U, lambda x: _entropy_wave(x, t))


# (p, n_seg pair, t_end, dt): even p needs finer cells before the observed
# order settles at p + 1 (2.53 at n = 4 -> 8, 2.91 at 8 -> 16 in 2D)
WAVE_2D = {1: ((2, 4), 0.05, 2e-3), 2: ((8, 16), 0.03, 5e-4), 3: ((2, 4), 0.05, 1e-3)}


@pytest.mark.parametrize("p", [1, 2, 3])
def test_entropy_wave_design_order_2d_two_levels(p):
    """Design order p + 1 (Sec. 5.1, the conclusion's optimal-order claim) on
    a 2-level forest: 2x2 roots of the periodic unit square with one root
    refined, cells halved by doubling n_seg; a fixed small time step keeps
    the SSP-RK3 error below the spatial one."""
    ns, t_end, dt = WAVE_2D[p]
    errs = []
    for n in ns:
        w = W.lattice_forest(2, 2, 1.0, n)
        w["refine"] = [[(0, 1, (0, 0))]]
        errs.append(_wave_error(w, p, t_end, dt))
    order = math.log2(errs[0] / errs[1])
    assert order > p + 0.8, (errs, order)


def test_entropy_wave_design_order_3d_two_levels_p1():
    """Design order p + 1 in 3D on a 2-level forest: 2^3 periodic roots, one
    refined, n_seg 2 -> 4."""
    errs = []
    for n in (2, 4):
        w = W.periodic_cube_forest(2, n_seg=n)
        w["refine"] = [[(0, 1, (0, 0, 0))]]
        errs.append(_wave_error(w, 1, 0.02, 2e-3))
    order = math.log2(errs[0] / errs[1])
    assert order > 1.8, (errs, order)


def test_entropy_wave_design_order_3d_p3():
    """Design order p + 1 in 3D at p = 3: one periodic root, n_seg 2 -> 4."""
    errs = []
    for n in (2, 4):
        errs.append(_wave_error(W.periodic_cube_forest(1, n_seg=n), 3, 0.03, 1e-3))
    order = math.log2(errs[0] / errs[1])
    assert order > 3.8, (errs, order)
