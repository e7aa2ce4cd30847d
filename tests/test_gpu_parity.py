"""GPU parity: the CUDA path through the C ABI against the FP64 oracle, element
by element, on seeded inputs (random valid modal states and closed-form
initial conditions).  Tolerances: FP64 relative L2 <= 1e-12, FP32 <= 1e-5
(the bars the FP64 and FP32 forms are held to)."""
import copy

import numpy as np
import pytest

import workloads as W
from oracle import dg
from oracle import forest as FO

pytestmark = pytest.mark.gpu

TOL = {"fp64": 1e-12, "fp32": 1e-5}


@pytest.fixture(scope="module")
def dgf():
    import paper_2502_12620_gb300 as pkg
    pkg.lib()
    return pkg


def rel(a, b):
    return float(np.linalg.norm((np.asarray(a, float) - b).ravel()) / max(np.linalg.norm(np.ravel(b)), 1e-300))


def modal_gain(d, p):
    """Infinity norm of the map from values at the (p+1)^d Gauss points to
    the modal coefficients of the output (K_k = (2k+1)/2 sum_q w_q P_k(x_q)
    u_q per axis): the factor by which an error in the point values can grow
    in one modal coefficient (1, 5.2, 11.0, 18.0 for p = 0..3 in 3D)."""
    N = p + 1
    x, w = np.polynomial.legendre.leggauss(N)
    rows = [sum(abs((2 * k + 1) / 2 * w[q] * np.polynomial.legendre.legval(x[q], [0] * k + [1]))
                for q in range(N)) for k in range(N)]
    return max(rows) ** d


def assert_matches(L, Lo, prec, S, U):
    """Relative L2 over the whole array and, element by element, the largest
    deviation against the size of the terms summed into L at the Gauss
    points times the growth of the point-to-mode map (so one wrong face
    point in one leaf cannot hide in the global norm, while the round-off of
    a correct FP32 evaluation, which that map amplifies in the top modes at
    p = 3, stays inside the bound)."""
    tol = TOL["fp64" if prec == "fp64" else "fp32"]
    e = rel(L, Lo)
    assert e < tol, e
    emax = float(np.max(np.abs(np.asarray(L, float) - Lo)))
    bound = tol * term_scale(S, U) * modal_gain(S.d, S.p)
    assert emax < bound, (emax, bound)


def _pair(dgf, w, p, prec, cfl=0.1):
    f = dgf.Forest.from_workload(w, p=p, precision=prec, cfl=cfl)
    S = dg.Solver(FO.build(w), p, cfl=cfl)
    return f, S


SMALL = {
    "pair_2d": lambda: W.rotated_pair_2d(n_seg=4),
    "vortex_2d_n4": lambda: dict(W.vortex2d_forest(), n_seg=4, root_cell_nodes=None),
    "jitter_3d_n2": lambda: W.jitter3d_forest(seed=1, n_seg=2),
    "jitter_3d_n4": lambda: W.jitter3d_forest(seed=4, n_seg=4),
    "cube_rot_3d": lambda: W.periodic_cube_forest(2, n_seg=2, rotate_roots=True, seed=5),
    "outflow_2d": lambda: dict(W.lattice_forest(2, 2, 1.0, 4, periodic=False, jitter=0.1, seed=2),
                               refine=[[(0, 1, (0, 0))]]),
    "single_root_2d": lambda: W.single_root_2d(n_seg=4),
    "strip3_2d": lambda: W.three_root_strip_2d(n_seg=4),
}


def _small(case):
    w = SMALL[case]()
    if case == "vortex_2d_n4":
        w = W.lattice_forest(2, 4, 10.0, 4)
        w["refine"] = W.vortex2d_forest()["refine"]
    return w


@pytest.mark.parametrize("case", sorted(SMALL))
@pytest.mark.parametrize("p", [0, 1, 2, 3])
def test_guardcells_match_oracle(dgf, case, p):
    w = _small(case)
    if w["dim"] == 3 and p == 3 and case == "jitter_3d_n4":
        pytest.skip("covered by n2")
    f, S = _pair(dgf, w, p, dgf.FP64)
    U = W.random_modal_state(f.n_leaves, f.dim, f.n_seg, p, seed=p + 7)
    f.set_state(U)
    G = f.fill_guardcells()
    Go = S.fill_guardcells(U)
    assert rel(G, Go) < TOL["fp64"]


@pytest.mark.parametrize("case", sorted(SMALL))
@pytest.mark.parametrize("p", [0, 1, 2, 3])
@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_residual_matches_oracle(dgf, case, p, prec):
    w = _small(case)
    f, S = _pair(dgf, w, p, dgf.FP64 if prec == "fp64" else dgf.FP32)
    U = W.random_modal_state(f.n_leaves, f.dim, f.n_seg, p, seed=p + 11)
    f.set_state(U)
    Uin = U.astype(f.dtype).astype(np.float64)
    L = f.dg_residual()
    Lo = S.residual(Uin)
    assert_matches(L, Lo, prec, S, Uin)


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_free_stream_preserved(dgf, prec):
    w = W.jitter3d_forest(seed=2, n_seg=4)
    f = dgf.Forest.from_workload(w, p=2, precision=dgf.FP64 if prec == "fp64" else dgf.FP32)
    f.project(W.free_stream)
    L = f.dg_residual()
    scale = 1.0 / (0.25 / 4 / 2)  # |F| / h_min
    assert np.max(np.abs(L)) < (1e-11 if prec == "fp64" else 2e-4) * scale


@pytest.mark.parametrize("case", ["pair_2d", "jitter_3d_n2", "outflow_2d", "strip3_2d"])
def test_rk_steps_match_oracle(dgf, case):
    w = _small(case)
    f, S = _pair(dgf, w, 2, dgf.FP64, cfl=0.2)
    U = W.random_modal_state(f.n_leaves, f.dim, f.n_seg, 2, seed=3)
    f.set_state(U)
    dt_gpu = f.compute_dt()
    assert abs(dt_gpu - S.dt(U)) <= 1e-13 * S.dt(U)
    for _ in range(3):
        dt_o = S.dt(U)
        U = S.ssp_rk3_step(U, dt_o)
        f.rk_step()
    assert rel(f.get_state(), U) < TOL["fp64"]
    assert abs(f.time - 0) > 0


def test_totals_match_oracle_and_single_level_conservation(dgf):
    w = W.jitter3d_forest(seed=6, n_seg=2)
    w["refine"] = []
    f, S = _pair(dgf, w, 2, dgf.FP64)
    U = W.random_modal_state(f.n_leaves, 3, 2, 2, seed=8)
    f.set_state(U)
    T0 = f.conserved_totals()
    assert np.allclose(T0, S.totals(U), rtol=1e-13, atol=1e-15)
    for _ in range(5):
        f.rk_step()
    T1 = f.conserved_totals()
    assert np.max(np.abs(T1 - T0)) / np.max(np.abs(T0)) < 1e-13


def test_vortex2d_100_steps_matches_oracle(dgf):
    """The 2D FP64 vortex workload (28 leaves, p=2, CFL 0.1, 100 steps)."""
    w = W.vortex2d_forest()
    f, S = _pair(dgf, w, 2, dgf.FP64, cfl=0.1)
    f.project(W.isentropic_vortex)
    Ug = f.get_state()
    U = S.project(W.isentropic_vortex)
    assert rel(Ug, U) < 1e-13
    U, t = S.run(U, 100)
    for _ in range(100):
        f.rk_step()
    assert abs(f.time - t) < 1e-12 * t
    assert rel(f.get_state(), U) < TOL["fp64"]
    # against the exact translated vortex (context: discretisation error)
    err = S.l2_error(f.get_state().astype(np.float64), lambda x: W.vortex_exact(x, t))
    assert err < 5e-3


def term_scale(S, U):
    """Size of the individual terms summed into L: max |F(u)| * 2 / h_min.
    A near-equilibrium state (most of the vortex domain is free stream) has a
    residual far smaller than its terms, so round-off is measured against
    the terms, not against |L|."""
    from oracle.euler import physical_flux
    F = 0.0
    hmin = np.inf
    for li in range(len(S.leaves)):
        uq = np.einsum("qm,vmc->cqv", S.ops.Phi, U[li])
        F = max(F, float(np.max(np.abs(physical_flux(uq)))))
        J, _ = S.geo_vol[li]
        hmin = min(hmin, float(np.min(np.einsum("q,cq->c", S.ops.wq, J) ** (1 / S.d))))
    return F * 2.0 / hmin


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_jitter3d_full_size_residual_matches_oracle(dgf, prec):
    """Full 3D jittered workload (71 leaves, 36,352 cells, p=2) in the launch
    configuration the benchmark uses, on the vortex state it times."""
    w = W.jitter3d_forest(seed=0)
    f, S = _pair(dgf, w, 2, dgf.FP64 if prec == "fp64" else dgf.FP32)
    assert f.n_leaves == 71
    f.project(lambda x: W.isentropic_vortex(x, scale=10.0))
    U = f.get_state().astype(np.float64)
    L = f.dg_residual()
    Lo = S.residual(U)
    err = float(np.max(np.abs(L - Lo)))
    assert err < TOL[prec] * term_scale(S, U), (err, rel(L, Lo))
    # one explicit stage with the CFL step: the solution bar itself
    dt = S.dt(U)
    assert rel(U + dt * L, U + dt * Lo) < TOL[prec] * 1e-2


def test_refine_then_coarsen_restores_state(dgf):
    """restriction(prolongation(u)) = u through the ABI (Sec. 3.4)."""
    w = W.jitter3d_forest(seed=5, n_seg=2)
    w["refine"] = [w["refine"][0]]
    f = dgf.Forest.from_workload(w, p=2)
    U0 = W.random_modal_state(f.n_leaves, 3, 2, 2, seed=4)
    f.set_state(U0)
    L0 = f.n_leaves
    f.refine([5, 40])
    assert f.n_leaves > L0
    o = FO.build(w)
    o.refine([o.leaves()[5], o.leaves()[40]])
    T, O = f.leaf_table(), o.leaf_table()
    assert np.array_equal(T["nbr"], O["nbr"])
    S0 = dg.Solver(FO.build(w), 2)
    S1 = dg.Solver(o, 2)
    assert rel(f.get_state(), S1.regrid_state(S0, U0)) < 1e-12
    new = [i for i, k in enumerate(o.leaves()) if k not in set(S0.leaves)]
    f.coarsen(new)
    assert f.n_leaves == L0
    assert rel(f.get_state(), U0) < 1e-12


def test_nonfinite_state_sets_status_word(dgf):
    w = W.rotated_pair_2d(n_seg=2)
    f = dgf.Forest.from_workload(w, p=1)
    U = W.random_modal_state(f.n_leaves, 2, 2, 1, seed=0)
    U[2, 0, 0, 1] = -1.0  # negative density in one cell
    f.set_state(U)
    assert f.status_word(reset=True) == -4
    f.rk_step()
    assert f.status_word() == -4


# ----------------------------------------------------- compensated FP32 form
@pytest.mark.parametrize("case", ["pair_2d", "jitter_3d_n2"])
def test_compensated_residual_and_steps_match_oracle(dgf, case):
    w = _small(case)
    f, S = _pair(dgf, w, 2, dgf.FP32_COMP, cfl=0.2)
    U = W.random_modal_state(f.n_leaves, f.dim, f.n_seg, 2, seed=9)
    f.set_state(U)
    assert rel(f.get_state(), U) < 1e-15  # the state itself is FP64
    assert_matches(f.dg_residual(), S.residual(U), "fp32", S, U)
    for _ in range(3):
        U = S.ssp_rk3_step(U, S.dt(U))
        f.rk_step()
    assert rel(f.get_state(), U) < TOL["fp32"]


def test_compensated_state_drifts_less_than_plain_fp32(dgf):
    """Over many steps the FP64-accumulated state stays closer to the FP64
    path than the plain FP32 state does (both run the residual in FP32)."""
    w = W.lattice_forest(2, 2, 10.0, 8)
    runs = {}
    for name, prec in (("fp64", dgf.FP64), ("fp32", dgf.FP32), ("comp", dgf.FP32_COMP)):
        f = dgf.Forest.from_workload(w, p=2, precision=prec, cfl=0.1)
        f.project(W.isentropic_vortex)
        for _ in range(300):
            f.rk_step()
        runs[name] = f.get_state().astype(np.float64)
    e32 = rel(runs["fp32"], runs["fp64"])
    ec = rel(runs["comp"], runs["fp64"])
    assert ec < TOL["fp32"] and e32 < TOL["fp32"]
    assert ec < 0.5 * e32, (ec, e32)


# ----------------------------------------------------- tiling invariance
@pytest.mark.parametrize("prec,kernel", [("fp32", "pair"), ("fp32", "classic"), ("fp64", "classic"),
                                         ("fp32_comp", "classic")])
def test_chunk_length_does_not_change_bits(dgf, prec, kernel, monkeypatch):
    """The stage kernel's z-chunk length (a tiling choice, tuned by timing)
    leaves every bit of the residual and of the stepped state unchanged, also
    with a ragged last chunk, so results are reproducible run to run; for
    each stage kernel (the cell-pair FP32 kernel and the layer-sweep one)."""
    w = W.jitter3d_forest(seed=2)
    U0 = W.random_modal_state(71, 3, 8, 2, seed=11)
    monkeypatch.setenv("DGF_STAGE_KERNEL", kernel)
    out = []
    for z in (8, 4, 3, 1):
        monkeypatch.setenv("DGF_ZCHUNK", str(z))
        f = dgf.Forest.from_workload(w, p=2, precision=prec)
        assert f.tuning()["zchunk"] == z and f.tuning()["stage_kernel"] == kernel
        f.set_state(U0)
        R = f.dg_residual()
        f.run(2)
        out.append((R, f.get_state()))
        f.close()
    for R, U in out[1:]:
        assert np.array_equal(R, out[0][0]) and np.array_equal(U, out[0][1])


@pytest.mark.parametrize("prec,kernel", [("fp32", "pair"), ("fp32", "classic"), ("fp64", "classic")])
def test_stage_grid_does_not_change_bits(dgf, prec, kernel, monkeypatch):
    """The stage grid (persistent CTAs walking the work items, or one CTA per
    item; a launch choice the autotuner times) leaves every bit unchanged."""
    w = W.jitter3d_forest(seed=2)
    U0 = W.random_modal_state(71, 3, 8, 2, seed=12)
    monkeypatch.setenv("DGF_STAGE_KERNEL", kernel)
    monkeypatch.setenv("DGF_ZCHUNK", "2")
    out = []
    for grid in ("persistent", "items"):
        monkeypatch.setenv("DGF_STAGE_GRID", grid)
        f = dgf.Forest.from_workload(w, p=2, precision=prec)
        assert f.tuning()["stage_grid"] == grid
        f.set_state(U0)
        R = f.dg_residual()
        f.run(2)
        out.append((R, f.get_state()))
        f.close()
    assert np.array_equal(out[0][0], out[1][0]) and np.array_equal(out[0][1], out[1][1])


# ----------------------------------------------------- mortar mode (R15)
@pytest.mark.parametrize("case", sorted(SMALL))
@pytest.mark.parametrize("p", [0, 1, 2, 3])
@pytest.mark.parametrize("prec", ["fp64", "fp32", "fp32_comp"])
def test_mortar_residual_matches_oracle(dgf, case, p, prec):
    w = _small(case)
    if prec == "fp32_comp" and p != 2:
        pytest.skip("compensated form: p = 2 covers the mortar path")
    pr = {"fp64": dgf.FP64, "fp32": dgf.FP32, "fp32_comp": dgf.FP32_COMP}[prec]
    f = dgf.Forest.from_workload(w, p=p, precision=pr, nonconforming="mortar")
    S = dg.Solver(FO.build(w), p, nonconforming="mortar")
    U = W.random_modal_state(f.n_leaves, f.dim, f.n_seg, p, seed=p + 21)
    f.set_state(U)
    Uin = U.astype(f.dtype).astype(np.float64)
    L = f.dg_residual()
    Lo = S.residual(Uin)
    assert_matches(L, Lo, prec, S, Uin)


@pytest.mark.parametrize("case", ["pair_2d", "jitter_3d_n4"])
def test_mortar_steps_conserve_totals(dgf, case):
    """Mortar mode: the totals stay constant to round-off across level jumps
    on the GPU (FP64), the paper's scheme drifts, and the steps follow the
    oracle."""
    w = _small(case)
    drift = {}
    for mode in ("mortar", "paper"):
        f = dgf.Forest.from_workload(w, p=2, precision=dgf.FP64, cfl=0.2, nonconforming=mode)
        U = W.random_modal_state(f.n_leaves, f.dim, f.n_seg, 2, seed=5)
        f.set_state(U)
        T0 = f.conserved_totals()
        for _ in range(4):
            f.rk_step()
        drift[mode] = np.max(np.abs(f.conserved_totals() - T0)) / np.max(np.abs(T0))
        if mode == "mortar":
            S = dg.Solver(FO.build(w), 2, cfl=0.2, nonconforming="mortar")
            Uo = U
            for _ in range(4):
                Uo = S.ssp_rk3_step(Uo, S.dt(Uo))
            assert rel(f.get_state(), Uo) < TOL["fp64"]
    assert drift["mortar"] < 1e-14 and drift["paper"] > 1e-10, drift


def test_mortar_free_stream(dgf):
    w = W.jitter3d_forest(seed=2, n_seg=4)
    for prec, tol in ((dgf.FP64, 1e-11), (dgf.FP32, 2e-4)):
        f = dgf.Forest.from_workload(w, p=2, precision=prec, nonconforming="mortar")
        f.project(W.free_stream)
        assert np.max(np.abs(f.dg_residual())) < tol * (1.0 / (0.25 / 4 / 2))  # |F| / h_min


# ----------------------------------------------------- row slabs (FP64 p = 3)
@pytest.mark.parametrize("mode", ["paper", "mortar"])
def test_fp64_p3_row_slabs_match_oracle(dgf, mode):
    """FP64 at p = 3 with 8^3-cell blocks sweeps each layer in slabs of rows
    (a whole layer's buffers exceed the shared memory of a CTA); the slab
    edges take the neighbouring rows' traces from memory.  Residual and steps
    against the oracle on a jittered, rotated forest with a level jump."""
    w = W.lattice_forest(3, 2, 1.0, 8, jitter=0.1, rotate_roots=True, seed=4)
    w["refine"] = [[(0, 1, (0, 0, 0))]]
    f = dgf.Forest.from_workload(w, p=3, precision=dgf.FP64, cfl=0.2, nonconforming=mode)
    S = dg.Solver(FO.build(w), 3, cfl=0.2, nonconforming=mode)
    U = W.random_modal_state(f.n_leaves, 3, 8, 3, seed=13)
    f.set_state(U)
    assert rel(f.dg_residual(), S.residual(U)) < TOL["fp64"]
    f.rk_step()
    U1 = S.ssp_rk3_step(U, S.dt(U))
    assert rel(f.get_state(), U1) < TOL["fp64"]


# ----------------------------------------------------- prescribed-state boundaries
@pytest.mark.parametrize("dim", [2, 3])
@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_prescribed_state_boundaries_match_oracle(dgf, dim, prec):
    """Root faces without a neighbour tagged at random as outflow or as a
    prescribed far-field state: guard cells, residual and RK steps against
    the oracle on a jittered, refined, non-periodic forest."""
    w = W.lattice_forest(dim, 2, 1.0, 4 if dim == 2 else 2, periodic=False, jitter=0.1, seed=6,
                         rotate_roots=True)
    w["refine"] = [[(0, 1, (0,) * dim)]]
    R = len(w["root_corners"])
    tags = np.random.default_rng(dim).integers(0, 2, size=(R, 2 * dim)).astype(np.int32)
    state = W.free_stream(np.zeros((1, dim)), state=(1.1, 0.4, -0.1, 0.2, 0.9)[: dim + 1] + (0.9,))[0]
    pr = dgf.FP64 if prec == "fp64" else dgf.FP32
    f = dgf.Forest.from_workload(w, p=2, precision=pr, cfl=0.2)
    f.set_boundary(tags, state)
    S = dg.Solver(FO.build(w), 2, cfl=0.2, boundary=(tags.tolist(), state))
    U = W.random_modal_state(f.n_leaves, dim, f.n_seg, 2, seed=17).astype(f.dtype).astype(np.float64)
    f.set_state(U)
    if prec == "fp64":
        assert rel(f.fill_guardcells(), S.fill_guardcells(U)) < TOL["fp64"]
    assert_matches(f.dg_residual(), S.residual(U), prec, S, U)
    for _ in range(2):
        U = S.ssp_rk3_step(U, S.dt(U))
        f.rk_step()
    assert rel(f.get_state(), U) < TOL[prec]
