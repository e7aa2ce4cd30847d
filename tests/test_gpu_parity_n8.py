"""GPU parity at n_seg = 8, the block size of every benchmark, adaptive and
serving run.  Each precision and degree instantiates its own stage kernel
(threads per CTA, CTAs per SM, shared-memory layout; FP32 at p = 3 fills
225 KB of shared memory, FP32 at p <= 1 runs four small CTAs per SM), so each
configuration those runs launch is compared here with the FP64 oracle: the
residual element by element and one SSP-RK3 time increment, in the paper's
level-jump scheme and in the mortar repair.

The forest: two roots of 8^3 cells side by side (periodic, seeded +-10 %
node jitter, seeded rotations of both root frames), the first refined once,
so every face kind meets the kernel: same level through rotations, finer and
coarser neighbours across the level jump, and the self-glued periodic faces.
"""
import numpy as np
import pytest

import workloads as W
from oracle import dg
from oracle import forest as FO

from test_gpu_parity import TOL, assert_matches, rel

pytestmark = pytest.mark.gpu

# (precision, p, stage kernel): FP32 at p = 1, 2 has two stage kernels (the
# cell-pair kernel and the layer-sweep kernel; the autotuner picks one by
# timing), both are compared, and at p = 1 the cell-pair kernel's two CTA
# shapes (four and five CTAs per SM)
CONFIGS = [("fp32", 1, "pair"), ("fp32", 1, "pair5"), ("fp32", 1, "classic"), ("fp32", 2, "pair"),
           ("fp32", 2, "classic"),
           ("fp32", 3, "classic"), ("fp64", 1, "classic"), ("fp64", 2, "classic"), ("fp32_comp", 2, "classic")]


@pytest.fixture(scope="module")
def dgf():
    import paper_2502_12620_gb300 as pkg
    pkg.lib()
    return pkg


def two_root_forest():
    w = W.lattice_forest(3, (2, 1, 1), 1.0, 8, jitter=0.1, rotate_roots=True, seed=3)
    w["refine"] = [[(0, 1, (0, 0, 0))]]
    return w


@pytest.mark.parametrize("mode", ["paper", "mortar"])
@pytest.mark.parametrize("prec,p,kernel", CONFIGS)
def test_n8_residual_and_step_match_oracle(dgf, prec, p, kernel, mode, monkeypatch):
    monkeypatch.setenv("DGF_STAGE_KERNEL", kernel)
    w = two_root_forest()
    pr = {"fp64": dgf.FP64, "fp32": dgf.FP32, "fp32_comp": dgf.FP32_COMP}[prec]
    f = dgf.Forest.from_workload(w, p=p, precision=pr, cfl=0.2, nonconforming=mode)
    assert f.n_leaves == 9 and f.n_seg == 8 and f.tuning()["stage_kernel"] == kernel
    S = dg.Solver(FO.build(w), p, cfl=0.2, nonconforming=mode)
    U = W.random_modal_state(f.n_leaves, 3, 8, p, seed=10 * p + (mode == "mortar"))
    if prec == "fp32":
        U = U.astype(np.float32).astype(np.float64)  # the state the FP32 path holds
    f.set_state(U)
    assert_matches(f.dg_residual(), S.residual(U), prec, S, U)
    dt = S.dt(U)
    assert abs(f.compute_dt() - dt) <= (1e-13 if prec == "fp64" else 1e-5) * dt
    f.rk_step()
    assert f.tuning()["stage_kernel"] == kernel
    U1 = S.ssp_rk3_step(U, dt)
    assert rel(f.get_state(), U1) < TOL["fp64" if prec == "fp64" else "fp32"]
    assert f.status_word() == 0
    f.close()


@pytest.mark.parametrize("mode", ["paper", "mortar"])
def test_n8_pair_cta_shapes_give_the_same_bits(dgf, mode, monkeypatch):
    """The cell-pair kernel's two CTA shapes at p = 1 are one source compiled
    with different register budgets: the same residual and time step, bit
    for bit, on the jittered rotated forest with a level jump."""
    w = two_root_forest()
    U = W.random_modal_state(9, 3, 8, 1, seed=21).astype(np.float32).astype(np.float64)
    out = []
    for kernel in ("pair", "pair5"):
        monkeypatch.setenv("DGF_STAGE_KERNEL", kernel)
        f = dgf.Forest.from_workload(w, p=1, precision=dgf.FP32, cfl=0.2, nonconforming=mode)
        assert f.tuning()["stage_kernel"] == kernel
        f.set_state(U)
        R = f.dg_residual()
        f.rk_step()
        f.rk_step()
        out.append((R, f.get_state()))
        f.close()
    assert np.array_equal(out[0][0], out[1][0]) and np.array_equal(out[0][1], out[1][1])
