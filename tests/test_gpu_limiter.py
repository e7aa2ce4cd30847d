"""GPU positivity limiter (reading R17) through the C ABI against the oracle:
one application to a stressed state, and blast steps with the limiter after
every stage (which break down without it)."""
import numpy as np
import pytest

import workloads as W
from oracle import dg
from oracle import forest as FO
from oracle import limiter as LIM
from oracle.euler import primitives

pytestmark = pytest.mark.gpu

TOL = {"fp64": 1e-12, "fp32": 1e-5}
EPS = 1e-6


@pytest.fixture(scope="module")
def dgf():
    import paper_2502_12620_gb300 as pkg
    pkg.lib()
    return pkg


def rel(a, b):
    return float(np.linalg.norm((np.asarray(a, float) - b).ravel()) / max(np.linalg.norm(np.ravel(b)), 1e-300))


def _stressed(S, seed):
    rng = np.random.default_rng(seed)
    U = W.random_modal_state(len(S.leaves), S.d, S.n, S.p, seed=seed)
    for li in range(len(S.leaves)):
        for c in rng.choice(U.shape[3], size=2, replace=False):
            U[li, :, 1:, c] *= 25.0
    return U


@pytest.mark.parametrize("case", ["jitter_3d", "pair_2d", "cube_3d"])
@pytest.mark.parametrize("p", [1, 2, 3])
@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_limit_matches_oracle(dgf, case, p, prec):
    w = {"jitter_3d": lambda: W.jitter3d_forest(seed=1, n_seg=2),
         "pair_2d": lambda: W.rotated_pair_2d(n_seg=4),
         "cube_3d": lambda: W.periodic_cube_forest(2, n_seg=4, rotate_roots=True, seed=3)}[case]()
    f = dgf.Forest.from_workload(w, p=p, precision=dgf.FP64 if prec == "fp64" else dgf.FP32)
    S = dg.Solver(FO.build(w), p)
    U = _stressed(S, seed=p).astype(f.dtype).astype(np.float64)
    V, changed, bad = LIM.positivity_limit(S, U, EPS)
    assert changed > 0 and bad == 0
    f.set_state(U)
    assert f.status_word(reset=True) == -4  # the stressed state has negative points
    f.set_limiter(EPS)
    f.limit()
    assert f.status_word() == 0
    assert rel(f.get_state(), V) < TOL[prec]


@pytest.mark.parametrize("p", [1, 2])
def test_blast_steps_with_limiter_match_oracle(dgf, p):
    w = W.lattice_forest(3, 2, 1.0, 2, rotate_roots=True, seed=1)
    ic = lambda x: W.blast(x, (0.3, 0.3, 0.3), r0=0.15, width=0.08)
    S = dg.Solver(FO.build(w), p, limiter=EPS)
    U = LIM.positivity_limit(S, S.project(ic), EPS)[0]
    f = dgf.Forest.from_workload(w, p=p, precision=dgf.FP64)
    f.set_state(U)
    f.set_limiter(EPS)
    for _ in range(3):
        U = S.ssp_rk3_step(U, S.dt(U))
        f.rk_step()
    assert f.status_word() == 0
    assert rel(f.get_state(), U) < 1e-10


def test_blast_fp32_runs_positive_with_limiter_only(dgf):
    w = W.lattice_forest(3, 2, 1.0, 2, rotate_roots=True, seed=1)
    ic = lambda x: W.blast(x, (0.3, 0.3, 0.3), r0=0.15, width=0.08)
    for p in (1, 2):
        if p == 1:  # p = 1: negative face traces from the start; breaks down without the limiter
            g = dgf.Forest.from_workload(w, p=p, precision=dgf.FP32)
            g.project(ic)
            g.run(10)
            assert g.status_word() != 0
            assert g.time < 1.0  # no CFL value from a broken state: dt is 0, time stops
        f = dgf.Forest.from_workload(w, p=p, precision=dgf.FP32)
        f.project(ic)
        f.set_limiter(1e-5)
        f.limit()
        f.status_word(reset=True)  # the projected initial data may have had negative face points
        T0 = f.conserved_totals()
        f.run(10)
        assert f.status_word() == 0
        Phi = dg.Ops(3, p).Phi
        uq = np.einsum("qm,lvmc->lcqv", Phi, f.get_state().astype(np.float64))
        r, _, pr = primitives(uq)
        assert r.min() > 0 and pr.min() > 0
        T1 = f.conserved_totals()
        assert np.max(np.abs(T1 - T0)[[0, 4]] / np.abs(T0)[[0, 4]]) < 1e-5


def test_limiter_refused_for_compensated_form(dgf):
    f = dgf.Forest.from_workload(W.rotated_pair_2d(n_seg=2), p=1, precision=dgf.FP32_COMP)
    with pytest.raises(dgf.DgfError) as e:
        f.set_limiter(1e-6)
    assert e.value.code == -8
