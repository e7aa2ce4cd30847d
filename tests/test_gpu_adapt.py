"""GPU adaptation (reading R16) through the C ABI against the oracle: the
refinement indicator, one adaptation step (same leaves bit for bit, state
transferred on the device by copy / split / combine) on affine and jittered
forests, and refine-all-then-coarsen-all returning the original state."""
import numpy as np
import pytest

import workloads as W
from oracle import adapt as A
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


def _tables_equal(f, S):
    T, O = f.leaf_table(), S.F.leaf_table()
    return all(np.array_equal(T[k].astype(np.int64), O[k].astype(np.int64))
               for k in ("root", "level", "pos", "kind", "nbr", "orient"))


def _gap_threshold(g, lo=0.25, hi=0.75):
    """A threshold in the widest gap between sorted indicator values in the
    middle of the range, so a rounding difference cannot flip a decision."""
    v = np.unique(np.round(g, 12))
    i0, i1 = int(len(v) * lo), max(int(len(v) * hi), int(len(v) * lo) + 1)
    gaps = np.diff(v[i0:i1 + 1])
    j = int(np.argmax(gaps))
    return 0.5 * (v[i0 + j] + v[i0 + j + 1]), gaps[j]


CASES = {
    "blast_affine_3d": (lambda: W.lattice_forest(3, 2, 1.0, 2, rotate_roots=True, seed=1),
                        lambda x: W.blast(x, (0.3, 0.3, 0.3), r0=0.15, width=0.08)),
    "blast_jitter_3d": (lambda: W.jitter3d_forest(seed=2, n_seg=2),
                        lambda x: W.blast(x, (0.45, 0.5, 0.55), r0=0.2, width=0.1)),
    "vortex_2d": (lambda: dict(W.lattice_forest(2, 4, 10.0, 4), refine=[[(5, 1, (0, 0))]]),
                  W.isentropic_vortex),
}


@pytest.mark.parametrize("case", sorted(CASES))
@pytest.mark.parametrize("prec", ["fp64", "fp32"])
@pytest.mark.parametrize("p", [1, 2])
def test_indicator_matches_oracle(dgf, case, prec, p):
    mk, ic = CASES[case]
    w = mk()
    f = dgf.Forest.from_workload(w, p=p, precision=dgf.FP64 if prec == "fp64" else dgf.FP32)
    S = dg.Solver(FO.build(w), p)
    U = S.project(ic)
    f.set_state(U)
    got = f.indicator()
    want = A.indicator(S, U.astype(f.dtype).astype(np.float64))
    assert np.max(np.abs(got - want)) <= TOL[prec] * (1 + np.max(want)) * 10


@pytest.mark.parametrize("case", sorted(CASES))
@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_adapt_matches_oracle(dgf, case, prec):
    mk, ic = CASES[case]
    w = mk()
    p = 2
    f = dgf.Forest.from_workload(w, p=p, precision=dgf.FP64 if prec == "fp64" else dgf.FP32)
    S = dg.Solver(FO.build(w), p)
    U = S.project(ic).astype(f.dtype).astype(np.float64)
    f.set_state(U)
    # refine step
    g = A.indicator(S, U)
    thr, gap = _gap_threshold(g)
    assert gap > 1e-6 * max(1.0, thr)
    counts = f.adapt(thr, -1.0, 3)
    S1, U1, nr, nc = A.adapt(S, U, thr, -1.0, 3)
    assert counts == (nr, nc) and nr > 0 and _tables_equal(f, S1)
    assert rel(f.get_state(), U1) < TOL[prec]
    # coarsen step from the device state
    U1g = f.get_state().astype(np.float64)
    g1 = A.indicator(S1, U1g)
    cthr, gap = _gap_threshold(g1, 0.3, 0.9)
    counts = f.adapt(np.inf, cthr, 3)
    S2, U2, nr2, nc2 = A.adapt(S1, U1g, np.inf, cthr, 3)
    assert counts == (nr2, nc2) and _tables_equal(f, S2)
    assert rel(f.get_state(), U2) < TOL[prec]
    assert np.max(np.abs(f.conserved_totals() - S2.totals(U2))) < TOL[prec] * np.max(np.abs(S2.totals(U2)))


@pytest.mark.parametrize("case", ["blast_affine_3d", "blast_jitter_3d"])
def test_refine_all_then_coarsen_all_restores_state(dgf, case):
    mk, ic = CASES[case]
    w = mk()
    f = dgf.Forest.from_workload(w, p=2, precision=dgf.FP64)
    f.project(ic)
    U0, L0 = f.get_state(), f.n_leaves

    def keys():
        T = f.leaf_table()
        return [(int(r), int(l), tuple(int(x) for x in p)) for r, l, p in zip(T["root"], T["level"], T["pos"])]
    orig = set(keys())
    assert f.adapt(-1.0, -1.0, 4) == (L0, 0) and f.n_leaves == 8 * L0
    # coarsen only what the refinement made (indicator 0 there, 1 on the
    # original leaves); one pass coarsens what balance allows in canonical
    # order, so with mixed levels a group beside still-finer blocks waits
    passes = 0
    while f.n_leaves > L0 and passes < 4:
        g = np.array([1.0 if k in orig else 0.0 for k in keys()])
        nr, nc = f.adapt(np.inf, 0.5, 4, indicator=g)
        assert nr == 0 and nc > 0
        passes += 1
    assert set(keys()) == orig and passes == (1 if case == "blast_affine_3d" else 2)
    assert rel(f.get_state(), U0) < 1e-12


def test_adapt_then_steps_run(dgf):
    """An adapted forest keeps stepping (tables, graphs and the CFL value are
    rebuilt), FP32."""
    mk, _ = CASES["blast_affine_3d"]
    w = mk()
    for prec in (dgf.FP32, dgf.FP64):
        f = dgf.Forest.from_workload(w, p=1, precision=prec)
        f.project(W.smooth_state)
        g = f.indicator()
        nr, _ = f.adapt(float(np.median(g)), -1.0, 3)
        assert nr > 0
        for _ in range(5):
            f.rk_step()
        assert f.status_word() == 0 and f.time > 0
        # the same steps on the oracle's adapted forest
        if prec == dgf.FP64:
            S = dg.Solver(FO.build(w), 1)
            U = S.project(W.smooth_state)
            S1, U1, _, _ = A.adapt(S, U, float(np.median(A.indicator(S, U))), -1.0, 3)
            for _ in range(5):
                U1 = S1.ssp_rk3_step(U1, S1.dt(U1))
            assert rel(f.get_state(), U1) < TOL["fp64"]


@pytest.mark.parametrize("p", [1, 3])
def test_transfer_at_n8_matches_oracle(dgf, p):
    """State transfer of a refinement and a coarsening at the block size of
    the adaptive runs (8^3 cells) and p = 1, 3, FP32, against the oracle's
    data inheritance (Sec. 3.4): split children (Eqs. (11)-(12)) and
    combined parents (Eqs. (13)-(14)) of a blast profile."""
    w = W.periodic_cube_forest(2)
    ic = lambda x: W.blast(x, (0.4, 0.5, 0.55), r0=0.2, width=0.05)
    f = dgf.Forest.from_workload(w, p=p, precision=dgf.FP32)
    S = dg.Solver(FO.build(w), p)
    U = S.project(ic).astype(np.float32).astype(np.float64)
    f.set_state(U)
    g = np.zeros(8)
    g[[0, 5]] = 1.0
    assert f.adapt(0.5, -1.0, 3, indicator=g) == (2, 0)
    S1, U1, nr, nc = A.adapt(S, U, 0.5, -1.0, 3, g=g)
    assert nr == 2 and _tables_equal(f, S1)
    assert rel(f.get_state(), U1) < TOL["fp32"]
    # coarsen the first refined root again
    T = f.leaf_table()
    g1 = np.array([0.0 if (int(T["root"][i]) == 0 and int(T["level"][i]) == 2) else 1.0
                   for i in range(f.n_leaves)])
    U1g = f.get_state().astype(np.float64)
    nr2, nc2 = f.adapt(np.inf, 0.5, 3, indicator=g1)
    S2, U2, _, _ = A.adapt(S1, U1g, np.inf, 0.5, 3, g=g1)
    assert nc2 == 1 and _tables_equal(f, S2)
    assert rel(f.get_state(), U2) < TOL["fp32"]
