"""Batches of forests (dgf_batch_*): every forest of a batch advanced by one
launch of each kernel per stage.  A forest's result in a batch is bit for bit
the one it gets alone in a batch (its work items do its own arithmetic and it
keeps its own time step and end time), and it agrees with the single-forest
time step within the FP32 tolerance; members at their end time stay
unchanged.  Degrees 1 and 2 run the cell-pair kernel, degree 3 the
layer-sweep kernel; affine and curved (jittered) members are mixed."""
import numpy as np
import pytest

import workloads as W

pytestmark = pytest.mark.gpu

TOL = 1e-5


@pytest.fixture(scope="module")
def dgf():
    import paper_2502_12620_gb300 as pkg
    pkg.lib()
    return pkg


def rel(a, b):
    return float(np.linalg.norm((np.asarray(a, float) - b).ravel()) / np.linalg.norm(np.ravel(b)))


def _members(dgf, p):
    """(workload, end time) of three members: an affine cube of 2^3 roots, a
    jittered 2-root forest with a level jump, a single affine root."""
    two = W.lattice_forest(3, (2, 1, 1), 1.0, 8, jitter=0.1, rotate_roots=True, seed=3)
    two["refine"] = [[(0, 1, (0, 0, 0))]]
    return [(W.periodic_cube_forest(2), 0.004), (two, 0.003), (W.periodic_cube_forest(1), 0.005)]


def _forest(dgf, w, p):
    f = dgf.Forest.from_workload(w, p=p, precision=dgf.FP32, cfl=0.2)
    f.project(lambda x: W.smooth_state(x))
    return f


@pytest.mark.parametrize("p", [1, 2, 3])
def test_batch_equals_alone_and_single_forest(dgf, p):
    specs = _members(dgf, p)
    # together
    fs = [_forest(dgf, w, p) for w, _ in specs]
    b = dgf.Batch()
    b.set(fs, [t for _, t in specs])
    for _ in range(60):
        b.step(5)
        b.sync()
        if all(f.time >= t for f, (_, t) in zip(fs, specs)):
            break
    together = [(f.get_state(), f.step_count, f.time) for f in fs]
    assert all(f.status_word() == 0 for f in fs)
    b.close()
    for (w, t), (U, n, tt) in zip(specs, together):
        assert tt == t and n > 1
        # alone in a batch: bit for bit
        f = _forest(dgf, w, p)
        b1 = dgf.Batch()
        b1.set([f], [t])
        while f.time < t:
            b1.step(5)
            b1.sync()
        assert f.step_count == n and np.array_equal(f.get_state(), U)
        b1.close()
        f.close()
        # the single-forest time step: same steps, FP32 tolerance
        f = _forest(dgf, w, p)
        while f.time < t:
            f.rk_step(t)
        assert f.step_count == n and abs(f.time - t) < 1e-15
        assert rel(U, f.get_state().astype(np.float64)) < TOL
        f.close()
    for f in fs:
        f.close()


def test_batch_refuses_unsupported_members(dgf):
    import paper_2502_12620_gb300 as pkg
    b = dgf.Batch()
    f64 = dgf.Forest.from_workload(W.periodic_cube_forest(1), p=1, precision=dgf.FP64)
    f64.project(W.smooth_state)
    with pytest.raises(pkg.DgfError):
        b.set([f64], [0.01])
    f2d = dgf.Forest.from_workload(W.rotated_pair_2d(n_seg=4), p=1, precision=dgf.FP32)
    f2d.project(W.smooth_x_state)
    with pytest.raises(pkg.DgfError):
        b.set([f2d], [0.01])
    b.close()
    f64.close()
    f2d.close()


def test_batched_server_mixed_equals_alone(dgf):
    """Continuous batching through the serving loop: solves of degrees 1..3
    arriving together share one batch per degree; each result equals the
    solve run alone through the same path."""
    from paper_2502_12620_gb300.serve import Request, Server
    specs = [(W.periodic_cube_forest(2), 1, 0.004), (W.periodic_cube_forest(1), 1, 0.006),
             (W.periodic_cube_forest(2), 2, 0.003), (W.periodic_cube_forest(1), 3, 0.002),
             (W.periodic_cube_forest(2), 3, 0.0015), (W.periodic_cube_forest(1), 2, 0.005)]
    reqs = [Request(i, 0.0, w, p, t, W.smooth_state, dgf.FP32) for i, (w, p, t) in enumerate(specs)]
    srv = Server(hbm_budget=8 << 30, max_active=6, steps_per_round=4, batched=True)
    res = srv.run(reqs, keep_state=True)
    for r, q in zip(res, reqs):
        alone = Server(hbm_budget=8 << 30, max_active=1, steps_per_round=4, batched=True).run([q], keep_state=True)[0]
        assert r.status == 0 and r.t == q.t_end
        assert r.steps == alone.steps and np.array_equal(r.state, alone.state), r.rid


@pytest.mark.parametrize("p", [1, 2, 3])
def test_batch_chunk_length_changes_no_bit(dgf, p, monkeypatch):
    """The batch's z-chunk length (chosen from its total block count, or
    fixed by DGF_ZCHUNK) is a tiling choice: whole blocks, a ragged chunk of
    3 layers and single layers give the same states bit for bit."""
    specs = _members(dgf, p)
    outs = []
    for z in (8, 3, 1):
        monkeypatch.setenv("DGF_ZCHUNK", str(z))
        fs = [_forest(dgf, w, p) for w, _ in specs]
        b = dgf.Batch()
        b.set(fs, [t for _, t in specs])
        b.step(6)
        b.sync()
        outs.append([f.get_state() for f in fs])
        assert all(f.status_word() == 0 for f in fs)
        b.close()
        for f in fs:
            f.close()
    for o in outs[1:]:
        for a, c in zip(o, outs[0]):
            assert np.array_equal(a, c)
