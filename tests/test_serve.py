"""Continuous batching of independent solves.

Host logic (admission by footprint and slot count, first-come-first-served
order, step accounting) runs on CPU with stand-in solves; on the GPU every
solve served in a mix must equal, bit for bit, the same solve run alone, and
an increment at t = t_end must leave the state unchanged."""
import math

import numpy as np
import pytest

import workloads as W
from paper_2502_12620_gb300 import FP32, FP32_COMP, FP64
from paper_2502_12620_gb300.serve import Request, Server, footprint_bytes, summarize


class FakeClock:
    def __init__(self):
        self.t = 0.0

    def __call__(self):
        return self.t

    def sleep(self, dt):
        self.t += max(dt, 1e-4)


class FakeSolve:
    """Advances time by a fixed dt per step; every stream is always idle."""
    log = []

    def __init__(self, req, clock, dt=0.01, nbytes=None):
        self.req, self.clock, self.dt = req, clock, dt
        self.t, self.steps, self.dof = 0.0, 0, 100
        self.device_bytes = nbytes if nbytes is not None else footprint_bytes(req.workload, req.p, req.precision)
        FakeSolve.log.append(("admit", req.rid))

    def enqueue(self, k):
        for _ in range(k):
            d = min(self.dt, self.req.t_end - self.t)
            if d > 0:
                self.t += d
                self.steps += 1
        self.clock.t += 1e-3 * k

    def idle(self):
        return True

    def progress(self):
        return self.t, self.steps

    def finish(self, keep_state):
        FakeSolve.log.append(("finish", self.req.rid))
        return None, 0


def _req(rid, arrival, B=2, p=1, t_end=0.1):
    return Request(rid, arrival, W.periodic_cube_forest(B, n_seg=2), p, t_end, None, FP32)


def test_footprint_monotone():
    fixed = 1 << 20
    small = footprint_bytes(W.periodic_cube_forest(2, n_seg=8), 1) - fixed
    big = footprint_bytes(W.periodic_cube_forest(4, n_seg=8), 1) - fixed
    p3 = footprint_bytes(W.periodic_cube_forest(2, n_seg=8), 3) - fixed
    assert big == 8 * small  # proportional to the leaf count
    assert p3 > 6 * small
    assert footprint_bytes(W.periodic_cube_forest(2, n_seg=8), 1, FP64) - fixed > 1.5 * small
    # three FP32 copies of 64 roots x 512 cells x 8 modes x 5 variables
    assert small > 3 * 8 * 512 * 8 * 5 * 4


def test_admission_budget_and_order():
    clock = FakeClock()
    FakeSolve.log = []
    reqs = [_req(i, 0.001 * i, t_end=0.05 + 0.01 * (i % 3)) for i in range(10)]
    one = footprint_bytes(reqs[0].workload, 1)
    srv = Server(hbm_budget=int(2.5 * one), max_active=8, steps_per_round=3,
                 build_workers=0, solve_factory=lambda r: FakeSolve(r, clock), clock=clock, sleep=clock.sleep)
    res = srv.run(reqs)
    assert srv.peak_active == 2 and srv.peak_bytes <= srv.budget
    admits = [rid for ev, rid in FakeSolve.log if ev == "admit"]
    assert admits == list(range(10))  # first come, first served
    for r, q in zip(res, reqs):
        assert r.rid == q.rid and abs(r.t - q.t_end) < 1e-12
        assert r.steps == math.ceil(q.t_end / 0.01 - 1e-9)
        assert r.finished >= r.admitted >= r.arrival - 1e-12
    s = summarize(res, clock.t)
    assert s["requests"] == 10 and s["p99_s"] >= s["p50_s"] > 0


def test_slot_limit_and_oversize():
    clock = FakeClock()
    FakeSolve.log = []
    reqs = [_req(i, 0.0) for i in range(6)] + [_req(6, 0.0, B=3)]
    srv = Server(hbm_budget=10 ** 12, max_active=4, steps_per_round=4,
                 build_workers=0, solve_factory=lambda r: FakeSolve(r, clock), clock=clock, sleep=clock.sleep)
    srv.run(reqs)
    assert srv.peak_active == 4
    # a request larger than the whole budget is admitted once it is alone
    clock = FakeClock()
    FakeSolve.log = []
    small = footprint_bytes(reqs[0].workload, 1)
    srv = Server(hbm_budget=small, max_active=4, build_workers=0, solve_factory=lambda r: FakeSolve(r, clock),
                 clock=clock, sleep=clock.sleep)
    res = srv.run([_req(0, 0.0), _req(1, 0.0, B=3), _req(2, 0.0)])
    assert srv.peak_active == 1 and [r.rid for r in res] == [0, 1, 2]
    ev = FakeSolve.log
    assert ev.index(("finish", 0)) < ev.index(("admit", 1)) < ev.index(("finish", 1)) < ev.index(("admit", 2))


def test_arrivals_wait():
    clock = FakeClock()
    FakeSolve.log = []
    reqs = [_req(0, 0.5), _req(1, 0.2)]
    srv = Server(hbm_budget=10 ** 12, build_workers=0, solve_factory=lambda r: FakeSolve(r, clock), clock=clock,
                 sleep=clock.sleep)
    res = srv.run(reqs)
    assert [ev for ev in FakeSolve.log if ev[0] == "admit"] == [("admit", 1), ("admit", 0)]
    assert res[0].admitted >= 0.5 and res[1].admitted >= 0.2


def test_serving_mix_recipe():
    R = W.serving_mix(256, seed=3)
    arr = np.array([r["arrival"] for r in R])
    assert np.all(np.diff(arr) > 0)
    assert 256 / 20.0 * 0.7 < arr[-1] < 256 / 20.0 * 1.3  # Poisson, rate 20/s
    blocks = np.array([r["B"] ** 3 for r in R])
    assert blocks.min() >= 27 and blocks.max() <= 21 ** 3
    assert {r["p"] for r in R} == {1, 2, 3}
    assert 0.3 < np.mean([r["kind"] == "blast" for r in R]) < 0.7
    assert all(0.05 <= r["t_end"] <= 0.5 for r in R)
    again = W.serving_mix(256, seed=3)  # seeded: the same stream every time
    assert all(a["arrival"] == b["arrival"] and a["B"] == b["B"] and a["p"] == b["p"]
               and np.array_equal(a["centre"], b["centre"]) for a, b in zip(R, again))


# ------------------------------------------------- batched mode (host logic)
class FakeForest:
    """Time, step count and status of one batch member (a stand-in)."""

    def __init__(self, dt, fail_at=None):
        self.dt, self.fail_at = dt, fail_at
        self.t, self.steps, self.status, self.t_end = 0.0, 0, 0, math.inf


class FakeBatch:
    """Advances every member like the library's batch: dt clipped to the
    member's end time, nothing once it is there; a member may turn
    non-finite (status -4) at a given step, after which its dt is 0."""
    made = []

    def __init__(self, clock):
        self.clock, self.members, self.steps_log, self.sets = clock, [], [], []
        FakeBatch.made.append(self)

    def set(self, forests, t_ends):
        self.members = list(forests)
        self.sets.append(len(forests))
        for f, t in zip(forests, t_ends):
            f.t_end = t

    def step(self, k):
        self.steps_log.append(k)
        for _ in range(k):
            for f in self.members:
                d = min(f.dt, f.t_end - f.t) if f.status == 0 else 0.0
                if d > 0:
                    f.t += d
                    f.steps += 1
                    if f.fail_at is not None and f.steps >= f.fail_at:
                        f.status = -4
        self.clock.t += 1e-4 * k

    def idle(self):
        return True

    def progress(self):
        return (np.array([f.t for f in self.members]), np.array([f.steps for f in self.members], np.int64),
                np.array([f.status for f in self.members], np.int32))

    def sync(self):
        pass

    def close(self):
        pass


class FakeBatchSolve:
    """A batched solve: its forest is advanced by the batch only."""

    def __init__(self, req, dt=0.01, fail_at=None):
        self.req, self.f, self.dof = req, FakeForest(dt, fail_at), 100
        self.device_bytes = footprint_bytes(req.workload, req.p, req.precision)

    def enqueue(self, k):
        raise AssertionError("a batched solve is never stepped on its own stream")

    def finish(self, keep_state):
        return None, self.f.status


def _fake_steps(t_end, dt=0.01):
    """Steps the fakes take to reach t_end (the same clipped accumulation)."""
    t, n = 0.0, 0
    while min(dt, t_end - t) > 0:
        t += min(dt, t_end - t)
        n += 1
    return n


def _breq(rid, arrival, p=1, t_end=0.05, precision=FP32):
    return Request(rid, arrival, W.periodic_cube_forest(2, n_seg=8), p, t_end, None, precision)


def _batched_server(clock, factory, **kw):
    return Server(hbm_budget=10 ** 12, max_active=6, build_workers=0, solve_factory=factory, clock=clock,
                  sleep=clock.sleep, batched=True, batch_steps=8, batch_factory=lambda: FakeBatch(clock), **kw)


def test_batched_mode_groups_by_degree_and_finishes_every_solve_at_its_end_time():
    clock = FakeClock()
    FakeBatch.made = []
    reqs = [_breq(i, 0.002 * i, p=1 + i % 2, t_end=0.03 + 0.07 * (i % 4)) for i in range(10)]
    res = _batched_server(clock, lambda r: FakeBatchSolve(r)).run(reqs)
    for r, q in zip(res, reqs):
        assert r.status == 0 and abs(r.t - q.t_end) < 1e-12
        assert r.steps == _fake_steps(q.t_end)
    assert len(FakeBatch.made) == 2  # one batch per degree (all small)
    for b in FakeBatch.made:
        assert all(8 <= k <= 64 for k in b.steps_log)  # rounds of batch_steps .. 8 batch_steps
        assert b.sets[0] >= 1 and max(b.sets) <= 6


def test_batched_mode_retires_a_failed_member_and_serves_the_rest():
    clock = FakeClock()
    FakeBatch.made = []
    reqs = [_breq(i, 0.0, t_end=0.2) for i in range(4)]
    res = _batched_server(clock, lambda r: FakeBatchSolve(r, fail_at=3 if r.rid == 1 else None)).run(reqs)
    assert [r.status for r in res] == [0, -4, 0, 0]
    assert res[1].steps == 3 and res[1].t < reqs[1].t_end
    assert all(abs(r.t - 0.2) < 1e-12 and r.steps == _fake_steps(0.2) for i, r in enumerate(res) if i != 1)


def test_batched_mode_keeps_other_solves_on_their_own_streams():
    clock = FakeClock()
    FakeBatch.made = []
    FakeSolve.log = []
    reqs = [_breq(0, 0.0), _breq(1, 0.0, precision=FP64), _req(2, 0.0)]  # FP32 8^3, FP64 8^3, FP32 2^3 blocks
    factory = lambda r: FakeBatchSolve(r) if r.rid == 0 else FakeSolve(r, clock)
    res = _batched_server(clock, factory).run(reqs)
    assert all(r.status == 0 and abs(r.t - q.t_end) < 1e-12 for r, q in zip(res, reqs))
    assert len(FakeBatch.made) == 1 and FakeBatch.made[0].sets[0] == 1
    assert {rid for ev, rid in FakeSolve.log if ev == "finish"} == {1, 2}


# ------------------------------------------------------------------ GPU
def _gpu_requests():
    # a mix of dimensions, degrees, precisions and refinement
    v2 = W.vortex2d_forest()
    c2 = W.periodic_cube_forest(2, n_seg=4)
    c3 = W.periodic_cube_forest(3, n_seg=2)
    j = W.jitter3d_forest(seed=1, n_seg=2)
    v2i = lambda x: W.isentropic_vortex(x)
    sm = lambda x: W.smooth_state(x)
    return [
        Request(0, 0.0, v2, 2, 0.05, v2i, FP32),
        Request(1, 0.0, c2, 1, 0.02, sm, FP32),
        Request(2, 0.0, c2, 3, 0.01, sm, FP32),
        Request(3, 0.0, j, 2, 0.01, sm, FP32_COMP),
        Request(4, 0.0, c3, 2, 0.015, sm, FP64),
        Request(5, 0.0, v2, 1, 0.04, v2i, FP64),
    ]


@pytest.mark.gpu
def test_mixed_equals_alone():
    from paper_2502_12620_gb300 import Forest
    reqs = _gpu_requests()
    alone = []
    for q in reqs:
        f = Forest.from_workload(q.workload, p=q.p, precision=q.precision)
        f.project(q.init)
        n = 0
        while f.time < q.t_end:
            f.rk_step(q.t_end)
            n += 1
            assert n < 10000
        alone.append((f.get_state(), f.step_count, f.time))
        f.close()
    srv = Server(hbm_budget=4 << 30, max_active=6, steps_per_round=5)
    res = srv.run(reqs, keep_state=True)
    assert srv.peak_active == 6
    for r, (U, steps, t) in zip(res, alone):
        assert r.status == 0
        assert r.steps == steps and r.t == t
        assert r.state.dtype == U.dtype and np.array_equal(r.state, U), r.rid


@pytest.mark.gpu
def test_footprint_estimate_matches_allocation():
    from paper_2502_12620_gb300 import Forest
    for w, p, prec in [(W.periodic_cube_forest(4, n_seg=8), 1, FP32),
                       (W.periodic_cube_forest(2, n_seg=8), 3, FP32),
                       (W.jitter3d_forest(seed=0), 2, FP32_COMP),
                       (W.periodic_cube_forest(2, n_seg=8), 2, FP64)]:
        f = Forest.from_workload(w, p=p, precision=prec)
        f.project(W.smooth_state)
        f.rk_step()
        actual = f.device_bytes
        est = footprint_bytes(w, p, prec)
        f.close()
        assert 0.8 * actual < est < 1.25 * actual, (p, prec, est, actual)


@pytest.mark.gpu
@pytest.mark.parametrize("prec", [FP32, FP32_COMP, FP64])
def test_step_past_t_end_is_identity(prec):
    from paper_2502_12620_gb300 import Forest
    f = Forest.from_workload(W.periodic_cube_forest(2, n_seg=4), p=2, precision=prec)
    f.project(W.smooth_state)
    t_end = 0.004
    while f.time < t_end:
        f.rk_step(t_end)
    U, n = f.get_state(), f.step_count
    assert f.time == t_end and n > 0
    for _ in range(3):
        assert f.rk_step(t_end, return_dt=True) == 0.0
    assert np.array_equal(f.get_state(), U) and f.step_count == n and f.time == t_end
    # the kept CFL minimum lets the march continue past the old end time
    f.rk_step(2 * t_end)
    assert f.time > t_end and f.step_count == n + 1 and f.status_word() == 0
    f.set_time(0.0)
    assert f.step_count == 0
    f.close()


def test_batch_round_length_follows_the_first_member_to_finish():
    from types import SimpleNamespace as NS
    srv = Server(hbm_budget=1 << 30, batched=True, batch_steps=8)
    a = NS(t0=0.0, req=NS(t_end=1.0))  # dt 0.05 so far: 10 steps left
    b = NS(t0=0.0, req=NS(t_end=1.0))  # dt 0.01 so far: 90 steps left
    c = NS(t0=0.0, req=NS(t_end=1.0))  # just joined: no steps yet
    prog = {id(a): (0.5, 10), id(b): (0.1, 10)}
    assert srv._round_steps([a, b], prog) == 10
    assert srv._round_steps([b], prog) == 64         # at most 8 rounds of batch_steps
    assert srv._round_steps([a, b, c], prog) == 8    # a new member: batch_steps
    assert srv._round_steps([NS(t0=0.0, req=NS(t_end=0.52))], {}) == 8
    done = NS(t0=0.0, req=NS(t_end=0.5))
    assert srv._round_steps([done], {id(done): (0.5, 10)}) == 8  # at least batch_steps
