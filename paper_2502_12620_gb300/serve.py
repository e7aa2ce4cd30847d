"""Continuous batching of independent DG solves on one GPU (host scheduler).

Requests arrive over time; a request is admitted, first come first served, as
soon as a slot is free and its device footprint fits the memory budget.  An
admitted solve keeps its forest and state resident on the GPU until it
reaches its end time, and runs on its own CUDA stream: the scheduler enqueues
a few time steps on every stream that has drained, so the steps of different
solves overlap on the device while the host looks at the next one.  Each
solve's arithmetic is the one it does alone (own buffers and graphs,
deterministic kernels, and an increment at t = t_end is the identity), so
its result does not depend on what else runs beside it.

With batched=True, the admitted 3D FP32 solves of 8^3-cell blocks are
advanced together instead: one library batch per degree and size class
(below / above large_dof unknowns, so that small solves do not wait for the
rounds of large ones), so each stage of
every such solve goes through one launch of the guard-trace kernel and one
of the persistent stage kernel (a single CUDA graph per batch membership;
admitting or retiring a solve rewrites the batch's device work descriptors).
Each solve keeps its own time step and end time; its result is the one it
gets alone in a batch.  Other solves keep their own streams.

All GPU work goes through the library; this module decides what to admit and
how many time steps to enqueue next.
"""
from __future__ import annotations

import dataclasses
import math
import threading
import time
from concurrent.futures import ThreadPoolExecutor

import numpy as np

from . import FP32, FP32_COMP, FP64, Batch, Forest


@dataclasses.dataclass
class Request:
    rid: int
    arrival: float          # seconds after the start of the run
    workload: dict          # forest description (dim, n_seg, nodes, root_corners, ...)
    p: int
    t_end: float
    init: object            # fun(x[..., d]) -> conserved values, ("nodal", values at the
                            # quadrature points), ("device", fn) with fn(forest) setting the
                            # state itself (e.g. from values computed on the GPU), or a
                            # modal state array
    precision: int = FP32


@dataclasses.dataclass
class Result:
    rid: int
    arrival: float
    admitted: float
    finished: float
    steps: int              # time increments with dt > 0
    dof: int                # scalar unknowns of the solve
    t: float
    status: int = 0
    device_bytes: int = 0
    state: np.ndarray = None

    @property
    def time_to_solution(self):
        return self.finished - self.arrival


def leaf_count(workload):
    """Leaves after the description's refinement batches (no 2:1 closure
    refinements are counted: the workloads' batches are balanced)."""
    leaves = len(workload["root_corners"])
    for batch in workload.get("refine", []):
        leaves += len(batch) * ((1 << workload["dim"]) - 1)
    return leaves


def footprint_bytes(workload, p, precision=FP32):
    """Device bytes a solve holds while resident, estimated before it is
    built: three stage buffers (for the compensated form two more in FP64
    and u^n split into two FP32 arrays),
    the cell map coefficients and cell sizes in the compute precision and in
    FP64, the guard traces and modal guard cells, the per-leaf tables and
    1 MiB for the finer-face operators and scalars."""
    d, n = workload["dim"], workload["n_seg"]
    L = leaf_count(workload)
    nc, N = n ** d, p + 1
    M = N ** d
    es = 8 if precision == FP64 else 4
    dof = L * nc * M * (d + 2)
    state = 3 * dof * es + (2 * dof * 8 + 2 * dof * 4 if precision == FP32_COMP else 0)
    geo = L * nc * (((1 << d) - 1) * d + 1) * (es + 8)
    faces = L * 2 * d * (d + 2) * n ** (d - 1)
    guard = faces * N ** (d - 1) * es + faces * M * (es + 8)
    return int(state + geo + guard + L * 2 * d * 40 + (1 << 20))


# solve and initial-value streams take precedence over batch streams
# (created at the default, lowest priority): the kernels of a solve being
# built get SMs as soon as CTAs of a running batch stage retire
PRIORITY = -1
_INIT_STREAMS = {}
_INIT_LOCK = threading.Lock()


def init_stream(device=0):
    """The stream on which solves compute their initial values, shared by
    the build workers, so that torch's cached blocks of one build serve the
    next (a stream of its own per solve would grow a pool per solve)."""
    import torch
    with _INIT_LOCK:
        s = _INIT_STREAMS.get(device)
        if s is None:
            s = _INIT_STREAMS[device] = torch.cuda.Stream(device=device, priority=PRIORITY)
    return s


def reserve_init_memory(nbytes, device=0):
    """Grow torch's cached pool of the initial-value stream by nbytes."""
    import torch
    with torch.cuda.stream(init_stream(device)):
        t = torch.empty(int(nbytes), dtype=torch.uint8, device=torch.device("cuda", device))
        del t


class GpuSolve:
    """One admitted request: a forest on its own stream."""

    def __init__(self, req, device=0):
        import torch
        self.req = req
        self.stream = torch.cuda.Stream(device=device, priority=PRIORITY)
        self.f = Forest.from_workload(req.workload, p=req.p, precision=req.precision, device=device)
        self.f.set_stream(self.stream)
        with torch.cuda.stream(init_stream(device)):  # initial values (the binding waits for them)
            if callable(req.init):
                self.f.project(req.init)
            elif isinstance(req.init, tuple) and req.init[0] == "nodal":
                self.f.set_state_nodal(req.init[1])
            elif isinstance(req.init, tuple) and req.init[0] == "device":
                req.init[1](self.f)
            else:
                self.f.set_state(req.init)
        self.dof = self.f.n_leaves * self.f.nv * self.f.M * self.f.nc

    @property
    def device_bytes(self):
        return self.f.device_bytes

    def enqueue(self, k):
        for _ in range(k):
            self.f.rk_step(self.req.t_end)

    def idle(self):
        return self.stream.query()

    def progress(self):
        return self.f.time, self.f.step_count

    def failed(self):
        """A non-finite state stops the solve's clock (its time increment is
        0 from then on), so it is retired as failed instead of waited for."""
        return self.f.status_word() != 0

    def finish(self, keep_state):
        state = self.f.get_state() if keep_state else None
        status = self.f.status_word()
        self.f.close()
        return state, status


class Server:
    """Admits requests by footprint and advances the admitted solves together.

    hbm_budget bounds the summed device bytes of the resident solves (by the
    estimate while a solve is being built, by its actual allocation after); a
    request larger than the whole budget runs alone.  steps_per_round is the
    most time steps enqueued on one stream at a time.  With build_workers > 0
    new solves are built (forest, initial state, first steps) on worker
    threads, so the streams already admitted keep getting work meanwhile.
    With batched=True, 3D FP32 solves of 8^3-cell blocks join the batch of
    their degree and size class (batch_factory() makes one; default: the
    library's Batch) and advance in rounds of batch_steps to 8 batch_steps
    steps; the others keep a stream each."""

    def __init__(self, device=0, hbm_budget=None, max_active=16, steps_per_round=8,
                 build_workers=2, solve_factory=None, clock=time.perf_counter, sleep=time.sleep,
                 batched=False, batch_steps=8, large_dof=64 << 20, batch_factory=None):
        self.device = device
        if hbm_budget is None:
            import torch
            free, _ = torch.cuda.mem_get_info(device)
            hbm_budget = int(0.5 * free)
        self.budget = int(hbm_budget)
        self.max_active = int(max_active)
        self.steps_per_round = int(steps_per_round)
        self.build_workers = int(build_workers)
        self.factory = solve_factory or (lambda req: GpuSolve(req, device))
        self.clock = clock
        self.sleep = sleep
        self.peak_active = 0
        self.peak_bytes = 0
        self.batched = bool(batched)
        self.batch_steps = int(batch_steps)
        self.large_dof = int(large_dof)
        self.groups = {}  # (degree, large) -> _Group (batched mode)
        self.batch_factory = batch_factory or (lambda: Batch(self.device))

    def _next_k(self, s, t, steps):
        """Steps to enqueue next: the predicted remainder (from the mean dt so
        far), at least one, at most steps_per_round."""
        if steps == 0:
            return self.steps_per_round
        dt = (t - s.t0) / steps
        if not dt > 0:
            return self.steps_per_round
        rem = math.ceil((s.req.t_end - t) / dt)
        return max(1, min(self.steps_per_round, rem))

    @staticmethod
    def batchable(req):
        w = req.workload
        return w["dim"] == 3 and w["n_seg"] == 8 and req.precision == FP32

    def _build(self, req):
        s = self.factory(req)
        s.req, s.t0 = req, 0.0
        s.batched = self.batched and self.batchable(req)
        if not s.batched:
            s.enqueue(self.steps_per_round)
        return s

    def _group_key(self, s):
        """Batches by degree and size class: a small solve does not wait for
        the rounds of large ones (a round is batch_steps steps of every
        member of the batch)."""
        return (s.req.p, s.dof > self.large_dof)

    def _serve_groups(self, results, keep_state, t0):
        """Batched mode: retire finished members, take in new ones, and
        enqueue the next round of steps on every batch that has drained.
        Returns (progressed, bytes released)."""
        progressed, freed = False, 0
        for g in self.groups.values():
            if not g.batch.idle():
                continue
            changed = False
            ts, nsteps, stats = g.batch.progress() if g.members else ((), (), ())
            prog = {id(s): (float(t), int(k)) for s, t, k in zip(g.members, ts, nsteps)}
            for s, t, steps, stw in list(zip(g.members, ts, nsteps, stats)):
                t, steps = float(t), int(steps)
                if t >= s.req.t_end or stw != 0:
                    state, status = s.finish(keep_state)
                    results[s.req.rid] = Result(s.req.rid, s.req.arrival, s.admitted, self.clock() - t0,
                                                steps, s.dof, t, status, s.bytes, state)
                    s.done = True
                    freed += s.bytes
                    g.members.remove(s)
                    changed = progressed = True
            if g.joining:
                g.members.extend(g.joining)
                g.joining = []
                changed = True
            if changed:
                g.batch.set([s.f for s in g.members], [s.req.t_end for s in g.members])
            if g.members:
                g.batch.step(self._round_steps(g.members, prog))
                progressed = True
        return progressed, freed

    def _round_steps(self, members, prog):
        """Steps of a batch's next round: the fewest predicted remaining steps
        of any member (from its mean dt so far), so that the first member to
        finish is retired when the round ends; at least batch_steps (also for
        a member without steps yet), at most 8 batch_steps."""
        k = 8 * self.batch_steps
        for s in members:
            t, steps = prog.get(id(s), (0.0, 0))
            dt = (t - s.t0) / steps if steps > 0 else 0.0
            rem = math.ceil((s.req.t_end - t) / dt) if dt > 0 else self.batch_steps
            k = min(k, rem)
        return max(self.batch_steps, k)

    def run(self, requests, keep_state=False, deadline=None):
        """Serve `requests` (arrival times relative to the call); returns the
        per-request results in request order.  With a deadline (seconds), the
        run stops admitting once it is passed, retires the active solves where
        they are (status -100) and reports the requests never admitted with
        status -101."""
        pending = sorted(requests, key=lambda r: (r.arrival, r.rid))
        queue, building, active, results = [], [], [], {}
        used = 0
        pool = ThreadPoolExecutor(self.build_workers) if self.build_workers > 0 else None
        t0 = self.clock()
        try:
            while pending or queue or building or active:
                now = self.clock() - t0
                if deadline is not None and now > deadline and not building:
                    for g in self.groups.values():
                        g.batch.sync()
                    for s in active:
                        if getattr(s, "done", False):
                            continue
                        t, steps = s.progress()
                        state, _ = s.finish(keep_state)
                        results[s.req.rid] = Result(s.req.rid, s.req.arrival, s.admitted, now, steps, s.dof, t,
                                                    -100, s.bytes, state)
                    for r in pending + queue:
                        results[r.rid] = Result(r.rid, r.arrival, now, now, 0, 0, 0.0, -101)
                    break
                while pending and pending[0].arrival <= now:
                    queue.append(pending.pop(0))
                # admission: first come first served, by slot count and footprint
                while queue and len(active) + len(building) < self.max_active:
                    est = footprint_bytes(queue[0].workload, queue[0].p, queue[0].precision)
                    if (active or building) and used + est > self.budget:
                        break
                    req = queue.pop(0)
                    used += est
                    item = [None, req, est, self.clock() - t0]
                    if pool is not None:
                        item[0] = pool.submit(self._build, req)
                    else:
                        item[0] = self._build(req)
                    building.append(item)
                progressed = False
                for item in building:
                    fut, req, est, adm = item
                    if pool is not None:
                        if not fut.done():
                            continue
                        s = fut.result()  # a failed build raises here
                    else:
                        s = fut
                    s.admitted = adm
                    s.bytes = s.device_bytes or est
                    used += s.bytes - est
                    active.append(s)
                    if getattr(s, "batched", False):
                        key = self._group_key(s)
                        if key not in self.groups:
                            self.groups[key] = _Group(self.batch_factory())
                        self.groups[key].joining.append(s)
                    item[0] = None
                    progressed = True
                building = [it for it in building if it[0] is not None]
                self.peak_active = max(self.peak_active, len(active) + len(building))
                self.peak_bytes = max(self.peak_bytes, used)
                if self.groups:
                    pg, freed = self._serve_groups(results, keep_state, t0)
                    progressed = progressed or pg
                    used -= freed
                for s in active:
                    if getattr(s, "batched", False) or not s.idle():
                        continue
                    progressed = True
                    t, steps = s.progress()
                    if t >= s.req.t_end or _failed(s):
                        state, status = s.finish(keep_state)
                        results[s.req.rid] = Result(s.req.rid, s.req.arrival, s.admitted, self.clock() - t0,
                                                    steps, s.dof, t, status, s.bytes, state)
                        s.done = True
                        used -= s.bytes
                    else:
                        s.enqueue(self._next_k(s, t, steps))
                active = [s for s in active if not getattr(s, "done", False)]
                if not progressed:
                    wait = 2e-4
                    if not active and not building and not queue and pending:
                        wait = max(0.0, min(0.01, pending[0].arrival - (self.clock() - t0)))
                    self.sleep(wait)
        finally:
            if pool is not None:
                pool.shutdown(wait=True)
            for g in self.groups.values():
                g.batch.close()
            self.groups = {}
        return [results[r.rid] for r in requests]


def _failed(s):
    f = getattr(s, "failed", None)
    return bool(f()) if f is not None else False


@dataclasses.dataclass
class _Group:
    """The solves of one degree and size class advanced by one library batch."""
    batch: object
    members: list = dataclasses.field(default_factory=list)
    joining: list = dataclasses.field(default_factory=list)


def summarize(results, wall):
    tts = np.array([r.time_to_solution for r in results])
    updates = sum(r.dof * 3 * r.steps for r in results)  # three RK stages per step
    return {"requests": len(results), "p50_s": float(np.percentile(tts, 50)),
            "p99_s": float(np.percentile(tts, 99)), "wall_s": wall,
            "dof_updates_per_s": updates / wall}
