"""Continuous-batching request server for independent bidomain simulations.

Requests (independent tissue simulations of different mesh size, membrane
model and stimulus protocol) arrive over time.  The server
  * admits a queued request as soon as a slot is free and its device
    footprint (``bd_footprint_bytes``) fits in the remaining HBM budget; the
    handle is built (host assembly, AMG set-up, upload) by a worker thread,
    so admission never stalls the requests already on the GPU,
  * keeps every admitted simulation resident on the GPU and keeps all of them
    advancing at once, in one of two forms:
      - per-request streams: whenever a simulation's enqueued steps have
        completed (non-blocking ``bd_query``), its next chunk of steps is
        enqueued (graph replays), so the work of different requests overlaps
        on the device;
      - batched (``batched=True``): resident simulations of the same group
        (the executor's group_key: membrane model and mesh size, the packing
        the batch autotuner prefers) advance together, a chunk at a time,
        through ``bd_batch_step`` -- one launch per phase over their
        concatenated nodes -- each group on its own stream and at its own
        pace; a request admitted meanwhile joins its group at that group's
        next chunk boundary,
  * completes a request when it has simulated its end time, reading its
    activation map, and frees its slot and memory for the queue.

Latency = completion time - arrival time ("time to activation map").  The
scheduler is written against a small executor interface so its admission,
ordering and batching logic can be tested on the CPU with a virtual-clock
executor.
"""
from __future__ import annotations

import concurrent.futures as cf
import dataclasses
import time
from typing import Any, Callable, Dict, List, Optional, Sequence

import numpy as np


@dataclasses.dataclass
class Job:
    rid: int
    arrival: float          # seconds on the executor's clock
    n_nodes: int
    n_steps: int
    payload: Any = None     # executor-specific description (e.g. a Workload)


@dataclasses.dataclass
class Completion:
    rid: int
    arrival: float
    admitted: float
    finished: float
    n_nodes: int
    n_steps: int
    result: Any = None

    @property
    def latency(self) -> float:
        return self.finished - self.arrival


class _Ready:
    """An already completed preparation (executors without a worker pool)."""

    def __init__(self, value):
        self.value = value

    def done(self) -> bool:
        return True

    def result(self):
        return self.value


class Executor:
    """Interface the scheduler drives.  prepare() must not block (it may hand
    the handle's construction to a worker); advance*/ready* must not block."""

    def now(self) -> float: ...
    def footprint(self, job: Job) -> int: ...
    def prepare(self, job: Job) -> Any: ...                   # future-like: done(), result() -> handle
    def advance(self, h: Any, n_steps: int) -> None: ...      # per-request form
    def ready(self, h: Any) -> bool: ...
    def group_key(self, job: Job) -> Any: ...                 # batched form: jobs batched together (None: alone)
    def advance_group(self, hs: Sequence[Any], n_steps: int) -> None: ...
    def group_ready(self, hs: Sequence[Any]) -> bool: ...
    def finish(self, h: Any) -> Any: ...
    def release(self, h: Any) -> None: ...
    def idle(self) -> None: ...                               # nothing ready: yield / sleep
    def wait_until(self, t: float) -> None: ...


class Server:
    def __init__(self, executor: Executor, max_slots: int = 8, hbm_budget: int = 64 << 30,
                 chunk_steps: int = 50, batched: bool = False, max_solo: Optional[int] = None):
        """max_solo (batched form): at most this many requests served alone
        advance at a time (in admission order); the others wait, built,
        until one completes.  None: no limit."""
        self.ex = executor
        self.max_solo = max_solo
        self.max_slots = max_slots
        self.budget = hbm_budget
        self.chunk = chunk_steps
        self.batched = batched

    def run(self, jobs: List[Job]) -> List[Completion]:
        """Open loop: each job arrives at its own time."""
        return self._serve(sorted(jobs, key=lambda j: (j.arrival, j.rid)), None)

    def run_closed(self, jobs: List[Job], clients: int) -> List[Completion]:
        """Closed loop: `clients` clients each keep one request outstanding;
        a client submits its next job (in list order) when its previous one
        completes.  The jobs' own arrival times are ignored."""
        return self._serve(list(jobs), clients)

    def _serve(self, queue: List[Job], clients: Optional[int]) -> List[Completion]:
        qi = 0
        total = len(queue)
        waiting: List[Job] = []
        starting: Dict[int, dict] = {}    # admitted, handle being built
        active: Dict[int, dict] = {}
        used = 0
        done: List[Completion] = []
        groups: Dict[Any, dict] = {}      # batched form: the chunk in flight, per group
        if clients is not None:           # closed loop: the first `clients` jobs arrive now
            t0 = self.ex.now()
            for _ in range(min(clients, total)):
                queue[qi] = dataclasses.replace(queue[qi], arrival=t0)
                waiting.append(queue[qi])
                qi += 1
        while len(done) < total:
            now = self.ex.now()
            if clients is None:
                while qi < total and queue[qi].arrival <= now:
                    waiting.append(queue[qi])
                    qi += 1
            # admission: FIFO, by free slot and footprint; the handle is built by a worker
            while waiting and len(active) + len(starting) < self.max_slots:
                j = waiting[0]
                fp = self.ex.footprint(j)
                if fp > self.budget:
                    raise ValueError(f"request {j.rid} needs {fp} bytes, more than the whole budget")
                if used + fp > self.budget:
                    break
                waiting.pop(0)
                used += fp
                starting[j.rid] = {"job": j, "fut": self.ex.prepare(j), "fp": fp, "admitted": self.ex.now()}
            progressed = False
            for rid in list(starting):
                st = starting[rid]
                if st["fut"].done():
                    progressed = True
                    a = {"job": st["job"], "h": st["fut"].result(), "fp": st["fp"], "steps": 0,
                         "admitted": st["admitted"]}
                    del starting[rid]
                    active[rid] = a
                    a["solo"] = not self.batched or self.ex.group_key(a["job"]) is None
                    a["running"] = False
            # requests served alone start (in admission order) while the
            # solo limit allows
            running = sum(1 for a in active.values() if a["solo"] and a["running"])
            for rid in sorted(active, key=lambda r: (active[r]["admitted"], r)):
                a = active[rid]
                if not a["solo"] or a["running"]:
                    continue
                if self.batched and self.max_solo is not None and running >= self.max_solo:
                    break
                a["running"] = True
                running += 1
                progressed = True
                n = min(self.chunk, a["job"].n_steps)
                self.ex.advance(a["h"], n)
                a["steps"] = n

            def complete(rid):
                nonlocal used, qi
                a = active.pop(rid)
                j = a["job"]
                res = self.ex.finish(a["h"])
                done.append(Completion(j.rid, j.arrival, a["admitted"], self.ex.now(), j.n_nodes, j.n_steps, res))
                self.ex.release(a["h"])
                used -= a["fp"]
                if clients is not None and qi < total:      # the client's next request
                    queue[qi] = dataclasses.replace(queue[qi], arrival=self.ex.now())
                    waiting.append(queue[qi])
                    qi += 1

            if self.batched:
                for key in list(groups):
                    g = groups[key]
                    if self.ex.group_ready(g["hs"]):
                        progressed = True
                        for rid in g["rids"]:
                            active[rid]["steps"] += g["n"]
                            if active[rid]["steps"] >= active[rid]["job"].n_steps:
                                complete(rid)
                        del groups[key]
                idle_members: Dict[Any, List[int]] = {}
                busy = {rid for g in groups.values() for rid in g["rids"]}
                for rid in sorted(active):
                    if rid not in busy and not active[rid]["solo"]:
                        idle_members.setdefault(self.ex.group_key(active[rid]["job"]), []).append(rid)
                for key, rids in idle_members.items():
                    if key in groups:
                        continue                  # joins at this group's next chunk
                    n = min([self.chunk] + [active[r]["job"].n_steps - active[r]["steps"] for r in rids])
                    hs = [active[r]["h"] for r in rids]
                    self.ex.advance_group(hs, n)
                    groups[key] = {"rids": rids, "hs": hs, "n": n}
                    progressed = True
            # requests served alone (every one in the per-request form; in the
            # batched form those whose group key is None)
            for rid in list(active):
                a = active[rid]
                if not a["solo"] or not a["running"] or not self.ex.ready(a["h"]):
                    continue
                progressed = True
                j = a["job"]
                if a["steps"] >= j.n_steps:
                    complete(rid)
                else:
                    n = min(self.chunk, j.n_steps - a["steps"])
                    self.ex.advance(a["h"], n)
                    a["steps"] += n
            if not progressed:
                if not active and not starting and not waiting and qi < total and clients is None:
                    self.ex.wait_until(queue[qi].arrival)
                else:
                    self.ex.idle()
        return done


def summarize(done: List[Completion], wall: Optional[float] = None) -> dict:
    """Latency percentiles and throughput; `offered` is the work of all
    requests over the span of their arrivals, `served` the completed work over
    the span from the first arrival to the last completion."""
    lat = np.array([c.latency for c in done]) * 1e3
    t0 = min(c.arrival for c in done)
    t1 = max(c.finished for c in done)
    span = wall if wall is not None else (t1 - t0)
    work = float(sum(c.n_nodes * c.n_steps for c in done))
    arr = sorted(c.arrival for c in done)
    arr_span = arr[-1] - arr[0]
    offered = work / arr_span if arr_span > 0 else float("inf")
    served = work / span if span > 0 else float("nan")
    return {"requests": len(done), "p50_ms": float(np.percentile(lat, 50)),
            "p99_ms": float(np.percentile(lat, 99)), "mean_ms": float(lat.mean()),
            "node_steps_per_s": served, "offered_node_steps_per_s": offered,
            "served_over_offered": served / offered if np.isfinite(offered) else float("nan"), "span_s": span}


def fifo_schedule(jobs: Sequence[Job], service_s: Sequence[float]) -> List[Completion]:
    """Exact single-server FIFO queue: job i (in arrival order) starts when it
    has arrived and the previous one has finished, and takes service_s[i]."""
    order = sorted(range(len(jobs)), key=lambda i: (jobs[i].arrival, jobs[i].rid))
    t = -np.inf
    out = []
    for i in order:
        j = jobs[i]
        start = max(t, j.arrival)
        t = start + float(service_s[i])
        out.append(Completion(j.rid, j.arrival, start, t, j.n_nodes, j.n_steps))
    return out


# ---------------------------------------------------------------------------
# executors
# ---------------------------------------------------------------------------

class GpuExecutor(Executor):
    """Real executor over the C ABI: one handle (and stream) per request,
    built by `workers` threads (the C calls release the interpreter lock).

    payload of a Job is a workloads.Workload; ``options`` builds bd_opts_t.
    In the batched form a group (same membrane model and mesh size) advances
    a chunk at a time with bd_batch_step on its first handle's stream;
    meshes of at least ``solo_nodes`` nodes (None: no limit) are served
    alone on their own streams (one request fills the GPU's persistent
    solver kernels; batching it would only add graph captures)."""

    def __init__(self, options: Callable[[], Any], dt: float, n_sdc_nodes: int = 3, n_sweeps: int = 2,
                 workers: int = 2, solo_nodes: Optional[int] = None):
        from . import binding
        self.b = binding
        self.options = options
        self.dt = dt
        self.M = n_sdc_nodes
        self.K = n_sweeps
        self.solo_nodes = solo_nodes
        self.t0 = time.perf_counter()
        self.pool = cf.ThreadPoolExecutor(max_workers=workers)

    def now(self) -> float:
        return time.perf_counter() - self.t0

    def footprint(self, job: Job) -> int:
        w = job.payload
        return self.b.footprint_bytes(w.xyz, w.elems, w.model, self.options(), w.elem_bath)

    def prepare(self, job: Job):
        return self.pool.submit(self.b.simulation_from_workload, job.payload, self.options())

    def advance(self, h, n_steps: int) -> None:
        for _ in range(n_steps):
            h.step(self.dt, self.M, self.K)

    def ready(self, h) -> bool:
        return h.ready()

    def group_key(self, job: Job):
        if self.solo_nodes is not None and job.n_nodes >= self.solo_nodes:
            return None
        return (job.payload.model, job.n_nodes)

    def advance_group(self, hs, n_steps: int) -> None:
        for _ in range(n_steps):
            self.b.batch_step(hs, self.dt, self.M, self.K)

    def group_ready(self, hs) -> bool:
        return all(h.ready() for h in hs)

    def finish(self, h):
        return h.activation_times()

    def release(self, h) -> None:
        h.close()

    def idle(self) -> None:
        time.sleep(0.0002)

    def wait_until(self, t: float) -> None:
        d = t - self.now()
        if d > 0:
            time.sleep(d)

    def close(self) -> None:
        self.pool.shutdown(wait=True)


class VirtualExecutor(Executor):
    """Deterministic stand-in with a virtual clock: a request advances at
    ``rate`` node-steps/s shared equally among the active requests
    (processor sharing), its footprint is ``bytes_per_node`` per node, and
    its handle takes ``setup`` seconds of a worker to build; requests of at
    least ``solo_nodes`` nodes are not batched (None: every one is)."""

    def __init__(self, rate: float = 1e9, bytes_per_node: int = 2000, quantum: float = 1e-3, setup: float = 0.0,
                 solo_nodes: Optional[int] = None):
        self.t = 0.0
        self.solo_nodes = solo_nodes
        self.grouped: List[List[int]] = []      # rids of every group chunk launched
        self.max_busy_solo = 0                  # most requests of solo size with work at once
        self.rate = rate
        self.bpn = bytes_per_node
        self.quantum = quantum
        self.setup = setup
        self.live: Dict[int, dict] = {}
        self.started: List[int] = []
        self.max_live = 0
        self._next = 0

    class _Build:
        def __init__(self, ex, job):
            self.ex, self.job, self.at = ex, job, ex.t + ex.setup
            self.h = None

        def done(self) -> bool:
            return self.ex.t >= self.at - 1e-12

        def result(self):
            if self.h is None:
                ex = self.ex
                self.h = ex._next
                ex._next += 1
                ex.live[self.h] = {"job": self.job, "work": 0.0}
                ex.max_live = max(ex.max_live, len(ex.live))
            return self.h

    def now(self) -> float:
        return self.t

    def footprint(self, job: Job) -> int:
        return job.n_nodes * self.bpn

    def prepare(self, job: Job):
        self.started.append(job.rid)
        return self._Build(self, job)

    def advance(self, h, n_steps: int) -> None:
        st = self.live[h]
        st["work"] += n_steps * st["job"].n_nodes

    def ready(self, h) -> bool:
        return self.live[h]["work"] <= 1e-9

    def group_key(self, job: Job):
        if self.solo_nodes is not None and job.n_nodes >= self.solo_nodes:
            return None
        return job.n_nodes

    def advance_group(self, hs, n_steps: int) -> None:
        self.grouped.append([self.live[h]["job"].rid for h in hs])
        for h in hs:
            self.advance(h, n_steps)

    def group_ready(self, hs) -> bool:
        return all(self.ready(h) for h in hs)

    def _tick(self, dt: float) -> None:
        busy = [st for st in self.live.values() if st["work"] > 1e-9]
        if self.solo_nodes is not None:
            nsolo = sum(1 for st in busy if st["job"].n_nodes >= self.solo_nodes)
            self.max_busy_solo = max(self.max_busy_solo, nsolo)
        if busy:
            share = self.rate * dt / len(busy)
            for st in busy:
                st["work"] = max(0.0, st["work"] - share)
        self.t += dt

    def idle(self) -> None:
        self._tick(self.quantum)

    def wait_until(self, t: float) -> None:
        while self.t < t:
            self._tick(min(self.quantum, t - self.t + 1e-12))

    def finish(self, h):
        return self.live[h]["job"].rid

    def release(self, h) -> None:
        del self.live[h]
