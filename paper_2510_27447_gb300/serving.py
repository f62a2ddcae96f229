"""Continuous-batching request server for independent bidomain simulations.

Requests (independent tissue simulations of different mesh size, membrane
model and stimulus protocol) arrive over time.  The server
  * admits a queued request as soon as a slot is free and its device
    footprint (``bd_footprint_bytes``) fits in the remaining HBM budget,
  * keeps every admitted simulation resident on the GPU, each on its own CUDA
    stream, and keeps all of them advancing at once: whenever a simulation's
    enqueued steps have completed (non-blocking ``bd_query``), the next chunk of
    steps is enqueued (graph replays), so the work of different requests
    overlaps on the device,
  * completes a request when it has simulated its end time, reading its
    activation map, and frees its slot and memory for the queue.

Latency = completion time - arrival time ("time to activation map").  The
scheduler is written against a small executor interface so its admission and
ordering logic can be tested on the CPU with a virtual-clock executor.
"""
from __future__ import annotations

import dataclasses
import heapq
import time
from typing import Any, Callable, Dict, List, Optional

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


class Executor:
    """Interface the scheduler drives (all methods except advance/ready may block)."""

    def now(self) -> float: ...
    def footprint(self, job: Job) -> int: ...
    def start(self, job: Job) -> Any: ...
    def advance(self, h: Any, n_steps: int) -> None: ...      # enqueue, must not block
    def ready(self, h: Any) -> bool: ...                      # must not block
    def finish(self, h: Any) -> Any: ...
    def release(self, h: Any) -> None: ...
    def idle(self) -> None: ...                               # nothing ready: yield / sleep


class Server:
    def __init__(self, executor: Executor, max_slots: int = 8, hbm_budget: int = 64 << 30,
                 chunk_steps: int = 50):
        self.ex = executor
        self.max_slots = max_slots
        self.budget = hbm_budget
        self.chunk = chunk_steps

    def run(self, jobs: List[Job]) -> List[Completion]:
        queue = sorted(jobs, key=lambda j: (j.arrival, j.rid))
        qi = 0
        waiting: List[Job] = []            # arrived, not admitted (FIFO)
        active: Dict[int, dict] = {}
        used = 0
        done: List[Completion] = []
        total = len(queue)
        while len(done) < total:
            now = self.ex.now()
            while qi < total and queue[qi].arrival <= now:
                waiting.append(queue[qi])
                qi += 1
            # admission: FIFO, by free slot and footprint
            while waiting and len(active) < self.max_slots:
                j = waiting[0]
                fp = self.ex.footprint(j)
                if fp > self.budget:
                    raise ValueError(f"request {j.rid} needs {fp} bytes, more than the whole budget")
                if used + fp > self.budget:
                    break
                waiting.pop(0)
                h = self.ex.start(j)
                used += fp
                active[j.rid] = {"job": j, "h": h, "fp": fp, "steps": 0, "admitted": self.ex.now()}
                n = min(self.chunk, j.n_steps)
                self.ex.advance(h, n)
                active[j.rid]["steps"] = n
            progressed = False
            for rid in list(active):
                a = active[rid]
                if not self.ex.ready(a["h"]):
                    continue
                progressed = True
                j = a["job"]
                if a["steps"] >= j.n_steps:
                    res = self.ex.finish(a["h"])
                    done.append(Completion(j.rid, j.arrival, a["admitted"], self.ex.now(), j.n_nodes,
                                           j.n_steps, res))
                    self.ex.release(a["h"])
                    used -= a["fp"]
                    del active[rid]
                else:
                    n = min(self.chunk, j.n_steps - a["steps"])
                    self.ex.advance(a["h"], n)
                    a["steps"] += n
            if not progressed:
                if not active and not waiting and qi < total:
                    self.ex.wait_until(queue[qi].arrival)
                else:
                    self.ex.idle()
        return done


def summarize(done: List[Completion], wall: Optional[float] = None) -> dict:
    lat = np.array([c.latency for c in done]) * 1e3
    t0 = min(c.arrival for c in done)
    t1 = max(c.finished for c in done)
    span = wall if wall is not None else (t1 - t0)
    work = float(sum(c.n_nodes * c.n_steps for c in done))
    return {"requests": len(done), "p50_ms": float(np.percentile(lat, 50)),
            "p99_ms": float(np.percentile(lat, 99)), "mean_ms": float(lat.mean()),
            "node_steps_per_s": work / span if span > 0 else float("nan"), "span_s": span}


# ---------------------------------------------------------------------------
# executors
# ---------------------------------------------------------------------------

class GpuExecutor(Executor):
    """Real executor over the C ABI: one handle (and stream) per request.

    payload of a Job is a workloads.Workload; ``options`` builds bd_opts_t."""

    def __init__(self, options: Callable[[], Any], dt: float, n_sdc_nodes: int = 3, n_sweeps: int = 2):
        from . import binding
        self.b = binding
        self.options = options
        self.dt = dt
        self.M = n_sdc_nodes
        self.K = n_sweeps
        self.t0 = time.perf_counter()

    def now(self) -> float:
        return time.perf_counter() - self.t0

    def footprint(self, job: Job) -> int:
        w = job.payload
        return self.b.footprint_bytes(w.xyz, w.elems, w.model, self.options(), w.elem_bath)

    def start(self, job: Job):
        return self.b.simulation_from_workload(job.payload, self.options())

    def advance(self, h, n_steps: int) -> None:
        for _ in range(n_steps):
            h.step(self.dt, self.M, self.K)

    def ready(self, h) -> bool:
        return h.ready()

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


class VirtualExecutor(Executor):
    """Deterministic stand-in with a virtual clock: a request advances at
    ``rate`` node-steps/s shared equally among the active requests
    (processor sharing), its footprint is ``bytes_per_node`` per node."""

    def __init__(self, rate: float = 1e9, bytes_per_node: int = 2000, quantum: float = 1e-3):
        self.t = 0.0
        self.rate = rate
        self.bpn = bytes_per_node
        self.quantum = quantum
        self.live: Dict[int, dict] = {}
        self.started: List[int] = []
        self.max_live = 0
        self._next = 0

    def now(self) -> float:
        return self.t

    def footprint(self, job: Job) -> int:
        return job.n_nodes * self.bpn

    def start(self, job: Job):
        h = self._next
        self._next += 1
        self.live[h] = {"job": job, "work": 0.0}
        self.started.append(job.rid)
        self.max_live = max(self.max_live, len(self.live))
        return h

    def advance(self, h, n_steps: int) -> None:
        st = self.live[h]
        st["work"] += n_steps * st["job"].n_nodes

    def ready(self, h) -> bool:
        return self.live[h]["work"] <= 1e-9

    def _tick(self, dt: float) -> None:
        busy = [st for st in self.live.values() if st["work"] > 1e-9]
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
