"""Packing of many simulations into batched steps, chosen by timing.

``bd_batch_step`` advances a set of compatible handles (same membrane model,
precision and device) by one launch per phase over their concatenated nodes.
How a set of handles is split into such batches -- one batch per model, one
per mesh size, or batches of at most k handles sorted by size -- trades
launch count against load balance (a batch's loop runs while its slowest
system iterates).  ``BatchRunner`` picks the packing by timing each candidate
on the live handles for a few steps, once per shape class (model, precision
and the multiset of mesh sizes), restoring every handle's state afterwards so
the tuning leaves the simulations where they were.

``OptionTuner`` chooses a single handle's layout and thread mapping the same
way: the storage form of long-row AMG levels (SELL-32 or CSR), the threads
per CSR row, the SELL-32/4 vector-load copy (streaming handles) or the
solver block size (persistent handles), timed once per shape class.
"""
from __future__ import annotations

import time
from typing import Dict, List, Sequence, Tuple

from . import binding


def _groups(sims, key) -> List[List[int]]:
    out: Dict[object, List[int]] = {}
    for i, s in enumerate(sims):
        out.setdefault(key(s), []).append(i)
    return list(out.values())


def candidate_packings(sims: Sequence[binding.Simulation]) -> Dict[str, List[List[int]]]:
    """Candidate splits of the handles into batches (lists of indices); a
    batch never mixes membrane models or precisions."""
    base = lambda s: (s.model, s.opts.precision)
    by_model = _groups(sims, base)
    cands = {"model": by_model,
             "size": _groups(sims, lambda s: (base(s), s.N))}
    for k in (4, 8, 16):
        packs = []
        for g in by_model:
            g = sorted(g, key=lambda i: sims[i].N)
            packs += [g[j:j + k] for j in range(0, len(g), k)]
        if len(packs) not in {len(v) for v in cands.values()}:
            cands[f"cap{k}"] = packs
    return cands


def shape_class(sims: Sequence[binding.Simulation]) -> Tuple:
    return tuple(sorted((s.model, s.opts.precision, s.N) for s in sims))


class BatchRunner:
    """Steps a set of handles with batched launches in the packing the tuner
    chose for their shape class (cached across calls)."""

    def __init__(self, trial_steps: int = 2):
        self.trial_steps = trial_steps
        self.cache: Dict[Tuple, Tuple[str, List[float]]] = {}
        self.timings: Dict[Tuple, Dict[str, float]] = {}

    def _run(self, sims, packing, dt, M, K, steps):
        for _ in range(steps):
            for b in packing:
                binding.batch_step([sims[i] for i in b], dt, M, K)

    def tune(self, sims: Sequence[binding.Simulation], dt: float, M: int = 3, K: int = 2) -> str:
        key = shape_class(sims)
        if key in self.cache:
            return self.cache[key][0]
        cands = candidate_packings(sims)
        blobs = [s.get_state() for s in sims]
        times = {}
        for name, packing in cands.items():
            self._run(sims, packing, dt, M, K, 1)          # capture the graphs (untimed)
            for s in sims:
                s.sync()
            t0 = time.perf_counter()
            self._run(sims, packing, dt, M, K, self.trial_steps)
            for s in sims:
                s.sync()
            times[name] = (time.perf_counter() - t0) / self.trial_steps
            for s, b in zip(sims, blobs):
                s.set_state(b)
        best = min(times, key=times.get)
        self.cache[key] = (best, [times[best]])
        self.timings[key] = times
        return best

    def packing(self, sims: Sequence[binding.Simulation], dt: float, M: int = 3, K: int = 2) -> List[List[int]]:
        return candidate_packings(sims)[self.tune(sims, dt, M, K)]

    def step(self, sims: Sequence[binding.Simulation], dt: float, M: int = 3, K: int = 2, steps: int = 1) -> None:
        self._run(sims, self.packing(sims, dt, M, K), dt, M, K, steps)


# ---------------------------------------------------------------------------
# Layout and thread-mapping options of one handle, chosen by timing
# ---------------------------------------------------------------------------

def option_candidates(streaming: bool, precision: int) -> Dict[str, Dict[str, int]]:
    """Candidate option sets for one shape class.  Streaming handles (large
    operators) choose how the AMG levels with long rows are stored and read
    (SELL-32 by the size rule or CSR; lanes per CSR row from the mean row
    length or forced to 16 / 32) and, in mixed precision, the SELL-32/4
    vector-load copy; persistent handles choose the solver block size."""
    if streaming:
        c = {"auto": {}, "csr": {"wide_sell": -1}, "csr16": {"wide_sell": -1, "csr_lanes": 16},
             "csr32": {"wide_sell": -1, "csr_lanes": 32}}
        if precision == binding.MIXED:
            c["sell32"] = {"vec4": -1}
        return c
    return {"auto": {}, "block256": {"cg_block": 256}, "block1024": {"cg_block": 1024}}


class OptionTuner:
    """Times option candidates on a workload (a handle per candidate, one
    untimed step for the graph capture, then ``trial_steps`` timed steps from
    the same initial state) once per shape class (model, precision, nodes,
    stored entries, solver form) and caches the fastest."""

    def __init__(self, trial_steps: int = 2):
        self.trial_steps = trial_steps
        self.cache: Dict[Tuple, str] = {}
        self.timings: Dict[Tuple, Dict[str, float]] = {}

    def tune(self, w, base: Dict[str, int], dt: float, M: int = 3, K: int = 2) -> Dict[str, int]:
        """Options (base updated with the chosen candidate) for workload w."""
        probe = binding.simulation_from_workload(w, binding.default_options(**base))
        st = probe.stats()
        nnz = probe.nnz()
        probe.close()
        prec = base.get("precision", binding.FP64)
        key = (w.model, prec, int(w.n_nodes), int(nnz), int(st["streaming"]))
        cands = option_candidates(bool(st["streaming"]), prec)
        if key not in self.cache:
            times = {}
            for name, extra in cands.items():
                sim = binding.simulation_from_workload(w, binding.default_options(**{**base, **extra}))
                sim.step(dt, M, K)
                sim.sync()
                t0 = time.perf_counter()
                for _ in range(self.trial_steps):
                    sim.step(dt, M, K)
                sim.sync()
                times[name] = (time.perf_counter() - t0) / self.trial_steps
                sim.close()
            self.cache[key] = min(times, key=times.get)
            self.timings[key] = times
        return {**base, **cands[self.cache[key]]}
