#!/usr/bin/env python3
"""Throughput of the partitioned-SDC bidomain step on GB300.

Metric: node-steps/s of one partitioned-SDC time step (Algorithm 2: elliptic
solve, ROS2 predictor, SDC correction; 3 Gauss-Lobatto nodes, 2 sweeps) on
the TP06 epicardial sheet of 257 x 257 P1 nodes (66,049 nodes, 2.5 cm square,
fibres along x, dt = 0.02 ms, S1 strip x < 0.1 cm at t = 0, S2 on the corner
quadrant at 310 ms), timed from a developed state (t = 330 ms: the S2 front
running into the S1 wave's refractory tail), inputs resident in HBM.
`value` is the mixed-precision path, `fp64` the pure FP64 path.  Further
legs: the TP06 3-D slab of 201 x 201 x 51 nodes (HBM-bound; its own
roofline), the LR91 bidomain-bath sheet of the paper's Sec. 4, the serving
stream, and the FP64 oracle on the host cores.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

N > 1 runs one independent replica per GPU under torchrun (the method has no
data-path exchange: each GPU steps its own simulation); rank 0 prints one
JSON line.

Two helpers for profiling runs:
  python bench.py --profile-workload {sheet,slab,lv,bath} [--side N] [--lv-h H] [--steps K]
      steps one workload K times (no timing) so that a profiler can capture it;
  python bench.py --summarize-launches launches.csv
      prints the per-kernel launches, total time and share of an
      `ncu --metrics gpu__time_duration.sum --csv` launch list as a table.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

WORKLOAD = "tp06_sheet_257x257"
SIDE, LENGTH, DT, M_NODES, K_SWEEPS = 257, 2.5, 0.02, 3, 2
S2_MS, S2_SIDE = 310.0, 1.25
SAMPLE_SIDE = 33          # oracle sample: 33 x 33 nodes at the same spacing


# ---------------------------------------------------------------------------
# oracle legs (CPU): cpu_baseline and --impl reference
# ---------------------------------------------------------------------------

def oracle_sample_problem():
    import numpy as np
    from oracle import bidomain as OB
    from oracle import tp06 as OT
    from paper_2510_27447_gb300 import workloads as W
    h = LENGTH / (SIDE - 1)
    w = W.sheet(SAMPLE_SIDE, h * (SAMPLE_SIDE - 1), W.TP06_EPI, DT, 1)
    cell = OT.model()
    P = OB.Bidomain(w.xyz, w.elems, w.fibers, w.sigma, w.chi, w.cm, cell, w.stimuli, pin_node=0)
    X = np.repeat(cell.initial()[:, None], w.n_nodes, axis=1)
    return P, X, w.n_nodes


def oracle_rate(warmup: int, steps: int, seconds: float) -> dict:
    import numpy as np
    P, X, n = oracle_sample_problem()
    u = np.zeros(n)
    for k in range(warmup):
        X, u, _ = P.step(X, u, k * DT, DT, M_NODES, K_SWEEPS)
    t0 = time.perf_counter()
    done = 0
    while done < steps or (seconds > 0 and time.perf_counter() - t0 < seconds):
        X, u, _ = P.step(X, u, (warmup + done) * DT, DT, M_NODES, K_SWEEPS)
        done += 1
        if seconds > 0 and done >= steps and time.perf_counter() - t0 >= seconds:
            break
    el = time.perf_counter() - t0
    return {"value": n * done / el, "steps": done, "seconds": el, "nodes": n}


def run_oracle_processes(procs: int, warmup: int, steps: int, seconds: float) -> dict:
    """`procs` independent single-threaded oracle processes on the same
    sample at once (the oracle's sparse direct solves run on one thread, so
    the host's cores are used by running one problem per core); the rate is
    the node-steps of all processes over the longest one's time."""
    env = dict(os.environ)
    for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
        env[k] = "1"
    cmd = [sys.executable, os.path.abspath(__file__), "--oracle-sample", "--warmup", str(warmup),
           "--steps", str(steps), "--seconds", str(seconds)]
    ps = [subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.PIPE, text=True, env=env)
          for _ in range(procs)]
    res = []
    for p in ps:
        out, err = p.communicate(timeout=900)
        if p.returncode != 0:
            raise RuntimeError(err[-2000:])
        res.append(json.loads(out.strip().splitlines()[-1]))
    secs = max(r["seconds"] for r in res)
    units = sum(r["nodes"] * r["steps"] for r in res)
    return {"value": units / secs, "steps": min(r["steps"] for r in res), "seconds": secs,
            "nodes": res[0]["nodes"], "processes": procs}


def sample_text(res: dict) -> str:
    who = "1 process" if res.get("processes", 1) == 1 else f"{res['processes']} concurrent processes"
    return (f"FP64 oracle (numpy/scipy, sparse direct solves), TP06 sheet of {SAMPLE_SIDE}x{SAMPLE_SIDE} "
            f"nodes at the 257x257 grid spacing, dt={DT} ms, M={M_NODES}, K={K_SWEEPS}, from the published "
            f"initial state with the S1 strip; {who} of 1 thread each, >= {res['steps']} steps in "
            f"{res['seconds']:.1f} s")


# ---------------------------------------------------------------------------
# clocks during the timed region
# ---------------------------------------------------------------------------

class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.lines = []
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except OSError:
            self.proc = None
        time.sleep(0.3)
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self) -> dict:
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx.append(float(parts[2]))
            except ValueError:
                continue
            for nm, val in zip(names, parts[5:9]):
                if val.lower() == "active":
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


# ---------------------------------------------------------------------------
# roofline bookkeeping
# ---------------------------------------------------------------------------

def kernel_source_hash() -> str:
    h = hashlib.sha256()
    for f in ("pcg.cu", "amg.cu", "mixed.cu", "stream.cu", "stream2.cu", "stream_rows.cuh", "sparse.cuh",
              "vcycle.cuh", "bd_internal.h"):
        path = os.path.join(ROOT, "paper_2510_27447_gb300", "csrc", f)
        if os.path.exists(path):
            with open(path, "rb") as fh:
                h.update(fh.read())
    return h.hexdigest()[:16]


def load_traffic(key: str, alg_bytes_per_launch: float = 0.0):
    """DRAM bytes per launch of a kernel from the committed ncu summary, if
    the solver sources are unchanged since it was captured (else None).  An
    entry holds either the bytes of one launch or, for a solve made of a
    chain of kernels captured on a smaller case, the ratio of DRAM bytes to
    algorithmic bytes over whole iterations, applied here to the launch's
    algorithmic bytes (traffic grows with the bytes the iterations move)."""
    try:
        with open(os.path.join(ROOT, "profiles", "traffic.json")) as fh:
            e = json.load(fh).get(key)
        if e and e.get("source_hash") == kernel_source_hash():
            if "dram_over_algorithmic" in e:
                return round(e["dram_over_algorithmic"] * alg_bytes_per_launch) if alg_bytes_per_launch else None
            return e.get("bytes_per_launch")
    except (OSError, ValueError):
        pass
    return None


def measured_peaks() -> dict:
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            return json.load(fh)
    except (OSError, ValueError):
        return {}


def l2_copy_gbs(torch, stream) -> float:
    """Bandwidth of a copy whose source and destination (2 x 24 MB) stay in
    L2 (129 MB): read + write bytes per second, best of 5 runs of 50 copies."""
    a = torch.empty(6 * 1024 * 1024, dtype=torch.float32, device="cuda").fill_(1.0)
    b = torch.empty_like(a)
    best = 0.0
    with torch.cuda.stream(stream):
        for _ in range(10):
            b.copy_(a)
        for _ in range(5):
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            for _ in range(50):
                b.copy_(a)
            e1.record(stream)
            e1.synchronize()
            best = max(best, 50 * 2 * a.numel() * 4 / (e0.elapsed_time(e1) / 1e3) / 1e9)
    return best


def solver_roofline(prof: dict, kind: str = "pcg_elliptic") -> dict:
    """Algorithmic bytes and achieved GB/s of one solver kind from a profile
    of whole steps: Krylov-level bytes by the per-SpMV and per-iteration
    model, the V-cycle levels by the same per-SpMV model (listed apart), the
    dense coarse solve apart and not counted."""
    idx = 0 if kind == "pcg_elliptic" else 1
    launches = prof["launches"][kind]
    avg_s = prof["ms"][kind] / launches / 1e3
    krylov = prof["alg_bytes"][idx] / launches
    vcyc = prof["vcycle_bytes"] / launches if idx == 0 else 0.0
    coarse = prof["coarse_bytes"] / launches if idx == 0 else 0.0
    its = prof["cg_iters"][idx] / launches
    return {"kernel": kind, "avg_launch_ms": round(avg_s * 1e3, 4),
            "krylov_bytes_per_launch": round(krylov), "vcycle_bytes_per_launch": round(vcyc),
            "coarse_dense_bytes_per_launch": round(coarse),
            "achieved_gbs": round((krylov + vcyc) / avg_s / 1e9, 1),
            "krylov_only_gbs": round(krylov / avg_s / 1e9, 1),
            "cg_iters_per_launch": round(its, 1),
            "per_iteration_us": round(avg_s * 1e6 / its, 2) if its > 0 else None}


def shares(prof: dict) -> dict:
    tot = sum(prof["ms"].values())
    return {k: round(v / tot, 4) for k, v in prof["ms"].items()}


# ---------------------------------------------------------------------------
# GPU legs
# ---------------------------------------------------------------------------

def headline_workload():
    from paper_2510_27447_gb300 import workloads as W
    return W.sheet(SIDE, LENGTH, W.TP06_EPI, DT, 1, s2=(S2_MS, S2_SIDE), name=WORKLOAD)


def timed(sim, torch, stream, flush, steps: int, dt: float) -> list:
    ms = []
    for _ in range(steps):
        flush.add_(1.0)                       # evict L2 between timed steps
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record(stream)
        sim.step(dt, M_NODES, K_SWEEPS)
        b.record(stream)
        b.synchronize()
        ms.append(a.elapsed_time(b))
    return ms


def developed_state(w, torch, stream, dev_ms: float):
    """State blob of the headline sheet at t = dev_ms, stepped from the
    published initial state on the mixed path (S1 at 0, S2 at 310 ms)."""
    import numpy as np
    from paper_2510_27447_gb300 import binding
    with torch.cuda.stream(stream):
        opts = binding.default_options(precision=binding.MIXED, stream=stream.cuda_stream)
        sim = binding.simulation_from_workload(w, opts)
        for _ in range(int(round(dev_ms / DT))):
            sim.step(DT, M_NODES, K_SWEEPS)
        sim.sync()
        blob = sim.get_state()
        v, _ = sim.fields()
        sim.close()
    return blob, {"t_ms": dev_ms, "depolarised_frac": round(float(np.mean(v > -60.0)), 3),
                  "v_range_mV": [round(float(v.min()), 1), round(float(v.max()), 1)]}


def e2e_rate(sim, torch, blob: bytes, steps: int) -> dict:
    """Same metric through the C ABI with host buffers: every step uploads the
    state blob from pinned host memory, steps, and reads v and u back."""
    import ctypes as C
    from paper_2510_27447_gb300 import binding
    L = binding.lib()
    nb = len(blob)
    host = torch.empty(nb, dtype=torch.uint8, pin_memory=True)
    host.numpy()[:] = memoryview(blob)
    vout = torch.empty(sim.NT, dtype=torch.float64, pin_memory=True)
    uout = torch.empty(sim.N, dtype=torch.float64, pin_memory=True)
    dp = C.POINTER(C.c_double)
    t0 = time.perf_counter()
    for _ in range(steps):
        rc = L.bd_set_state(sim.h, C.c_void_p(host.data_ptr()), nb)
        if rc:
            raise binding.BdError(rc, "set_state")
        sim.step(DT, M_NODES, K_SWEEPS)
        rc = L.bd_get_fields(sim.h, C.cast(C.c_void_p(vout.data_ptr()), dp),
                             C.cast(C.c_void_p(uout.data_ptr()), dp), None)
        if rc:
            raise binding.BdError(rc, "get_fields")
    el = time.perf_counter() - t0
    return {"value": sim.N * steps / el, "unit": "node-steps/s", "h2d_bytes_per_step": nb,
            "d2h_bytes_per_step": 8 * (sim.NT + sim.N)}


def per_solve(st0, st1, key):
    return round((st1[f"cg_iters_{key}"] - st0[f"cg_iters_{key}"]) /
                 max(1, st1[f"cg_solves_{key}"] - st0[f"cg_solves_{key}"]), 1)


def slab_leg(args, torch, stream, flush, peaks) -> dict:
    """Config 2: TP06 in the 2 x 2 x 0.5 cm slab (201 x 201 x 51 nodes,
    Kuhn tetrahedra, -60..+60 deg transmural fibres, gates perturbed by
    +-2 % with PCG64(2)), dt = 0.025 ms, 3 Lobatto nodes, 2 sweeps, mixed and
    FP64, timed from t = 2 ms (S1 front formed).  Its operators (30.4M
    entries) do not fit in L2: the solver rooflines are against HBM."""
    from paper_2510_27447_gb300 import binding, workloads as W
    t0 = time.perf_counter()
    rest = binding.rest_state(W.TP06_EPI)
    w = W.config2(rest=rest, gate_rows=list(range(1, 13)))
    out = {"workload": w.name, "nodes": w.n_nodes, "dt_ms": w.dt, "mesh_s": round(time.perf_counter() - t0, 1),
           "start": "t = 2 ms from the seeded perturbed initial state (S1 plane x < 0.1 cm at 0 ms)"}
    blob = None
    hbm = peaks.get("hbm_gbs", 6800.0)
    for name, prec in (("mixed", binding.MIXED), ("fp64", binding.FP64)):
        with torch.cuda.stream(stream):
            t0 = time.perf_counter()
            opts = binding.default_options(precision=prec, stream=stream.cuda_stream)
            sim = binding.simulation_from_workload(w, opts)
            setup = time.perf_counter() - t0
            if blob is None:
                for _ in range(int(round(2.0 / w.dt))):
                    sim.step(w.dt, M_NODES, K_SWEEPS)
                sim.sync()
                blob = sim.get_state()
            else:
                sim.set_state(blob)
            for _ in range(args.warmup):
                sim.step(w.dt, M_NODES, K_SWEEPS)
            sim.sync()
            st0 = sim.stats()
            torch.cuda.synchronize()
            ms = timed(sim, torch, stream, flush, args.slab_steps, w.dt)
            sim.sync()
            st1 = sim.stats()
            prof = sim.profile_steps(w.dt, M_NODES, K_SWEEPS, 2)
            sim.close()
        t = sum(ms) / len(ms)
        out[name] = {"ms_per_step": round(t, 3), "value": round(w.n_nodes / (t / 1e3), 1),
                     "setup_s": round(setup, 1), "cg_iters_e": per_solve(st0, st1, "e"),
                     "cg_iters_p": per_solve(st0, st1, "p"), "kernel_share": shares(prof),
                     "elliptic": solver_roofline(prof, "pcg_elliptic"),
                     "parabolic": solver_roofline(prof, "pcg_parabolic"),
                     "solver_tier": st1["solver_tier"], "amg_levels": st1["amg_levels"]}
    m = out["mixed"]["elliptic"]
    out["roofline"] = {"kernel": "pcg_elliptic (mixed)", "bound": "hbm", "achieved": m["achieved_gbs"],
                       "peak": hbm, "unit": "GB/s", "frac": round(m["achieved_gbs"] / hbm, 4),
                       "traffic": load_traffic("slab_pcg_elliptic", m["krylov_bytes_per_launch"] +
                                               m["vcycle_bytes_per_launch"]),
                       "peak_source": "measured" if "hbm_gbs" in peaks else "fallback",
                       "parabolic_frac": round(out["mixed"]["parabolic"]["achieved_gbs"] / hbm, 4)}
    out["steps"] = args.slab_steps
    return out


def bath_leg(args, torch, stream, flush) -> dict:
    """The bidomain-bath run of Sec. 4 (801^2 nodes over [-1, 7]^2, tissue
    [0, 6]^2 with 601^2 nodes, LR91, 3 Lobatto nodes, 2 sweeps) at its maximum
    step dt = 0.05 ms, from rest + S1: node-steps/s over all nodes (the unit
    the paper's 34 h for 600 ms on 2 x 28 cores converts to: 641,601 x 12,000
    steps / 122,400 s = 6.29e4 node-steps/s, if every step is the maximum)."""
    from paper_2510_27447_gb300 import binding, workloads as W
    w = W.bath_paper_2d()
    out = {"workload": w.name, "nodes": w.n_nodes, "tissue_nodes": w.n_tissue, "dt_ms": w.dt,
           "sigma_bath": w.sbath, "paper_rate_node_steps_per_s": 6.29e4}
    for name, prec in (("mixed", binding.MIXED), ("fp64", binding.FP64)):
        with torch.cuda.stream(stream):
            opts = binding.default_options(precision=prec, stream=stream.cuda_stream, pin_node=w.pin_node)
            sim = binding.simulation_from_workload(w, opts)
            for _ in range(args.warmup):
                sim.step(w.dt, M_NODES, K_SWEEPS)
            sim.sync()
            st0 = sim.stats()
            torch.cuda.synchronize()
            ms = timed(sim, torch, stream, flush, args.bath_steps, w.dt)
            sim.sync()
            st1 = sim.stats()
            sim.close()
        t = sum(ms) / len(ms)
        out[name] = {"ms_per_step": round(t, 3), "value": round(w.n_nodes / (t / 1e3), 1),
                     "cg_iters_e": per_solve(st0, st1, "e"), "cg_iters_p": per_solve(st0, st1, "p")}
    out["steps"] = args.bath_steps
    return out


def lv_leg(args, torch, stream, flush, peaks) -> dict:
    """The 3-D bidomain-bath configuration: TP06 in a truncated prolate LV
    shell inside a box bath (jittered Kuhn lattice, h = args.lv_h cm in the
    shell's bounding box, coarser bath margins), dt = 0.025 ms, 3 Lobatto
    nodes, 2 sweeps, mixed and FP64, from rest + apical pacing."""
    from paper_2510_27447_gb300 import binding, workloads as W
    t0 = time.perf_counter()
    w = W.lv_shell_bath(h=args.lv_h)
    out = {"workload": w.name, "nodes": w.n_nodes, "tissue_nodes": w.n_tissue, "elements": int(len(w.elems)),
           "dt_ms": w.dt, "sigma_bath": w.sbath, "mesh_s": round(time.perf_counter() - t0, 1)}
    for name, prec in (("mixed", binding.MIXED), ("fp64", binding.FP64)):
        with torch.cuda.stream(stream):
            t0 = time.perf_counter()
            opts = binding.default_options(precision=prec, stream=stream.cuda_stream, pin_node=w.pin_node)
            sim = binding.simulation_from_workload(w, opts)
            setup = time.perf_counter() - t0
            for _ in range(args.warmup):
                sim.step(w.dt, M_NODES, K_SWEEPS)
            sim.sync()
            st0 = sim.stats()
            torch.cuda.synchronize()
            ms = timed(sim, torch, stream, flush, args.lv_steps, w.dt)
            sim.sync()
            st1 = sim.stats()
            prof = sim.profile_steps(w.dt, M_NODES, K_SWEEPS, 2)
            sim.close()
        t = sum(ms) / len(ms)
        out[name] = {"ms_per_step": round(t, 3), "value": round(w.n_nodes / (t / 1e3), 1),
                     "setup_s": round(setup, 1), "cg_iters_e": per_solve(st0, st1, "e"),
                     "cg_iters_p": per_solve(st0, st1, "p"), "kernel_share": shares(prof),
                     "elliptic": solver_roofline(prof, "pcg_elliptic"),
                     "parabolic": solver_roofline(prof, "pcg_parabolic")}
    hbm = peaks.get("hbm_gbs", 6800.0)
    m = out["mixed"]["elliptic"]
    out["roofline"] = {"kernel": "pcg_elliptic (mixed)", "bound": "hbm", "achieved": m["achieved_gbs"],
                       "peak": hbm, "unit": "GB/s", "frac": round(m["achieved_gbs"] / hbm, 4),
                       "traffic": load_traffic("lv_pcg_elliptic", m["krylov_bytes_per_launch"] +
                                               m["vcycle_bytes_per_launch"]),
                       "peak_source": "measured" if "hbm_gbs" in peaks else "fallback",
                       "parabolic_frac": round(out["mixed"]["parabolic"]["achieved_gbs"] / hbm, 4)}
    out["steps"] = args.lv_steps
    return out


def batch_leg(args) -> dict:
    """Batched execution (bd_batch_step) of args.batch_requests independent
    requests of the serving stream's shape (sides 33/65/129, LR91/TP06 50/50,
    jittered conductivities), each timed for args.batch_steps steps of
    dt = 0.02 ms: one launch per phase over the concatenated nodes of a batch,
    packed by the autotuner, against the same requests stepped one at a time
    (each its own graph) in the same precision."""
    from paper_2510_27447_gb300 import binding, workloads as W
    from paper_2510_27447_gb300.batching import BatchRunner
    reqs = W.request_stream(args.batch_requests, 40.0, seed=5, sides=(33, 65, 129), t_end=10.0)
    ws = [W.request_workload(r) for r in reqs]
    dt, steps, warm = 0.02, args.batch_steps, 3
    nodes = sum(w.n_nodes for w in ws)
    out = {"requests": len(ws), "nodes": nodes, "sides": [33, 65, 129], "steps": steps,
           "models": {"lr91": sum(w.model == W.LR91 for w in ws), "tp06": sum(w.model == W.TP06_EPI for w in ws)}}
    for name, prec in (("mixed", binding.MIXED), ("fp64", binding.FP64)):
        opts = lambda: binding.default_options(precision=prec)
        el = 0.0
        for w in ws:
            sim = binding.simulation_from_workload(w, opts())
            for _ in range(warm):
                sim.step(dt, M_NODES, K_SWEEPS)
            sim.sync()
            t0 = time.perf_counter()
            for _ in range(steps):
                sim.step(dt, M_NODES, K_SWEEPS)
            sim.sync()
            el += time.perf_counter() - t0
            sim.close()
        alone = nodes * steps / el
        sims = [binding.simulation_from_workload(w, opts()) for w in ws]
        runner = BatchRunner()
        t0 = time.perf_counter()
        best = runner.tune(sims, dt, M_NODES, K_SWEEPS)
        tune_s = time.perf_counter() - t0
        runner.step(sims, dt, M_NODES, K_SWEEPS, warm)
        for s in sims:
            s.sync()
        t0 = time.perf_counter()
        runner.step(sims, dt, M_NODES, K_SWEEPS, steps)
        for s in sims:
            s.sync()
        bt = time.perf_counter() - t0
        packing = runner.packing(sims, dt, M_NODES, K_SWEEPS)
        key = list(runner.timings)[0]
        for s in sims:
            s.close()
        out[name] = {"batched_node_steps_per_s": round(nodes * steps / bt, 1),
                     "one_at_a_time_node_steps_per_s": round(alone, 1),
                     "speedup": round(alone and (nodes * steps / bt) / alone, 2),
                     "batched_ms_per_step": round(1e3 * bt / steps, 3),
                     "packing": best, "batches": len(packing), "tune_s": round(tune_s, 2),
                     "candidate_ms_per_step": {k: round(1e3 * v, 3) for k, v in runner.timings[key].items()}}
    return out


def serve_leg(args) -> dict:
    """The serving stream: args.serve_requests Poisson(40/s) arrivals (the
    request recipe of the 512-request workload: sides 33/65/129/257,
    LR91/TP06 50/50, jittered conductivities, strip and S2 positions), each
    simulated for args.serve_ms ms at dt = 0.02 ms, mixed precision:
      batched     resident requests below args.serve_solo_nodes nodes advance
                  together through bd_batch_step, one batch per (model, mesh
                  size), joining at 10-step chunk boundaries; larger ones run
                  alone on their own streams, one at a time (16 slots in all);
      streams     each resident request on its own stream (8 slots);
      closed      the batched form with 16 clients keeping one request each
                  outstanding;
      one at a time, mixed and FP64: every request's service time (handle
                  set-up + its steps) measured on the GPU alone, the FIFO
                  queue of the same arrivals computed from them exactly.
    Handles are built by worker threads in every served form."""
    from paper_2510_27447_gb300 import binding, serving as S, workloads as W
    sides = (33, 65, 129, 257)
    reqs = W.request_stream(args.serve_requests, 40.0, seed=4, sides=sides, t_end=args.serve_ms)

    def jobs():
        return [S.Job(r.rid, r.arrival_s, r.side ** 2, int(round(args.serve_ms / r.dt)), W.request_workload(r))
                for r in reqs]
    js = jobs()
    out = {"requests": len(reqs), "rate_per_s": 40.0, "sides": list(sides), "t_end_ms": args.serve_ms,
           "work_node_steps": int(sum(j.n_nodes * j.n_steps for j in js))}

    def record(sm, wall):
        return {"p50_ms": round(sm["p50_ms"], 2), "p99_ms": round(sm["p99_ms"], 2),
                "node_steps_per_s": round(sm["node_steps_per_s"], 1),
                "offered_node_steps_per_s": round(sm["offered_node_steps_per_s"], 1),
                "served_over_offered": round(sm["served_over_offered"], 4), "wall_s": round(wall, 2)}
    mixed = lambda: binding.default_options(precision=binding.MIXED)          # noqa: E731
    out["solo_nodes"] = args.serve_solo_nodes
    solo = args.serve_solo_nodes if args.serve_solo_nodes > 0 else None
    for name, batched, slots, chunk in (("batched_mixed", True, 16, 10), ("streams_mixed", False, 8, 25)):
        ex = S.GpuExecutor(mixed, dt=0.02, solo_nodes=solo)
        t0 = time.perf_counter()
        done = S.Server(ex, max_slots=slots, hbm_budget=64 << 30, chunk_steps=chunk, batched=batched,
                        max_solo=1).run(jobs())
        wall = time.perf_counter() - t0
        ex.close()
        out[name] = record(S.summarize(done), wall)
        out[name]["slots"] = slots
        out[name]["chunk_steps"] = chunk
    ex = S.GpuExecutor(mixed, dt=0.02, solo_nodes=solo)
    t0 = time.perf_counter()
    done = S.Server(ex, max_slots=16, hbm_budget=64 << 30, chunk_steps=10, batched=True,
                    max_solo=1).run_closed(jobs(), 16)
    wall = time.perf_counter() - t0
    ex.close()
    sm = S.summarize(done)
    out["closed_batched_mixed"] = {"clients": 16, "p50_ms": round(sm["p50_ms"], 2), "p99_ms": round(sm["p99_ms"], 2),
                                   "node_steps_per_s": round(sm["node_steps_per_s"], 1), "wall_s": round(wall, 2)}
    for name, prec in (("one_at_a_time_mixed", binding.MIXED), ("one_at_a_time_fp64", binding.FP64)):
        service = []
        for j in js:
            t0 = time.perf_counter()
            sim = binding.simulation_from_workload(j.payload, binding.default_options(precision=prec))
            setup = time.perf_counter() - t0
            k = min(j.n_steps, 20)
            sim.step(0.02, M_NODES, K_SWEEPS)          # capture (part of the set-up)
            sim.sync()
            setup = time.perf_counter() - t0
            t1 = time.perf_counter()
            for _ in range(k):
                sim.step(0.02, M_NODES, K_SWEEPS)
            sim.sync()
            per_step = (time.perf_counter() - t1) / k
            sim.close()
            service.append(setup + per_step * j.n_steps)
        sm = S.summarize(S.fifo_schedule(js, service))
        out[name] = {"p50_ms": round(sm["p50_ms"], 2), "p99_ms": round(sm["p99_ms"], 2),
                     "node_steps_per_s": round(sm["node_steps_per_s"], 1),
                     "served_over_offered": round(sm["served_over_offered"], 4),
                     "service_s_total": round(sum(service), 2),
                     "method": "service time per request measured alone on the GPU (set-up + 20 timed steps "
                               "scaled to its step count); FIFO queue of the same arrivals computed exactly"}
    return out


def run_ours(args) -> None:
    import torch
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    if rank == 0:
        import __graft_entry__ as g
        g.build()
    if dist:
        dist.barrier()
    from paper_2510_27447_gb300 import binding
    from paper_2510_27447_gb300.replicas import whole_job_rate
    peaks = measured_peaks()
    stream = torch.cuda.Stream()
    flush = torch.zeros(64 * 1024 * 1024, dtype=torch.float32, device="cuda")   # 256 MB > L2
    l2_gbs = l2_copy_gbs(torch, stream)
    w = headline_workload()
    blob, dev = developed_state(w, torch, stream, args.dev_ms)
    results, profiles = {}, {}
    for name, prec in (("mixed", binding.MIXED), ("fp64", binding.FP64)):
        with torch.cuda.stream(stream):
            opts = binding.default_options(precision=prec, stream=stream.cuda_stream)
            sim = binding.simulation_from_workload(w, opts)
            sim.set_state(blob)
            for _ in range(args.warmup):
                sim.step(DT, M_NODES, K_SWEEPS)
            sim.sync()
            st0 = sim.stats()
            if dist:
                dist.barrier()
            torch.cuda.synchronize()
            with ClockSampler(local) as clk:
                ms = timed(sim, torch, stream, flush, args.steps, DT)
            torch.cuda.synchronize()
            sim.sync()
            st1 = sim.stats()
            rate, secs = whole_job_rate(sim.N * args.steps, sum(ms) / 1e3, device="cuda")
            results[name] = {"ms_per_step": secs * 1e3 / args.steps, "value": rate, "clocks": clk.summary(),
                             "launches": st1["kernel_launches"] - st0["kernel_launches"],
                             "cg_iters_e": per_solve(st0, st1, "e"), "cg_iters_p": per_solve(st0, st1, "p"),
                             "solver_tier": st1["solver_tier"], "amg_levels": st1["amg_levels"]}
            sim.set_state(blob)
            profiles[name] = sim.profile_steps(DT, M_NODES, K_SWEEPS, args.steps)
            if name == "mixed":
                results[name]["e2e"] = e2e_rate(sim, torch, blob, max(3, args.steps // 2))
            sim.close()
    if rank != 0:
        if dist:
            dist.destroy_process_group()
        return

    prof = profiles["mixed"]
    ell = solver_roofline(prof, "pcg_elliptic")
    hbm = peaks.get("hbm_gbs", 6800.0)
    # the headline sheet's operators and vectors (about 7 MB a matrix) live in
    # L2: its solver is bounded by L2 bandwidth and by the latency of its
    # dependent phases, not by HBM
    roof = {"kernel": "pcg_elliptic (mixed)", "bound": "l2", "achieved": ell["achieved_gbs"],
            "peak": round(l2_gbs, 1), "unit": "GB/s", "frac": round(ell["achieved_gbs"] / l2_gbs, 4),
            "traffic": load_traffic("sheet_pcg_elliptic"),
            "peak_source": "L2-resident copy measured in this run (2 x 24 MB, read + write)",
            "hbm_frac": round(ell["achieved_gbs"] / hbm, 4), "hbm_peak": hbm,
            "per_iteration_us": ell["per_iteration_us"], "cg_iters_per_launch": ell["cg_iters_per_launch"],
            "krylov_bytes_per_launch": ell["krylov_bytes_per_launch"],
            "vcycle_bytes_per_launch": ell["vcycle_bytes_per_launch"],
            "coarse_dense_bytes_per_launch": ell["coarse_dense_bytes_per_launch"],
            "avg_launch_ms": ell["avg_launch_ms"]}

    slab = None
    if args.slab_steps > 0:
        try:
            slab = slab_leg(args, torch, stream, flush, peaks)
        except Exception as e:  # noqa: BLE001
            slab = {"error": str(e)[:300]}
    bath = None
    if args.bath_steps > 0:
        try:
            bath = bath_leg(args, torch, stream, flush)
        except Exception as e:  # noqa: BLE001
            bath = {"error": str(e)[:300]}
    lv = None
    if args.lv_steps > 0:
        try:
            lv = lv_leg(args, torch, stream, flush, peaks)
        except Exception as e:  # noqa: BLE001
            lv = {"error": str(e)[:300]}
    batch = None
    if args.batch_requests > 0:
        try:
            batch = batch_leg(args)
        except Exception as e:  # noqa: BLE001
            batch = {"error": str(e)[:300]}
    serve = None
    if args.serve_requests > 0:
        try:
            serve = serve_leg(args)
        except Exception as e:  # noqa: BLE001
            serve = {"error": str(e)[:300]}

    base = None
    if world == 1 and not args.no_baseline:
        try:
            one = run_oracle_processes(1, 0, 1, 15.0)
            ncores = os.cpu_count() or 1
            allc = run_oracle_processes(ncores, 0, 1, 15.0)
            base = {"value": round(allc["value"], 2), "unit": "node-steps/s", "cores": ncores, "kind": "oracle",
                    "sample": sample_text(allc),
                    "single_thread": {"value": round(one["value"], 2), "cores": 1, "sample": sample_text(one)}}
        except Exception as e:  # noqa: BLE001
            base = {"value": None, "unit": "node-steps/s", "cores": None, "kind": "oracle",
                    "sample": f"failed: {e}"[:200]}

    mixed = results["mixed"]
    line = {
        "metric": "node-steps/s",
        "value": round(mixed["value"], 1),
        "unit": "node-steps/s",
        "n_gpus": world,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": round(mixed["ms_per_step"], 4),
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "mixed: f32 membrane model and Krylov iterations, f64 refinement and state",
        "data": "synthetic",
        "config": {"workload": WORKLOAD, "nodes": w.n_nodes, "model": "TP06 epicardial", "dt_ms": DT,
                   "sdc_nodes": M_NODES, "sweeps": K_SWEEPS,
                   "start": f"developed state at {args.dev_ms:g} ms (S1 strip at 0 ms, S2 corner quadrant at "
                            f"{S2_MS:g} ms), restored with bd_set_state before each leg",
                   "developed_state": dev,
                   "l2": "flushed between timed steps (256 MB write)", "parallelism": f"replicas x{world}"},
        "fp64": {"value": round(results["fp64"]["value"], 1),
                 "ms_per_step": round(results["fp64"]["ms_per_step"], 4), "dtype": "f64",
                 "kernel_share": shares(profiles["fp64"]),
                 "elliptic": solver_roofline(profiles["fp64"], "pcg_elliptic"),
                 "cg_iters_per_solve": {"elliptic": results["fp64"]["cg_iters_e"],
                                        "parabolic": results["fp64"]["cg_iters_p"]}},
        "e2e": {k: (round(v, 1) if isinstance(v, float) else v) for k, v in mixed["e2e"].items()},
        "gpu_launches": int(mixed["launches"]),
        "clocks": mixed["clocks"],
        "roofline": roof,
        "kernel_share": shares(prof),
        "parabolic": solver_roofline(prof, "pcg_parabolic"),
        "cg_iters_per_solve": {"elliptic": mixed["cg_iters_e"], "parabolic": mixed["cg_iters_p"]},
        "solver": {"tier": mixed["solver_tier"], "amg_levels": mixed["amg_levels"]},
        "cpu_baseline": base,
        "slab": slab,
        "bath": bath,
        "lv_shell_bath": lv,
        "batch": batch,
        "serve": serve,
    }
    print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()


def profile_workload(args) -> None:
    """Step one workload args.steps times and print the handle's counters."""
    from paper_2510_27447_gb300 import binding, workloads as W
    name = args.profile_workload
    if name == "sheet":
        w = W.sheet(args.side, LENGTH * (args.side - 1) / (SIDE - 1), W.TP06_EPI, DT, 1)
    elif name == "slab":
        w = W.config2() if args.side == SIDE else W.config2(args.side, args.side, (args.side - 1) // 4 + 1)
    elif name == "lv":
        w = W.lv_shell_bath(h=args.lv_h)
    else:
        w = W.bath_paper_2d()
    prec = binding.FP64 if args.precision == "fp64" else binding.MIXED
    sim = binding.simulation_from_workload(w, binding.default_options(precision=prec, pin_node=w.pin_node,
                                                                      streaming=args.streaming, vec4=args.vec4,
                                                                      wide_sell=args.wide_sell,
                                                                      pair_solve=args.pair_solve))
    for _ in range(args.steps):
        sim.step(w.dt, M_NODES, K_SWEEPS)
    sim.sync()
    out = {"workload": w.name, "nodes": int(w.n_nodes), "steps": args.steps, "vec4": args.vec4,
           "wide_sell": args.wide_sell, "pair_solve": args.pair_solve, "stats": sim.stats(),
           "amg": sim.amg_levels()}
    if args.profile_steps > 0:
        prof = sim.profile_steps(w.dt, M_NODES, K_SWEEPS, args.profile_steps)
        out["ms_per_step"] = round(sum(prof["ms"].values()) / args.profile_steps, 3)
        out["kernel_share"] = shares(prof)
        out["elliptic"] = solver_roofline(prof, "pcg_elliptic")
        out["parabolic"] = solver_roofline(prof, "pcg_parabolic")
    print(json.dumps(out))
    sim.close()


def _short_kernel_name(name: str) -> str:
    import re
    m = re.search(r"bd::\(anonymous namespace\)::(\w+)", name)
    if m:
        base = m.group(1)
        for tag in ("TP06", "LR91"):
            if tag in name:
                base += f"<{tag}" + (",float" if "float" in name else ",double")
                mode = re.search(r", \(int\)(\d)>", name) or re.search(r", (\d)>", name)
                if mode and base.startswith("ionic_kernel"):
                    base += f",mode{mode.group(1)}"
                base += ">"
                break
        return base
    if "at::" in name or "at_cuda" in name:
        return "torch:" + re.sub(r"<.*", "", name.split("at::")[-1])[:40]
    return name[:60]


def summarize_launches(path: str) -> None:
    """Markdown table of an ncu launch list: per kernel its launches, total
    device time and share of the listed time."""
    import csv
    from collections import defaultdict
    tot, cnt = defaultdict(float), defaultdict(int)
    with open(path) as fh:
        lines = [ln for ln in fh if ln.startswith('"')]
    scale = {"ns": 1e-3, "nsecond": 1e-3, "us": 1.0, "usecond": 1.0, "ms": 1e3, "msecond": 1e3}
    for row in csv.DictReader(lines):
        if row.get("Metric Name") != "gpu__time_duration.sum":
            continue
        k = _short_kernel_name(row["Kernel Name"])
        tot[k] += float(row["Metric Value"].replace(",", "")) * scale.get(row.get("Metric Unit", "ns"), 1e-3)
        cnt[k] += 1
    all_us = sum(tot.values())
    print("| kernel | launches | total us | share |")
    print("|---|---|---|---|")
    for k in sorted(tot, key=lambda x: -tot[x]):
        print(f"| `{k}` | {cnt[k]} | {tot[k]:.1f} | {100 * tot[k] / all_us:.2f}% |")
    print(f"| TOTAL | {sum(cnt.values())} | {all_us:.1f} | |")


def run_reference(args) -> None:
    """The oracle, as it stands, on the host cores: one single-threaded
    process per core on the bounded sample of the headline workload."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    ncores = os.cpu_count() or 1
    res = run_oracle_processes(ncores, args.warmup, args.steps, 0.0)
    val = round(res["value"], 3)
    line = {"impl": "reference", "metric": "node-steps/s", "value": val, "unit": "node-steps/s",
            "n_gpus": int(os.environ.get("WORLD_SIZE", "1")), "steps": res["steps"], "warmup": args.warmup,
            "ms_per_step": round(1e3 * res["seconds"] / res["steps"], 3), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD, "sample_nodes": res["nodes"], "model": "TP06 epicardial",
                       "dt_ms": DT, "sdc_nodes": M_NODES, "sweeps": K_SWEEPS, "processes": ncores},
            "cpu_baseline": {"value": val, "unit": "node-steps/s", "cores": ncores, "kind": "oracle",
                             "sample": sample_text(res)},
            "e2e": {"value": val, "unit": "node-steps/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--no-baseline", action="store_true")
    ap.add_argument("--dev-ms", type=float, default=330.0,
                    help="simulated time of the developed state the headline legs start from (ms)")
    ap.add_argument("--slab-steps", type=int, default=5,
                    help="timed steps of the 201x201x51 slab leg (0: skip)")
    ap.add_argument("--batch-requests", type=int, default=32,
                    help="requests of the batched-execution leg (0: skip)")
    ap.add_argument("--batch-steps", type=int, default=10, help="timed steps of the batched-execution leg")
    ap.add_argument("--serve-requests", type=int, default=64)
    ap.add_argument("--serve-ms", type=float, default=10.0)
    ap.add_argument("--serve-solo-nodes", type=int, default=50000,
                    help="serve leg, batched form: requests of at least this many nodes run alone (0: batch all)")
    ap.add_argument("--lv-steps", type=int, default=3,
                    help="timed steps of the 3-D LV-shell-in-bath leg (0: skip; mesh and set-up take ~1 min)")
    ap.add_argument("--lv-h", type=float, default=0.04, help="lattice spacing of the LV leg (cm)")
    ap.add_argument("--bath-steps", type=int, default=10,
                    help="timed steps of the 801^2 bidomain-bath leg (0: skip)")
    ap.add_argument("--profile-workload", choices=["sheet", "slab", "lv", "bath"],
                    help="step one workload --steps times for a profiler (no timing)")
    ap.add_argument("--side", type=int, default=SIDE,
                    help="--profile-workload: sheet side, or the slab's x/y nodes (z: (side-1)/4+1)")
    ap.add_argument("--precision", choices=["mixed", "fp64"], default="mixed")
    ap.add_argument("--vec4", type=int, default=0, choices=[-1, 0, 1],
                    help="--profile-workload: SELL-32/4 copy of the FP32 elliptic operator (bd_opts_t.vec4)")
    ap.add_argument("--wide-sell", type=int, default=0, choices=[-1, 0, 1],
                    help="--profile-workload: SELL-32 for AMG levels with long rows (bd_opts_t.wide_sell)")
    ap.add_argument("--pair-solve", type=int, default=0, choices=[-1, 0],
                    help="--profile-workload: a sweep's two elliptic solves as one (bd_opts_t.pair_solve)")
    ap.add_argument("--profile-steps", type=int, default=0,
                    help="--profile-workload: also time this many steps per kind (bd_profile_steps)")
    ap.add_argument("--streaming", type=int, default=0, choices=[-1, 0, 1, 2],
                    help="--profile-workload: solver form (bd_opts_t.streaming)")
    ap.add_argument("--summarize-launches", metavar="CSV", help="summarise an ncu launch list")
    ap.add_argument("--oracle-sample", action="store_true", help=argparse.SUPPRESS)
    ap.add_argument("--seconds", type=float, default=0.0, help=argparse.SUPPRESS)
    args = ap.parse_args()
    if args.summarize_launches:
        summarize_launches(args.summarize_launches)
        return
    if args.profile_workload:
        profile_workload(args)
        return
    if args.oracle_sample:
        import numpy as np
        np.seterr(all="ignore")
        print(json.dumps(oracle_rate(args.warmup, args.steps, args.seconds)))
        return
    if args.warmup < 3 and args.impl == "ours":
        ap.error("--warmup must be >= 3")
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
