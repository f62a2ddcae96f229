"""ctypes binding of the C ABI in include/bd.h (argument marshalling only).

Every computation happens in libbd.so.  If the library has not been built
the first call raises ``LibraryMissing``; there is no fallback.
"""
from __future__ import annotations

import ctypes as C
import os
from typing import Optional, Sequence

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "_lib", "libbd.so")

BD_OK = 0
ERRORS = {-1: "BD_ERR_ARG", -2: "BD_ERR_OOM", -3: "BD_ERR_CUDA", -4: "BD_ERR_NOT_CONVERGED",
          -5: "BD_ERR_NONFINITE", -6: "BD_ERR_INDEFINITE", -7: "BD_ERR_TIMEOUT"}
FP64, MIXED = 0, 1
LR91, LR91_PAPER_MOD, TP06_EPI = 0, 1, 2

EXPORTS = ["bd_default_options", "bd_create", "bd_add_stimulus", "bd_set_initial", "bd_step",
           "bd_batch_step", "bd_sync", "bd_clear_status", "bd_activation_times", "bd_get_fields",
           "bd_device_fields", "bd_get_state", "bd_set_state", "bd_footprint_bytes", "bd_get_stats",
           "bd_reset_stats", "bd_num_nodes", "bd_num_states", "bd_last_error", "bd_destroy",
           "bd_ionic_eval", "bd_ionic_pattern", "bd_rest_state", "bd_operator_csr",
           "bd_solve_elliptic", "bd_profile_steps", "bd_solve_elliptic_noalloc", "bd_query",
           "bd_step_adaptive", "bd_get_time", "bd_num_tissue_nodes", "bd_step_decoupled",
           "bd_selftest_wait_timeout", "bd_struct_sizes", "bd_amg_level"]


class LibraryMissing(RuntimeError):
    pass


class BdError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"{ERRORS.get(code, code)}: {msg}")
        self.code = code


class Mesh(C.Structure):
    _fields_ = [("dim", C.c_int), ("n_nodes", C.c_int64), ("n_elems", C.c_int64),
                ("xyz", C.POINTER(C.c_double)), ("elems", C.POINTER(C.c_int32)),
                ("fiber", C.POINTER(C.c_double)), ("elem_bath", C.POINTER(C.c_uint8))]


class Cond(C.Structure):
    _fields_ = [("sil", C.c_double), ("sit", C.c_double), ("sel", C.c_double),
                ("set", C.c_double), ("chi", C.c_double), ("cm", C.c_double), ("sbath", C.c_double)]


ALLOC_FN = C.CFUNCTYPE(C.c_void_p, C.c_size_t, C.c_void_p)
FREE_FN = C.CFUNCTYPE(None, C.c_void_p, C.c_void_p)


class Opts(C.Structure):
    _fields_ = [("precision", C.c_int), ("mass_lumped", C.c_int), ("pin_node", C.c_int),
                ("sdc_correction", C.c_int), ("cg_tol_e", C.c_double), ("cg_tol_p", C.c_double),
                ("cg_cap_e", C.c_int), ("cg_cap_p", C.c_int), ("sweep_tol", C.c_double),
                ("v_act_mV", C.c_double), ("spd_margin", C.c_double), ("use_graph", C.c_int),
                ("elliptic_precond", C.c_int), ("amg_coarse_max", C.c_int), ("cg_block", C.c_int),
                ("cg_grid", C.c_int),
                ("alloc", ALLOC_FN), ("free", FREE_FN), ("alloc_ctx", C.c_void_p),
                ("stream", C.c_void_p), ("cg_cluster", C.c_int), ("solver_tier", C.c_int),
                ("streaming", C.c_int), ("vec4", C.c_int), ("csr_lanes", C.c_int), ("wide_sell", C.c_int),
                ("pair_solve", C.c_int)]


class Stats(C.Structure):
    _fields_ = [(k, C.c_int64) for k in ("steps", "sweeps", "cg_iters_e", "cg_solves_e",
                                          "cg_iters_p", "cg_solves_p", "spd_clamps", "ionic_evals",
                                          "kernel_launches", "solver_block_bound", "solver_tier",
                                          "amg_levels", "amg_coarse_rows", "streaming")]


KERNEL_KINDS = ("pcg_elliptic", "pcg_parabolic", "ionic", "field", "combine", "finish")


class Profile(C.Structure):
    _fields_ = [("ms", C.c_double * 6), ("launches", C.c_int64 * 6), ("cg_iters", C.c_int64 * 2),
                ("cg_solves", C.c_int64 * 2), ("outer_iters", C.c_int64 * 2), ("nnz", C.c_int64),
                ("alg_bytes", C.c_double * 2), ("vcycle_bytes", C.c_double), ("coarse_bytes", C.c_double)]


_lib = None


def lib():
    """Load libbd.so once; raises LibraryMissing if it was not built."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise LibraryMissing(f"{LIB_PATH} not found: build it with paper_2510_27447_gb300.build.build()")
    L = C.CDLL(LIB_PATH)
    P = C.POINTER
    dp, ip, u8p = P(C.c_double), P(C.c_int32), P(C.c_uint8)
    sig = {
        "bd_default_options": (None, [P(Opts)]),
        "bd_create": (C.c_int, [P(Mesh), P(Cond), C.c_int, P(Opts), P(C.c_void_p)]),
        "bd_add_stimulus": (C.c_int, [C.c_void_p, u8p, C.c_double, C.c_double, C.c_double]),
        "bd_set_initial": (C.c_int, [C.c_void_p, dp, dp]),
        "bd_step": (C.c_int, [C.c_void_p, C.c_double, C.c_int, C.c_int]),
        "bd_step_decoupled": (C.c_int, [C.c_void_p, C.c_double]),
        "bd_selftest_wait_timeout": (C.c_int, [C.c_void_p]),
        "bd_batch_step": (C.c_int, [P(C.c_void_p), C.c_int, C.c_double, C.c_int, C.c_int]),
        "bd_sync": (C.c_int, [C.c_void_p]),
        "bd_query": (C.c_int, [C.c_void_p]),
        "bd_step_adaptive": (C.c_int, [C.c_void_p, C.c_double, C.c_double, C.c_int, C.c_int, dp, dp,
                                       P(C.c_int)]),
        "bd_get_time": (C.c_int, [C.c_void_p, dp, P(C.c_int64)]),
        "bd_clear_status": (None, [C.c_void_p]),
        "bd_activation_times": (C.c_int, [C.c_void_p, dp, C.c_int64]),
        "bd_get_fields": (C.c_int, [C.c_void_p, dp, dp, dp]),
        "bd_device_fields": (C.c_int, [C.c_void_p, P(C.c_void_p), P(C.c_void_p)]),
        "bd_get_state": (C.c_int, [C.c_void_p, C.c_void_p, P(C.c_size_t)]),
        "bd_set_state": (C.c_int, [C.c_void_p, C.c_void_p, C.c_size_t]),
        "bd_footprint_bytes": (C.c_size_t, [P(Mesh), C.c_int, P(Opts)]),
        "bd_get_stats": (C.c_int, [C.c_void_p, P(Stats)]),
        "bd_struct_sizes": (C.c_int, [P(C.c_size_t)] * 4),
        "bd_reset_stats": (C.c_int, [C.c_void_p]),
        "bd_num_nodes": (C.c_int64, [C.c_void_p]),
        "bd_num_tissue_nodes": (C.c_int64, [C.c_void_p]),
        "bd_num_states": (C.c_int, [C.c_int]),
        "bd_last_error": (C.c_char_p, [C.c_void_p]),
        "bd_destroy": (None, [C.c_void_p]),
        "bd_ionic_eval": (C.c_int, [C.c_int, C.c_int, C.c_int64, dp, dp, C.c_double, dp, dp]),
        "bd_ionic_pattern": (C.c_int, [C.c_int, P(C.c_uint32)]),
        "bd_rest_state": (C.c_int, [C.c_int, dp]),
        "bd_operator_csr": (C.c_int, [C.c_void_p, C.c_int, P(C.c_int64), ip, ip, dp]),
        "bd_solve_elliptic": (C.c_int, [C.c_void_p, dp, dp, dp, P(C.c_int)]),
        "bd_profile_steps": (C.c_int, [C.c_void_p, C.c_double, C.c_int, C.c_int, C.c_int, P(Profile)]),
        "bd_solve_elliptic_noalloc": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, P(C.c_int)]),
        "bd_amg_level": (C.c_int, [C.c_void_p, C.c_int, P(C.c_int64)]),
    }
    for name, (res, args) in sig.items():
        fn = getattr(L, name)
        fn.restype = res
        fn.argtypes = args
    _lib = L
    return L


def _dp(a: Optional[np.ndarray]):
    if a is None:
        return None
    return a.ctypes.data_as(C.POINTER(C.c_double))


def _check(rc: int, handle=None):
    if rc != BD_OK:
        msg = lib().bd_last_error(handle)
        raise BdError(rc, msg.decode() if msg else "")


def default_options(**kw) -> Opts:
    o = Opts()
    lib().bd_default_options(C.byref(o))
    for k, v in kw.items():
        if not hasattr(o, k):
            raise KeyError(k)
        setattr(o, k, v)
    return o


def num_states(model: int) -> int:
    return int(lib().bd_num_states(model))


def rest_state(model: int) -> np.ndarray:
    x = np.zeros(num_states(model))
    _check(lib().bd_rest_state(model, _dp(x)))
    return x


def ionic_pattern(model: int) -> np.ndarray:
    m = np.zeros(num_states(model), dtype=np.uint32)
    _check(lib().bd_ionic_pattern(model, m.ctypes.data_as(C.POINTER(C.c_uint32))))
    return m


def ionic_eval(model: int, X: np.ndarray, istim: Optional[np.ndarray] = None, cm: float = 1.0,
               precision: int = FP64, jacobian: bool = True):
    """Node field f (ns, n) and, optionally, node Jacobians (n, ns, ns)."""
    X = np.ascontiguousarray(X, dtype=np.float64)
    ns, n = X.shape
    f = np.empty((ns, n))
    J = np.empty((n, ns, ns)) if jacobian else None
    ist = None if istim is None else np.ascontiguousarray(istim, dtype=np.float64)
    _check(lib().bd_ionic_eval(model, precision, n, _dp(X), _dp(ist), cm, _dp(f), _dp(J)))
    return (f, J) if jacobian else f


def mesh_struct(xyz: np.ndarray, elems: np.ndarray, fibers: Optional[np.ndarray],
                elem_bath: Optional[np.ndarray] = None):
    xyz = np.ascontiguousarray(xyz, dtype=np.float64)
    elems = np.ascontiguousarray(elems, dtype=np.int32)
    fib = None if fibers is None else np.ascontiguousarray(fibers, dtype=np.float64)
    bath = None if elem_bath is None else np.ascontiguousarray(elem_bath, dtype=np.uint8)
    if bath is not None and bath.shape != (elems.shape[0],):
        raise ValueError("elem_bath must have one byte per element")
    m = Mesh(xyz.shape[1], xyz.shape[0], elems.shape[0], _dp(xyz),
             elems.ctypes.data_as(C.POINTER(C.c_int32)), _dp(fib),
             None if bath is None else bath.ctypes.data_as(C.POINTER(C.c_uint8)))
    return m, (xyz, elems, fib, bath)


def footprint_bytes(xyz, elems, model: int, opts: Optional[Opts] = None, elem_bath=None) -> int:
    m, keep = mesh_struct(xyz, elems, None, elem_bath)
    return int(lib().bd_footprint_bytes(C.byref(m), model, C.byref(opts) if opts else None))


class Simulation:
    """One bidomain handle (bd_state_t)."""

    def __init__(self, xyz, elems, fibers, sigma: Sequence[float], chi: float, cm: float,
                 model: int, opts: Optional[Opts] = None, stimuli=(), elem_bath=None,
                 sbath: float = 0.0):
        L = lib()
        m, self._keep = mesh_struct(xyz, elems, fibers, elem_bath)
        cond = Cond(*[float(x) for x in sigma], float(chi), float(cm), float(sbath))
        self.opts = opts if opts is not None else default_options()
        h = C.c_void_p()
        _check(L.bd_create(C.byref(m), C.byref(cond), model, C.byref(self.opts), C.byref(h)))
        self.h = h
        self.model = model
        self.N = int(L.bd_num_nodes(h))             # all nodes (u)
        self.NT = int(L.bd_num_tissue_nodes(h))     # tissue nodes (v, membrane state)
        self.ns = num_states(model)
        for s in stimuli:
            self.add_stimulus(s.mask, s.t_on, s.duration, s.amplitude)

    def close(self):
        if getattr(self, "h", None):
            lib().bd_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def add_stimulus(self, mask, t_on, duration, amplitude):
        mk = np.ascontiguousarray(mask, dtype=np.uint8)
        if mk.shape == (self.N,) and self.NT < self.N:
            if np.any(mk[self.NT:]):
                raise ValueError("a stimulus mask may only cover tissue nodes")
            mk = np.ascontiguousarray(mk[:self.NT])
        if mk.shape != (self.NT,):
            raise ValueError("mask must have one byte per (tissue) node")
        _check(lib().bd_add_stimulus(self.h, mk.ctypes.data_as(C.POINTER(C.c_uint8)),
                                     float(t_on), float(duration), float(amplitude)), self.h)

    def set_initial(self, X: np.ndarray, u: Optional[np.ndarray] = None):
        X = np.ascontiguousarray(X, dtype=np.float64)
        if X.shape != (self.ns, self.NT):
            raise ValueError(f"X must be ({self.ns}, {self.NT})")
        uu = None if u is None else np.ascontiguousarray(u, dtype=np.float64)
        _check(lib().bd_set_initial(self.h, _dp(X), _dp(uu)), self.h)

    def step(self, dt: float, n_sdc_nodes: int = 3, n_sweeps: int = 2):
        _check(lib().bd_step(self.h, float(dt), int(n_sdc_nodes), int(n_sweeps)), self.h)

    def sync(self):
        _check(lib().bd_sync(self.h), self.h)

    def step_decoupled(self, dt: float):
        """One CN-RK2 step (decoupled strategy, Strang splitting)."""
        _check(lib().bd_step_decoupled(self.h, float(dt)), self.h)

    def step_adaptive(self, dt_max: float, tol: float, n_sdc_nodes: int = 3, n_sweeps: int = 2):
        """One accepted adaptive step; returns (dt taken, error estimate, rejections)."""
        dt = C.c_double(0.0)
        err = C.c_double(0.0)
        rej = C.c_int(0)
        _check(lib().bd_step_adaptive(self.h, float(dt_max), float(tol), int(n_sdc_nodes), int(n_sweeps),
                                      C.byref(dt), C.byref(err), C.byref(rej)), self.h)
        return dt.value, err.value, rej.value

    def time(self):
        """(simulated time in ms, completed steps)."""
        t = C.c_double(0.0)
        n = C.c_int64(0)
        _check(lib().bd_get_time(self.h, C.byref(t), C.byref(n)), self.h)
        return t.value, n.value

    def ready(self) -> bool:
        """True when all enqueued steps have completed (never blocks)."""
        r = lib().bd_query(self.h)
        if r < 0:
            _check(r, self.h)
        return r == 1

    def clear_status(self):
        lib().bd_clear_status(self.h)

    def fields(self, full: bool = False):
        v = np.empty(self.NT)
        u = np.empty(self.N)
        X = np.empty((self.ns, self.NT)) if full else None
        _check(lib().bd_get_fields(self.h, _dp(v), _dp(u), _dp(X)), self.h)
        return (v, u, X) if full else (v, u)

    def activation_times(self) -> np.ndarray:
        out = np.empty(self.NT)
        _check(lib().bd_activation_times(self.h, _dp(out), self.NT), self.h)
        return out

    def get_state(self) -> bytes:
        n = C.c_size_t(0)
        _check(lib().bd_get_state(self.h, None, C.byref(n)), self.h)
        buf = C.create_string_buffer(n.value)
        _check(lib().bd_get_state(self.h, buf, C.byref(n)), self.h)
        return buf.raw

    def set_state(self, blob: bytes):
        buf = C.create_string_buffer(blob, len(blob))
        _check(lib().bd_set_state(self.h, buf, len(blob)), self.h)

    def amg_levels(self) -> list:
        """Per AMG level: {A, R, P: (rows, stored entries, form)}; form 0 SELL-32,
        -1 wide SELL-32, k > 0 CSR with k threads per row (bd_amg_level)."""
        out, buf = [], (C.c_int64 * 9)()
        L = lib()
        for level in range(self.stats()["amg_levels"]):
            _check(L.bd_amg_level(self.h, level, buf), self.h)
            v = list(buf)
            out.append({"A": tuple(v[0:3]), "R": tuple(v[3:6]), "P": tuple(v[6:9])})
        return out

    def stats(self) -> dict:
        s = Stats()
        _check(lib().bd_get_stats(self.h, C.byref(s)), self.h)
        return {k: int(getattr(s, k)) for k, _ in Stats._fields_}

    def profile_steps(self, dt: float, n_sdc_nodes: int, n_sweeps: int, n_steps: int) -> dict:
        p = Profile()
        _check(lib().bd_profile_steps(self.h, float(dt), int(n_sdc_nodes), int(n_sweeps),
                                      int(n_steps), C.byref(p)), self.h)
        return {"ms": dict(zip(KERNEL_KINDS, list(p.ms))),
                "launches": dict(zip(KERNEL_KINDS, [int(x) for x in p.launches])),
                "cg_iters": [int(p.cg_iters[0]), int(p.cg_iters[1])],
                "cg_solves": [int(p.cg_solves[0]), int(p.cg_solves[1])],
                "outer_iters": [int(p.outer_iters[0]), int(p.outer_iters[1])], "nnz": int(p.nnz),
                "alg_bytes": [float(p.alg_bytes[0]), float(p.alg_bytes[1])],
                "vcycle_bytes": float(p.vcycle_bytes), "coarse_bytes": float(p.coarse_bytes),
                "nodes": self.N, "tissue_nodes": self.NT}

    def reset_stats(self):
        _check(lib().bd_reset_stats(self.h), self.h)

    def nnz(self) -> int:
        """Stored entries of the shared operator pattern (of A_ie)."""
        n = C.c_int64(0)
        _check(lib().bd_operator_csr(self.h, 1, C.byref(n), None, None, None), self.h)
        return int(n.value)

    def operator(self, which: int):
        """(rowptr, col, val) of A_i (0), A_ie (1), M (2); M_L (3) as a vector."""
        nnz = C.c_int64(0)
        L = lib()
        _check(L.bd_operator_csr(self.h, which, C.byref(nnz), None, None, None), self.h)
        if which == 3:
            val = np.empty(self.N)
            _check(L.bd_operator_csr(self.h, 3, C.byref(nnz), None, None, _dp(val)), self.h)
            return val
        rp = np.empty(self.N + 1, dtype=np.int32)
        col = np.empty(nnz.value, dtype=np.int32)
        val = np.empty(nnz.value)
        ip = C.POINTER(C.c_int32)
        _check(L.bd_operator_csr(self.h, which, C.byref(nnz), rp.ctypes.data_as(ip),
                                 col.ctypes.data_as(ip), _dp(val)), self.h)
        return rp, col, val

    def solve_elliptic(self, v: np.ndarray, u_guess: Optional[np.ndarray] = None):
        v = np.ascontiguousarray(v, dtype=np.float64)
        g = None if u_guess is None else np.ascontiguousarray(u_guess, dtype=np.float64)
        u = np.empty(self.N)
        it = C.c_int(0)
        _check(lib().bd_solve_elliptic(self.h, _dp(v), _dp(g), _dp(u), C.byref(it)), self.h)
        return u, it.value


def batch_step(sims: Sequence[Simulation], dt: float, n_sdc_nodes: int = 3, n_sweeps: int = 2):
    arr = (C.c_void_p * len(sims))(*[s.h for s in sims])
    _check(lib().bd_batch_step(arr, len(sims), float(dt), int(n_sdc_nodes), int(n_sweeps)))


def simulation_from_workload(w, opts: Optional[Opts] = None) -> Simulation:
    """Handle for a paper_2510_27447_gb300.workloads.Workload."""
    o = opts if opts is not None else default_options(cg_tol_e=w.cg_tol, pin_node=w.pin_node)
    sim = Simulation(w.xyz, w.elems, w.fibers, w.sigma, w.chi, w.cm, w.model, o, w.stimuli,
                     elem_bath=getattr(w, "elem_bath", None), sbath=getattr(w, "sbath", 0.0))
    if w.initial is not None:
        sim.set_initial(w.initial)
    return sim
