"""bd_solve_elliptic_noalloc: the allocation-free elliptic solve.

Some callers cannot allocate GPU memory in the middle of their work -- they
run under an external memory budget or allocator, or in a latency-critical
loop where cudaMalloc/cudaFree (which can synchronise the whole device) is
not acceptable.  For them the library offers an elliptic solve whose CG
scratch lives in a fixed device array of the library.  These tests check that
it returns what the oracle's direct solve and the allocating
bd_solve_elliptic return, on two calls in a row (the scratch keeps the
previous call's contents); that a step whose device-side sweep test closed
the remaining sweeps does not turn it into a no-op; that it covers bath
nodes; that a mixed-precision AMG handle still gets the FP64 Jacobi answer;
and that meshes above its fixed size are refused.

The file is collected last so that a run stopping at the first failure has
run every other test before it.
"""
import ctypes

import numpy as np
import pytest

from gpu_util import gpu_sim, oracle_problem
from paper_2510_27447_gb300 import binding
from paper_2510_27447_gb300 import workloads as W

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def _noalloc(sim, v_dev, guess_dev, u_dev):
    it = ctypes.c_int(-1)
    rc = binding.lib().bd_solve_elliptic_noalloc(
        sim.h, ctypes.c_void_p(v_dev.data_ptr()),
        ctypes.c_void_p(guess_dev.data_ptr()) if guess_dev is not None else None,
        ctypes.c_void_p(u_dev.data_ptr()), ctypes.byref(it))
    if rc != 0:
        raise binding.BdError(rc, binding.lib().bd_last_error(sim.h).decode())
    return it.value


def _rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def _bump(xyz, n):
    x, y = xyz[:n, 0], xyz[:n, 1]
    return -80.0 + 100.0 * np.exp(-30.0 * ((x - 0.3) ** 2 + (y - 0.6) ** 2))


def _dev(a):
    return torch.tensor(np.ascontiguousarray(a), dtype=torch.float64, device="cuda")


def test_noalloc_solve_matches_oracle_and_allocating_solve_on_two_calls():
    w = W.sheet(65, 1.0, W.LR91, 0.02, 1)
    sim = gpu_sim(w, cg_tol_e=1e-13, elliptic_precond=0)
    v = _bump(w.xyz, w.n_nodes)
    u_orc = oracle_problem(w).elliptic(v)
    u_ref, it_ref = sim.solve_elliptic(v)
    v_dev = _dev(v)
    u_dev = torch.empty_like(v_dev)
    torch.cuda.synchronize()
    for _ in range(2):
        u_dev.fill_(float("nan"))
        torch.cuda.synchronize()
        it = _noalloc(sim, v_dev, None, u_dev)
        u = u_dev.cpu().numpy()
        assert np.all(np.isfinite(u))
        assert _rel(u, u_orc) < 1e-9          # the oracle's direct solve is the authority
        assert _rel(u, u_ref) < 1e-10
        assert u[0] == 0.0
        assert it == it_ref
    # warm start from the answer: converges at once to the same solution
    g_dev = _dev(u_ref)
    torch.cuda.synchronize()
    it = _noalloc(sim, v_dev, g_dev, u_dev)
    assert it <= 2 and _rel(u_dev.cpu().numpy(), u_orc) < 1e-9
    sim.close()


def test_noalloc_solve_after_a_step_whose_sweep_test_closed_the_gate():
    # a huge sweep_tol stops every step after its first sweep on the device,
    # leaving the sweep gate closed when the step ends
    w = W.sheet(33, 0.5, W.LR91, 0.02, 1)
    sim = gpu_sim(w, cg_tol_e=1e-13, cg_tol_p=1e-12, elliptic_precond=0, sweep_tol=1e6)
    sim.step(w.dt, 3, 2)
    sim.sync()
    assert sim.stats()["sweeps"] == 1
    v = _bump(w.xyz, w.n_nodes)
    u_orc = oracle_problem(w).elliptic(v)
    v_dev = _dev(v)
    u_dev = torch.full_like(v_dev, float("nan"))
    torch.cuda.synchronize()
    for _ in range(2):
        it = _noalloc(sim, v_dev, None, u_dev)
        assert it > 0
        assert _rel(u_dev.cpu().numpy(), u_orc) < 1e-9
    u_ref, _ = sim.solve_elliptic(v)
    assert _rel(u_dev.cpu().numpy(), u_ref) < 1e-10
    sim.close()


def test_noalloc_solve_on_a_bath_mesh():
    w = W.bath_sheet(24, -0.25, 1.25, 0.0, 1.0, W.LR91_PAPER_MOD, 0.05, 1, strip=0.1,
                     s1_amp=80.0, s1_dur=1.0)
    sim = gpu_sim(w, cg_tol_e=1e-12, elliptic_precond=0)
    assert sim.NT < sim.N
    v = _bump(w.xyz, w.n_tissue)
    u_orc = oracle_problem(w).elliptic(v)
    u_ref, _ = sim.solve_elliptic(v)
    # the bath entries of v are finite and multiplied by zero
    vfull = np.concatenate([v, np.full(w.n_nodes - w.n_tissue, 7.0)])
    v_dev = _dev(vfull)
    u_dev = torch.empty_like(v_dev)
    torch.cuda.synchronize()
    for _ in range(2):
        u_dev.fill_(float("nan"))
        torch.cuda.synchronize()
        _noalloc(sim, v_dev, None, u_dev)
        u = u_dev.cpu().numpy()
        assert u[w.pin_node] == 0.0
        assert _rel(u, u_orc) < 1e-9
        assert _rel(u, u_ref) < 1e-9
        assert np.ptp(u[w.n_tissue:]) > 1e-3 * np.ptp(u)
    sim.close()


def test_noalloc_solve_on_a_mixed_amg_handle_is_the_fp64_jacobi_solve():
    w = W.sheet(65, 1.0, W.TP06_EPI, 0.02, 1)
    sim = gpu_sim(w, precision=binding.MIXED, cg_tol_e=1e-12, elliptic_precond=1)
    st = sim.stats()
    assert st["amg_levels"] >= 1
    v = _bump(w.xyz, w.n_nodes)
    u_orc = oracle_problem(w).elliptic(v)
    v_dev = _dev(v)
    u_dev = torch.empty_like(v_dev)
    torch.cuda.synchronize()
    for _ in range(2):
        u_dev.fill_(float("nan"))
        torch.cuda.synchronize()
        _noalloc(sim, v_dev, None, u_dev)
        assert _rel(u_dev.cpu().numpy(), u_orc) < 1e-10
    sim.close()


def test_noalloc_refuses_meshes_above_its_fixed_size():
    n = 363                       # 131,769 nodes > BD_NOALLOC_MAX_NODES = 131,072
    w = W.sheet(n, 1.0, W.LR91, 0.02, 1)
    sim = binding.Simulation(w.xyz, w.elems, w.fibers, w.sigma, w.chi, w.cm, w.model)
    v_dev = torch.zeros(sim.N, dtype=torch.float64, device="cuda")
    u_dev = torch.zeros_like(v_dev)
    torch.cuda.synchronize()
    with pytest.raises(binding.BdError) as e:
        _noalloc(sim, v_dev, None, u_dev)
    assert e.value.code == -1
    sim.close()
