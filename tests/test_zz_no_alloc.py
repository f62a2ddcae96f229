"""bd_solve_elliptic_noalloc: the allocation-free elliptic solve.

Some callers cannot allocate GPU memory in the middle of their work -- they
run under an external memory budget or allocator, or in a latency-critical
loop where cudaMalloc/cudaFree (which can synchronise the whole device) is
not acceptable.  For them the library offers an elliptic solve whose CG
scratch lives in a fixed device array of the library.  These tests check that
it returns what the allocating bd_solve_elliptic returns, on two calls in a
row (the scratch keeps the previous call's contents), and that meshes above
its fixed size are refused.
"""
import ctypes

import numpy as np
import pytest

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


def test_noalloc_solve_matches_allocating_solve_on_two_calls():
    w = W.sheet(65, 1.0, W.LR91, 0.02, 1)
    sim = binding.Simulation(w.xyz, w.elems, w.fibers, w.sigma, w.chi, w.cm, w.model,
                             binding.default_options(cg_tol_e=1e-13, elliptic_precond=0))
    xyz = w.xyz
    v = -80.0 + 100.0 * np.exp(-30.0 * ((xyz[:, 0] - 0.3) ** 2 + (xyz[:, 1] - 0.6) ** 2))
    u_ref, it_ref = sim.solve_elliptic(v)
    v_dev = torch.tensor(v, dtype=torch.float64, device="cuda")
    u_dev = torch.empty_like(v_dev)
    torch.cuda.synchronize()
    for _ in range(2):
        u_dev.fill_(float("nan"))
        torch.cuda.synchronize()
        it = _noalloc(sim, v_dev, None, u_dev)
        u = u_dev.cpu().numpy()
        assert np.all(np.isfinite(u))
        assert _rel(u, u_ref) < 1e-10
        assert u[0] == 0.0
        assert it == it_ref
    # warm start from the answer: converges at once to the same solution
    g_dev = torch.tensor(u_ref, dtype=torch.float64, device="cuda")
    torch.cuda.synchronize()
    it = _noalloc(sim, v_dev, g_dev, u_dev)
    assert it <= 2 and _rel(u_dev.cpu().numpy(), u_ref) < 1e-10
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
