"""GPU parity of the building blocks against the FP64 oracle: membrane model
field and Jacobian (A4), assembled operators (A0), elliptic solve (A1-A2)."""
import numpy as np
import pytest
import scipy.sparse as sp

from gpu_util import gpu_sim, oracle_cell, oracle_problem, rel
from paper_2510_27447_gb300 import binding
from paper_2510_27447_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def _states(cell, n, seed):
    rng = np.random.default_rng(seed)
    x0 = cell.initial()
    X = np.repeat(x0[:, None], n, axis=1)
    X[0] = rng.uniform(-90.0, 45.0, n)
    for r in cell.gate_rows:
        X[r] = rng.uniform(0.01, 0.99, n)
    for r in range(1 + len(cell.gate_rows), cell.ns):
        X[r] = x0[r] * rng.uniform(0.7, 1.3, n)
    # include the switch points and removable singularities exactly
    X[0, :6] = [-40.0, -47.13, -77.0, 15.0, -100.0, 0.0]
    return X


@pytest.mark.parametrize("model", [W.LR91, W.LR91_PAPER_MOD, W.TP06_EPI])
def test_ionic_field_and_jacobian_fp64(model):
    cell = oracle_cell(model)
    X = _states(cell, 1000, 1)           # 1000 nodes: several blocks and a ragged tail
    ist = np.where(np.arange(1000) % 3 == 0, 80.0, 0.0)
    f, J = binding.ionic_eval(model, X, ist)
    fo = cell.field(X, ist).real
    Jo = np.transpose(cell.jacobian(X, ist), (2, 0, 1))
    scale = np.abs(fo).max(axis=1, keepdims=True) + 1e-300
    assert np.max(np.abs(f - fo) / scale) < 1e-12
    jscale = np.abs(Jo).max(axis=2, keepdims=True) + 1e-300
    assert np.max(np.abs(J - Jo) / jscale) < 1e-10


@pytest.mark.parametrize("model", [W.LR91, W.TP06_EPI])
def test_ionic_field_fp32_mixed(model):
    cell = oracle_cell(model)
    X = _states(cell, 512, 2)
    f = binding.ionic_eval(model, X, None, precision=binding.MIXED, jacobian=False)
    fo = cell.field(X, np.zeros(512)).real
    scale = np.abs(fo).max(axis=1, keepdims=True) + 1e-300
    assert np.max(np.abs(f - fo) / scale) < 2e-4


@pytest.mark.parametrize("dim", [2, 3])
def test_assembled_operators_match_oracle(dim):
    if dim == 2:
        w = W.sheet(23, 1.3, W.LR91, 0.02, 1)
    else:
        xyz, tets = W.slab_grid(9, 7, 5, 1.0, 0.8, 0.4)
        fib = W.fibers_transmural(xyz, tets, 0.0, 0.4, -60, 60)
        w = W.Workload("slab", xyz, tets, fib, W.CONFIG0_SIGMA, 2000.0, 1.0, W.TP06_EPI, [], 0.025, 1)
    sim = gpu_sim(w)
    ops = oracle_problem(w).ops
    for which, ref in ((0, ops.A_i), (1, ops.A_ie), (2, ops.M)):
        rp, col, val = sim.operator(which)
        A = sp.csr_matrix((val, col, rp), shape=ref.shape)
        ref = ref.tocsr()
        ref.sort_indices()
        np.testing.assert_array_equal(A.indptr, ref.indptr)
        np.testing.assert_array_equal(A.indices, ref.indices)
        np.testing.assert_allclose(A.data, ref.data, rtol=1e-13, atol=1e-15 * np.abs(ref.data).max())
    np.testing.assert_allclose(sim.operator(3), ops.M_L, rtol=1e-14)
    sim.close()


@pytest.mark.parametrize("pin", [0, 37, -1])
def test_elliptic_solve_matches_direct_solve(pin):
    w = W.sheet(33, 1.0, W.LR91, 0.02, 1)
    sim = gpu_sim(w, cg_tol_e=1e-13, pin_node=pin)
    P = oracle_problem(w, pin=pin)
    xyz = w.xyz
    v = -80 + 100 * np.exp(-30 * ((xyz[:, 0] - 0.3) ** 2 + (xyz[:, 1] - 0.6) ** 2))
    u_ref = P.elliptic(v)
    u, it = sim.solve_elliptic(v)
    assert it > 10
    assert rel(u, u_ref) < 1e-10
    if pin >= 0:
        assert u[pin] == 0.0
    else:
        assert abs(u.mean()) < 1e-12 * np.abs(u).max()
    # warm start from the answer converges at once to the same solution
    u2, it2 = sim.solve_elliptic(v, u_guess=u)
    assert it2 <= 2 and rel(u2, u_ref) < 1e-10
    sim.close()


def test_equal_anisotropy_closed_form_on_gpu():
    lam = 0.6
    w = W.sheet(41, 1.0, W.LR91, 0.02, 1, sigma=(3.0, 0.31, lam * 3.0, lam * 0.31))
    sim = gpu_sim(w, cg_tol_e=1e-13, pin_node=5)
    v = np.random.default_rng(0).uniform(-90, 30, w.n_nodes)
    u, _ = sim.solve_elliptic(v)
    want = -v / (1 + lam)
    want -= want[5]
    np.testing.assert_allclose(u, want, atol=1e-9)
    sim.close()


@pytest.mark.parametrize("side", [65, 129])
def test_amg_preconditioned_elliptic_solve(side):
    """The AMG-preconditioned CG (the paper's elliptic preconditioner class)
    reaches the same solution as the direct solve and as Jacobi-PCG, with an
    iteration count that does not grow with the mesh."""
    w = W.sheet(side, 1.0, W.LR91, 0.02, 1)
    xyz = w.xyz
    v = -80 + 100 * np.exp(-30 * ((xyz[:, 0] - 0.3) ** 2 + (xyz[:, 1] - 0.6) ** 2))
    u_ref = oracle_problem(w).elliptic(v)
    sim_a = gpu_sim(w, cg_tol_e=1e-13, elliptic_precond=1)
    sim_j = gpu_sim(w, cg_tol_e=1e-13, elliptic_precond=0)
    ua, ita = sim_a.solve_elliptic(v)
    uj, itj = sim_j.solve_elliptic(v)
    assert rel(ua, u_ref) < 1e-10 and rel(uj, u_ref) < 1e-10
    assert ita < 45 and ita * 8 < itj
    sim_a.close()
    sim_j.close()
