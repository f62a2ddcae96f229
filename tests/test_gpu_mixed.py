"""Mixed-precision path (FP32 membrane model and Krylov iterations, FP64
iterative refinement of the elliptic solve, FP64 state): error against the
FP64 oracle within the stated tolerances -- relative L2 of v and u <= 1e-3,
activation times within 0.1 ms, conduction velocity within 1 %."""
import os

import numpy as np
import pytest

from gpu_util import gpu_sim, oracle_problem, rel, rest_X
from oracle import bidomain as OB
from paper_2510_27447_gb300 import binding
from paper_2510_27447_gb300 import workloads as W

pytestmark = pytest.mark.gpu

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "config0_10ms.npz")


@pytest.mark.parametrize("precond", [0, 1])
def test_mixed_elliptic_refinement_reaches_fp64_accuracy(precond):
    w = W.sheet(129, 1.0, W.LR91, 0.02, 1)
    xyz = w.xyz
    v = -80 + 100 * np.exp(-30 * ((xyz[:, 0] - 0.3) ** 2 + (xyz[:, 1] - 0.6) ** 2))
    u_ref = oracle_problem(w).elliptic(v)
    sim = gpu_sim(w, precision=binding.MIXED, cg_tol_e=1e-12, elliptic_precond=precond)
    u, it = sim.solve_elliptic(v)
    assert rel(u, u_ref) < 1e-9
    sim.close()


@pytest.mark.parametrize("model,side,steps", [(W.LR91, 17, 30), (W.TP06_EPI, 11, 15)])
def test_mixed_step_within_tolerance(model, side, steps):
    w = W.sheet(side, 0.04 * (side - 1) / 2, model, 0.02, steps, strip=0.06)
    X0 = rest_X(w)
    Xo, uo, _ = OB.run(oracle_problem(w), X0, steps, w.dt, 3, 2)
    sim = gpu_sim(w, precision=binding.MIXED)
    sim.set_initial(X0)
    for _ in range(steps):
        sim.step(w.dt)
    v, u, X = sim.fields(full=True)
    sim.close()
    assert rel(v, Xo[0]) < 1e-3
    assert rel(u, uo) < 1e-3


def test_mixed_config0_meets_stated_tolerances():
    ref = np.load(GOLDEN)
    w = W.config0()
    sim = binding.simulation_from_workload(w, binding.default_options(precision=binding.MIXED, pin_node=0))
    sim.set_initial(ref["X0"])
    for _ in range(w.n_steps):
        sim.step(w.dt, w.n_sdc_nodes, w.n_sweeps)
    v, u = sim.fields()
    ta = sim.activation_times()
    sim.close()
    assert rel(v, ref["X"][0]) < 1e-3
    assert rel(u, ref["u"]) < 1e-3
    act = ~np.isnan(ref["t_act"])
    np.testing.assert_array_equal(np.isnan(ta), ~act)
    assert np.max(np.abs(ta[act] - ref["t_act"][act])) < 0.1
    cv = OB.conduction_velocity(w.xyz, ta, 0.5, 0.3)
    cv_ref = OB.conduction_velocity(w.xyz, ref["t_act"], 0.5, 0.3)
    assert abs(cv - cv_ref) / cv_ref < 0.01


@pytest.mark.parametrize("force,tier", [(0, 1), (1, 0), (3, 2)])
def test_mixed_amg_steps_in_every_solver_tier(force, tier):
    """Mixed steps on a mesh with an AMG hierarchy (the sweep-2 elliptic pair
    runs in the two-RHS kernel) in each register tier, forced where the mesh
    would not pick it: within the mixed tolerance of the FP64 oracle."""
    w = W.sheet(41, 0.4, W.LR91, 0.02, 10, strip=0.06)
    X0 = rest_X(w)
    Xo, uo, _ = OB.run(oracle_problem(w), X0, w.n_steps, w.dt, 3, 2)
    sim = gpu_sim(w, precision=binding.MIXED, solver_tier=force)
    st = sim.stats()
    assert st["solver_tier"] == tier and st["amg_levels"] >= 1, st
    sim.set_initial(X0)
    for _ in range(w.n_steps):
        sim.step(w.dt)
    v, u, X = sim.fields(full=True)
    sim.close()
    assert rel(v, Xo[0]) < 1e-3 and rel(u, uo) < 1e-3
