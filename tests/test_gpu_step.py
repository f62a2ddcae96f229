"""GPU parity of whole partitioned-SDC steps (Algorithm 2; rows A1-A10)
against the FP64 oracle, plus handle behaviour."""
import numpy as np
import pytest

from gpu_util import gpu_sim, oracle_problem, rel, rest_X
from oracle import bidomain as OB
from paper_2510_27447_gb300 import binding
from paper_2510_27447_gb300 import workloads as W

pytestmark = pytest.mark.gpu

TIGHT = dict(cg_tol_e=1e-13, cg_tol_p=1e-13)


def _run_both(w, steps, M=3, K=2, correction=True, lumped=False, **opt):
    X0 = rest_X(w)
    P = oracle_problem(w, mass_lumped=lumped)
    Xo, uo, to = OB.run(P, X0, steps, w.dt, M, K, correction)
    sim = gpu_sim(w, sdc_correction=int(correction), mass_lumped=int(lumped), **TIGHT, **opt)
    sim.set_initial(X0)
    for _ in range(steps):
        sim.step(w.dt, M, K)
    v, u, X = sim.fields(full=True)
    ta = sim.activation_times()
    st = sim.stats()
    sim.close()
    return (X, u, ta, st), (Xo, uo, to)


@pytest.mark.parametrize("M,K,corr", [(3, 2, True), (2, 2, True), (2, 1, False), (3, 3, True)])
def test_lr91_sheet_matches_oracle(M, K, corr):
    # 17 x 17 = 289 nodes: two CUDA blocks of the node kernels, ragged tail
    w = W.sheet(17, 0.4, W.LR91, 0.02, 30, strip=0.06)
    (X, u, ta, st), (Xo, uo, to) = _run_both(w, 30, M, K, corr)
    assert rel(X, Xo) < 1e-10
    assert rel(u, uo) < 1e-8
    assert X[0].max() > -20.0                     # the strip has depolarised
    np.testing.assert_array_equal(np.isnan(ta), np.isnan(to))
    np.testing.assert_allclose(ta[~np.isnan(ta)], to[~np.isnan(to)], atol=1e-9)
    assert st["cg_solves_p"] == 30 * K * (2 * (M - 1) + ((M - 1) if corr else 0))


def test_lr91_paper_params_lumped_mass():
    w = W.sheet(15, 0.3, W.LR91_PAPER_MOD, 0.05, 12, strip=0.05)
    (X, u, _, _), (Xo, uo, _) = _run_both(w, 12, 3, 2, True, lumped=True)
    assert rel(X, Xo) < 1e-10 and rel(u, uo) < 1e-8


def test_tp06_sheet_matches_oracle():
    w = W.sheet(11, 0.2, W.TP06_EPI, 0.02, 15, strip=0.04)
    (X, u, _, _), (Xo, uo, _) = _run_both(w, 15, 3, 2, True)
    assert rel(X, Xo) < 1e-10
    assert rel(u, uo) < 1e-8
    for r in range(14, 19):          # concentrations, each row separately
        assert rel(X[r], Xo[r]) < 1e-10


def test_tp06_slab_3d_matches_oracle():
    xyz, tets = W.slab_grid(7, 6, 4, 0.3, 0.25, 0.15)
    fib = W.fibers_transmural(xyz, tets, 0.0, 0.15, -60, 60)
    stim = [W.Stimulus(W.nodes_x_below(xyz, 0.06), 0.0, 1.0, 80.0)]
    w = W.Workload("slab", xyz, tets, fib, W.CONFIG0_SIGMA, 2000.0, 1.0, W.TP06_EPI, stim, 0.025, 8)
    (X, u, _, _), (Xo, uo, _) = _run_both(w, 8, 3, 2, True)
    assert rel(X, Xo) < 1e-10 and rel(u, uo) < 1e-8


def test_rest_state_is_fixed_point_on_gpu():
    w = W.sheet(9, 0.3, W.LR91, 0.02, 5)
    w.stimuli = []
    sim = gpu_sim(w, **TIGHT)
    X0 = rest_X(w)
    sim.set_initial(X0)
    for _ in range(5):
        sim.step(w.dt)
    v, u, X = sim.fields(full=True)
    np.testing.assert_allclose(X, X0, rtol=1e-12, atol=1e-15)
    assert np.max(np.abs(u)) < 1e-10
    sim.close()


def _gpu_run(w, steps, **opt):
    sim = gpu_sim(w, **opt)
    for _ in range(steps):
        sim.step(w.dt)
    out = sim.fields(full=True)
    sim.close()
    return out


def test_graph_replay_and_eager_are_bit_identical_and_deterministic():
    w = W.sheet(21, 0.5, W.LR91, 0.02, 10, strip=0.06)
    a = _gpu_run(w, 10, use_graph=1)
    b = _gpu_run(w, 10, use_graph=0)
    c = _gpu_run(w, 10, use_graph=1)
    for x, y, z in zip(a, b, c):
        np.testing.assert_array_equal(x, y)
        np.testing.assert_array_equal(x, z)


def test_checkpoint_resume_is_bitwise():
    w = W.sheet(13, 0.3, W.LR91, 0.02, 10, strip=0.05)
    sim = gpu_sim(w)
    for _ in range(4):
        sim.step(w.dt)
    blob = sim.get_state()
    for _ in range(4):
        sim.step(w.dt)
    first = sim.fields(full=True)
    t1 = sim.activation_times()
    sim.set_state(blob)
    for _ in range(4):
        sim.step(w.dt)
    second = sim.fields(full=True)
    np.testing.assert_array_equal(first[2], second[2])
    np.testing.assert_array_equal(first[1], second[1])
    np.testing.assert_array_equal(np.isnan(t1), np.isnan(sim.activation_times()))
    sim.close()


def test_invalid_inputs_and_iteration_cap_are_reported():
    w = W.sheet(9, 0.3, W.LR91, 0.02, 2)
    sim = gpu_sim(w)
    X = rest_X(w)
    X[0, 3] = np.nan
    with pytest.raises(binding.BdError) as e:
        sim.set_initial(X)
    assert e.value.code == -1
    with pytest.raises(binding.BdError):
        sim.step(-1.0)
    with pytest.raises(binding.BdError):
        sim.step(0.02, 4, 2)
    sim.close()
    # an iteration cap of one parabolic CG iteration is reported as not converged
    sim = gpu_sim(w, cg_cap_p=1, cg_tol_p=1e-14)
    sim.step(w.dt)
    with pytest.raises(binding.BdError) as e:
        sim.sync()
    assert e.value.code == -4
    sim.clear_status()
    sim.sync()
    sim.close()


def test_sweep_tolerance_matches_oracle():
    """Algorithm 2's stopping test ||X^k - X^(k-1)|| < tol (max norm, last
    Lobatto node), decided on the device: same sweep counts and states as the
    oracle with the same tolerance."""
    w = W.sheet(15, 0.3, W.LR91_PAPER_MOD, 0.05, 12, strip=0.05)
    X0 = rest_X(w)
    P = oracle_problem(w)
    X, u = X0.copy(), np.zeros(w.n_nodes)
    sweeps = 0
    for n in range(12):
        X, u, k = P.step(X, u, n * w.dt, w.dt, 3, 6, True, sweep_tol=1e-3)
        sweeps += k
    sim = gpu_sim(w, sweep_tol=1e-3, **TIGHT)
    sim.set_initial(X0)
    for _ in range(12):
        sim.step(w.dt, 3, 6)
    v, ug, Xg = sim.fields(full=True)
    st = sim.stats()
    sim.close()
    assert 12 < sweeps < 72                 # the test stopped some, not all, steps early
    assert st["sweeps"] == sweeps
    assert rel(Xg, X) < 1e-10 and rel(ug, u) < 1e-8


@pytest.mark.parametrize("cluster", [0, 8, 16])
def test_solver_launch_modes_match_oracle(cluster):
    """The persistent CG kernels as a cooperative grid (device-wide barriers)
    or as one thread-block cluster (hardware cluster barriers): same
    solutions within the solver tolerance."""
    w = W.sheet(17, 0.4, W.LR91, 0.02, 10, strip=0.06)
    (X, u, ta, st), (Xo, uo, to) = _run_both(w, 10, 3, 2, True, cg_cluster=cluster)
    assert rel(X, Xo) < 1e-10 and rel(u, uo) < 1e-8
    for prec in (binding.FP64, binding.MIXED):
        sim = gpu_sim(w, precision=prec, cg_cluster=cluster, cg_tol_e=1e-12)
        v = -80 + 100 * np.exp(-30 * ((w.xyz[:, 0] - 0.1) ** 2 + (w.xyz[:, 1] - 0.3) ** 2))
        u1, _ = sim.solve_elliptic(v)
        sim.close()
        assert rel(u1, oracle_problem(w).elliptic(v)) < 1e-9


def test_device_barrier_wait_is_bounded():
    """A device-wide barrier whose partner block never arrives gives up after
    its bound (about two seconds of device time), reports BD_ERR_TIMEOUT, and
    leaves the handle usable."""
    import time
    w = W.sheet(9, 0.2, W.LR91, 0.02, 3, strip=0.05)
    sim = gpu_sim(w)
    t0 = time.perf_counter()
    rc = binding.lib().bd_selftest_wait_timeout(sim.h)
    el = time.perf_counter() - t0
    assert rc == -7 and 1.0 < el < 30.0, (rc, el)
    for _ in range(3):
        sim.step(w.dt)
    v, u = sim.fields()
    sim.close()
    assert np.all(np.isfinite(v)) and np.all(np.isfinite(u))


@pytest.mark.parametrize("cg_block,coarse_max,force,tier", [(512, 0, 0, 1), (1024, 0, 0, 0), (512, 3000, 0, 1),
                                                             (512, 0, 1, 0), (512, 0, 3, 2)])
def test_amg_solver_builds_match_oracle(cg_block, coarse_max, force, tier):
    """The AMG-preconditioned elliptic CG in every register build of the
    solver kernels (tier 0: 1024-thread launch bound; tier 1: 512-thread
    bound, chosen when the rows fit one block per SM; tier 2: the mixed AMG
    kernels at two 1024-thread blocks per SM, chosen for meshes of a million
    rows and forced here) and with a dense coarse level too wide for the
    shared-memory staging of its right-hand side (2,827 rows): FP64 and mixed
    solutions within the solver tolerance of the oracle's direct solve.  The
    handle's counters show which build and hierarchy ran; the coarse levels
    use several lanes per row here."""
    w = W.sheet(129, 1.25, W.LR91, 0.02, 1)
    v = -80 + 100 * np.exp(-30 * ((w.xyz[:, 0] - 0.4) ** 2 + (w.xyz[:, 1] - 0.7) ** 2))
    ref = oracle_problem(w).elliptic(v)
    for prec in (binding.FP64, binding.MIXED):
        sim = gpu_sim(w, precision=prec, cg_block=cg_block, amg_coarse_max=coarse_max, cg_tol_e=1e-11,
                      solver_tier=force)
        st = sim.stats()
        want = 0 if (tier == 2 and prec == binding.FP64) else tier    # tier 2 differs only in mixed AMG kernels
        assert st["solver_tier"] == want and st["amg_levels"] >= 1, st
        assert st["solver_block_bound"] == (512 if want == 1 else 1024), st
        if coarse_max:
            assert st["amg_coarse_rows"] > 1536, st
        u, it = sim.solve_elliptic(v)
        sim.close()
        assert 0 < it < 200 and rel(u, ref) < 1e-9, (prec, it, rel(u, ref))


def test_solver_tier_option_is_checked():
    """solver_tier outside 0..3, or the 512-thread tier with 1024-thread
    blocks, is refused with BD_ERR_ARG before any solve."""
    w = W.sheet(9, 0.2, W.LR91, 0.02, 3, strip=0.05)
    for opt in (dict(solver_tier=4), dict(solver_tier=-1), dict(solver_tier=2, cg_block=1024)):
        with pytest.raises(binding.BdError) as e:
            gpu_sim(w, **opt)
        assert binding.ERRORS[e.value.code] == "BD_ERR_ARG", e.value
