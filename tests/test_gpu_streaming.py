"""The streaming solver form (chains of full-occupancy kernels with the CG
loops on the device as CUDA-graph conditional nodes), forced on meshes small
enough for the oracle: the elliptic constraint (Eq. (3.15)) with AMG and
Jacobi preconditioning in FP64 and mixed precision, on a 2-D sheet, a 3-D
slab (coarse levels with long rows) and a bath mesh, and whole partitioned-SDC
steps (Algorithm 2) in graph replay and in eager launches, with the sweep test
of Algorithm 2 closing sweeps on the device."""
import numpy as np
import pytest

from gpu_util import gpu_sim, oracle_problem, rel, rest_X
from oracle import bidomain as OB
from paper_2510_27447_gb300 import binding
from paper_2510_27447_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def _bump(xyz, n):
    c = np.array([0.3, 0.6, 0.2][: xyz.shape[1]])
    return -80.0 + 100.0 * np.exp(-30.0 * np.sum((xyz[:n] - c) ** 2, axis=1))


def _slab():
    xyz, tets = W.slab_grid(21, 21, 11, 0.5, 0.5, 0.25)
    fib = W.fibers_transmural(xyz, tets, 0.0, 0.25, -60.0, 60.0)
    stim = [W.Stimulus(W.nodes_x_below(xyz, 0.05), 0.0, 1.0, W.STIM_AMP)]
    return W.Workload(name="slab_small", xyz=xyz, elems=tets, fibers=fib, sigma=W.CONFIG0_SIGMA, chi=2000.0,
                      cm=1.0, model=W.LR91, stimuli=stim, dt=0.02, n_steps=8)


@pytest.mark.parametrize("prec", [binding.FP64, binding.MIXED])
@pytest.mark.parametrize("precond", [0, 1])
@pytest.mark.parametrize("mesh", ["sheet", "slab", "bath"])
def test_streaming_elliptic_solve_matches_oracle(prec, precond, mesh):
    if mesh == "sheet":
        w = W.sheet(65, 1.0, W.LR91, 0.02, 1)
    elif mesh == "slab":
        w = _slab()
    else:
        w = W.bath_sheet(48, -0.25, 1.25, 0.0, 1.0, W.LR91_PAPER_MOD, 0.05, 1, strip=0.1, s1_amp=80.0,
                         s1_dur=1.0)
    v = _bump(w.xyz, w.n_tissue)
    u_ref = oracle_problem(w).elliptic(v)
    sim = gpu_sim(w, precision=prec, cg_tol_e=1e-11, elliptic_precond=precond, streaming=1)
    st = sim.stats()
    assert st["streaming"] == 1
    if precond:
        assert st["amg_levels"] >= 1
    for _ in range(2):                       # the second solve reuses every scalar and workspace
        u, it = sim.solve_elliptic(v)
        assert u[w.pin_node] == 0.0
        assert rel(u, u_ref) < 1e-8, (rel(u, u_ref), it)
        assert it > 0
    # a warm start from the answer converges at once
    u2, it2 = sim.solve_elliptic(v, u_guess=u)
    assert it2 <= 2 and rel(u2, u_ref) < 1e-8
    sim.close()


@pytest.mark.parametrize("graph", [1, 0])
def test_streaming_fp64_steps_match_oracle(graph):
    w = W.sheet(41, 0.4, W.LR91, 0.02, 10, strip=0.06)
    X0 = rest_X(w)
    Xo, uo, to = OB.run(oracle_problem(w), X0, w.n_steps, w.dt, 3, 2)
    sim = gpu_sim(w, cg_tol_e=1e-13, cg_tol_p=1e-13, streaming=1, use_graph=graph)
    sim.set_initial(X0)
    for _ in range(w.n_steps):
        sim.step(w.dt, 3, 2)
    v, u, X = sim.fields(full=True)
    ta = sim.activation_times()
    st = sim.stats()
    sim.close()
    assert st["streaming"] == 1 and st["amg_levels"] >= 1
    assert rel(X, Xo) < 1e-9
    assert rel(u, uo) < 1e-9
    act = ~np.isnan(to)
    np.testing.assert_array_equal(np.isnan(ta), ~act)
    np.testing.assert_allclose(ta[act], to[act], atol=1e-6)


def test_streaming_mixed_steps_on_a_slab_within_tolerance():
    w = _slab()
    X0 = rest_X(w)
    Xo, uo, _ = OB.run(oracle_problem(w), X0, w.n_steps, w.dt, 3, 2)
    sim = gpu_sim(w, precision=binding.MIXED, streaming=1)
    sim.set_initial(X0)
    for _ in range(w.n_steps):
        sim.step(w.dt, 3, 2)
    v, u, X = sim.fields(full=True)
    st = sim.stats()
    sim.close()
    assert st["streaming"] == 1 and st["amg_levels"] >= 1
    assert rel(v, Xo[0]) < 1e-3
    assert rel(u, uo) < 1e-3


def test_streaming_matches_persistent_and_counts_its_launches():
    """Same FP64 steps through both solver forms (same tolerance): the
    states agree to the solver tolerance, and the streaming form's launch
    counter grows with the iterations run on the device."""
    w = W.sheet(41, 0.4, W.TP06_EPI, 0.02, 6, strip=0.06)
    X0 = rest_X(w)
    out = {}
    for form in (-1, 1):
        sim = gpu_sim(w, cg_tol_e=1e-12, cg_tol_p=1e-12, streaming=form)
        sim.set_initial(X0)
        for _ in range(w.n_steps):
            sim.step(w.dt, 3, 2)
        out[form] = (sim.fields(full=True), sim.stats())
        sim.close()
    (v0, u0, X0s), s0 = out[-1]
    (v1, u1, X1s), s1 = out[1]
    assert s0["streaming"] == 0 and s1["streaming"] == 1
    assert rel(X1s, X0s) < 1e-9 and rel(u1, u0) < 1e-8
    # every CG iteration launches at least two kernels in the streaming form
    assert s1["kernel_launches"] > 2 * (s1["cg_iters_e"] + s1["cg_iters_p"]) > 0


def test_streaming_sweep_test_closes_sweeps_on_the_device():
    """Algorithm 2's stopping test with the solves in streaming form: a closed
    sweep gate turns the remaining sweeps' solves into no-ops on the device
    (the workload of the persistent form's sweep test)."""
    w = W.sheet(15, 0.3, W.LR91_PAPER_MOD, 0.05, 12, strip=0.05)
    X0 = rest_X(w)
    P = oracle_problem(w)
    X, u = X0.copy(), np.zeros(w.n_nodes)
    sweeps = 0
    for n in range(w.n_steps):
        X, u, k = P.step(X, u, n * w.dt, w.dt, 3, 6, True, sweep_tol=1e-3)
        sweeps += k
    sim = gpu_sim(w, cg_tol_e=1e-13, cg_tol_p=1e-13, streaming=1, sweep_tol=1e-3)
    sim.set_initial(X0)
    for _ in range(w.n_steps):
        sim.step(w.dt, 3, 6)
    _, ug, Xg = sim.fields(full=True)
    st = sim.stats()
    sim.close()
    assert w.n_steps < sweeps < 6 * w.n_steps
    assert st["sweeps"] == sweeps
    assert rel(Xg, X) < 1e-10 and rel(ug, u) < 1e-8


@pytest.mark.parametrize("form", [-1, 1])
def test_profiled_steps_time_every_kind_and_advance_like_steps(form):
    """bd_profile_steps replays each step as a graph with event nodes around
    every launch (or streaming solve): every kind gets device time, the solve
    counts match the counters, and the state advances as bd_step does."""
    w = W.sheet(33, 0.5, W.TP06_EPI, 0.02, 4, strip=0.1)
    X0 = rest_X(w)
    sims = [gpu_sim(w, precision=binding.MIXED, streaming=form) for _ in range(2)]
    for s in sims:
        s.set_initial(X0)
    for _ in range(w.n_steps):
        sims[0].step(w.dt, 3, 2)
    st0 = sims[1].stats()
    prof = sims[1].profile_steps(w.dt, 3, 2, w.n_steps)
    st1 = sims[1].stats()
    assert all(prof["ms"][k] > 0.0 for k in ("pcg_elliptic", "pcg_parabolic", "ionic", "field", "combine"))
    assert prof["cg_solves"][0] == st1["cg_solves_e"] - st0["cg_solves_e"] > 0
    assert prof["cg_iters"][1] == st1["cg_iters_p"] - st0["cg_iters_p"] > 0
    assert prof["alg_bytes"][0] > 0 and prof["alg_bytes"][1] > 0
    a = sims[0].fields(full=True)[2]
    b = sims[1].fields(full=True)[2]
    assert np.array_equal(a, b)          # same kernels, same order: bit for bit
    for s in sims:
        s.close()


def test_host_driven_loops_give_the_same_bits_as_graph_loops():
    """streaming = 2 runs the same kernels with the loop decisions read back
    by the host (a form profilers can capture launch by launch): the same
    bits as the device-side loops."""
    w = W.sheet(41, 0.4, W.TP06_EPI, 0.02, 5, strip=0.06)
    X0 = rest_X(w)
    out = []
    for form in (1, 2):
        sim = gpu_sim(w, precision=binding.MIXED, streaming=form)
        sim.set_initial(X0)
        for _ in range(w.n_steps):
            sim.step(w.dt, 3, 2)
        out.append(sim.fields(full=True))
        sim.close()
    for a, b in zip(out[0], out[1]):
        assert np.array_equal(a, b)


def test_vector_load_layout_gives_the_same_solves():
    """The SELL-32/4 copy of the FP32 elliptic operator (16-byte loads of
    four entries of a row) adds each row's entries in the SELL-32 order: the
    mixed steps on a slab agree with the plain layout and with the oracle."""
    w = _slab()
    X0 = rest_X(w)
    out = {}
    for v4 in (0, 1, -1):           # 1: the AMG level operators use the copy too, whatever their size
        sim = gpu_sim(w, precision=binding.MIXED, streaming=1, vec4=v4)
        sim.set_initial(X0)
        for _ in range(w.n_steps):
            sim.step(w.dt, 3, 2)
        out[v4] = sim.fields(full=True)
        sim.close()
    Xo, uo, _ = OB.run(oracle_problem(w), X0, w.n_steps, w.dt, 3, 2)
    v1, u1, _ = out[-1]
    for v4 in (0, 1):
        v0, u0, _ = out[v4]
        assert rel(v0, v1) < 1e-6 and rel(u0, u1) < 1e-6
        assert rel(v0, Xo[0]) < 1e-3 and rel(u0, uo) < 1e-3


@pytest.mark.parametrize("prec", [binding.FP64, binding.MIXED])
@pytest.mark.parametrize("form", [(0, 0), (1, 0), (-1, 4), (-1, 16), (-1, 32), (-1, 256)])
def test_every_coarse_level_row_form_solves_the_elliptic_system(prec, form):
    """The AMG levels of a 3-D slab have rows longer than 32 entries: stored
    as SELL-32 (wide_sell = 1, thread per row), by the size rule (0), or as
    CSR read by 4 to 32 lanes per row or a whole block per row (csr_lanes
    forced on every CSR level).  Every form gives the oracle's solution of
    Eq. (3.15)."""
    wide, lanes = form
    w = _slab()
    v = _bump(w.xyz, w.n_tissue)
    u_ref = oracle_problem(w).elliptic(v)
    sim = gpu_sim(w, precision=prec, cg_tol_e=1e-11, elliptic_precond=1, streaming=1, wide_sell=wide,
                  csr_lanes=lanes)
    st = sim.stats()
    assert st["amg_levels"] >= 1
    levels = sim.amg_levels()
    forms = [L[k][2] for L in levels for k in "ARP"]
    for lv, L in enumerate(levels):
        assert L["P"][0] == L["A"][0]                                   # P_l: fine rows
        nxt = levels[lv + 1]["A"][0] if lv + 1 < len(levels) else st["amg_coarse_rows"]
        assert L["R"][0] == nxt                                         # R_l: coarse rows
        assert min(L[k][1] for k in "ARP") > 0
    if wide == -1:
        assert -1 not in forms and any(f > 0 for f in forms)            # long rows are CSR here
    if wide == 1:
        assert -1 in forms
    if lanes:
        assert all(f == lanes for f in forms if f > 0)
    u, it = sim.solve_elliptic(v)
    sim.close()
    assert u[w.pin_node] == 0.0 and it > 0
    assert rel(u, u_ref) < 1e-8, (rel(u, u_ref), it)


def test_option_tuner_times_every_candidate_and_keeps_the_results():
    """The option tuner times each layout / thread-mapping candidate once per
    shape class and returns options whose steps agree with the default ones
    (the candidates change only summation order)."""
    from paper_2510_27447_gb300.batching import OptionTuner, option_candidates
    w = _slab()
    X0 = rest_X(w)
    w.initial = X0
    base = {"precision": binding.FP64, "streaming": 1, "pin_node": w.pin_node, "cg_tol_e": 1e-12,
            "cg_tol_p": 1e-12}
    tuner = OptionTuner(trial_steps=1)
    opts = tuner.tune(w, base, w.dt)
    assert len(tuner.timings) == 1
    (key, times), = tuner.timings.items()
    assert set(times) == set(option_candidates(True, binding.FP64))
    assert tuner.tune(w, base, w.dt) == opts and len(tuner.timings) == 1      # cached
    out = []
    for o in (base, opts):
        sim = gpu_sim(w, **o)
        sim.set_initial(X0)
        for _ in range(3):
            sim.step(w.dt, 3, 2)
        out.append(sim.fields(full=True))
        sim.close()
    assert rel(out[1][0], out[0][0]) < 1e-9 and rel(out[1][1], out[0][1]) < 1e-8


def _bath_small():
    # 625 nodes (289 tissue): the tissue rows' columns reach into the bath
    return W.bath_sheet(24, -0.25, 1.25, 0.0, 1.0, W.LR91_PAPER_MOD, 0.05, 12, strip=0.1, s1_amp=80.0,
                        s1_dur=1.0)


@pytest.mark.parametrize("prec", [binding.FP64, binding.MIXED])
def test_streaming_steps_on_a_bath_mesh_match_oracle(prec):
    """Whole steps of the streaming form on a bidomain-bath mesh (the path of
    the LV-shell leg): the parabolic solves over the tissue rows of the
    shared pattern, the elliptic solve over tissue and bath."""
    w = _bath_small()
    X0 = rest_X(w)
    Xo, uo, to = OB.run(oracle_problem(w), X0, w.n_steps, w.dt, 3, 2)
    tight = dict(cg_tol_e=1e-13, cg_tol_p=1e-13) if prec == binding.FP64 else {}
    sim = gpu_sim(w, precision=prec, streaming=1, **tight)
    sim.set_initial(X0)
    for _ in range(w.n_steps):
        sim.step(w.dt, 3, 2)
    v, u, X = sim.fields(full=True)
    ta = sim.activation_times()
    st = sim.stats()
    sim.close()
    assert st["streaming"] == 1 and X.shape == (8, w.n_tissue) and u.shape == (w.n_nodes,)
    assert X[0].max() > -20.0
    if prec == binding.FP64:
        assert rel(X, Xo) < 1e-9 and rel(u, uo) < 1e-8
        np.testing.assert_array_equal(np.isnan(ta), np.isnan(to))
        np.testing.assert_allclose(ta[~np.isnan(ta)], to[~np.isnan(to)], atol=1e-6)
    else:
        assert rel(v, Xo[0]) < 1e-3 and rel(u, uo) < 1e-3


def test_streaming_steps_on_the_lv_shell_in_a_bath_match_oracle():
    """The 3-D bidomain-bath geometry on a coarse lattice with the AMG
    hierarchy, TP06, streaming form, FP64 and mixed."""
    w = W.lv_shell_bath(h=0.35, n_steps=3)
    X0 = rest_X(w)
    Xo, uo, _ = OB.run(oracle_problem(w), X0, 3, w.dt, 3, 2)
    for prec, tx, tu in ((binding.FP64, 1e-9, 1e-8), (binding.MIXED, 1e-4, 1e-3)):
        tight = dict(cg_tol_e=1e-13, cg_tol_p=1e-13) if prec == binding.FP64 else {}
        sim = gpu_sim(w, precision=prec, streaming=1, **tight)
        sim.set_initial(X0)
        for _ in range(3):
            sim.step(w.dt)
        v, u, X = sim.fields(full=True)
        st = sim.stats()
        sim.close()
        assert st["streaming"] == 1 and st["amg_levels"] >= 1
        assert rel(X, Xo) < tx and rel(u, uo) < tu, prec
