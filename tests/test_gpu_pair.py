"""The two-system elliptic solve of the streaming form: from the second sweep
on, Algorithm 2 (Sec. 3.3.2) solves the elliptic constraint at two
Gauss-Lobatto nodes, and one chain of kernels serves both right-hand sides,
loading each operator entry once (bd_opts_t.pair_solve), in mixed precision
and in FP64.  Each system gets
what the single-system chain gives it, to the solver tolerance; whole steps
match the oracle on a slab and on a bidomain-bath sheet; the host-driven
loops give the same bits as the graph loops; the device-side sweep test
closes a pair's sweeps as it closes single solves; the profile counts a
shared operator pass once."""
import numpy as np
import pytest

from gpu_util import gpu_sim, oracle_problem, rel, rest_X
from oracle import bidomain as OB
from paper_2510_27447_gb300 import binding
from paper_2510_27447_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def _slab(n_steps=8):
    # 4,851 nodes: a smoothed-aggregation hierarchy with long-row coarse levels
    xyz, tets = W.slab_grid(21, 21, 11, 0.5, 0.5, 0.25)
    fib = W.fibers_transmural(xyz, tets, 0.0, 0.25, -60.0, 60.0)
    stim = [W.Stimulus(W.nodes_x_below(xyz, 0.05), 0.0, 1.0, W.STIM_AMP)]
    return W.Workload(name="slab_small", xyz=xyz, elems=tets, fibers=fib, sigma=W.CONFIG0_SIGMA, chi=2000.0,
                      cm=1.0, model=W.LR91, stimuli=stim, dt=0.02, n_steps=n_steps)


def _bath():
    # 1,681 nodes (tissue in the middle third): above the dense-solve limit,
    # so the elliptic system over tissue and bath gets an AMG hierarchy
    return W.bath_sheet(40, -0.25, 1.25, 0.0, 1.0, W.LR91_PAPER_MOD, 0.05, 8, strip=0.1, s1_amp=80.0,
                        s1_dur=1.0)


def _run(w, X0, steps, K=2, **opt):
    opt.setdefault("precision", binding.MIXED)
    sim = gpu_sim(w, streaming=opt.pop("streaming", 1), **opt)
    sim.set_initial(X0)
    for _ in range(steps):
        sim.step(w.dt, 3, K)
    f = sim.fields(full=True)
    st = sim.stats()
    sim.close()
    return f, st


@pytest.mark.parametrize("mesh", ["slab", "bath"])
def test_pair_solve_matches_single_solves_and_the_oracle(mesh):
    w = _slab() if mesh == "slab" else _bath()
    X0 = rest_X(w)
    (vp, up, Xp), sp = _run(w, X0, w.n_steps, cg_tol_e=1e-11)
    (vs, us, Xs), ss = _run(w, X0, w.n_steps, cg_tol_e=1e-11, pair_solve=-1)
    assert sp["streaming"] == 1 and sp["amg_levels"] >= 1
    # the same solves, one chain for each pair: fewer launches
    assert sp["cg_solves_e"] == ss["cg_solves_e"] > 0
    assert sp["kernel_launches"] < ss["kernel_launches"]
    assert abs(sp["cg_iters_e"] - ss["cg_iters_e"]) <= 0.05 * ss["cg_iters_e"]
    # the elliptic solutions agree to the FP64-refined tolerance; the FP32
    # parabolic solves (relative tolerance 1e-6) carry the difference on
    assert rel(up, us) < 1e-5 and rel(Xp, Xs) < 1e-5
    Xo, uo, _ = OB.run(oracle_problem(w), X0, w.n_steps, w.dt, 3, 2)
    assert Xp[0].max() > -75.0                   # the stimulus has depolarised its nodes (rest: -84.5 mV)
    assert rel(vp, Xo[0]) < 1e-3 and rel(up, uo) < 1e-3


@pytest.mark.parametrize("mesh", ["slab", "bath"])
def test_fp64_pair_solve_matches_single_solves_and_the_oracle(mesh):
    """The paper's precision: FP64 inner iterations on both systems."""
    w = _slab() if mesh == "slab" else _bath()
    X0 = rest_X(w)
    tight = dict(precision=binding.FP64, cg_tol_e=1e-13, cg_tol_p=1e-13)
    (vp, up, Xp), sp = _run(w, X0, w.n_steps, **tight)
    (vs, us, Xs), ss = _run(w, X0, w.n_steps, pair_solve=-1, **tight)
    assert sp["streaming"] == 1 and sp["amg_levels"] >= 1
    assert sp["cg_solves_e"] == ss["cg_solves_e"] > 0
    assert sp["kernel_launches"] < ss["kernel_launches"]
    assert rel(up, us) < 1e-9 and rel(Xp, Xs) < 1e-10
    Xo, uo, _ = OB.run(oracle_problem(w), X0, w.n_steps, w.dt, 3, 2)
    assert rel(Xp, Xo) < 1e-9 and rel(up, uo) < 1e-8


@pytest.mark.parametrize("prec", [binding.MIXED, binding.FP64])
def test_pair_host_driven_loops_give_the_same_bits_as_graph_loops(prec):
    """streaming = 2 launches the pair's kernels eagerly and reads both
    systems' decisions back on the host: the same bits as the conditional
    graph loops."""
    w = _slab(3)
    X0 = rest_X(w)
    out = [_run(w, X0, 3, streaming=form, precision=prec)[0] for form in (1, 2)]
    for a, b in zip(out[0], out[1]):
        assert np.array_equal(a, b)


def test_sweep_test_closes_pair_sweeps_on_the_device():
    """Up to six sweeps with the device-side sweep test: a pair skips its
    work once the test has closed the sweep, as two single solves do."""
    w = _slab(4)
    X0 = rest_X(w)
    (_, up, Xp), sp = _run(w, X0, 4, K=6, sweep_tol=1e-3, cg_tol_e=1e-11)
    (_, us, Xs), ss = _run(w, X0, 4, K=6, sweep_tol=1e-3, cg_tol_e=1e-11, pair_solve=-1)
    assert sp["sweeps"] == ss["sweeps"] < 4 * 6
    assert sp["cg_solves_e"] == ss["cg_solves_e"]
    assert rel(up, us) < 1e-5 and rel(Xp, Xs) < 1e-5


@pytest.mark.parametrize("prec", [binding.MIXED, binding.FP64])
def test_profile_counts_a_shared_operator_pass_once(prec):
    w = _slab(3)
    X0 = rest_X(w)
    prof = {}
    for pair in (0, -1):
        sim = gpu_sim(w, precision=prec, streaming=1, pair_solve=pair)
        sim.set_initial(X0)
        prof[pair] = sim.profile_steps(w.dt, 3, 2, 3)
        sim.close()
    p, q = prof[0], prof[-1]
    assert p["cg_solves"][0] == q["cg_solves"][0] > 0
    assert p["ms"]["pcg_elliptic"] > 0.0
    # the pair's algorithmic bytes drop by the shared operator passes only:
    # the vector streams of both systems remain
    assert 0.5 * q["alg_bytes"][0] < p["alg_bytes"][0] < q["alg_bytes"][0]
    assert 0.3 * q["vcycle_bytes"] < p["vcycle_bytes"] < q["vcycle_bytes"]
    assert p["coarse_bytes"] < q["coarse_bytes"]


def test_pair_solve_option_is_checked():
    w = _slab(1)
    with pytest.raises(binding.BdError):
        gpu_sim(w, precision=binding.MIXED, streaming=1, pair_solve=1)
