"""Decoupled CN-RK2 strategy on the GPU (Sec. 3.3.3) against the FP64
oracle: Strang splitting of the node reaction (explicit midpoint half steps)
and the Crank-Nicolson diffusion, elliptic constraint last."""
import numpy as np
import pytest

from gpu_util import gpu_sim, oracle_problem, rel, rest_X
from oracle import decoupled as D
from paper_2510_27447_gb300 import binding
from paper_2510_27447_gb300 import workloads as W

pytestmark = pytest.mark.gpu

TIGHT = dict(cg_tol_e=1e-13, cg_tol_p=1e-13)


def _run_both(w, steps, dt, **opt):
    X0 = rest_X(w)
    Xo, uo, to = D.run_cnrk2(oracle_problem(w), X0, steps, dt)
    sim = gpu_sim(w, **opt)
    sim.set_initial(X0)
    for _ in range(steps):
        sim.step_decoupled(dt)
    v, u, X = sim.fields(full=True)
    ta = sim.activation_times()
    st = sim.stats()
    sim.close()
    return (X, u, ta, st), (Xo, uo, to)


@pytest.mark.parametrize("model,side,length,dt,steps", [(W.LR91, 17, 0.4, 0.01, 80),
                                                       (W.TP06_EPI, 11, 0.2, 0.002, 300)])
def test_cnrk2_matches_oracle(model, side, length, dt, steps):
    w = W.sheet(side, length, model, dt, steps, strip=0.06)
    (X, u, ta, st), (Xo, uo, to) = _run_both(w, steps, dt, **TIGHT)
    assert X[0].max() > -40.0                     # the strip has depolarised
    assert rel(X, Xo) < 1e-10 and rel(u, uo) < 1e-8
    np.testing.assert_array_equal(np.isnan(ta), np.isnan(to))
    np.testing.assert_allclose(ta[~np.isnan(ta)], to[~np.isnan(to)], atol=1e-9)
    assert st["cg_solves_p"] == steps and st["cg_solves_e"] == steps


def test_cnrk2_with_bath_matches_oracle():
    w = W.bath_sheet(24, -0.25, 1.25, 0.0, 1.0, W.LR91_PAPER_MOD, 0.01, 40, strip=0.1,
                     s1_amp=80.0, s1_dur=1.0)
    (X, u, ta, _), (Xo, uo, to) = _run_both(w, 40, 0.01, **TIGHT)
    assert rel(X, Xo) < 1e-10 and rel(u, uo) < 1e-8


def test_cnrk2_mixed_precision_within_tolerance():
    w = W.sheet(17, 0.4, W.LR91, 0.01, 80, strip=0.06)
    (X, u, _, _), (Xo, uo, _) = _run_both(w, 80, 0.01, precision=binding.MIXED)
    assert rel(X[0], Xo[0]) < 1e-3 and rel(u, uo) < 1e-3


def test_cnrk2_graph_replay_equals_eager():
    w = W.sheet(17, 0.4, W.LR91, 0.01, 20, strip=0.06)
    out = []
    for g in (1, 0):
        s = gpu_sim(w, use_graph=g)
        for _ in range(20):
            s.step_decoupled(0.01)
        out.append(s.fields(full=True))
        s.close()
    for a, b in zip(*out):
        np.testing.assert_array_equal(a, b)


def test_cnrk2_streaming_form_matches_oracle():
    """The decoupled scheme's diffusion and elliptic solves in the streaming
    form (the form large meshes take)."""
    w = W.sheet(17, 0.4, W.LR91, 0.01, 80, strip=0.06)
    (X, u, ta, st), (Xo, uo, to) = _run_both(w, 80, 0.01, streaming=1, **TIGHT)
    assert st["streaming"] == 1
    assert X[0].max() > -40.0
    assert rel(X, Xo) < 1e-9 and rel(u, uo) < 1e-8
    np.testing.assert_array_equal(np.isnan(ta), np.isnan(to))
    np.testing.assert_allclose(ta[~np.isnan(ta)], to[~np.isnan(to)], atol=1e-6)
