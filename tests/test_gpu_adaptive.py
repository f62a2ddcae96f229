"""Adaptive time stepping on the GPU (embedded ROS2 estimate, Sec. 3.3.2):
same accepted steps, rejections and states as the oracle's controller."""
import numpy as np
import pytest

from oracle import bidomain as OB
from paper_2510_27447_gb300 import workloads as W

from gpu_util import gpu_sim, oracle_problem, rel, rest_X

pytestmark = pytest.mark.gpu

TIGHT = dict(cg_tol_e=1e-12, cg_tol_p=1e-12)


def _sheet():
    return W.sheet(15, 0.3, W.LR91_PAPER_MOD, 0.05, 30, strip=0.05)


def test_adaptive_steps_match_oracle():
    w = _sheet()
    X0 = rest_X(w)
    P = oracle_problem(w)
    X, u, t, ta, dts, rej = OB.run_adaptive(P, X0, 30, 0.05, 1e-2)
    sim = gpu_sim(w, **TIGHT)
    sim.set_initial(X0)
    gdts, grej = [], 0
    for _ in range(30):
        dt, err, r = sim.step_adaptive(0.05, 1e-2)
        assert err <= 1.0 or dt == 0.05 / 128
        gdts.append(dt)
        grej += r
    tg, n = sim.time()
    _, ug, Xg = sim.fields(full=True)
    tag = sim.activation_times()
    sim.close()
    assert rej > 0 and min(dts) < 0.05          # the controller did shrink and reject
    assert gdts == dts and grej == rej
    assert n == 30 and tg == pytest.approx(t, abs=1e-12)
    assert rel(Xg, X) < 1e-9 and rel(ug, u) < 1e-7
    fin = ~np.isnan(ta)
    assert np.array_equal(fin, ~np.isnan(tag))
    assert np.max(np.abs(tag[fin] - ta[fin]), initial=0.0) < 1e-8


def test_adaptive_resume_is_bitwise():
    """The state blob carries the clock and the next adaptive step."""
    w = _sheet()
    X0 = rest_X(w)
    a = gpu_sim(w)
    a.set_initial(X0)
    for _ in range(12):
        a.step_adaptive(0.05, 1e-2)
    blob = a.get_state()
    ref = [a.step_adaptive(0.05, 1e-2) for _ in range(10)]
    _, _, Xa = a.fields(full=True)
    ta, na = a.time()
    a.close()
    b = gpu_sim(w)
    b.set_state(blob)
    got = [b.step_adaptive(0.05, 1e-2) for _ in range(10)]
    _, _, Xb = b.fields(full=True)
    tb, nb = b.time()
    b.close()
    assert got == ref and (ta, na) == (tb, nb) and np.array_equal(Xa, Xb)


def test_adaptive_mixed_precision_tracks_fp64():
    w = _sheet()
    X0 = rest_X(w)
    out = []
    for prec in (0, 1):
        s = gpu_sim(w, precision=prec)
        s.set_initial(X0)
        dts = [s.step_adaptive(0.05, 1e-2)[0] for _ in range(30)]
        _, _, Xs = s.fields(full=True)
        s.close()
        out.append((dts, Xs))
    # same step sequence up to decisions taken within FP32 rounding of err = 1
    assert sum(out[0][0]) == pytest.approx(sum(out[1][0]), rel=0.1)
    assert np.all(np.isfinite(out[1][1]))


def test_adaptive_steps_in_the_streaming_form_match_oracle():
    """The adaptive controller on a handle whose solves take the streaming
    form: the same accepted steps and rejections as the oracle."""
    w = _sheet()
    X0 = rest_X(w)
    X, u, t, ta, dts, rej = OB.run_adaptive(oracle_problem(w), X0, 30, 0.05, 1e-2)
    sim = gpu_sim(w, streaming=1, **TIGHT)
    sim.set_initial(X0)
    gdts, grej = [], 0
    for _ in range(30):
        dt, err, r = sim.step_adaptive(0.05, 1e-2)
        gdts.append(dt)
        grej += r
    _, ug, Xg = sim.fields(full=True)
    st = sim.stats()
    sim.close()
    assert st["streaming"] == 1
    assert gdts == dts and grej == rej
    assert rel(Xg, X) < 1e-8 and rel(ug, u) < 1e-7
