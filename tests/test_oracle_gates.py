"""Gate pins of the oracle's membrane models (Sec. 2): all twelve gates of
the TP06 epicardial cell, the slow ones (j, f, f2, Xr1, Xs, fCass) included,
and the six gates of LR91 (m, h, j, d, f, X; written as rates,
dx/dt = alpha (1 - x) - beta x, so x_inf = alpha / (alpha + beta) and
tau = 1 / (alpha + beta), with alpha, beta >= 0).

  * The gate rows of the vector field that the step integrates are the
    relaxations dx/dt = (x_inf - x) / tau.  Each row is affine in its own
    gate, so two evaluations of the field give its slope -1/tau and its zero
    x_inf without reading any formula; they must be the pair that
    gate_inf_tau returns for that gate (a rate wired to the wrong gate, or
    a row that depends on another gate, fails).
  * Hodgkin-Huxley gating fixes, whatever the constants: x_inf in [0, 1],
    tau > 0 and finite; activation gates (m, d, r, Xr1, Xs) open with
    depolarisation and inactivation gates (h, j, f, f2, s, Xr2) close, each
    x_inf monotone over -100..60 mV and spanning most of its range there;
    fCass inactivates as the subspace calcium rises.  A sign error in an
    exponent's argument reverses a gate's direction.

The complex-step Jacobian and the charge-conservation identity test
derivatives and bookkeeping; the biomarker bands test the whole cell.
None of them sees a single slow gate's direction or wiring.
"""
import numpy as np
import pytest

from oracle import lr91, tp06

GATES = ("m", "h", "j", "d", "f", "f2", "s", "r", "Xr1", "Xr2", "Xs", "fCass")
OPENS = ("m", "d", "r", "Xr1", "Xs")                 # activation: x_inf rises with V
CLOSES = ("h", "j", "f", "f2", "s", "Xr2")            # inactivation: x_inf falls with V


def _states(n, seed):
    rng = np.random.default_rng(seed)
    cell = tp06.model()
    X = np.repeat(cell.initial()[:, None], n, axis=1)
    X[0] = rng.uniform(-95.0, 45.0, n)
    X[1:13] = rng.uniform(0.05, 0.95, (12, n))
    X[18] = X[18] * rng.uniform(0.5, 50.0, n)        # subspace calcium over two decades
    return cell, X


def test_gate_rows_of_the_field_are_the_published_relaxations():
    cell, X = _states(400, 3)
    f0 = cell.field(X, 0.0)
    it = cell.gate_inf_tau(X[0], X[18])
    for k, name in enumerate(GATES):
        row = 1 + k
        Xd = X.copy()
        Xd[row] += 0.25
        f1 = cell.field(Xd, 0.0)
        slope = (f1[row] - f0[row]) / 0.25
        tau = -1.0 / slope
        xinf = X[row] + tau * f0[row]
        np.testing.assert_allclose(tau, it[k][1], rtol=1e-9, err_msg=name)
        np.testing.assert_allclose(xinf, it[k][0], rtol=1e-9, atol=1e-12, err_msg=name)
        # the row depends on no other gate
        for other in range(1, 13):
            if other == row:
                continue
            Xo = X.copy()
            Xo[other] += 0.25
            np.testing.assert_array_equal(cell.field(Xo, 0.0)[row], f0[row], err_msg=f"{name} <- {other}")


@pytest.mark.parametrize("name", [g for g in GATES if g != "fCass"])
def test_voltage_gates_are_bounded_and_open_or_close_with_depolarisation(name):
    V = np.linspace(-100.0, 60.0, 1601)
    cass = np.full_like(V, 1e-4)
    k = GATES.index(name)
    xinf, tau = tp06.model().gate_inf_tau(V, cass)[k]
    assert np.all(np.isfinite(xinf)) and np.all(np.isfinite(tau))
    assert np.all(tau > 0.0)
    assert np.all((xinf >= 0.0) & (xinf <= 1.0))
    d = np.diff(xinf)
    if name in OPENS:
        assert np.all(d >= 0.0) and xinf[-1] - xinf[0] > 0.5
    else:
        assert name in CLOSES
        assert np.all(d <= 0.0) and xinf[0] - xinf[-1] > 0.5


def test_fcass_inactivates_as_subspace_calcium_rises():
    cass = np.logspace(-5, 0, 501)                    # mM
    V = np.full_like(cass, -20.0)
    xinf, tau = tp06.model().gate_inf_tau(V, cass)[GATES.index("fCass")]
    assert np.all(tau > 0.0) and np.all(np.isfinite(tau))
    assert np.all((xinf >= 0.0) & (xinf <= 1.0))
    assert np.all(np.diff(xinf) <= 0.0) and xinf[0] - xinf[-1] > 0.5
    # voltage plays no part in it
    other = tp06.model().gate_inf_tau(np.full_like(cass, 30.0), cass)[GATES.index("fCass")]
    np.testing.assert_array_equal(other[0], xinf)


LR91_GATES = ("m", "h", "j", "d", "f", "X")
LR91_OPENS = ("m", "d", "X")
LR91_CLOSES = ("h", "j", "f")


@pytest.mark.parametrize("paper", [False, True])
def test_lr91_gate_rows_of_the_field_are_the_rate_relaxations(paper):
    cell = lr91.model(paper)
    rng = np.random.default_rng(5)
    n = 400
    X = np.repeat(cell.initial()[:, None], n, axis=1)
    X[0] = rng.uniform(-95.0, 45.0, n)
    X[1:7] = rng.uniform(0.05, 0.95, (6, n))
    f0 = cell.field(X, 0.0)
    rates = cell.rates(X[0])
    for k, name in enumerate(LR91_GATES):
        row = 1 + k
        a, b = rates[k]
        Xd = X.copy()
        Xd[row] += 0.25
        slope = (cell.field(Xd, 0.0)[row] - f0[row]) / 0.25
        np.testing.assert_allclose(-slope, a + b, rtol=1e-9, err_msg=name)
        np.testing.assert_allclose(X[row] - f0[row] / slope, a / (a + b), rtol=1e-9, atol=1e-12, err_msg=name)
        for other in range(1, 7):
            if other != row:
                Xo = X.copy()
                Xo[other] += 0.25
                np.testing.assert_array_equal(cell.field(Xo, 0.0)[row], f0[row], err_msg=f"{name} <- {other}")


@pytest.mark.parametrize("name", LR91_GATES)
def test_lr91_gates_are_bounded_and_open_or_close_with_depolarisation(name):
    V = np.linspace(-100.0, 60.0, 1601)
    a, b = lr91.model().rates(V)[LR91_GATES.index(name)]
    assert np.all(np.isfinite(a)) and np.all(np.isfinite(b))
    assert np.all(a >= 0.0) and np.all(b >= 0.0) and np.all(a + b > 0.0)
    xinf = a / (a + b)
    d = np.diff(xinf)
    if name in LR91_OPENS:
        assert np.all(d >= 0.0) and xinf[-1] - xinf[0] > 0.5
    else:
        assert name in LR91_CLOSES
        assert np.all(d <= 0.0) and xinf[0] - xinf[-1] > 0.5
