"""Pins of the oracle's partitioned SDC step (Sec. 3.3.2, Algorithm 2)."""
import numpy as np
import pytest
from scipy.integrate import solve_ivp

from oracle import bidomain as B
from oracle import cell as C
from oracle import lr91, tp06
from paper_2510_27447_gb300 import workloads as W

SIG = (3.0, 0.31, 2.0, 1.35)


class LinearCell(C.CellModel):
    """f(X) = diag(lam) X: the scalar test equation on every component."""
    def __init__(self, lam):
        self.lam = np.asarray(lam, dtype=np.float64)
        self.ns = len(lam)
        self.names = tuple(f"x{k}" for k in range(self.ns))
        self.gate_rows = ()

    def initial(self):
        return np.ones(self.ns)

    def currents(self, X, i_stim):
        return -self.lam[0] * X[0], self.lam[1:, None] * X[1:]


def _problem(cell, n=5, stim=(), lumped=False, pin=0, sigma=SIG, length=1.0):
    xyz, tri = W.square_grid(n, length)
    return B.Bidomain(xyz, tri, W.fibers_along_x(len(tri), 2), sigma, 2000.0, 1.0, cell,
                      stim, pin_node=pin, mass_lumped=lumped)


def test_integration_matrix_values_and_exactness():
    S3 = B.integration_matrix(B.lobatto_nodes(3))
    np.testing.assert_allclose(S3, [[5 / 24, 1 / 3, -1 / 24], [-1 / 24, 1 / 3, 5 / 24]], atol=1e-15)
    np.testing.assert_allclose(B.integration_matrix(B.lobatto_nodes(2)), [[0.5, 0.5]], atol=1e-16)
    c = B.lobatto_nodes(3)
    for deg in range(3):
        vals = c ** deg
        exact = (c[1:] ** (deg + 1) - c[:-1] ** (deg + 1)) / (deg + 1)
        np.testing.assert_allclose(S3 @ vals, exact, atol=1e-15)


def test_ros2_matches_closed_form_stability_function():
    lam = np.array([-3.0, -50.0, -0.2])
    P = _problem(LinearCell(lam))
    X = np.repeat(np.array([1.3, -0.7, 2.0])[:, None], P.N, axis=1)
    u = np.zeros(P.N)
    for h in (0.01, 0.1, 1.0):
        out = P.ros2(X, h, u, np.zeros(P.N))
        want = B.ros2_amplification(lam * h)[:, None] * X
        np.testing.assert_allclose(out, want, rtol=1e-12, atol=1e-13)
    # L-stability and second order of R itself
    assert abs(B.ros2_amplification(-1e12)) < 1e-10
    # local error R(z) - e^z = O(z^3): halving z divides it by 8 (order 2)
    e1 = abs(B.ros2_amplification(1e-2) - np.exp(1e-2))
    e2 = abs(B.ros2_amplification(5e-3) - np.exp(5e-3))
    assert 7.5 < e1 / e2 < 8.5


def test_sdc_step_two_nodes_closed_form():
    """M = 2, Eq. (3.20) on y' = lambda y with u = 0: every sweep recomputes
    the same predictor, so X^{n+1}/X^n = R + (1 - R + z (1 + R)/2)/(1 - z)."""
    lam = np.array([-2.0, -40.0])
    P = _problem(LinearCell(lam))
    X = np.repeat(np.array([0.8, 1.5])[:, None], P.N, axis=1)
    for h in (0.02, 0.3):
        out, u, _ = P.step(X, np.zeros(P.N), 0.0, h, n_sdc_nodes=2, n_sweeps=2)
        z = lam * h
        R = B.ros2_amplification(z)
        G = R + (1 - R + z * (1 + R) / 2) / (1 - z)
        np.testing.assert_allclose(out, G[:, None] * X, rtol=1e-12)
        assert np.max(np.abs(u)) < 1e-12


def test_equal_anisotropy_closed_form_elliptic():
    lam = 0.6
    sig = (3.0, 0.31, lam * 3.0, lam * 0.31)
    P = _problem(lr91.model(), n=9, sigma=sig, pin=4)
    v = np.random.default_rng(3).uniform(-90, 30, P.N)
    u = P.elliptic(v)
    want = -v / (1 + lam)
    want -= want[4]
    np.testing.assert_allclose(u, want, rtol=0, atol=1e-11)
    assert u[4] == 0.0


def test_elliptic_uniqueness_pin_and_mean():
    P0 = _problem(lr91.model(), n=9, pin=0)
    Pm = _problem(lr91.model(), n=9, pin=-1)
    x, y = P0.ops.M_L, None
    v = -80 + 100 * np.exp(-20 * np.sum((W.square_grid(9, 1.0)[0] - 0.3) ** 2, axis=1))
    u0 = P0.elliptic(v)
    um = Pm.elliptic(v)
    assert u0[0] == 0.0
    assert abs(um.mean()) < 1e-13
    np.testing.assert_allclose(u0 - um, np.full(P0.N, u0.mean() - um.mean()), atol=1e-11)
    # the constraint itself holds
    r = P0.ops.A_ie @ u0 + P0.ops.A_i @ v
    assert np.max(np.abs(r)) < 1e-12 * np.max(np.abs(P0.ops.A_i @ v))


def test_rest_state_is_a_fixed_point():
    cellm = lr91.model()
    P = _problem(cellm, n=5)
    X = np.repeat(cellm.rest_state()[:, None], P.N, axis=1)
    out, u, _ = P.step(X, np.zeros(P.N), 0.0, 0.02)
    np.testing.assert_allclose(out, X, rtol=1e-12, atol=1e-15)
    assert np.max(np.abs(u)) < 1e-10


def _single_cell_reference(cellm, x0, t_end, amp, dur):
    def rhs(t, x):
        return cellm.field(x[:, None], np.array([amp if t < dur else 0.0]))[:, 0].real

    def jac(t, x):
        return cellm.jacobian(x[:, None], np.array([amp if t < dur else 0.0]))[:, :, 0]
    a = solve_ivp(rhs, (0, dur), x0, method="Radau", jac=jac, rtol=1e-12, atol=1e-14)
    b = solve_ivp(rhs, (dur, t_end), a.y[:, -1], method="Radau", jac=jac, rtol=1e-12, atol=1e-14)
    return b.y[:, -1]


@pytest.mark.parametrize("n_nodes", [2, 3])
def test_zero_dimensional_reduction_second_order(n_nodes):
    """Uniform state + uniform stimulus: u = 0, every node follows the
    single-cell ODE and the step integrates it to second order.  The stimulus
    is sub-threshold so that v stays below the -40 mV switch of the h and j
    rates: across that jump of the right-hand side any fixed-step method
    loses its order."""
    cellm = lr91.model(True)
    x0 = cellm.rest_state()
    t_end, amp, dur = 2.0, 20.0, 1.0
    ref = _single_cell_reference(cellm, x0, t_end, amp, dur)
    assert ref[0] < -45.0
    errs = []
    for dt in (0.1, 0.05, 0.025):
        P = _problem(cellm, n=2, stim=[B.Stim(np.ones(4, np.uint8), 0.0, dur, amp)])
        X0 = np.repeat(x0[:, None], P.N, axis=1)
        X, u, _ = B.run(P, X0, int(round(t_end / dt)), dt, n_nodes, 2)
        assert np.max(np.abs(u)) < 1e-9
        assert np.max(np.abs(X - X[:, :1])) < 1e-9 * np.max(np.abs(X))
        errs.append(abs(X[0, 0] - ref[0]))       # v, the quantity of Table 4.1
    rates = np.log2(np.array(errs[:-1]) / np.array(errs[1:]))
    assert np.all(rates > 1.7), (errs, rates)


def _order(n_nodes, correction):
    cellm = lr91.model(True)
    P = _problem(cellm, n=7, stim=[])
    xyz, _ = W.square_grid(7, 1.0)
    P.stimuli = [B.Stim(W.nodes_x_below(xyz, 0.3), 0.0, 1.0, 40.0)]
    X0 = np.repeat(cellm.rest_state()[:, None], P.N, axis=1)

    def run(dt):
        return B.run(P, X0, int(round(0.5 / dt)), dt, n_nodes, 2, correction)[0][0]
    ref = run(0.1 / 64)
    errs = np.array([np.linalg.norm(run(dt) - ref) / np.linalg.norm(ref)
                     for dt in (0.05, 0.025, 0.0125)])
    return np.log2(errs[:-1] / errs[1:])


def test_partitioned_order_with_and_without_sdc():
    """Table 4.1: about second order with the SDC correction, first order
    without (Algorithm 1), for the relative L2 error of v at t = 0.5 ms
    (self-convergence; sub-threshold stimulus, see above)."""
    with_sdc = _order(2, True)
    without = _order(2, False)
    assert with_sdc[-1] > 1.7, with_sdc
    assert 0.7 < without[-1] < 1.3, without
    assert with_sdc[-1] - without[-1] > 0.6


@pytest.mark.slow
def test_partitioned_order_three_lobatto_nodes():
    rates = _order(3, True)
    assert rates[-1] > 1.8, rates


def test_gates_stay_in_unit_interval_during_upstroke():
    cellm = tp06.model()
    xyz, tri = W.square_grid(7, 0.3)
    P = B.Bidomain(xyz, tri, W.fibers_along_x(len(tri), 2), SIG, 2000.0, 1.0, cellm,
                   [B.Stim(W.nodes_x_below(xyz, 0.06), 0.0, 1.0, 80.0)])
    X = np.repeat(cellm.initial()[:, None], P.N, axis=1)
    u = np.zeros(P.N)
    rows = list(cellm.gate_rows)
    for n in range(60):
        X, u, _ = P.step(X, u, n * 0.05, 0.05)
        g = X[rows]
        assert g.min() > -1e-9 and g.max() < 1 + 1e-9
    assert X[0].max() > 0.0     # the stimulated corner has depolarised


def test_activation_time_interpolation():
    t = np.full(3, np.nan)
    B.activation_update(t, np.array([-40.0, -20.0, -50.0]), np.array([-20.0, 10.0, -45.0]), 1.0, 0.5)
    assert t[0] == pytest.approx(1.25)
    assert np.isnan(t[1]) and np.isnan(t[2])
    B.activation_update(t, np.array([-35.0, -35.0, -35.0]), np.array([0.0, 0.0, 0.0]), 2.0, 0.5)
    assert t[0] == pytest.approx(1.25)       # first crossing is kept
    assert t[1] == pytest.approx(2.0 + 0.5 * 5 / 35)


def test_stimulus_window():
    P = _problem(lr91.model(), n=3, stim=[B.Stim(np.ones(9, np.uint8), 1.0, 1.0, 80.0)])
    dt = 0.02
    on = [bool(P.i_stim(n * dt, dt)[0]) for n in range(200)]
    assert on.index(True) == 50 and sum(on) == 50


# ---------------------------------------------------------------------------
# adaptive stepping: embedded ROS2 estimate and step controller
# ---------------------------------------------------------------------------

def _embedded_amplification(z):
    """X_hat = X + k1/gamma on y' = lambda y: k1 = gamma z X/(1 - gamma z),
    so X_hat/X = (1 + (1 - gamma) z)/(1 - gamma z), a first-order method."""
    g = B.GAMMA
    return (1.0 + (1.0 - g) * z) / (1.0 - g * z)


def test_embedded_estimate_closed_form():
    lam = np.array([-3.0, -50.0, -0.2])
    P = _problem(LinearCell(lam))
    x = np.array([1.3, -0.7, 2.0])
    X = np.repeat(x[:, None], P.N, axis=1)
    tol = 1e-3
    P.adaptive_tol = tol
    for h in (0.01, 0.1, 1.0):
        # M = 2: the last sweep's predictor is one ROS2 step of length h
        P.step(X, np.zeros(P.N), 0.0, h, n_sdc_nodes=2, n_sweeps=2)
        z = lam * h
        R, Rh = B.ros2_amplification(z), _embedded_amplification(z)
        want = np.max(np.abs((R - Rh) * x) / (tol * (1.0 + np.abs(R * x))))
        assert P.last_err == pytest.approx(want, rel=1e-10)
        # M = 3: two sub-steps of h/2, the second from the first's result
        P.step(X, np.zeros(P.N), 0.0, h, n_sdc_nodes=3, n_sweeps=1)
        z2 = z / 2
        R2, Rh2 = B.ros2_amplification(z2), _embedded_amplification(z2)
        x1 = R2 * x
        e1 = np.abs((R2 - Rh2) * x) / (tol * (1.0 + np.abs(x1)))
        e2 = np.abs((R2 - Rh2) * x1) / (tol * (1.0 + np.abs(R2 * x1)))
        assert P.last_err == pytest.approx(max(e1.max(), e2.max()), rel=1e-10)
    # the embedded method is of order one: local error O(z^2)
    r = abs(_embedded_amplification(1e-3) - np.exp(1e-3)) / abs(_embedded_amplification(5e-4) - np.exp(5e-4))
    assert 3.9 < r < 4.1


def test_embedded_estimate_scales_with_h_squared_on_lr91():
    """A smooth sub-threshold phase: halving the step divides the estimate by
    about four (difference of a second- and a first-order solution).  The
    steps are long enough for v to dominate the maximum; below about 0.005 ms
    the stiff m gate (time constant of microseconds) takes over, whose
    estimate is not yet in its asymptotic range."""
    cellm = lr91.model(True)
    P = _problem(cellm, n=4, stim=[B.Stim(np.ones(16, np.uint8), 0.0, 5.0, 15.0)])
    P.adaptive_tol = 1.0
    X = np.repeat(cellm.rest_state()[:, None], P.N, axis=1)
    errs = []
    for h in (0.04, 0.02, 0.01):
        P.step(X, np.zeros(P.N), 0.0, h, n_sdc_nodes=2, n_sweeps=1)
        errs.append(P.last_err)
    r = np.array(errs[:-1]) / np.array(errs[1:])
    assert np.all((r > 3.5) & (r < 4.5)), (errs, r)


def test_controller_ladder_and_factor():
    assert B.ladder_step(0.05, 0.05, 8) == 0.05
    assert B.ladder_step(0.05, 0.049, 8) == 0.025
    assert B.ladder_step(0.05, 0.0125, 8) == 0.0125
    assert B.ladder_step(0.05, 1e-9, 8) == 0.05 / 128
    assert B.ladder_step(0.05, 1.0, 8) == 0.05
    assert B.controller_factor(0.0) == 2.0
    assert B.controller_factor(0.01) == 2.0
    assert B.controller_factor(1.0) == pytest.approx(0.9)
    assert B.controller_factor(4.0) == pytest.approx(0.5)
    assert B.controller_factor(100.0) == 0.5


def test_adaptive_limits_reduce_to_fixed_steps():
    """tol -> infinity: every step dt_max, identical to the fixed-step march;
    tol -> 0: the first step is rejected down the whole ladder (7 times),
    then every step stays on the smallest rung."""
    cellm = lr91.model(True)
    stim = [B.Stim(np.ones(16, np.uint8), 0.0, 1.0, 30.0)]
    P = _problem(cellm, n=4, stim=stim)
    X0 = np.repeat(cellm.rest_state()[:, None], P.N, axis=1)
    X, u, t, ta, dts, rej = B.run_adaptive(P, X0, 5, 0.05, 1e30)
    Xf, uf, _ = B.run(_problem(cellm, n=4, stim=stim), X0, 5, 0.05)
    assert dts == [0.05] * 5 and rej == 0 and t == pytest.approx(0.25)
    np.testing.assert_array_equal(X, Xf)
    X, u, t, ta, dts, rej = B.run_adaptive(P, X0, 3, 0.05, 1e-30)
    assert dts == [0.05 / 128] * 3 and rej == 7
    Xf, uf, _ = B.run(_problem(cellm, n=4, stim=stim), X0, 3, 0.05 / 128)
    np.testing.assert_array_equal(X, Xf)
