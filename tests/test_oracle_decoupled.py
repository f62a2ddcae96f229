"""Pins of the CN-RK2 oracle (decoupled strategy, Sec. 3.3.3)."""
import numpy as np
import pytest
import scipy.linalg as sla
from scipy.integrate import solve_ivp

from oracle import bidomain as B
from oracle import cell as C
from oracle import decoupled as D
from oracle import lr91
from paper_2510_27447_gb300 import workloads as W

SIG = (3.0, 0.31, 2.0, 1.35)


class ZeroCell(C.CellModel):
    """No membrane dynamics: the reaction sub-steps are the identity."""
    ns = 2
    names = ("v", "y")
    gate_rows = ()

    def initial(self):
        return np.zeros(2)

    def currents(self, X, i_stim):
        return 0.0 * X[0], 0.0 * X[1:]


def _problem(cell, n=6, stim=(), sigma=SIG, lumped=False):
    xyz, tri = W.square_grid(n, 1.0)
    return B.Bidomain(xyz, tri, W.fibers_along_x(len(tri), 2), sigma, 2000.0, 1.0, cell, stim,
                      pin_node=0, mass_lumped=lumped)


@pytest.mark.parametrize("lumped", [False, True])
def test_crank_nicolson_factor_on_generalised_eigenmodes(lumped):
    """Zero reaction, u^n = 0: one step multiplies each generalised
    eigenvector A_i phi = mu M phi by (1 - z/2)/(1 + z/2), z = dt mu."""
    P = _problem(ZeroCell(), lumped=lumped)
    mu, phi = sla.eigh(P.ops.A_i.toarray(), P.M_v.toarray())
    dt = 0.7
    for k in (0, 3, 11, len(mu) - 1):
        X = np.zeros((2, P.N))
        X[0] = phi[:, k]
        X[1] = 0.25
        X1, _ = D.cnrk2_step(P, X, np.zeros(P.N), 0.0, dt)
        z = dt * mu[k]
        np.testing.assert_allclose(X1[0], (1 - z / 2) / (1 + z / 2) * phi[:, k], atol=1e-11)
        assert np.all(X1[1] == 0.25)


def test_zero_dimensional_reduction_second_order():
    """Uniform state and stimulus: the diffusion step is the identity, u = 0
    and every node follows two midpoint-rule half steps of the single-cell
    ODE per step: second order against a Radau reference."""
    cellm = lr91.model(True)
    x0 = cellm.rest_state()
    t_end, amp, dur = 2.0, 20.0, 1.0

    def rhs(t, x):
        return cellm.field(x[:, None], np.array([amp if t < dur else 0.0]))[:, 0].real
    a = solve_ivp(rhs, (0, dur), x0, method="Radau", rtol=1e-12, atol=1e-14)
    ref = solve_ivp(rhs, (dur, t_end), a.y[:, -1], method="Radau", rtol=1e-12, atol=1e-14).y[:, -1]
    errs = []
    for dt in (0.02, 0.01, 0.005):
        P = _problem(cellm, n=2, stim=[B.Stim(np.ones(4, np.uint8), 0.0, dur, amp)])
        X0 = np.repeat(x0[:, None], P.N, axis=1)
        X, u, _ = D.run_cnrk2(P, X0, int(round(t_end / dt)), dt)
        assert np.max(np.abs(u)) < 1e-9
        errs.append(abs(X[0, 0] - ref[0]))
    rates = np.log2(np.array(errs[:-1]) / np.array(errs[1:]))
    assert np.all(rates > 1.8), (errs, rates)


@pytest.mark.slow
def test_cnrk2_conduction_velocity_matches_biomarker_table():
    """Sec. 4's LR91 biomarker table lists CV = 27.52 cm/s for CN-RK2 (the
    same as the partitioned strategy) on the setup of the SDC pin."""
    cellm = lr91.model(True)
    xyz, tri = W.rect_grid(61, 3, 0.6, 0.02)
    P = B.Bidomain(xyz, tri, W.fibers_along_x(len(tri), 2), (3.0, 3.0, 3.0, 3.0), 2000.0, 1.0,
                   cellm, [B.Stim(W.nodes_x_below(xyz, 0.051), 0.0, 1.0, 80.0)], pin_node=0)
    X0 = np.repeat(cellm.rest_state()[:, None], P.N, axis=1)
    _, _, t_act = D.run_cnrk2(P, X0, 2500, 0.01)
    cv = 1000.0 * B.conduction_velocity(xyz, t_act, 0.01, 0.15)
    assert abs(cv - 27.52) / 27.52 < 0.10, cv
