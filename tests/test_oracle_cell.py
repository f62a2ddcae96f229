"""Pins of the oracle's membrane models (Sec. 2, LR91 and TP06)."""
import numpy as np
import pytest

from oracle import cell, lr91, tp06


def test_exprel_series_and_limit():
    z = np.array([0.0, 1e-12, -1e-8, 0.05, -0.0999, 0.1, -0.1, 0.5, -3.0, 12.0])
    want = np.where(z == 0, 1.0, np.expm1(z) / np.where(z == 0, 1.0, z))
    np.testing.assert_allclose(cell.exprel(z), want, rtol=2e-15)
    # derivative at 0 is 1/2, second derivative 1/3 (series 1 + z/2 + z^2/6 ...)
    h = 1e-30
    assert cell.exprel(np.array([1j * h])).imag[0] / h == pytest.approx(0.5, rel=1e-15)


def _random_states(model, n, seed):
    rng = np.random.Generator(np.random.PCG64(seed))
    x0 = model.initial()
    X = np.repeat(x0[:, None], n, axis=1)
    X[0] = rng.uniform(-90.0, 40.0, n)
    for r in model.gate_rows:
        X[r] = rng.uniform(0.02, 0.98, n)
    for r in range(1 + len(model.gate_rows), model.ns):
        X[r] = x0[r] * rng.uniform(0.7, 1.3, n)
    # keep away from the -40 mV switch of h, j where the field is not smooth
    X[0] = np.where(np.abs(X[0] + 40.0) < 0.5, -41.0, X[0])
    return X


@pytest.mark.parametrize("model", [lr91.model(), lr91.model(True), tp06.model()],
                         ids=["lr91", "lr91_paper", "tp06"])
def test_complex_step_jacobian_matches_central_differences(model):
    X = _random_states(model, 12, 7)
    ist = np.zeros(X.shape[1])
    J = model.jacobian(X, ist)
    for k in range(model.ns):
        h = 1e-6 * np.maximum(np.abs(X[k]), 1e-3)
        Xp = X.copy(); Xp[k] += h
        Xm = X.copy(); Xm[k] -= h
        fd = (model.field(Xp, ist) - model.field(Xm, ist)) / (2 * h)
        scale = np.abs(J).max(axis=1) + 1e-300      # row scale per node
        err = np.abs(fd - J[:, k, :]) / scale
        assert err.max() < 1e-6, (k, err.max())


@pytest.mark.parametrize("v_sing,model", [(-47.13, lr91.model()), (-77.0, lr91.model()),
                                          (15.0, tp06.model())])
def test_removable_singularities_are_smooth(v_sing, model):
    x0 = model.initial()
    X = np.repeat(x0[:, None], 5, axis=1)
    X[0] = v_sing + np.array([-1e-3, -1e-9, 0.0, 1e-9, 1e-3])
    f = model.field(X, np.zeros(5))
    assert np.all(np.isfinite(f))
    # continuity across the singular point and a derivative equal to the chord slope
    np.testing.assert_allclose(f[:, 1:4], f[:, 2:3].repeat(3, axis=1), rtol=1e-8, atol=1e-12)
    J = model.jacobian(X[:, 2:3], np.zeros(1))[:, 0, 0]
    chord = (f[:, 4] - f[:, 0]) / 2e-3
    np.testing.assert_allclose(J, chord, rtol=1e-5, atol=1e-9)


def test_lr91_rest_state():
    m = lr91.model()
    xr = m.rest_state()
    assert np.max(np.abs(m.field(xr[:, None], np.zeros(1)))) < 1e-12
    # the 1991 article's resting potential is about -84 mV
    assert -86.0 < xr[0] < -83.0
    (am, bm), (ah, bh), (aj, bj), (ad, bd), (af, bf), (ax, bx) = m.rates(np.array([xr[0]]))
    np.testing.assert_allclose(xr[1:7], [a[0] / (a[0] + b[0]) for a, b in
                                         [(am, bm), (ah, bh), (aj, bj), (ad, bd), (af, bf), (ax, bx)]],
                               rtol=1e-10)


def test_tp06_charge_conservation_identity():
    """Charge carried by the concentration fluxes equals the membrane charge
    for any state: Cap dV/dt = F (V_c (dKi + dNai + 2 dCai_tot) + 2 V_sr dCaSR_tot
    + 2 V_ss dCaSS_tot), the buffered totals obtained by dividing the free
    derivatives by the rapid-buffer factors.  A wrong sign or a dropped flux
    in any concentration equation breaks it."""
    m = tp06.model()
    X = _random_states(m, 50, 11)
    ist = np.linspace(0.0, 80.0, 50)
    f = m.field(X, ist).real
    ki, nai, cai, casr, cass = (f[14], f[15], f[16], f[17], f[18])
    b_c = 1.0 / (1.0 + tp06.BUF_C * tp06.K_BUF_C / (X[16] + tp06.K_BUF_C) ** 2)
    b_sr = 1.0 / (1.0 + tp06.BUF_SR * tp06.K_BUF_SR / (X[17] + tp06.K_BUF_SR) ** 2)
    b_ss = 1.0 / (1.0 + tp06.BUF_SS * tp06.K_BUF_SS / (X[18] + tp06.K_BUF_SS) ** 2)
    ion = tp06.F_C * (tp06.V_C * (ki + nai + 2 * cai / b_c) + 2 * tp06.V_SR * casr / b_sr
                      + 2 * tp06.V_SS * cass / b_ss)
    mem = tp06.CAP * f[0]
    np.testing.assert_allclose(ion, mem, rtol=1e-9, atol=1e-9 * np.abs(mem).max())


def test_tp06_initial_state_is_near_rest():
    m = tp06.model()
    f = m.field(m.initial()[:, None], np.zeros(1))[:, 0]
    assert abs(f[0]) < 0.01           # mV/ms
    assert np.max(np.abs(f[1:])) < 5e-3
