"""Node-wise membrane dynamics shared by the oracle's cell models.

Test infrastructure only (see the package docstring).

Sec. 2 writes the membrane dynamics at each point as
    dv/dt = ... - I_ion(v, w, c) + I_stim,   dc/dt = S(v, w, c),   dw/dt = G(v, w)
(Eqs. (2.2)-(2.4)).  With the state of one node X = (v, y), y = (w, c), this
module forms the node vector field
    f(X) = ( -(I_ion(X) - I_stim)/C_m ,  g(X) ),    g = (G, S),
and its Jacobian df/dX, which the paper's Rosenbrock method uses exactly
("exact derivatives", Sec. 3.3.2).

The oracle obtains the Jacobian by complex-step differentiation
(Squire & Trapp, SIAM Review 40, 1998; Martins, Sturdza & Alonso, ACM TOMS 29,
2003): for a real-analytic f, df/dx_k = Im f(x + i h e_k) / h with no
subtractive cancellation, exact to rounding for h = 1e-30.  Every model
function is therefore written so that it accepts complex arrays: branches
test the real part, and singular quotients use ``exprel`` below.  This is an
independent route to the same derivatives the CUDA library computes by
forward-mode differentiation.

Pins (tests/test_oracle_cell.py): complex-step Jacobian against central
finite differences; exprel against its series and against expm1; gate bounds;
rest state is a zero of f.
"""
from __future__ import annotations

import numpy as np

H_CS = 1e-30   # complex-step size


def exprel(z):
    """(exp(z) - 1) / z with its limit 1 at z = 0.

    Near z = 0 the quotient is replaced by its Taylor series
    sum_k z^k / (k+1)!  (11 terms, truncation < 3e-18 for |Re z| < 0.1);
    elsewhere the quotient is evaluated directly.  Both forms are analytic,
    so the complex-step derivative stays exact.
    """
    z = np.asarray(z)
    small = np.abs(z.real) < 0.1
    zs = np.where(small, z, 0.0)
    series = np.zeros_like(zs)
    term = np.ones_like(zs)
    fact = 1.0
    for k in range(11):
        fact *= (k + 1)
        series = series + term / fact
        term = term * zs
    zb = np.where(small, 1.0, z)
    direct = (np.exp(zb) - 1.0) / zb
    return np.where(small, series, direct)


class CellModel:
    """Interface of a membrane model in the oracle.

    Subclasses define ``ns``, ``names``, ``gate_rows``, ``initial()`` and
    ``currents(X, i_stim) -> (I_ion, g)`` where X is [ns, N] (real or complex),
    I_ion is [N] in uA/cm^2 (per unit membrane area at C_m = 1 uF/cm^2) and
    g is [ns-1, N].
    """
    ns: int
    names: tuple
    gate_rows: tuple

    def initial(self) -> np.ndarray:
        raise NotImplementedError

    def currents(self, X, i_stim):
        raise NotImplementedError

    # -- node vector field and its Jacobian ---------------------------------
    def field(self, X, i_stim, cm: float = 1.0):
        """f(X) = (-(I_ion - I_stim)/C_m, g(X)), shape [ns, N]."""
        I_ion, g = self.currents(X, i_stim)
        out = np.empty((self.ns,) + np.shape(X[0]), dtype=np.result_type(X, I_ion, g))
        out[0] = -(I_ion - i_stim) / cm
        out[1:] = g
        return out

    def jacobian(self, X, i_stim, cm: float = 1.0) -> np.ndarray:
        """df/dX by complex step, shape [ns, ns, N] (row = component of f)."""
        X = np.asarray(X, dtype=np.float64)
        ns, n = X.shape
        J = np.empty((ns, ns, n))
        for k in range(ns):
            Xc = X.astype(np.complex128)
            Xc[k] += 1j * H_CS
            J[:, k, :] = self.field(Xc, i_stim, cm).imag / H_CS
        return J

    def rest_state(self, x0=None, tol=1e-13, max_iter=60) -> np.ndarray:
        """Zero of the single-cell field f(X) = 0 (no stimulus) by Newton's
        method from the published initial values."""
        x = np.array(self.initial() if x0 is None else x0, dtype=np.float64).reshape(self.ns, 1)
        for _ in range(max_iter):
            f = self.field(x, np.zeros(1)).real
            J = self.jacobian(x, np.zeros(1))[:, :, 0]
            dx = np.linalg.solve(J, -f[:, 0])
            x[:, 0] += dx
            if np.max(np.abs(dx) / np.maximum(np.abs(x[:, 0]), 1e-12)) < tol:
                break
        return x[:, 0]
