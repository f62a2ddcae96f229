"""Partitioned bidomain time step with spectral deferred correction (oracle).

Test infrastructure only (see the package docstring).  Plain FP64, every
linear system solved as written with a sparse direct factorisation.

Semi-discrete system (Sec. 3.2-3.3, Eqs. (3.10)-(3.11)):
    A_ie u = -A_i v                           (elliptic constraint)
    Mt dX/dt = F(X, u),   X = (v, y)          (parabolic PDE + ODEs)
with, per node i and the node field f = (f_v, f_y) of ``cell.py``,
    F_v(X, u) = -A_i (v + u) + M_L f_v(X),    F_y(X) = M_L f_y(X),
    Mt = diag(M, M_L, ..., M_L).
Reading (the paper uses consistent M_c, M_w, Eq. (3.8)-(3.9)): the reaction
terms and the ODE rows use the lumped mass M_L, only dv/dt keeps the
consistent M (``mass_lumped=True`` uses M_L there too).  This keeps every
ODE node-local and the condensed v-system symmetric.

ROS2 (Eq. (3.13)-(3.14), s = 2, p = 2, L-stable).  The paper cites Lang 2001
and prints no coefficients; the reading here is the two-stage method of
Verwer, Spee, Blom & Hundsdorfer (SIAM J. Sci. Comput. 20, 1999) in the
paper's form: gamma = 1 + 1/sqrt(2), a21 = 1/gamma, c21 = 2/gamma,
m = (3/(2 gamma), 1/(2 gamma)), embedded m_hat = (1/gamma, 0):
    (Mt/(gamma h) - W) k1 = F(X, u)
    (Mt/(gamma h) - W) k2 = F(X + k1/gamma, u) - (2/(gamma h)) Mt k1
    X_new = X + 3/(2 gamma) k1 + 1/(2 gamma) k2,   X_hat = X + k1/gamma.
On y' = lambda y the step is R(z) = (1 + (1 - 2 gamma) z)/(1 - gamma z)^2.

SDC correction (Eq. (3.17)-(3.20)).  For two quadrature nodes {t^n, t^n+1}
Eq. (3.20) reads
    (Mt - tau J(X~)) eps = Mt X^n - Mt X~ + tau/2 (F(X^n, u^n) + F(X~, u^n+1)).
It is applied here on M Gauss-Lobatto nodes c_0 = 0 < ... < c_{M-1} = 1
(M = 2 is exactly Eq. (3.20)); with dt_m = tau (c_{m+1} - c_m) and the
spectral integration matrix S_{m,j} = tau * int_{c_m}^{c_{m+1}} l_j(s) ds,
    (Mt - dt_m W(X~_{m+1})) eps_{m+1} = Mt (X_m^new - X~_{m+1}) + sum_j S_{m,j} F(X~_j, u_j),
    X_{m+1}^new = X~_{m+1} + eps_{m+1}.

Algorithm 2 (partitioned strategy with SDC), inner iteration k:
  1. solve the elliptic equation (3.15) with the previous iterate's v at
     every node m >= 1 (u_0 = u^n);
  2. predict X~ with ROS2 on each sub-interval from X^n, with u_{m+1} fixed;
  3. correct (above);
  4. stop after n_sweeps iterations or when max|X^k - X^{k-1}| < sweep_tol.
Output X^{n+1} = X_{M-1}, u^{n+1} = u_{M-1} of the last iteration.
With correction=False this is Algorithm 1 (partitioned strategy without SDC).

W-matrix safeguard (a reading; the paper solves with BiCGSTAB and needs no
symmetry): per node the Schur complement of the node block onto v,
    s_i = -j_vv - j_vy (alpha I - j_yy)^{-1} j_yv,
is raised to at least -margin alpha lambda_M (margin = ``spd_margin``, 0.9 by
default; lambda_M = 1 lumped, 1/4 for P1 triangles, 1/5 for P1 tetrahedra:
the smallest generalised eigenvalue of (M, M_L) on one element, so
M >= lambda_M M_L) by adding the difference to -j_vv.  This keeps
alpha M + A_i + M_L diag(s) positive definite.  The modified matrix is a W
matrix in the sense of W-methods, for which ROS2 stays second order; the
floor only acts at finite steps, since s_i is bounded while alpha grows as
the step shrinks.  Both the oracle and the CUDA path apply the same rule.
``w_shift`` (0 by default, a test hook) subtracts a constant from the (v, v)
entry of every node block, an h-independent W perturbation.

Elliptic constraint (Eq. (3.15), Sec. 2 Dirichlet part left unstated): u is
the solution of A_ie u = -A_i v with u[pin] = 0 (pin >= 0), or with zero
nodal mean (pin < 0); solved by eliminating the pinned row and column.

Bidomain-bath (Sec. 4, "Results for Bidomain-Bath"; the paper states no
equations for it): the tissue nodes, numbered first, carry X; u lives on all
nodes and solves A_ie u = -A_i v, where A_ie includes the bath stiffness and
A_i vanishes outside the tissue (see ``fem.py``).  The parabolic and ODE rows
are those above, restricted to the tissue nodes, with u taken there.

Adaptive step (Sec. 3.3.2: the embedded X_hat "determines the future step";
Sec. 4 runs use a maximum step of 0.05 ms): ``run_adaptive`` below.

Stimulus: I_stim,i = sum over stimuli of amplitude * mask_i when
t_on <= t^n < t_on + duration (t^n = n tau, 1e-9 tau tolerance), constant
over the step.

Activation time: first upward crossing of v_act (default -30 mV) between two
steps, linearly interpolated; NaN if the node never crosses.

Pins (tests/test_oracle_bidomain.py): ROS2 closed form R(z); S integrates
polynomials of degree <= M-1 exactly; 0-D reduction against a fine RK4 /
Radau single-cell run with observed order 2; equal-anisotropy closed form
u = -v/(1 + lambda); observed temporal order ~2 with SDC and ~1 without
(Table 4.1's slopes); rest-state fixed point; u uniqueness; conduction
velocity against Sec. 4's biomarker table.
"""
from __future__ import annotations

import dataclasses
from typing import List, Optional, Sequence

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from . import fem

GAMMA = 1.0 + 1.0 / np.sqrt(2.0)


# ---------------------------------------------------------------------------
# quadrature
# ---------------------------------------------------------------------------

def lobatto_nodes(m: int) -> np.ndarray:
    """Gauss-Lobatto nodes on [0, 1]: {0, 1} for M = 2, {0, 1/2, 1} for M = 3."""
    if m == 2:
        return np.array([0.0, 1.0])
    if m == 3:
        return np.array([0.0, 0.5, 1.0])
    raise ValueError("n_sdc_nodes must be 2 or 3")


def integration_matrix(c: np.ndarray) -> np.ndarray:
    """S[m, j] = int_{c_m}^{c_{m+1}} l_j(s) ds for the Lagrange basis l_j on
    the nodes c (unit interval); exact integration of the interpolant."""
    M = len(c)
    S = np.zeros((M - 1, M))
    for j in range(M):
        others = [c[k] for k in range(M) if k != j]
        poly = np.poly1d(others, r=True) / np.prod([c[j] - o for o in others])
        P = np.polyint(poly)
        for m in range(M - 1):
            S[m, j] = P(c[m + 1]) - P(c[m])
    return S


def ros2_amplification(z):
    """Stability function of ROS2 on y' = lambda y, z = lambda h."""
    return (1.0 + (1.0 - 2.0 * GAMMA) * z) / (1.0 - GAMMA * z) ** 2


# ---------------------------------------------------------------------------
# problem
# ---------------------------------------------------------------------------

@dataclasses.dataclass
class Stim:
    mask: np.ndarray
    t_on: float
    duration: float
    amplitude: float


class Bidomain:
    """Discrete bidomain problem on a P1 mesh (oracle)."""

    def __init__(self, xyz, elems, fibers, sigma, chi, cm, cell, stimuli: Sequence = (),
                 pin_node: int = 0, mass_lumped: bool = False, elem_bath=None,
                 sigma_b: float = 0.0):
        ops = fem.assemble(np.asarray(xyz, np.float64), np.asarray(elems),
                           np.asarray(fibers, np.float64), sigma, chi, cm, elem_bath, sigma_b)
        # tissue nodes (those of tissue elements) are numbered first: v and the
        # membrane state live on them, u on all nodes (bidomain-bath, Sec. 4)
        self.N_all = xyz.shape[0]
        NT = self.N_all
        if elem_bath is not None:
            tis = np.zeros(self.N_all, dtype=bool)
            tis[np.asarray(elems)[np.asarray(elem_bath) == 0].ravel()] = True
            NT = int(tis.sum())
            if not np.all(tis[:NT]):
                raise ValueError("tissue nodes must be numbered before bath nodes")
        self.A_i_rect = ops.A_i[:, :NT].tocsr()         # -A_i v on every node (elliptic rhs)
        self.ops = fem.Operators(A_i=ops.A_i[:NT, :NT].tocsr(), A_ie=ops.A_ie,
                                 M=ops.M[:NT, :NT].tocsr(), M_L=ops.M_L[:NT].copy())
        self.cell = cell
        self.cm = float(cm)
        self.N = NT
        self.ns = cell.ns
        self.dim = xyz.shape[1]
        self.mass_lumped = mass_lumped
        self.M_v = sp.diags(self.ops.M_L).tocsr() if mass_lumped else self.ops.M
        self.lambda_M = 1.0 if mass_lumped else (0.25 if self.dim == 2 else 0.2)
        self.stimuli = [Stim(np.asarray(s.mask), float(s.t_on), float(s.duration),
                             float(s.amplitude)) for s in stimuli]
        self.pin = pin_node
        keep = np.ones(self.N_all, dtype=bool)
        self.pin_row = pin_node if pin_node >= 0 else 0
        keep[self.pin_row] = False
        self.keep = keep
        self.ell_lu = spla.splu(self.ops.A_ie[keep][:, keep].tocsc())
        self.spd_margin = 0.9      # floor factor of the condensed diagonal (0 disables)
        self.w_shift = 0.0         # test hook: W_vv = J_vv - w_shift
        self.clamp_count = 0
        self.adaptive_tol = 0.0    # > 0: step() records the embedded error estimate
        self.last_err = 0.0

    # -- data ----------------------------------------------------------------
    def i_stim(self, t: float, dt: float) -> np.ndarray:
        out = np.zeros(self.N)
        eps = 1e-9 * dt
        for s in self.stimuli:
            if (t - s.t_on) > -eps and (t - s.t_on - s.duration) < -eps:
                out += s.amplitude * s.mask[:self.N]
        return out

    def Mt(self, X: np.ndarray) -> np.ndarray:
        out = np.empty_like(X)
        out[0] = self.M_v @ X[0]
        out[1:] = self.ops.M_L[None, :] * X[1:]
        return out

    def F(self, X: np.ndarray, u: np.ndarray, istim: np.ndarray) -> np.ndarray:
        """F(X, u) of Eq. (3.11)."""
        f = self.cell.field(X, istim, self.cm).real
        out = np.empty_like(X)
        out[0] = -(self.ops.A_i @ (X[0] + u[:self.N])) + self.ops.M_L * f[0]
        out[1:] = self.ops.M_L[None, :] * f[1:]
        return out

    # -- elliptic constraint ---------------------------------------------------
    def elliptic(self, v: np.ndarray) -> np.ndarray:
        """u with A_ie u = -A_i v and u[pin] = 0 (or zero mean if pin < 0);
        u on every node (tissue and bath), v on the tissue nodes."""
        b = -(self.A_i_rect @ v)
        u = np.zeros(self.N_all)
        u[self.keep] = self.ell_lu.solve(b[self.keep])
        if self.pin < 0:
            u -= u.mean()
        return u

    # -- W matrix and shifted solves -----------------------------------------
    def node_blocks(self, X: np.ndarray, istim: np.ndarray, alpha: float) -> np.ndarray:
        """Exact node Jacobian df/dX [ns, ns, N] with the Schur-complement
        safeguard applied to the (v, v) entry for the shift alpha."""
        j = self.cell.jacobian(X, istim, self.cm)
        n1 = self.ns - 1
        A = alpha * np.eye(n1)[:, :, None] - j[1:, 1:, :]
        A_b = np.transpose(A, (2, 0, 1))
        w = np.linalg.solve(A_b, np.transpose(j[1:, 0:1, :], (2, 0, 1)))[:, :, 0]  # [N, n1]
        s = -j[0, 0, :] - np.einsum("kn,nk->n", j[0, 1:, :], w)
        if self.spd_margin > 0.0:
            s_min = -self.spd_margin * alpha * self.lambda_M
            clamp = s < s_min
            self.clamp_count += int(clamp.sum())
            j[0, 0, :] -= np.where(clamp, s_min - s, 0.0)
        j[0, 0, :] -= self.w_shift
        return j

    def shifted_solve(self, alpha: float, j: np.ndarray, rhs: np.ndarray) -> np.ndarray:
        """Solve (alpha Mt - W) k = rhs, W = [[-A_i, 0], [0, 0]] + M_L * j,
        as one sparse system over all ns*N unknowns (state-major order)."""
        N, ns = self.N, self.ns
        ML = self.ops.M_L
        blocks = [[None] * ns for _ in range(ns)]
        for a in range(ns):
            for b in range(ns):
                d = -ML * j[a, b, :]
                if a == b:
                    d = d + alpha * ML
                if a == 0 and b == 0:
                    blocks[a][b] = (alpha * self.M_v + self.ops.A_i + sp.diags(-ML * j[0, 0, :])).tocsr()
                elif np.any(d != 0.0):
                    blocks[a][b] = sp.diags(d)
        for a in range(ns):
            if blocks[a][a] is None:
                blocks[a][a] = sp.csr_matrix((N, N))
        A = sp.bmat(blocks, format="csc")
        x = spla.spsolve(A, rhs.reshape(-1))
        return np.asarray(x).reshape(ns, N)

    # -- ROS2 ----------------------------------------------------------------
    def ros2(self, X: np.ndarray, h: float, u: np.ndarray, istim: np.ndarray) -> np.ndarray:
        alpha = 1.0 / (GAMMA * h)
        j = self.node_blocks(X, istim, alpha)
        k1 = self.shifted_solve(alpha, j, self.F(X, u, istim))
        r2 = self.F(X + k1 / GAMMA, u, istim) - (2.0 / (GAMMA * h)) * self.Mt(k1)
        k2 = self.shifted_solve(alpha, j, r2)
        X_new = X + (1.5 / GAMMA) * k1 + (0.5 / GAMMA) * k2
        # embedded first-order solution X_hat = X + m_hat . k, m_hat = (1/gamma, 0)
        # (Eq. (3.14)); its distance from X_new is the local error estimate
        self.last_embedded = X + k1 / GAMMA
        return X_new

    # -- one time step (Algorithm 2) -----------------------------------------
    def step(self, X: np.ndarray, u_n: np.ndarray, t: float, dt: float,
             n_sdc_nodes: int = 3, n_sweeps: int = 2, correction: bool = True,
             sweep_tol: float = 0.0):
        c = lobatto_nodes(n_sdc_nodes)
        M = len(c)
        S = dt * integration_matrix(c)
        dts = dt * np.diff(c)
        istim = self.i_stim(t, dt)
        Xk = [X.copy() for _ in range(M)]
        u: List[Optional[np.ndarray]] = [u_n] + [None] * (M - 1)
        sweeps = 0
        for k in range(n_sweeps):
            sweeps += 1
            for m in range(1, M):
                u[m] = self.elliptic(Xk[m][0])
            Xt = [X]
            err = 0.0
            for m in range(M - 1):
                Xt.append(self.ros2(Xt[m], dts[m], u[m + 1], istim))
                if self.adaptive_tol > 0.0:
                    E = np.abs(Xt[m + 1] - self.last_embedded)
                    err = max(err, float(np.max(E / (self.adaptive_tol * (1.0 + np.abs(Xt[m + 1]))))))
            self.last_err = err
            if correction:
                Fq = [self.F(Xt[jn], u[jn], istim) for jn in range(M)]
                new = [X]
                for m in range(M - 1):
                    R = self.Mt(new[m] - Xt[m + 1]) + sum(S[m, jn] * Fq[jn] for jn in range(M))
                    alpha = 1.0 / dts[m]
                    jb = self.node_blocks(Xt[m + 1], istim, alpha)
                    eps = self.shifted_solve(alpha, jb, R / dts[m])
                    new.append(Xt[m + 1] + eps)
            else:
                new = Xt
            delta = float(np.max(np.abs(new[M - 1] - Xk[M - 1])))
            Xk = new
            if sweep_tol > 0.0 and delta < sweep_tol:
                break
        return Xk[M - 1], u[M - 1], sweeps


# ---------------------------------------------------------------------------
# driver and biomarkers
# ---------------------------------------------------------------------------

def activation_update(t_act: np.ndarray, v_old: np.ndarray, v_new: np.ndarray,
                      t_old: float, dt: float, v_act: float = -30.0) -> None:
    """First upward crossing of v_act inside (t_old, t_old + dt], linearly
    interpolated; only nodes without an activation time are updated."""
    cross = np.isnan(t_act) & (v_old < v_act) & (v_new >= v_act)
    frac = (v_act - v_old[cross]) / (v_new[cross] - v_old[cross])
    t_act[cross] = t_old + frac * dt


def run(problem: Bidomain, X0: np.ndarray, n_steps: int, dt: float, n_sdc_nodes: int = 3,
        n_sweeps: int = 2, correction: bool = True, u0: Optional[np.ndarray] = None,
        v_act: float = -30.0, callback=None):
    """March n_steps steps from X0 (u0 = 0 if not given); returns
    (X, u, activation_times)."""
    X = np.array(X0, dtype=np.float64, copy=True)
    u = np.zeros(problem.N_all) if u0 is None else np.array(u0, dtype=np.float64)
    t_act = np.full(problem.N, np.nan)
    for n in range(n_steps):
        t = n * dt
        Xn, un, _ = problem.step(X, u, t, dt, n_sdc_nodes, n_sweeps, correction)
        activation_update(t_act, X[0], Xn[0], t, dt, v_act)
        X, u = Xn, un
        if callback is not None:
            callback(n + 1, X, u)
    return X, u, t_act


# ---------------------------------------------------------------------------
# adaptive time step from the embedded ROS2 solution (Sec. 3.3.2, Eq. (3.14))
# ---------------------------------------------------------------------------
#
# Reading (the paper states only that the second solution "determines the
# future time step", with a maximum step of 0.05 ms in its reentry runs):
#   error   err = max over the last sweep's ROS2 sub-steps, nodes and state
#           variables of |X_new - X_hat| / (tol (1 + |X_new|))
#   accept  err <= 1 (or the smallest step of the ladder is reached)
#   next    dt * min(2, max(0.5, 0.9 err^(-1/2))) (the embedded solution is of
#           order 1), rounded down to the ladder dt_max 2^-k, k = 0..ladder-1
#   reject  err > 1: the step is repeated from X^n with the step so chosen
#           (at least one rung smaller)

def ladder_step(dt_max: float, dt_want: float, ladder: int) -> float:
    """Largest dt_max 2^-k (k < ladder) not above dt_want (the smallest rung
    if none is)."""
    for k in range(ladder):
        d = dt_max * 0.5 ** k
        if d <= dt_want * (1.0 + 1e-12):
            return d
    return dt_max * 0.5 ** (ladder - 1)


def controller_factor(err: float) -> float:
    if err <= 0.0:
        return 2.0
    return min(2.0, max(0.5, 0.9 * err ** -0.5))


def run_adaptive(problem: Bidomain, X0: np.ndarray, n_steps: int, dt_max: float, tol: float,
                 n_sdc_nodes: int = 3, n_sweeps: int = 2, ladder: int = 8, v_act: float = -30.0):
    """n_steps accepted adaptive steps from X0 (u0 = 0); returns
    (X, u, t, activation_times, accepted dts, rejections)."""
    X = np.array(X0, dtype=np.float64, copy=True)
    u = np.zeros(problem.N_all)
    t = 0.0
    t_act = np.full(problem.N, np.nan)
    dt = dt_max
    dts, rejected = [], 0
    problem.adaptive_tol = tol
    for _ in range(n_steps):
        while True:
            Xn, un, _ = problem.step(X, u, t, dt, n_sdc_nodes, n_sweeps, True)
            err = problem.last_err
            smallest = dt <= dt_max * 0.5 ** (ladder - 1) * (1.0 + 1e-12)
            if err <= 1.0 or smallest:
                break
            rejected += 1
            dt = min(ladder_step(dt_max, dt * controller_factor(err), ladder), dt * 0.5)
        activation_update(t_act, X[0], Xn[0], t, dt, v_act)
        X, u = Xn, un
        t = t + dt
        dts.append(dt)
        dt = ladder_step(dt_max, min(dt_max, dt * controller_factor(err)), ladder)
    problem.adaptive_tol = 0.0
    return X, u, t, t_act, dts, rejected


def conduction_velocity(xyz: np.ndarray, t_act: np.ndarray, y_line: float,
                        x_min: float, tol: float = 1e-9) -> float:
    """Least-squares slope of distance over activation time along the line
    y = y_line for activated nodes with x > x_min (cm/ms)."""
    sel = (np.abs(xyz[:, 1] - y_line) < tol) & (xyz[:, 0] > x_min) & ~np.isnan(t_act)
    x = xyz[sel, 0]
    t = t_act[sel]
    A = np.stack([t, np.ones_like(t)], axis=1)
    slope = np.linalg.lstsq(A, x, rcond=None)[0][0]
    return float(slope)
