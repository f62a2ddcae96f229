"""Decoupled CN-RK2 strategy (oracle): the paper's reference decoupled scheme.

Test infrastructure only (see the package docstring).

Sec. 3.3.3 (Strang splitting, Crank-Nicolson diffusion, second-order
Runge-Kutta reaction), one step t^n -> t^n + dt:
  1. reaction half step: the node ODE system dX/dt = f(X) over dt/2 with the
     explicit midpoint rule, X* = X^n + (dt/2) f(X^n + (dt/4) f(X^n));
  2. diffusion: one Crank-Nicolson step of M dv/dt = -A_i (v + u^n),
     (M + dt/2 A_i) v** = (M - dt/2 A_i) v* - dt A_i u^n, the other states
     unchanged;
  3. reaction half step from (v**, y*) as in 1, giving X^{n+1};
  4. elliptic constraint A_ie u^{n+1} = -A_i v^{n+1}.

Readings (the printed equations carry typos):
  * the reaction sub-steps are node-local ODE steps: the mass matrix written
    beside I_ion cancels against the mass-weighted reaction term of the
    semi-discrete system (Eqs. (3.6)-(3.9));
  * the "+" between the gate and concentration arguments is a ","; all
    states are advanced together by the midpoint rule;
  * the stimulus enters the reaction sub-steps through the node field f
    (constant over the step, as in the partitioned step), not the diffusion
    step where the paper prints it: the TP06 model carries the stimulus in
    dK_i/dt too, which only the reaction sub-steps see.  Both placements are
    consistent to second order.
  * M in step 2 is the parabolic mass M_v of ``bidomain.Bidomain`` (the
    consistent M, or M_L with ``mass_lumped``).
Each linear system is solved with a sparse direct factorisation.

Pins (tests/test_oracle_decoupled.py): the 0-D reduction converges to the
single-cell reference at order 2; on a reaction-free problem with an
infinitely conducting extracellular space each generalised eigenmode of
(A_i, M) is multiplied by the Crank-Nicolson factor (1 - z/2)/(1 + z/2),
z = dt mu; the conduction velocity agrees with the partitioned SDC step.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse.linalg as spla

from .bidomain import Bidomain, activation_update


def reaction_half_step(problem: Bidomain, X: np.ndarray, istim: np.ndarray, dt: float) -> np.ndarray:
    """Explicit midpoint rule over dt/2 on every node's ODE system."""
    h = 0.5 * dt
    f1 = problem.cell.field(X, istim, problem.cm).real
    f2 = problem.cell.field(X + 0.5 * h * f1, istim, problem.cm).real
    return X + h * f2


def cnrk2_step(problem: Bidomain, X: np.ndarray, u_n: np.ndarray, t: float, dt: float):
    """One CN-RK2 step; returns (X^{n+1}, u^{n+1})."""
    istim = problem.i_stim(t, dt)
    Xs = reaction_half_step(problem, X, istim, dt)
    A, Mv = problem.ops.A_i, problem.M_v
    lhs = (Mv + 0.5 * dt * A).tocsc()
    rhs = Mv @ Xs[0] - 0.5 * dt * (A @ Xs[0]) - dt * (A @ u_n[:problem.N])
    Xss = Xs.copy()
    Xss[0] = spla.spsolve(lhs, rhs)
    Xn1 = reaction_half_step(problem, Xss, istim, dt)
    return Xn1, problem.elliptic(Xn1[0])


def run_cnrk2(problem: Bidomain, X0: np.ndarray, n_steps: int, dt: float, v_act: float = -30.0):
    """March n_steps CN-RK2 steps from X0 with u = 0; returns (X, u, t_act)."""
    X = np.array(X0, dtype=np.float64, copy=True)
    u = np.zeros(problem.N_all)
    t_act = np.full(problem.N, np.nan)
    for n in range(n_steps):
        Xn, u = cnrk2_step(problem, X, u, n * dt, dt)
        activation_update(t_act, X[0], Xn[0], n * dt, dt, v_act)
        X = Xn
    return X, u, t_act
