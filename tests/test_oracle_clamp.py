"""Pins of the oracle's W-matrix safeguard (Sec. 3.3.2, the condensed
parabolic system; the floor on the condensed diagonal is a reading, see the
oracle's module docstring).

The safeguard raises the Schur complement s_i of a node block onto v to at
least -margin alpha lambda_M.  Its two ingredients are pinned independently:
  * lambda_M is the mass bound M >= lambda_M M_L, i.e. the smallest
    generalised eigenvalue of (M, M_L): 1/4 for P1 triangles, 1/5 for P1
    tetrahedra, 1 for the lumped mass.  A wrong constant (say 1/3 or 1/6)
    fails the single-element equality or the assembled-mesh bound;
  * the clamp itself: after it, the recomputed Schur complement equals the
    floor on the clamped nodes and the exact one elsewhere (a wrong sign
    doubles the distance instead of closing it), and the condensed matrix
    alpha M + A_i + M_L diag(s) is positive definite.
A run in which the clamp fires is the TP06 upstroke at the paper's largest
step (tau = 0.05 ms) with the two-node trapezoidal correction of
Eq. (3.20).  The modified matrix is a W matrix: ROS2 keeps its second order
for a W that differs from the exact Jacobian, which the last test observes on
the 0-D reduction with an h-independent perturbation of the (v, v) entry.
"""
import numpy as np
import pytest
import scipy.linalg as sla
import scipy.sparse as sp

from oracle import bidomain as B
from oracle import fem
from oracle import lr91, tp06
from paper_2510_27447_gb300 import workloads as W

SIG = (3.0, 0.31, 2.0, 1.35)


def _mass_pair(xyz, elems):
    ops = fem.assemble(xyz, elems, W.fibers_along_x(len(elems), xyz.shape[1]), SIG, 2000.0, 1.0)
    return ops.M.toarray(), ops.M_L


@pytest.mark.parametrize("dim", [2, 3])
def test_lambda_m_is_the_mass_bound(dim):
    if dim == 2:
        one = (np.array([[0.0, 0.0], [1.0, 0.2], [0.3, 0.9]]), np.array([[0, 1, 2]]))
        mesh = W.square_grid(7, 1.0)
        want = 0.25
    else:
        one = (np.array([[0.0, 0.0, 0.0], [1.0, 0.1, 0.0], [0.2, 0.8, 0.1], [0.1, 0.3, 0.7]]),
               np.array([[0, 1, 2, 3]]))
        mesh = W.slab_grid(4, 4, 3, 1.0, 1.0, 0.5)
        want = 0.2
    P = B.Bidomain(mesh[0], mesh[1], W.fibers_along_x(len(mesh[1]), dim), SIG, 2000.0, 1.0,
                   lr91.model(), [])
    assert P.lambda_M == want
    M, ML = _mass_pair(*one)
    ev = sla.eigh(M, np.diag(ML), eigvals_only=True)
    assert ev.min() == pytest.approx(want, rel=1e-12)      # attained on one element
    assert ev.max() == pytest.approx(1.0, rel=1e-12)
    M, ML = _mass_pair(*mesh)
    ev = sla.eigh(M, np.diag(ML), eigvals_only=True)
    assert ev.min() >= want * (1 - 1e-12)                  # holds after assembly
    assert ev.min() < want + 0.05                          # and is nearly tight
    Pl = B.Bidomain(mesh[0], mesh[1], W.fibers_along_x(len(mesh[1]), dim), SIG, 2000.0, 1.0,
                    lr91.model(), [], mass_lumped=True)
    assert Pl.lambda_M == 1.0


def _tp06_upstroke(steps, dt=0.05, M=2):
    cellm = tp06.model()
    xyz, tri = W.square_grid(9, 0.3)
    P = B.Bidomain(xyz, tri, W.fibers_along_x(len(tri), 2), SIG, 2000.0, 1.0, cellm,
                   [B.Stim(W.nodes_x_below(xyz, 0.06), 0.0, 1.0, 80.0)])
    X = np.repeat(cellm.initial()[:, None], P.N, axis=1)
    u = np.zeros(P.N)
    counts = []
    for n in range(steps):
        X, u, _ = P.step(X, u, n * dt, dt, M, 2)
        counts.append(P.clamp_count)
    return P, X, u, counts


def test_clamp_fires_on_the_tp06_upstroke_at_the_largest_step():
    P, X, u, counts = _tp06_upstroke(40)
    assert P.clamp_count > 0
    assert np.all(np.isfinite(X)) and X[0].max() > 0.0
    # the same run at tau = 0.02 ms with three Lobatto nodes never needs it
    P2, _, _, _ = _tp06_upstroke(100, dt=0.02, M=3)
    assert P2.clamp_count == 0


def _schur(j, alpha):
    n1 = j.shape[0] - 1
    A = np.transpose(alpha * np.eye(n1)[:, :, None] - j[1:, 1:, :], (2, 0, 1))
    w = np.linalg.solve(A, np.transpose(j[1:, 0:1, :], (2, 0, 1)))[:, :, 0]
    return -j[0, 0, :] - np.einsum("kn,nk->n", j[0, 1:, :], w)


def test_clamped_schur_complement_sits_on_the_floor_and_the_matrix_is_spd():
    P, _, _, counts = _tp06_upstroke(40)
    first = int(np.argmax(np.array(counts) > 0))       # first step with a clamp
    P, X, u, _ = _tp06_upstroke(first)                 # the state entering it
    dt = 0.05
    alpha = 1.0 / (B.GAMMA * dt)
    istim = P.i_stim(first * dt, dt)
    j_exact = P.cell.jacobian(X, istim, P.cm)
    s_exact = _schur(j_exact, alpha)
    floor = -P.spd_margin * alpha * P.lambda_M
    before = P.clamp_count
    j = P.node_blocks(X, istim, alpha)
    hit = s_exact < floor
    assert hit.any() and P.clamp_count - before == int(hit.sum())
    s = _schur(j, alpha)
    np.testing.assert_allclose(s[hit], floor, rtol=1e-9)
    np.testing.assert_array_equal(s[~hit], s_exact[~hit])
    np.testing.assert_array_equal(j[:, 1:], j_exact[:, 1:])      # only the (v, v) entry moves
    np.testing.assert_array_equal(j[1:, 0], j_exact[1:, 0])
    K = (alpha * P.M_v + P.ops.A_i + sp.diags(P.ops.M_L * s)).toarray()
    np.linalg.cholesky(0.5 * (K + K.T))                          # positive definite
    assert np.linalg.eigvalsh(alpha * P.M_v.toarray() + np.diag(P.ops.M_L * s)).min() > 0.0


@pytest.mark.parametrize("shift", [2.0, -2.0])
def test_ros2_stays_second_order_with_a_perturbed_w(shift):
    """0-D reduction (uniform state: u = 0, every node is the single cell),
    Algorithm 1 with one sweep: the step is ROS2 alone.  With
    W_vv = J_vv - shift the local errors change but the order stays 2."""
    from test_oracle_bidomain import _problem, _single_cell_reference
    cellm = lr91.model(True)
    x0 = cellm.rest_state()
    t_end, amp, dur = 2.0, 20.0, 1.0
    ref = _single_cell_reference(cellm, x0, t_end, amp, dur)

    def errs(ws):
        out = []
        for dt in (0.05, 0.025, 0.0125):
            P = _problem(cellm, n=2, stim=[B.Stim(np.ones(4, np.uint8), 0.0, dur, amp)])
            P.w_shift = ws
            X0 = np.repeat(x0[:, None], P.N, axis=1)
            X, _, _ = B.run(P, X0, int(round(t_end / dt)), dt, 2, 1, False)
            out.append(abs(X[0, 0] - ref[0]))
        return np.array(out)
    e = errs(shift)
    e0 = errs(0.0)
    assert np.all(e > 10 * e0)                 # the perturbation is felt
    rates = np.log2(e[:-1] / e[1:])
    assert rates[-1] > 1.8 and rates[-1] < 2.3, rates
