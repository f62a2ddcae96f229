"""Bidomain-bath coupling on the GPU (Sec. 4): operators, elliptic solves
over tissue + bath and whole partitioned-SDC steps against the FP64 oracle."""
import numpy as np
import pytest
import scipy.sparse as sp

from gpu_util import gpu_sim, oracle_problem, rel, rest_X
from oracle import bidomain as OB
from oracle import fem
from paper_2510_27447_gb300 import binding
from paper_2510_27447_gb300 import workloads as W

pytestmark = pytest.mark.gpu

TIGHT = dict(cg_tol_e=1e-13, cg_tol_p=1e-13)


def _small(model=W.LR91_PAPER_MOD, n_cells=24, dt=0.05, steps=12):
    # 625 nodes (289 tissue): several blocks of every kernel, ragged tails,
    # tissue rows whose columns reach into the bath
    return W.bath_sheet(n_cells, -0.25, 1.25, 0.0, 1.0, model, dt, steps, strip=0.1,
                        s1_amp=80.0, s1_dur=1.0)


def _v(w):
    x, y = w.xyz[:w.n_tissue, 0], w.xyz[:w.n_tissue, 1]
    return -80 + 100 * np.exp(-30 * ((x - 0.3) ** 2 + (y - 0.6) ** 2))


def test_bath_operators_match_oracle():
    w = _small()
    sim = gpu_sim(w)
    assert (sim.N, sim.NT) == (625, 289)
    ops = fem.assemble(w.xyz, w.elems, w.fibers, w.sigma, w.chi, w.cm, w.elem_bath, w.sbath)
    for which, ref in ((0, ops.A_i), (1, ops.A_ie), (2, ops.M)):
        rp, col, val = sim.operator(which)
        A = sp.csr_matrix((val, col, rp), shape=ref.shape).toarray()
        np.testing.assert_allclose(A, ref.toarray(), rtol=1e-13, atol=1e-15 * abs(ref).max())
    np.testing.assert_allclose(sim.operator(3), ops.M_L, rtol=1e-14, atol=0)
    sim.close()


@pytest.mark.parametrize("precond,n_cells", [(0, 24), (1, 96)])
def test_bath_elliptic_solve_matches_direct_solve(precond, n_cells):
    w = _small(n_cells=n_cells)
    v = _v(w)
    u_ref = oracle_problem(w).elliptic(v)
    sim = gpu_sim(w, cg_tol_e=1e-11, elliptic_precond=precond)
    u, it = sim.solve_elliptic(v)
    assert u.shape == (w.n_nodes,) and u[w.pin_node] == 0.0
    assert rel(u, u_ref) < 1e-9
    assert np.ptp(u[w.n_tissue:]) > 1e-3 * np.ptp(u)      # the bath carries a field
    sim.close()


@pytest.mark.parametrize("M,K", [(3, 2), (2, 1)])
def test_bath_steps_match_oracle(M, K):
    w = _small()
    X0 = rest_X(w)
    Xo, uo, to = OB.run(oracle_problem(w), X0, w.n_steps, w.dt, M, K)
    sim = gpu_sim(w, **TIGHT)
    sim.set_initial(X0)
    for _ in range(w.n_steps):
        sim.step(w.dt, M, K)
    v, u, X = sim.fields(full=True)
    ta = sim.activation_times()
    sim.close()
    assert X.shape == (8, w.n_tissue) and u.shape == (w.n_nodes,)
    assert X[0].max() > -20.0
    assert rel(X, Xo) < 1e-10 and rel(u, uo) < 1e-8
    np.testing.assert_array_equal(np.isnan(ta), np.isnan(to))
    np.testing.assert_allclose(ta[~np.isnan(ta)], to[~np.isnan(to)], atol=1e-9)


def test_bath_mixed_precision_within_tolerance():
    w = _small()
    X0 = rest_X(w)
    Xo, uo, _ = OB.run(oracle_problem(w), X0, w.n_steps, w.dt, 3, 2)
    sim = gpu_sim(w, precision=binding.MIXED)
    sim.set_initial(X0)
    for _ in range(w.n_steps):
        sim.step(w.dt)
    v, u = sim.fields()
    sim.close()
    assert rel(v, Xo[0]) < 1e-3 and rel(u, uo) < 1e-3


def test_bath_checkpoint_and_adaptive_step():
    w = _small()
    X0 = rest_X(w)
    a = gpu_sim(w)
    a.set_initial(X0)
    for _ in range(4):
        a.step_adaptive(0.05, 1e-2)
    blob = a.get_state()
    ref = [a.step_adaptive(0.05, 1e-2) for _ in range(4)]
    Xa = a.fields(full=True)
    a.close()
    b = gpu_sim(w)
    b.set_state(blob)
    got = [b.step_adaptive(0.05, 1e-2) for _ in range(4)]
    Xb = b.fields(full=True)
    b.close()
    assert got == ref
    for p, q in zip(Xa, Xb):
        np.testing.assert_array_equal(p, q)


def test_lv_shell_in_bath_matches_oracle():
    """The 3-D bidomain-bath geometry (truncated prolate LV shell, helical
    fibres, box bath) on a coarse jittered lattice: TP06 steps against the
    oracle, FP64 and mixed."""
    w = W.lv_shell_bath(h=0.35, n_steps=3)
    assert w.n_tissue < w.n_nodes and w.stimuli[0].mask.sum() > 0
    X0 = rest_X(w)
    Xo, uo, _ = OB.run(oracle_problem(w), X0, 3, w.dt, 3, 2)
    for prec, tx, tu in ((binding.FP64, 1e-10, 1e-8), (binding.MIXED, 1e-4, 1e-3)):
        sim = gpu_sim(w, precision=prec, **(TIGHT if prec == binding.FP64 else {}))
        sim.set_initial(X0)
        for _ in range(3):
            sim.step(w.dt)
        v, u, X = sim.fields(full=True)
        sim.close()
        assert rel(X, Xo) < tx and rel(u, uo) < tu, prec
