"""Batched steps (bd_batch_step): many independent simulations advanced by one
launch per phase over their concatenated nodes -- node-wise kernels over all
tissue nodes, every elliptic and parabolic solve one batched streaming solve
with per-simulation reductions, scalars, stopping tests and iteration caps --
captured as one graph per step shape.

A simulation's arithmetic in a batch does not depend on its companions: it
gives the same bits stepped alone (a batch of one) and in any batch.  Against
the oracle each member meets the FP64 gate (1e-9) and, mixed, the stated
tolerance (1e-3)."""
import numpy as np
import pytest

from gpu_util import gpu_sim, oracle_problem, rel, rest_X
from oracle import bidomain as OB
from paper_2510_27447_gb300 import binding
from paper_2510_27447_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def _sheets(model, sides, steps, dt=0.02):
    # 33^2 = 1,089 rows solve with Jacobi, larger sheets with the AMG
    # hierarchy: the batches mix both
    return [W.sheet(n, 0.02 * (n - 1) / 2, model, dt, steps, strip=0.06) for n in sides]


def _run(ws, batches, steps, **opt):
    sims = [gpu_sim(w, **opt) for w in ws]
    for s, w in zip(sims, ws):
        s.set_initial(rest_X(w))
    for _ in range(steps):
        for b in batches:
            binding.batch_step([sims[i] for i in b], ws[0].dt, 3, 2)
    out = [s.fields(full=True) + (s.activation_times(), s.stats()) for s in sims]
    for s in sims:
        s.close()
    return out


@pytest.mark.parametrize("prec", [binding.MIXED, binding.FP64])
def test_member_gives_the_same_bits_alone_and_batched(prec):
    ws = _sheets(W.TP06_EPI, (33, 41, 25, 57), 6)
    alone = _run(ws, [[0], [1], [2], [3]], 6, precision=prec)
    together = _run(ws, [[0, 1, 2, 3]], 6, precision=prec)
    regrouped = _run(ws, [[3, 1], [2, 0]], 6, precision=prec)
    for a, b, c in zip(alone, together, regrouped):
        for k in range(4):          # v, u, X, activation times
            assert np.array_equal(a[k], b[k], equal_nan=True)
            assert np.array_equal(a[k], c[k], equal_nan=True)
    assert together[1][4]["amg_levels"] >= 1 and together[0][4]["amg_levels"] == 0


def test_batched_fp64_members_match_oracle():
    ws = _sheets(W.LR91, (33, 41, 21), 10)
    got = _run(ws, [[0, 1, 2]], 10, cg_tol_e=1e-13, cg_tol_p=1e-13)
    for w, (v, u, X, ta, st) in zip(ws, got):
        Xo, uo, to = OB.run(oracle_problem(w), rest_X(w), w.n_steps, w.dt, 3, 2)
        assert rel(X, Xo) < 1e-9
        assert rel(u, uo) < 1e-9
        act = ~np.isnan(to)
        np.testing.assert_array_equal(np.isnan(ta), ~act)
        np.testing.assert_allclose(ta[act], to[act], atol=1e-6)
        assert st["steps"] == w.n_steps


def test_batched_mixed_members_within_tolerance():
    ws = _sheets(W.TP06_EPI, (41, 25, 33), 15)
    got = _run(ws, [[0, 1, 2]], 15, precision=binding.MIXED)
    for w, (v, u, X, ta, st) in zip(ws, got):
        Xo, uo, _ = OB.run(oracle_problem(w), rest_X(w), w.n_steps, w.dt, 3, 2)
        assert rel(v, Xo[0]) < 1e-3
        assert rel(u, uo) < 1e-3


def test_batch_with_a_bath_member_matches_oracle():
    wb = W.bath_sheet(24, -0.25, 1.25, 0.0, 1.0, W.LR91_PAPER_MOD, 0.05, 6, strip=0.1, s1_amp=80.0, s1_dur=1.0)
    ws = W.sheet(21, 0.2, W.LR91_PAPER_MOD, 0.05, 6, strip=0.06)
    sims = [gpu_sim(w, cg_tol_e=1e-12, cg_tol_p=1e-13) for w in (wb, ws)]
    for s, w in zip(sims, (wb, ws)):
        s.set_initial(rest_X(w))
    for _ in range(6):
        binding.batch_step(sims, 0.05, 3, 2)
    for s, w in zip(sims, (wb, ws)):
        v, u, X = s.fields(full=True)
        Xo, uo, _ = OB.run(oracle_problem(w), rest_X(w), 6, 0.05, 3, 2)
        assert rel(X, Xo) < 1e-9 and rel(u, uo) < 1e-8
        s.close()


def test_batch_rejects_mixed_models_and_sweep_tests():
    a = gpu_sim(W.sheet(9, 0.1, W.LR91, 0.02, 1))
    b = gpu_sim(W.sheet(9, 0.1, W.TP06_EPI, 0.02, 1))
    c = gpu_sim(W.sheet(9, 0.1, W.LR91, 0.02, 1), sweep_tol=1e-3)
    for pair in ([a, b], [a, c], [a, a]):
        with pytest.raises(binding.BdError) as e:
            binding.batch_step(pair, 0.02, 3, 2)
        assert e.value.code == -1
    for s in (a, b, c):
        s.close()
