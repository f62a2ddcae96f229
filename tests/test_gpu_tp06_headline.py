"""Parity of the headline configuration's model and solver path: TP06
epicardial on a 65 x 65 sheet at the bench sheet's spacing (h = 2.5/256 cm),
14 ms from the published initial state through the upstroke under the S1
strip, the front crossing the sheet and the start of the plateau behind it
(Sec. 3.3.2, Algorithm 2 with 3 Gauss-Lobatto nodes and 2 sweeps).

At 4,225 rows the elliptic solve runs with its AMG hierarchy (more rows than
the dense coarse level holds), in the 512-thread register tier, and on the
mixed path the second sweep's two elliptic solves run in the two-RHS kernel:
the solver path the bench times on the 257 x 257 sheet.

The expected values in tests/golden/tp06_sheet65_14ms.npz were written by
tests/golden/make_tp06_sheet65.py, which calls only the oracle.  Gates:
FP64 within 1e-9 relative L2 in v, u and the whole state (CG tolerances of
1e-13 on the GPU, direct solves in the oracle); mixed within the stated
tolerances -- 1e-3 relative L2 in v and u, activation times within 0.1 ms,
conduction velocity within 1 %.
"""
import os
import sys

import numpy as np
import pytest

from gpu_util import rel
from oracle import bidomain as OB
from paper_2510_27447_gb300 import binding

pytestmark = pytest.mark.gpu

HERE = os.path.dirname(os.path.abspath(__file__))
GOLDEN = os.path.join(HERE, "golden", "tp06_sheet65_14ms.npz")
sys.path.insert(0, os.path.join(HERE, "golden"))
import make_tp06_sheet65 as G  # noqa: E402


def _run(precision, **opt):
    ref = np.load(GOLDEN)
    w = G.workload()
    sim = binding.simulation_from_workload(w, binding.default_options(precision=precision, pin_node=0, **opt))
    st = sim.stats()
    assert st["amg_levels"] >= 1 and st["solver_tier"] == 1, st
    sim.set_initial(ref["X0"])
    for _ in range(G.SNAP):
        sim.step(G.DT, 3, 2)
    snap = sim.fields(full=True)
    for _ in range(G.STEPS - G.SNAP):
        sim.step(G.DT, 3, 2)
    v, u, X = sim.fields(full=True)
    ta = sim.activation_times()
    sim.close()
    return ref, w, snap, (v, u, X), ta


def test_tp06_sheet_fp64_matches_oracle_through_upstroke_and_plateau():
    ref, w, (v2, u2, X2), (v, u, X), ta = _run(binding.FP64, cg_tol_e=1e-13, cg_tol_p=1e-13)
    assert rel(X2, ref["X_2ms"]) < 1e-9 and rel(u2, ref["u_2ms"]) < 1e-9
    assert rel(v, ref["X"][0]) < 1e-9
    assert rel(u, ref["u"]) < 1e-9
    assert rel(X, ref["X"]) < 1e-9
    act = ~np.isnan(ref["t_act"])
    assert act.mean() > 0.9             # the front has crossed the sheet
    np.testing.assert_array_equal(np.isnan(ta), ~act)
    np.testing.assert_allclose(ta[act], ref["t_act"][act], atol=1e-6)


def test_tp06_sheet_mixed_meets_stated_tolerances():
    ref, w, (v2, u2, _), (v, u, X), ta = _run(binding.MIXED)
    assert rel(v2, ref["X_2ms"][0]) < 1e-3 and rel(u2, ref["u_2ms"]) < 1e-3
    assert rel(v, ref["X"][0]) < 1e-3
    assert rel(u, ref["u"]) < 1e-3
    act = ~np.isnan(ref["t_act"])
    np.testing.assert_array_equal(np.isnan(ta), ~act)
    assert np.max(np.abs(ta[act] - ref["t_act"][act])) < 0.1
    L = G.H * (G.SIDE - 1)
    cv = OB.conduction_velocity(w.xyz, ta, L / 2, 0.3)
    cv_ref = OB.conduction_velocity(w.xyz, ref["t_act"], L / 2, 0.3)
    assert abs(cv - cv_ref) / cv_ref < 0.01
