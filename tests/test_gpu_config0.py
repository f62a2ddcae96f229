"""FP64 parity gate on the 65 x 65 LR91 workload over 10 ms (500 steps).

The expected values in tests/golden/config0_10ms.npz were written by
tests/golden/make_config0.py, which calls only the oracle.  The GPU run uses
the same seeded inputs, the same initial state and CG tolerances of 1e-13,
and must match v and u to 1e-9 relative L2 and the activation times to
1e-6 ms.
"""
import os

import numpy as np
import pytest

from gpu_util import rel
from paper_2510_27447_gb300 import binding
from paper_2510_27447_gb300 import workloads as W

pytestmark = pytest.mark.gpu

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "config0_10ms.npz")


def test_config0_fp64_matches_oracle_over_10ms():
    ref = np.load(GOLDEN)
    w = W.config0()
    opts = binding.default_options(cg_tol_e=1e-13, cg_tol_p=1e-13, pin_node=0)
    sim = binding.simulation_from_workload(w, opts)
    sim.set_initial(ref["X0"])
    for _ in range(w.n_steps):
        sim.step(w.dt, w.n_sdc_nodes, w.n_sweeps)
    v, u, X = sim.fields(full=True)
    t_act = sim.activation_times()
    sim.close()
    assert rel(v, ref["X"][0]) < 1e-9
    assert rel(u, ref["u"]) < 1e-9
    assert rel(X, ref["X"]) < 1e-9
    act = ~np.isnan(ref["t_act"])
    assert act.sum() > 100            # the wave has crossed part of the sheet
    np.testing.assert_array_equal(np.isnan(t_act), ~act)
    np.testing.assert_allclose(t_act[act], ref["t_act"][act], atol=1e-6)
