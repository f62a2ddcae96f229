"""The W-matrix safeguard on the GPU (Sec. 3.3.2, condensed parabolic
system; the floor on the condensed diagonal is the reading the oracle's
docstring states): on the TP06 upstroke at the paper's largest step
(tau = 0.05 ms, two-node trapezoidal correction of Eq. (3.20)) the floor is
active on many nodes.  The FP64 GPU path must take the same clamps as the
oracle, node for node and step for step (the counters agree), and match its
states and u to 1e-10 relative L2."""
import numpy as np
import pytest

from gpu_util import gpu_sim, oracle_problem, rel
from oracle import bidomain as OB
from oracle import tp06 as OT
from paper_2510_27447_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("M", [2, 3])
def test_fp64_steps_with_active_clamps_match_oracle(M):
    dt = 0.05 if M == 2 else 0.1
    steps = 40 if M == 2 else 20
    w = W.sheet(9, 0.3, W.TP06_EPI, dt, steps, strip=0.06)
    X0 = np.repeat(OT.model().initial()[:, None], w.n_nodes, axis=1)
    P = oracle_problem(w)
    Xo, uo, to = OB.run(P, X0, steps, dt, M, 2)
    assert P.clamp_count > 0
    sim = gpu_sim(w, cg_tol_e=1e-13, cg_tol_p=1e-13)
    sim.set_initial(X0)
    for _ in range(steps):
        sim.step(dt, M, 2)
    v, u, X = sim.fields(full=True)
    st = sim.stats()
    sim.close()
    assert np.all(np.isfinite(X))
    assert st["spd_clamps"] == P.clamp_count, (st["spd_clamps"], P.clamp_count)
    assert rel(X, Xo) < 1e-10
    assert rel(u, uo) < 1e-10
