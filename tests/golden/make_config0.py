"""Write tests/golden/config0_10ms.npz with the FP64 oracle (and nothing else).

Workload: LR91 (1991 parameters) on the unit square, 65 x 65 P1 nodes,
fibres along x, sigma_i = (3.0, 0.31), sigma_e = (2.0, 1.35) mS/cm,
chi = 2000 /cm, C_m = 1 uF/cm^2, S1 = 80 uA/cm^2 for 1 ms on x < 0.1,
tau = 0.02 ms for 500 steps (10 ms), 3 Gauss-Lobatto nodes, 2 sweeps,
u pinned at node 0, starting from the oracle's LR91 rest state.

Stored: X0 (initial state), X (state at 10 ms), u (extracellular potential
at 10 ms), t_act (activation times, NaN where not activated).
Run:  python tests/golden/make_config0.py
"""
import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

from oracle import bidomain as OB  # noqa: E402
from oracle import lr91 as OL  # noqa: E402
from paper_2510_27447_gb300 import workloads as W  # noqa: E402


def main():
    w = W.config0()
    cell = OL.model()
    P = OB.Bidomain(w.xyz, w.elems, w.fibers, w.sigma, w.chi, w.cm, cell, w.stimuli, pin_node=0)
    X0 = np.repeat(cell.rest_state()[:, None], w.n_nodes, axis=1)
    t0 = time.time()
    X, u, t_act = OB.run(P, X0, w.n_steps, w.dt, w.n_sdc_nodes, w.n_sweeps)
    out = os.path.join(os.path.dirname(os.path.abspath(__file__)), "config0_10ms.npz")
    np.savez_compressed(out, X0=X0, X=X, u=u, t_act=t_act)
    print(f"wrote {out} in {time.time() - t0:.0f} s; activated {np.sum(~np.isnan(t_act))} nodes")


if __name__ == "__main__":
    main()
