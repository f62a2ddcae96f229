"""Write tests/golden/tp06_sheet65_14ms.npz with the FP64 oracle (and nothing else).

Workload: the bench's TP06-epicardial sheet cut down to 65 x 65 P1 nodes at
the same spacing (h = 2.5/256 cm, a 0.625 cm square), fibres along x,
sigma_i = (3.0, 0.31), sigma_e = (2.0, 1.35) mS/cm, chi = 2000 /cm,
C_m = 1 uF/cm^2, S1 = 80 uA/cm^2 for 1 ms on x < 0.1 cm, tau = 0.02 ms for
700 steps (14 ms: the upstroke under the stimulus, the front crossing the
sheet and the start of the plateau behind it), 3 Gauss-Lobatto nodes,
2 sweeps, u pinned at node 0, from the published TP06 initial values.
At 4,225 rows the GPU elliptic solve uses its AMG preconditioner (more rows
than the dense coarse level holds) and, on the mixed path, the two-RHS
kernel of the second sweep: the headline configuration's solver path.

Stored: X0 (initial state), X_2ms / u_2ms (step 100), X / u (step 700),
t_act (activation times at -30 mV, NaN where not activated).
Run:  python tests/golden/make_tp06_sheet65.py      (about 45 min, one core)
"""
import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

from oracle import bidomain as OB  # noqa: E402
from oracle import tp06 as OT  # noqa: E402
from paper_2510_27447_gb300 import workloads as W  # noqa: E402

SIDE, H, DT, STEPS, SNAP = 65, 2.5 / 256, 0.02, 700, 100


def workload():
    return W.sheet(SIDE, H * (SIDE - 1), W.TP06_EPI, DT, STEPS, name="tp06_sheet_65x65")


def main():
    w = workload()
    cell = OT.model()
    P = OB.Bidomain(w.xyz, w.elems, w.fibers, w.sigma, w.chi, w.cm, cell, w.stimuli, pin_node=0)
    X0 = np.repeat(cell.initial()[:, None], w.n_nodes, axis=1)
    snap = {}

    def keep(n, X, u):
        if n == SNAP:
            snap["X_2ms"], snap["u_2ms"] = X.copy(), u.copy()
        if n % 50 == 0:
            print(f"step {n}: v in [{X[0].min():.1f}, {X[0].max():.1f}]", flush=True)

    t0 = time.time()
    X, u, t_act = OB.run(P, X0, STEPS, DT, 3, 2, callback=keep)
    out = os.path.join(os.path.dirname(os.path.abspath(__file__)), "tp06_sheet65_14ms.npz")
    np.savez_compressed(out, X0=X0, X=X, u=u, t_act=t_act, **snap)
    print(f"wrote {out} in {time.time() - t0:.0f} s; activated {np.sum(~np.isnan(t_act))} nodes")


if __name__ == "__main__":
    main()
