"""Whole-chain pin: conduction velocity against the paper's biomarker table.

Sec. 4 ("Biomarkers", LR91 table): with the paper's LR91 parameter set
(G_si = 0.02, G_Na = 4.0, G_K = 0.423), isotropic intra- and extracellular
conductivities of 1.5e-3 (in our scaling sigma/(chi C_m) = 1.5e-3 cm^2/ms,
i.e. sigma = 3 mS/cm at chi = 2000 /cm, C_m = 1), a 100x100-element grid of
the unit square (h = 0.01 cm) and the partitioned strategy with SDC, the
paper reports CV = 27.52 cm/s.  The oracle, on P1 triangles of the same
spacing, must land within 10 %.  This pins the chi*C_m scaling of the
assembly, the LR91 transcription and the step together.
"""
import numpy as np
import pytest

from oracle import bidomain as B
from oracle import lr91
from paper_2510_27447_gb300 import workloads as W


@pytest.mark.slow
def test_lr91_paper_parameters_conduction_velocity():
    cellm = lr91.model(True)
    xyz, tri = W.rect_grid(61, 3, 0.6, 0.02)
    P = B.Bidomain(xyz, tri, W.fibers_along_x(len(tri), 2), (3.0, 3.0, 3.0, 3.0), 2000.0, 1.0,
                   cellm, [B.Stim(W.nodes_x_below(xyz, 0.051), 0.0, 1.0, 80.0)], pin_node=0)
    X0 = np.repeat(cellm.rest_state()[:, None], P.N, axis=1)
    # 10 ms: the front has crossed the 0.01-0.15 cm window by about 8 ms
    _, _, t_act = B.run(P, X0, 200, 0.05, 3, 2)
    window = (xyz[:, 0] >= 0.01) & (xyz[:, 0] <= 0.15)
    assert np.all(np.isfinite(t_act[window]))
    cv = 1000.0 * B.conduction_velocity(xyz, t_act, 0.01, 0.15)   # cm/s
    assert abs(cv - 27.52) / 27.52 < 0.10, cv
