"""Helpers shared by the GPU parity tests (inputs and oracle runs)."""
import numpy as np

from oracle import bidomain as OB
from oracle import lr91 as OL
from oracle import tp06 as OT
from paper_2510_27447_gb300 import binding
from paper_2510_27447_gb300 import workloads as W


def oracle_cell(model):
    if model == W.TP06_EPI:
        return OT.model()
    return OL.model(model == W.LR91_PAPER_MOD)


def oracle_problem(w, mass_lumped=False, pin=None):
    return OB.Bidomain(w.xyz, w.elems, w.fibers, w.sigma, w.chi, w.cm, oracle_cell(w.model),
                       w.stimuli, pin_node=w.pin_node if pin is None else pin,
                       mass_lumped=mass_lumped, elem_bath=w.elem_bath, sigma_b=w.sbath)


def rest_X(w):
    cell = oracle_cell(w.model)
    x = cell.initial() if w.model == W.TP06_EPI else cell.rest_state()
    return np.repeat(x[:, None], w.n_tissue, axis=1)


def gpu_sim(w, **opt):
    opt.setdefault("pin_node", w.pin_node)
    o = binding.default_options(**opt)
    return binding.Simulation(w.xyz, w.elems, w.fibers, w.sigma, w.chi, w.cm, w.model, o, w.stimuli,
                              elem_bath=w.elem_bath, sbath=w.sbath)


def rel(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / max(np.linalg.norm(b), 1e-300))
