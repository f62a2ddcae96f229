"""Step one synthetic workload a few times and print the handle's counters:
a small driver for profiling one configuration under a tool such as ncu.

usage: python -m paper_2510_27447_gb300.run_workload <workload> [options]

workloads: sheet (TP06 epicardial sheet of --n x --n nodes, 2.5 cm wide),
slab (config 2: TP06 201x201x51 Kuhn-lattice slab), lv (TP06 left-ventricle
shell in a box bath, lattice spacing --h cm), bath (LR91 bidomain-bath sheet
of 801 x 801 nodes).
"""
import argparse
import json

from . import binding
from . import workloads as W


def build(name: str, n: int, h: float):
    if name == "sheet":
        return W.sheet(n, 2.5 * (n - 1) / 256, W.TP06_EPI, 0.02, 1)
    if name == "slab":
        return W.config2()
    if name == "lv":
        return W.lv_shell_bath(h=h)
    if name == "bath":
        return W.bath_paper_2d()
    raise SystemExit(f"unknown workload {name!r}")


def main(argv=None) -> None:
    ap = argparse.ArgumentParser(description=__doc__.splitlines()[0])
    ap.add_argument("workload", choices=["sheet", "slab", "lv", "bath"])
    ap.add_argument("--n", type=int, default=257, help="sheet side (nodes)")
    ap.add_argument("--h", type=float, default=0.08, help="lattice spacing of the lv workload (cm)")
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--precision", choices=["mixed", "fp64"], default="mixed")
    a = ap.parse_args(argv)
    w = build(a.workload, a.n, a.h)
    prec = binding.MIXED if a.precision == "mixed" else binding.FP64
    sim = binding.simulation_from_workload(w, binding.default_options(precision=prec, pin_node=w.pin_node))
    for _ in range(a.steps):
        sim.step(w.dt)
    sim.sync()
    print(json.dumps({"workload": w.name, "nodes": int(w.n_nodes), "steps": a.steps, "stats": sim.stats()}))
    sim.close()


if __name__ == "__main__":
    main()
