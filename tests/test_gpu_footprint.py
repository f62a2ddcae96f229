"""bd_footprint_bytes against the device memory a handle actually takes
(bd_create and its first step, which adds the parabolic shift caches and
the step graph): the estimate used for admission control must not fall far
below the real footprint, nor exceed it grossly."""
import numpy as np
import pytest

from paper_2510_27447_gb300 import binding
from paper_2510_27447_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def _cases():
    slab = W.config2(101, 101, 26)
    sheet = W.sheet(257, 2.5, W.TP06_EPI, 0.02, 1)
    return [("slab mixed streaming", slab, dict(precision=binding.MIXED, streaming=1)),
            ("slab fp64 persistent", slab, dict(precision=binding.FP64, streaming=-1)),
            ("sheet mixed", sheet, dict(precision=binding.MIXED))]


@pytest.mark.parametrize("case", range(3))
def test_footprint_estimate_brackets_the_device_memory_taken(case):
    torch = pytest.importorskip("torch")
    name, w, o = _cases()[case]
    opts = binding.default_options(pin_node=w.pin_node, **o)
    est = binding.footprint_bytes(w.xyz, w.elems, w.model, opts, w.elem_bath)
    torch.cuda.init()
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    sim = binding.simulation_from_workload(w, opts)
    sim.step(w.dt, 3, 2)
    sim.sync()
    free1, _ = torch.cuda.mem_get_info()
    sim.close()
    used = free0 - free1
    ratio = est / used
    print(f"{name}: estimate {est / 2**20:.0f} MiB, taken {used / 2**20:.0f} MiB, ratio {ratio:.2f}")
    assert used > 0
    # measured on GB300: 1.04-1.18 (slab 101x101x26 mixed streaming / FP64,
    # 257^2 sheet mixed)
    assert 0.9 < ratio < 1.6, (name, est, used)
