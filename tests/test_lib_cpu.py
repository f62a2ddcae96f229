"""Host-side checks of the C-ABI library (no GPU needed)."""
import ctypes
import os
import re

import numpy as np
import pytest

from oracle import lr91, tp06
from paper_2510_27447_gb300 import binding, build

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    build.build()
    return binding.lib()


def _declared_symbols():
    text = open(os.path.join(ROOT, "include", "bd.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(bd_[a-z_]+)\s*\(", text)))


def test_library_exports_every_declared_symbol(lib):
    decl = _declared_symbols()
    assert len(decl) >= 20
    for name in decl:
        assert hasattr(lib, name), name
    assert sorted(binding.EXPORTS) == decl


def test_state_counts(lib):
    assert binding.num_states(binding.LR91) == 8
    assert binding.num_states(binding.TP06_EPI) == 19
    assert binding.num_states(7) == 0


@pytest.mark.parametrize("model,cell", [(binding.LR91, lr91.model()), (binding.TP06_EPI, tp06.model())],
                         ids=["lr91", "tp06"])
def test_compile_time_pattern_equals_detected_pattern(lib, model, cell):
    """The node-Jacobian sparsity compiled into the kernels (the CTSM blocks)
    equals the pattern detected on the oracle by complex-step derivatives at
    random states."""
    rng = np.random.default_rng(5)
    x0 = cell.initial()
    X = np.repeat(x0[:, None], 64, axis=1)
    X[0] = rng.uniform(-90, 40, 64)
    for r in range(1, cell.ns):
        X[r] = x0[r] * rng.uniform(0.5, 1.5, 64) if x0[r] > 0 else rng.uniform(0.01, 0.99, 64)
    for r in cell.gate_rows:
        X[r] = rng.uniform(0.02, 0.98, 64)
    J = cell.jacobian(X, np.full(64, 10.0))
    detected = np.zeros(cell.ns, dtype=np.uint32)
    for r in range(cell.ns):
        for c in range(cell.ns):
            if np.any(J[r, c] != 0.0):
                detected[r] |= np.uint32(1 << c)
    declared = binding.ionic_pattern(model)
    np.testing.assert_array_equal(declared, detected)


def test_lr91_rest_state_matches_oracle(lib):
    for model, paper in ((binding.LR91, False), (binding.LR91_PAPER_MOD, True)):
        np.testing.assert_allclose(binding.rest_state(model), lr91.model(paper).rest_state(),
                                   rtol=1e-11, atol=1e-15)


def test_tp06_rest_state_is_published_initial_values(lib):
    np.testing.assert_array_equal(binding.rest_state(binding.TP06_EPI), tp06.model().initial())


def test_bad_arguments_are_rejected_without_a_device(lib):
    m = binding.Mesh(4, 3, 1, None, None, None)
    h = ctypes.c_void_p()
    rc = lib.bd_create(ctypes.byref(m), None, 0, None, ctypes.byref(h))
    assert rc == -1 and not h.value
    assert b"" != lib.bd_last_error(None)


def test_footprint_scales_with_nodes(lib):
    from paper_2510_27447_gb300 import workloads as W
    jac = binding.default_options(elliptic_precond=0)
    a = binding.footprint_bytes(*W.square_grid(33), binding.LR91, jac)
    b = binding.footprint_bytes(*W.square_grid(65), binding.LR91, jac)
    c = binding.footprint_bytes(*W.square_grid(65), binding.TP06_EPI, jac)
    assert 3.5 < (b - 2**20) / (a - 2**20) < 4.2
    assert c > 1.5 * b


def test_footprint_follows_the_options(lib):
    """The estimate adds the AMG hierarchy, the FP32 copies of the mixed
    path and, for streaming handles, the SELL-32/4 copies."""
    from paper_2510_27447_gb300 import workloads as W
    g = W.square_grid(129)
    fp = lambda **o: binding.footprint_bytes(*g, binding.TP06_EPI, binding.default_options(**o))   # noqa: E731
    jac, amg = fp(elliptic_precond=0), fp(elliptic_precond=1)
    mixed = fp(elliptic_precond=1, precision=binding.MIXED)
    stream = fp(elliptic_precond=1, precision=binding.MIXED, streaming=1)
    plain = fp(elliptic_precond=1, precision=binding.MIXED, streaming=1, vec4=-1)
    assert jac < amg < mixed < plain < stream
    assert fp() == binding.footprint_bytes(*g, binding.TP06_EPI)       # NULL options = defaults


def test_bath_mesh_errors_are_host_side(lib):
    """Bath meshes are validated during host assembly, before any device
    call: tissue nodes must come first and the bath needs sbath > 0."""
    from paper_2510_27447_gb300 import workloads as W
    w = W.bath_sheet(8, -0.25, 1.25, 0.0, 1.0, W.LR91, 0.05, 1)
    cond = binding.Cond(*w.sigma, w.chi, w.cm, 0.0)
    h = ctypes.c_void_p()
    m, keep = binding.mesh_struct(w.xyz, w.elems, w.fibers, w.elem_bath)
    assert lib.bd_create(ctypes.byref(m), ctypes.byref(cond), 0, None, ctypes.byref(h)) == -1
    assert b"sbath" in lib.bd_last_error(None)
    # swap a tissue node with a bath node: the numbering rule is broken
    perm = np.arange(w.n_nodes)
    perm[[0, w.n_nodes - 1]] = perm[[w.n_nodes - 1, 0]]
    xyz = w.xyz[perm]
    inv = np.argsort(perm)
    elems = inv[w.elems].astype(np.int32)
    cond = binding.Cond(*w.sigma, w.chi, w.cm, 20.0)
    m, keep = binding.mesh_struct(xyz, elems, w.fibers, w.elem_bath)
    assert lib.bd_create(ctypes.byref(m), ctypes.byref(cond), 0, None, ctypes.byref(h)) == -1
    assert b"numbered before" in lib.bd_last_error(None)
    assert not h.value


def test_bath_footprint_counts_tissue_state_only(lib):
    from paper_2510_27447_gb300 import workloads as W
    w = W.bath_sheet(64, -0.25, 1.25, 0.0, 1.0, W.TP06_EPI, 0.05, 1)
    with_bath = binding.footprint_bytes(w.xyz, w.elems, binding.TP06_EPI, None, w.elem_bath)
    all_tissue = binding.footprint_bytes(w.xyz, w.elems, binding.TP06_EPI)
    assert with_bath < 0.7 * all_tissue


def test_struct_layouts_match_the_library(lib):
    """The binding's ctypes layouts of the public structs have the sizes the
    library was compiled with (a field added on one side only would shift
    every later field)."""
    sz = [ctypes.c_size_t(0) for _ in range(4)]
    assert lib.bd_struct_sizes(*[ctypes.byref(x) for x in sz]) == 0
    ours = [ctypes.sizeof(binding.Mesh), ctypes.sizeof(binding.Cond), ctypes.sizeof(binding.Opts),
            ctypes.sizeof(binding.Stats)]
    assert [x.value for x in sz] == ours


def _header_struct_fields():
    """Field names, in order, of every `typedef struct {...} NAME;` in bd.h."""
    text = open(os.path.join(ROOT, "include", "bd.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    out = {}
    for body, name in re.findall(r"typedef struct\s*\{(.*?)\}\s*(\w+)\s*;", text, flags=re.S):
        names = []
        for decl in body.split(";"):
            decl = " ".join(decl.split())
            if not decl:
                continue
            fp = re.search(r"\(\s*\*\s*(\w+)\s*\)", decl)            # function pointer
            if fp:
                names.append(fp.group(1))
                continue
            decl = re.sub(r"\[[^\]]*\]", "", decl)                    # array extents
            for part in decl.split(","):                               # int a, b;
                names.append(re.findall(r"(\w+)\s*$", part.strip())[0])
        out[name] = names
    return out


def test_binding_fields_follow_the_header_in_order():
    """The ctypes structs name the header's fields in the header's order (equal
    sizes alone would not catch two fields of one type swapped)."""
    fields = _header_struct_fields()
    pairs = {"bd_mesh_t": binding.Mesh, "bd_cond_t": binding.Cond, "bd_opts_t": binding.Opts,
             "bd_stats_t": binding.Stats, "bd_profile_t": binding.Profile}
    for cname, cls in pairs.items():
        assert [f[0] for f in cls._fields_] == fields[cname], cname
