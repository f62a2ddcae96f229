"""The synthetic input recipes: sizes of the paper's workloads (Sec. 4 and the
benchmark configurations), well-formed meshes, tissue-first numbering of the
bath meshes, seeded determinism.  Host only."""
import numpy as np
import pytest

from paper_2510_27447_gb300 import workloads as W


def _signed_measures(w):
    x = w.xyz[w.elems]
    if w.dim == 2:
        a, b = x[:, 1] - x[:, 0], x[:, 2] - x[:, 0]
        return 0.5 * (a[:, 0] * b[:, 1] - a[:, 1] * b[:, 0])
    a, b, c = x[:, 1] - x[:, 0], x[:, 2] - x[:, 0], x[:, 3] - x[:, 0]
    return np.einsum("ij,ij->i", a, np.cross(b, c)) / 6.0


def _check_mesh(w):
    assert w.elems.min() >= 0 and w.elems.max() < w.n_nodes
    assert len(np.unique(w.elems.ravel())) == w.n_nodes          # no orphan node
    vol = np.abs(_signed_measures(w))
    assert vol.min() > 0.0
    f = np.asarray(w.fibers).reshape(len(w.elems), w.dim)
    np.testing.assert_allclose(np.linalg.norm(f, axis=1), 1.0, rtol=1e-12)
    return vol


def test_headline_sheet_has_the_benchmark_size():
    w = W.config1()
    assert (w.n_nodes, len(w.elems), w.dt, w.model) == (257 * 257, 2 * 256 * 256, 0.02, W.TP06_EPI)
    vol = _check_mesh(w)
    assert vol.sum() == pytest.approx(2.5 * 2.5, rel=1e-12)      # the 2.5 cm square
    s1 = w.stimuli[0]
    assert s1.t_on == 0.0 and np.asarray(s1.mask)[w.xyz[:, 0] < 0.1].all()


def test_bath_run_of_section_4_has_the_paper_sizes_and_numbers_tissue_first():
    w = W.bath_paper_2d()
    assert w.n_nodes == 801 * 801 and w.n_tissue == 601 * 601
    assert w.sbath == W.BATH_SIGMA and w.dt == 0.05 and w.n_steps == 12000   # 600 ms
    _check_mesh(w)
    tis = np.zeros(w.n_nodes, dtype=bool)
    tis[w.elems[w.elem_bath == 0].ravel()] = True
    assert tis[:w.n_tissue].all() and not tis[w.n_tissue:].any()
    xt = w.xyz[:w.n_tissue]
    assert xt.min() >= -1e-12 and xt.max() <= 6.0 + 1e-12             # tissue [0, 6]^2
    assert w.xyz.min() == pytest.approx(-1.0) and w.xyz.max() == pytest.approx(7.0)


def test_slab_config_has_two_million_nodes():
    xyz, tets = W.slab_grid(201, 201, 51, 2.0, 2.0, 0.5)
    assert len(xyz) == 2060451
    w = W.Workload("s", xyz, tets, W.fibers_transmural(xyz, tets, 0.0, 0.5, -60.0, 60.0), W.CONFIG0_SIGMA,
                   2000.0, 1.0, W.TP06_EPI, [], 0.025, 1)
    vol = _check_mesh(w)
    assert vol.sum() == pytest.approx(2.0 * 2.0 * 0.5, rel=1e-10)


def test_lv_shell_in_a_bath_is_tissue_first_and_seeded():
    a = W.lv_shell_bath(h=0.3)
    b = W.lv_shell_bath(h=0.3)
    for x, y in ((a.xyz, b.xyz), (a.elems, b.elems), (a.elem_bath, b.elem_bath), (a.fibers, b.fibers)):
        np.testing.assert_array_equal(x, y)                          # same seed, same mesh
    _check_mesh(a)
    assert 0 < a.n_tissue < a.n_nodes
    tis = np.zeros(a.n_nodes, dtype=bool)
    tis[a.elems[a.elem_bath == 0].ravel()] = True
    assert tis[:a.n_tissue].all() and not tis[a.n_tissue:].any()


def test_request_stream_is_reproducible():
    r1 = W.request_stream(32, seed=4)
    r2 = W.request_stream(32, seed=4)
    assert [(q.arrival_s, q.side, q.model) for q in r1] == [(q.arrival_s, q.side, q.model) for q in r2]
    assert all(np.diff([q.arrival_s for q in r1]) >= 0)
    assert W.request_stream(32, seed=5)[0].arrival_s != r1[0].arrival_s
