"""Pins of the oracle's bidomain-bath coupling (Sec. 4, "Results for
Bidomain-Bath") against independent computations: the tissue-only mesh, the
whole-domain mesh, and the insulating / perfectly conducting bath limits."""
import numpy as np
import pytest
import scipy.sparse.linalg as spla

from oracle import bidomain as B
from oracle import fem, lr91
from paper_2510_27447_gb300 import workloads as W

SIG = (3.0, 0.31, 2.0, 1.35)


def _bath(n_cells=24, sbath=20.0, sigma=SIG):
    return W.bath_sheet(n_cells, -0.25, 1.25, 0.0, 1.0, W.LR91, 0.05, 10, sigma=sigma, sbath=sbath)


def _tissue_only(w):
    """The tissue elements as a mesh of their own (nodes 0..NT-1)."""
    nt = w.n_tissue
    t = w.elems[w.elem_bath == 0]
    assert t.max() < nt
    return w.xyz[:nt], t, w.fibers[w.elem_bath == 0]


def test_tissue_operators_equal_the_tissue_only_mesh():
    w = _bath()
    ops = fem.assemble(w.xyz, w.elems, w.fibers, SIG, 2000.0, 1.0, w.elem_bath, w.sbath)
    xt, tt, ft = _tissue_only(w)
    ref = fem.assemble(xt, tt, ft, SIG, 2000.0, 1.0)
    nt = w.n_tissue
    for a, b in ((ops.A_i, ref.A_i), (ops.M, ref.M)):
        np.testing.assert_allclose(a[:nt, :nt].toarray(), b.toarray(), atol=1e-15)
        assert abs(a[nt:, :]).sum() == 0.0 and abs(a[:, nt:]).sum() == 0.0
    np.testing.assert_allclose(ops.M_L[:nt], ref.M_L, rtol=1e-14)
    assert np.all(ops.M_L[nt:] == 0.0)
    # the area of the tissue square, not of the whole domain
    assert ops.M_L.sum() == pytest.approx(1.0, rel=1e-13)


def test_bath_with_matching_conductivity_is_the_whole_domain():
    """sigma_b I = sigma_i + sigma_e (isotropic): the extracellular operator of
    the bath mesh is the one of a whole-domain tissue mesh."""
    sig = (1.0, 1.0, 1.5, 1.5)
    w = _bath(sbath=2.5, sigma=sig)
    ops = fem.assemble(w.xyz, w.elems, w.fibers, sig, 2000.0, 1.0, w.elem_bath, 2.5)
    whole = fem.assemble(w.xyz, w.elems, w.fibers, sig, 2000.0, 1.0)
    np.testing.assert_allclose(ops.A_ie.toarray(), whole.A_ie.toarray(), atol=1e-15)
    # ... and a different bath conductivity changes exactly the bath elements
    ops2 = fem.assemble(w.xyz, w.elems, w.fibers, sig, 2000.0, 1.0, w.elem_bath, 5.0)
    d = (ops2.A_ie - ops.A_ie).toarray()
    bath_nodes = np.unique(w.elems[w.elem_bath == 1])
    assert np.all(d[np.setdiff1d(np.arange(w.n_nodes), bath_nodes)] == 0.0)


def _v_field(w):
    x, y = w.xyz[:w.n_tissue, 0], w.xyz[:w.n_tissue, 1]
    return -80.0 + 60.0 * np.exp(-((x - 0.3) ** 2 + (y - 0.6) ** 2) / 0.05)


def _problem(w, sbath):
    return B.Bidomain(w.xyz, w.elems, w.fibers, SIG, 2000.0, 1.0, lr91.model(True), (),
                      pin_node=w.pin_node, elem_bath=w.elem_bath, sigma_b=sbath)


def test_insulating_bath_limit_recovers_the_tissue_only_problem():
    w = _bath()
    v = _v_field(w)
    u = _problem(w, 1e-9).elliptic(v)[:w.n_tissue]
    xt, tt, ft = _tissue_only(w)
    P0 = B.Bidomain(xt, tt, ft, SIG, 2000.0, 1.0, lr91.model(True), (), pin_node=0)
    u0 = P0.elliptic(v)
    d = (u - u.mean()) - (u0 - u0.mean())
    assert np.max(np.abs(d)) < 1e-5 * np.max(np.abs(u0))
    # a conducting bath draws current: the tissue field differs markedly
    u20 = _problem(w, 20.0).elliptic(v)[:w.n_tissue]
    assert np.max(np.abs((u20 - u20.mean()) - (u0 - u0.mean()))) > 0.05 * np.max(np.abs(u0))


def test_perfectly_conducting_bath_limit_is_a_dirichlet_problem():
    """sigma_b -> infinity shorts the bath: u is constant on the bath and the
    interface, and in the tissue it solves A_ie u = -A_i v with that constant
    as Dirichlet data on the interface nodes."""
    w = _bath()
    v = _v_field(w)
    P = _problem(w, 1e9)
    u = P.elliptic(v)
    nt = w.n_tissue
    iface = np.intersect1d(np.unique(w.elems[w.elem_bath == 1]), np.arange(nt))
    assert np.ptp(u[nt:]) < 1e-6 * np.ptp(u[:nt])
    c = u[nt:].mean()
    xt, tt, ft = _tissue_only(w)
    ref = fem.assemble(xt, tt, ft, SIG, 2000.0, 1.0)
    inner = np.setdiff1d(np.arange(nt), iface)
    A = ref.A_ie.tocsr()
    rhs = -(ref.A_i @ v) - A[:, iface] @ np.full(len(iface), c)
    ud = np.full(nt, c)
    ud[inner] = spla.spsolve(A[inner][:, inner].tocsc(), rhs[inner])
    assert np.max(np.abs(u[:nt] - ud)) < 1e-5 * np.ptp(ud)


def test_uniform_tissue_state_ignores_the_bath():
    """Uniform state and stimulus over the whole tissue: A_i v = 0, so u = 0
    on every node and each tissue node follows the single-cell ODE."""
    w = _bath(n_cells=12)
    cell = lr91.model(True)
    nt = w.n_tissue
    mask = np.zeros(w.n_nodes, np.uint8)
    mask[:nt] = 1
    P = B.Bidomain(w.xyz, w.elems, w.fibers, SIG, 2000.0, 1.0, cell,
                   [B.Stim(mask, 0.0, 1.0, 30.0)], pin_node=w.pin_node,
                   elem_bath=w.elem_bath, sigma_b=w.sbath)
    X0 = np.repeat(cell.rest_state()[:, None], nt, axis=1)
    X, u, _ = B.run(P, X0, 10, 0.05)
    assert u.shape == (w.n_nodes,) and np.max(np.abs(u)) < 1e-9
    assert np.max(np.abs(X - X[:, :1])) < 1e-10 * np.max(np.abs(X))
    assert X[0, 0] > cell.rest_state()[0] + 1.0
