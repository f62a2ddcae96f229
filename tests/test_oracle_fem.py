"""Pins of the oracle's P1 assembly (Sec. 3.2, Eqs. (3.6)-(3.9))."""
import numpy as np
import scipy.sparse.linalg as spla

from oracle import fem
from paper_2510_27447_gb300 import workloads as W


def test_reference_triangle_closed_form():
    xyz = np.array([[0.0, 0.0], [1.0, 0.0], [0.0, 1.0]])
    tri = np.array([[0, 1, 2]])
    K = fem.stiffness(xyz, tri, np.array([[1.0, 0.0]]), 1.0, 1.0).toarray()
    M = fem.mass(xyz, tri).toarray()
    np.testing.assert_allclose(K, 0.5 * np.array([[2, -1, -1], [-1, 1, 0], [-1, 0, 1]]), atol=1e-15)
    np.testing.assert_allclose(M, np.array([[2, 1, 1], [1, 2, 1], [1, 1, 2]]) / 24.0, atol=1e-16)


def test_reference_tet_mass_and_anisotropic_stiffness():
    xyz = np.array([[0.0, 0, 0], [1, 0, 0], [0, 1, 0], [0, 0, 1]])
    tet = np.array([[0, 1, 2, 3]])
    M = fem.mass(xyz, tet).toarray()
    np.testing.assert_allclose(M, (np.ones((4, 4)) + np.eye(4)) / 120.0, atol=1e-16)
    # sigma = diag(3, 1, 1) (fibre along x): K_ab = |T| grad a . sigma grad b, |T| = 1/6
    K = fem.stiffness(xyz, tet, np.array([[1.0, 0, 0]]), 3.0, 1.0).toarray()
    G = np.array([[-1, -1, -1], [1, 0, 0], [0, 1, 0], [0, 0, 1.0]])
    np.testing.assert_allclose(K, G @ np.diag([3.0, 1, 1]) @ G.T / 6.0, atol=1e-15)


def _ops(xyz, el, fib, sigma=(3.0, 0.31, 2.0, 1.35)):
    return fem.assemble(xyz, el, fib, sigma, 2000.0, 1.0)


def test_null_space_symmetry_and_total_mass_2d():
    xyz, tri = W.square_grid(9, 2.5)
    ops = _ops(xyz, tri, W.fibers_along_x(len(tri), 2))
    one = np.ones(len(xyz))
    for A in (ops.A_i, ops.A_ie):
        assert np.max(np.abs(A @ one)) < 1e-15
        assert abs(A - A.T).max() < 1e-18
    assert abs(one @ (ops.M @ one) - 2.5 ** 2) < 1e-12
    np.testing.assert_allclose(ops.M_L.sum(), 2.5 ** 2, rtol=1e-14)


def test_null_space_and_volume_3d_rotated_fibres():
    xyz, tet = W.slab_grid(5, 4, 3, 2.0, 2.0, 0.5)
    fib = W.fibers_transmural(xyz, tet, 0.0, 0.5, -60.0, 60.0)
    ops = _ops(xyz, tet, fib)
    one = np.ones(len(xyz))
    assert np.max(np.abs(ops.A_ie @ one)) < 1e-15
    assert abs(ops.A_ie - ops.A_ie.T).max() < 1e-18
    np.testing.assert_allclose(one @ (ops.M @ one), 2.0 * 2.0 * 0.5, rtol=1e-13)
    # every interior triangular face is shared by exactly two tetrahedra
    faces = {}
    for t in tet:
        for drop in range(4):
            f = tuple(sorted(np.delete(t, drop)))
            faces[f] = faces.get(f, 0) + 1
    assert max(faces.values()) == 2


def test_equal_anisotropy_identity():
    xyz, tri = W.square_grid(7, 1.0)
    lam = 0.75
    si = (3.0, 0.31)
    ops = fem.assemble(xyz, tri, W.fibers_along_x(len(tri), 2),
                       (si[0], si[1], lam * si[0], lam * si[1]), 2000.0, 1.0)
    assert abs(ops.A_ie - (1.0 + lam) * ops.A_i).max() < 1e-17


def _mms_error(n, dim):
    """-div(sigma grad u) = f with Neumann data for u = prod cos(pi x_k);
    returns the discrete L2 error of the zero-mean Galerkin solution."""
    if dim == 2:
        xyz, el = W.square_grid(n, 1.0)
        fib = W.fibers_along_x(len(el), 2)
    else:
        xyz, el = W.slab_grid(n, n, n, 1.0, 1.0, 1.0)
        fib = W.fibers_along_x(len(el), 3)
    sl, st = 2.0, 0.5
    K = fem.stiffness(xyz, el, fib, sl, st)
    M = fem.mass(xyz, el)
    u = np.prod(np.cos(np.pi * xyz), axis=1)
    f = (sl + (dim - 1) * st) * np.pi ** 2 * u
    b = M @ f
    keep = np.arange(1, len(xyz))
    uh = np.zeros(len(xyz))
    uh[keep] = spla.spsolve(K[keep][:, keep].tocsc(), b[keep])
    one = np.ones(len(xyz))
    area = one @ (M @ one)
    uh -= (one @ (M @ uh)) / area
    e = uh - u
    return np.sqrt(e @ (M @ e))


def test_mms_second_order_2d():
    errs = [_mms_error(n, 2) for n in (9, 17, 33)]
    rates = np.log2(np.array(errs[:-1]) / np.array(errs[1:]))
    assert np.all(rates > 1.85), rates


def test_mms_second_order_3d():
    errs = [_mms_error(n, 3) for n in (5, 9, 17)]
    rates = np.log2(np.array(errs[:-1]) / np.array(errs[1:]))
    assert np.all(rates > 1.7), rates
