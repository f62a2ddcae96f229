"""P1 finite-element operators of the semi-discrete bidomain system (oracle).

Test infrastructure only (see the package docstring).

Sec. 3.2 ("Spatial Discretization"), Eqs. (3.6)-(3.9): with piecewise linear
basis functions w_i the stiffness matrices are
    A_ie = { ((sigma_i + sigma_e) grad w_i, grad w_j) },   A_i = { (sigma_i grad w_i, grad w_j) },
and the mass matrix is M = { (w_i, w_j) }.  The conductivity of each element is
the transversely isotropic tensor sigma = s_t I + (s_l - s_t) f f^T built from
the element's fibre direction f (Sec. 2: constant diagonal tensors in the
fibre frame).  The parabolic equation is divided by chi*C_m (surface-to-volume
ratio times membrane capacitance), so A_i and A_ie here are the stiffness
matrices scaled by 1/(chi*C_m): with sigma_il = 3 mS/cm, chi = 2000 /cm and
C_m = 1 uF/cm^2 the intracellular diffusivity is 1.5e-3 cm^2/ms, the value the
paper quotes in Sec. 4.

Every element matrix is formed from its definition (gradient of the
barycentric basis, exact integral of the product of two linear functions) and
scattered with scipy's COO->CSR summation.  The lumped mass M_L is the row sum
of M.

Bidomain-bath coupling (Sec. 4, "Results for Bidomain-Bath"): a bath element
has no intracellular space and no membrane; it adds sigma_b I (isotropic) to
the extracellular conductivity only.  Hence A_i, M and M_L collect tissue
elements only, and A_ie collects K(sigma_i + sigma_e) over the tissue plus
K(sigma_b I) over the bath -- the weak form of div((sigma_i + sigma_e) grad u
+ sigma_i grad v) = 0 in the tissue, div(sigma_b grad u) = 0 in the bath,
with u continuous and the normal currents balanced on the interface.

Pins (tests/test_oracle_fem.py): manufactured solution with observed O(h^2),
exact null space (A 1 = 0), total mass = area/volume, closed-form element
matrices of the reference triangle, and the equal-anisotropy identity
A_ie = (1 + lambda) A_i when sigma_e = lambda sigma_i.
"""
from __future__ import annotations

import dataclasses

import numpy as np
import scipy.sparse as sp


def _element_geometry(xyz: np.ndarray, elems: np.ndarray):
    """Return (measure[E], grads[E, d+1, d]) of P1 barycentric functions."""
    dim = xyz.shape[1]
    P = xyz[elems]                                # [E, d+1, d]
    B = np.transpose(P[:, 1:, :] - P[:, :1, :], (0, 2, 1))   # columns x_k - x_0, [E, d, d]
    det = np.linalg.det(B)
    fact = 2.0 if dim == 2 else 6.0
    meas = np.abs(det) / fact
    Binv = np.linalg.inv(B)                       # rows = grad(lambda_1..d)
    g = np.empty((len(elems), dim + 1, dim))
    g[:, 1:, :] = Binv
    g[:, 0, :] = -Binv.sum(axis=1)
    return meas, g


def _tensor(fibers: np.ndarray, s_l: float, s_t: float) -> np.ndarray:
    """sigma = s_t I + (s_l - s_t) f f^T per element, [E, d, d]."""
    dim = fibers.shape[1]
    f = fibers / np.linalg.norm(fibers, axis=1, keepdims=True)
    return s_t * np.eye(dim)[None] + (s_l - s_t) * np.einsum("ei,ej->eij", f, f)


def _scatter(elems: np.ndarray, local: np.ndarray, n: int) -> sp.csr_matrix:
    k = elems.shape[1]
    rows = np.repeat(elems, k, axis=1).ravel()
    cols = np.tile(elems, (1, k)).ravel()
    return sp.coo_matrix((local.ravel(), (rows, cols)), shape=(n, n)).tocsr()


def stiffness(xyz, elems, fibers, s_l, s_t) -> sp.csr_matrix:
    """K_ab = |T| grad(w_a)^T sigma grad(w_b), summed over elements."""
    meas, g = _element_geometry(xyz, elems)
    S = _tensor(fibers, s_l, s_t)
    local = meas[:, None, None] * np.einsum("eai,eij,ebj->eab", g, S, g)
    return _scatter(elems, local, xyz.shape[0])


def mass(xyz, elems) -> sp.csr_matrix:
    """M_ab = integral of w_a w_b = |T| (1 + delta_ab) / ((d+1)(d+2))."""
    dim = xyz.shape[1]
    meas, _ = _element_geometry(xyz, elems)
    k = dim + 1
    ref = (np.ones((k, k)) + np.eye(k)) / ((dim + 1) * (dim + 2))
    local = meas[:, None, None] * ref[None]
    return _scatter(elems, local, xyz.shape[0])


@dataclasses.dataclass
class Operators:
    A_i: sp.csr_matrix      # K(sigma_i) / (chi C_m)
    A_ie: sp.csr_matrix     # K(sigma_i + sigma_e) / (chi C_m)
    M: sp.csr_matrix        # consistent mass
    M_L: np.ndarray         # lumped mass (row sums of M)


def assemble(xyz, elems, fibers, sigma, chi, cm, elem_bath=None, sigma_b: float = 0.0) -> Operators:
    """Operators of Eqs. (3.6)-(3.7) for conductivities
    sigma = (s_il, s_it, s_el, s_et) in mS/cm; elements with elem_bath != 0
    are bath elements of isotropic conductivity sigma_b."""
    s_il, s_it, s_el, s_et = sigma
    scale = 1.0 / (chi * cm)
    if elem_bath is None:
        tis = np.ones(len(elems), dtype=bool)
    else:
        tis = np.asarray(elem_bath) == 0
    et, ft = elems[tis], fibers[tis]
    A_i = stiffness(xyz, et, ft, s_il, s_it) * scale
    A_ie = stiffness(xyz, et, ft, s_il + s_el, s_it + s_et) * scale
    M = mass(xyz, et)
    if not np.all(tis):
        eb, fb = elems[~tis], fibers[~tis]
        A_ie = A_ie + stiffness(xyz, eb, fb, sigma_b, sigma_b) * scale
    M_L = np.asarray(M.sum(axis=1)).ravel()
    return Operators(A_i=A_i.tocsr(), A_ie=A_ie.tocsr(), M=M.tocsr(), M_L=M_L)
