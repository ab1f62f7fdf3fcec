"""P1 finite elements on tetrahedra (oracle).

Test infrastructure only (see oracle/__init__.py).

For a tetrahedron with vertices x_0..x_3 the P1 basis functions are
phi_a(x) = c_a + g_a . x with phi_a(x_b) = delta_ab, i.e. the columns of the
inverse of the 4x4 matrix whose row b is [1, x_b].  From the gradients g_a and
the volume |K| the element contributes
  * stiffness  L_ab   = |K| g_a . g_b            (the -Delta term)
  * lumped mass m_a   = |K| / 4
  * divergence D_K E = sum_b g_b . E_b            (P1 divergence of a nodal field)
The stabilising Gauss-law term of the model problem, -grad div((eps-1) E)
(Sec. 2, eq. forward_prob, its note on spurious P1 solutions; Sec. 5,
eq. model1), has the weak form int div(lambda) div((eps-1) E) (Sec. 3,
eq. lagrangian_weak).  Reading: epsilon is nodal P1 and (eps-1)E is
interpolated nodally, so the term is D^T D S E with D stacked over elements
(row K weighted by sqrt|K|) and S = diag(eps - 1) per node.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp


def p1_geometry(coords: np.ndarray, tets: np.ndarray):
    """Gradients (T, 4, 3) and volumes (T,) of the P1 basis on each tet."""
    X = coords[tets]                                   # (T, 4, 3)
    A = np.concatenate([np.ones(X.shape[:2] + (1,)), X], axis=2)  # rows [1, x_b]
    C = np.linalg.inv(A)                               # column a -> [c_a, g_a]
    G = np.transpose(C[:, 1:, :], (0, 2, 1))           # (T, 4, 3): g_a
    vol = np.abs(np.linalg.det(X[:, 1:, :] - X[:, :1, :])) / 6.0
    return G, vol


def p1_stiffness(nn: int, tets, G, vol) -> sp.csr_matrix:
    rows = np.repeat(tets, 4, axis=1).ravel()
    cols = np.tile(tets, (1, 4)).ravel()
    vals = (vol[:, None, None] * np.einsum("tac,tbc->tab", G, G)).ravel()
    return sp.coo_matrix((vals, (rows, cols)), shape=(nn, nn)).tocsr()


def p1_lumped_mass(nn: int, tets, vol) -> np.ndarray:
    m = np.zeros(nn)
    np.add.at(m, tets.ravel(), np.repeat(vol / 4.0, 4))
    return m


def p1_divergence(nn: int, tets, G, vol) -> sp.csr_matrix:
    """D: one row per tet, columns c*nn + node for the three components of a
    component-major nodal field; row K scaled by sqrt|K| so that
    D^T D = sum_K |K| g g^T."""
    T = tets.shape[0]
    rows = np.repeat(np.arange(T), 12)
    cols = (np.arange(3)[None, None, :] * nn + tets[:, :, None]).reshape(T, 12).ravel()
    vals = (np.sqrt(vol)[:, None, None] * G).reshape(T, 12).ravel()
    return sp.coo_matrix((vals, (rows, cols)), shape=(T, 3 * nn)).tocsr()
