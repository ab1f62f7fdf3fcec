"""Finite-difference operators on the hexahedral grid (oracle).

Test infrastructure only (see oracle/__init__.py).

The outer region Omega_FDM is discretised on a structured hexahedral grid
(Sec. 5, Fig. 1).  Its operators are those of the trilinear hexahedral element
with vertex (trapezoidal) quadrature, which is the standard second-order
finite difference scheme: a 7-point Laplacian whose Neumann boundary rows are
the ghost-node rows.  In tensor-product form, with the 1-D pieces
  K1 = (1/h) tridiag(-1, 2, -1) with end rows (1, -1)   (1-D stiffness)
  W1 = diag(1/2, 1, ..., 1, 1/2)                         (trapezoid weights)
and M1 = h W1 (1-D lumped mass), the 3-D operators are
  L = K1 (x) M1 (x) M1 + M1 (x) K1 (x) M1 + M1 (x) M1 (x) K1   (stiffness)
  m = M1 (x) M1 (x) M1                               (lumped volume mass)
  b_face = M1 (x) M1 on the face's nodes             (lumped surface mass)
Reading: the boundary lives in the FDM region (the paper notes that the
model equation is the plain wave equation there and that Gamma lies in the
closure of Omega_FDM, Sec. 2), so the boundary rows and boundary masses are
the FD ones.  They coincide with the Kuhn-P1 rows everywhere except on the
twelve edges of the cube, where the Kuhn split is not mirror-symmetric.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp

from .grid import Grid


def _k1(n: int, h: float) -> sp.csr_matrix:
    main = np.full(n, 2.0)
    main[0] = main[-1] = 1.0
    off = np.full(n - 1, -1.0)
    return sp.diags([off, main, off], [-1, 0, 1], format="csr") / h


def _w1(n: int) -> np.ndarray:
    w = np.ones(n)
    w[0] = w[-1] = 0.5
    return w


def fd_laplacian(g: Grid) -> sp.csr_matrix:
    """Scalar FD stiffness L (node order i + n(j + n k), so the Kronecker
    factors run z (x) y (x) x)."""
    n, h = g.n, g.h
    K = _k1(n, h)
    W = sp.diags(h * _w1(n))
    L = (sp.kron(W, sp.kron(W, K)) + sp.kron(W, sp.kron(K, W))
         + sp.kron(K, sp.kron(W, W)))
    extra = g.nn - n ** 3            # nodes of a refined FEM mesh: no FD rows
    if extra:
        L = sp.block_diag((L, sp.csr_matrix((extra, extra))))
    return L.tocsr()


def fd_mass(g: Grid) -> np.ndarray:
    w = _w1(g.n)
    m = g.h ** 3 * np.kron(w, np.kron(w, w))
    return np.concatenate([m, np.zeros(g.nn - g.n ** 3)])


def fd_face_mass(g: Grid, face: str) -> np.ndarray:
    """Lumped surface mass of one face, as a full-length nodal vector (zero
    off the face)."""
    n, h = g.n, g.h
    w = _w1(n)
    sel = g.face_nodes(face)
    out = np.zeros(g.nn)
    ax_pair = {"x0": (1, 2), "x1": (1, 2), "y0": (0, 2), "y1": (0, 2),
               "bottom": (0, 1), "top": (0, 1)}[face]
    idx = np.stack([g.i_of, g.j_of, g.k_of], axis=1)
    out[sel] = h * h * w[idx[sel, ax_pair[0]]] * w[idx[sel, ax_pair[1]]]
    return out
