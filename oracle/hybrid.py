"""The hybrid FE/FD semi-discrete operator (oracle).

Test infrastructure only (see oracle/__init__.py).

Semi-discretising the stabilized model problem (Sec. 5, eq. model1, equal to
Sec. 2, eq. forward_prob, after moving terms) gives, per time t,

    M_eps E'' + C E' + K(eps) E = F,        K(eps) = I_3 (x) L + P D^T D S,

with
  * L      scalar stiffness: FEM rows (P1 on the Kuhn tets) on the nodes
           strictly inside the FEM cube, FD rows everywhere else;
  * M_eps  diag(m * eps) per component, m the lumped mass of the same rows;
  * C      diag(m * sigma + b_abs), b_abs the lumped surface mass of the faces
           that are absorbing at time t (first-order condition
           d_n E = -d_t E, eq. model1);
  * D      the P1 divergence over the FEM tets (fem.p1_divergence),
           S = diag(eps - 1), P = diag(1 on FEM rows): the stabilisation only
           enters the rows the FEM updates.
K is not symmetric when eps varies; its transpose, used by the adjoint, is
I_3 (x) L^T + S D^T D P.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp

from . import fdm, fem
from .grid import Grid


class HybridOperator:
    def __init__(self, g: Grid, eps_free: np.ndarray, sig_free: np.ndarray):
        self.g = g
        nn = g.nn
        free = g.free_nodes
        eps_free = np.asarray(eps_free, dtype=np.float64)
        sig_free = np.asarray(sig_free, dtype=np.float64)
        if eps_free.shape != free.shape or sig_free.shape != free.shape:
            raise ValueError("coefficients must be given on the free nodes")
        self.eps = np.ones(nn)
        self.sig = np.zeros(nn)
        self.eps[free] = eps_free
        self.sig[free] = sig_free
        self.s = self.eps - 1.0

        # FD rows everywhere, then FEM rows inside the FEM cube.
        L_fd = fdm.fd_laplacian(g)
        m_fd = fdm.fd_mass(g)
        self.tets = g.kuhn_tets()
        self.G, self.vol = fem.p1_geometry(g.coords, self.tets)
        L_fem = fem.p1_stiffness(nn, self.tets, self.G, self.vol)
        m_fem = fem.p1_lumped_mass(nn, self.tets, self.vol)
        self.fem_mask = g.fem_rows.astype(np.float64)
        P = sp.diags(self.fem_mask)
        Q = sp.diags(1.0 - self.fem_mask)
        self.L = (Q @ L_fd + P @ L_fem).tocsr()
        self.m = (1.0 - self.fem_mask) * m_fd + self.fem_mask * m_fem
        self.L_fd, self.L_fem, self.m_fd, self.m_fem = L_fd, L_fem, m_fd, m_fem
        self.LT = self.L.T.tocsr()
        self.D = fem.p1_divergence(nn, self.tets, self.G, self.vol)
        self.face_mass = {f: fdm.fd_face_mass(g, f)
                          for f in ("x0", "x1", "y0", "y1", "bottom", "top")}

    # E, mu: arrays of shape (3, nn), component-major.
    def apply_K(self, E: np.ndarray) -> np.ndarray:
        out = np.stack([self.L @ E[c] for c in range(3)])
        SE = (self.s[None, :] * E).ravel()
        stab = (self.D.T @ (self.D @ SE)).reshape(3, -1)
        return out + self.fem_mask[None, :] * stab

    def apply_KT(self, mu: np.ndarray) -> np.ndarray:
        out = np.stack([self.LT @ mu[c] for c in range(3)])
        Pmu = (self.fem_mask[None, :] * mu).ravel()
        stab = (self.D.T @ (self.D @ Pmu)).reshape(3, -1)
        return out + self.s[None, :] * stab

    def apply_DtD_masked(self, mu: np.ndarray) -> np.ndarray:
        """D^T D P mu, the factor that meets dS/deps in the gradient."""
        Pmu = (self.fem_mask[None, :] * mu).ravel()
        return (self.D.T @ (self.D @ Pmu)).reshape(3, -1)

    def sparse_K(self) -> sp.csr_matrix:
        """K as one (3nn x 3nn) sparse matrix, for tests on small grids."""
        nn = self.g.nn
        I3L = sp.kron(sp.identity(3), self.L)
        P3 = sp.diags(np.tile(self.fem_mask, 3))
        S3 = sp.diags(np.tile(self.s, 3))
        return (I3L + P3 @ (self.D.T @ self.D) @ S3).tocsr()

    def damping(self, absorbing_faces) -> np.ndarray:
        """Diagonal of C for the given set of absorbing faces."""
        c = self.m * self.sig
        for f in absorbing_faces:
            c = c + self.face_mass[f]
        return c
