"""Grid geometry and the Kuhn tetrahedral mesh of the FEM cube (oracle).

Test infrastructure only (see oracle/__init__.py).

Domain decomposition (Sec. 2 and Sec. 5, Fig. 1): Omega is split into an outer
region Omega_FDM, discretised by a structured hexahedral (finite difference)
grid, and an inner cube Omega_FEM, discretised by tetrahedra, with the FEM
boundary inside the FDM region.  Here Omega = [0,1]^3 carries n^3 grid nodes
(spacing h = 1/(n-1), node id i + n*(j + n*k), k = depth, top face k = n-1) and
the FEM cube is the node box [a, b]^3, centred.  Its tetrahedra are the six
Kuhn tetrahedra of every grid cube inside the box: for each permutation p of
the axes, the path 0 -> e_p0 -> e_p0+e_p1 -> (1,1,1).

Reading (the coupling is deferred by the paper to its reference [BL1]): FEM
rows are used for the nodes strictly inside the box, (a, b)^3; all other nodes
take FD rows; coefficients differ from vacuum only on the free nodes
[a+2, b-2]^3, so the FEM cube's outer two node layers carry epsilon = 1,
sigma = 0 as eq. epsilon_sigma_constraint requires of Omega_FDM.
"""
from __future__ import annotations

from itertools import permutations

import numpy as np


class Grid:
    def __init__(self, n: int, fem_n: int):
        if fem_n < 5 or fem_n > n - 2:
            raise ValueError("need 5 <= fem_n <= n-2")
        self.n = n
        self.h = 1.0 / (n - 1)
        self.fem_n = fem_n
        self.a = (n - fem_n) // 2
        self.b = self.a + fem_n - 1
        self.f0 = self.a + 2
        self.f1 = self.b - 2
        self.nn = n ** 3
        ijk = np.indices((n, n, n))  # [k, j, i] order of axes
        self.k_of = ijk[0].ravel()
        self.j_of = ijk[1].ravel()
        self.i_of = ijk[2].ravel()
        self.coords = np.stack([self.i_of, self.j_of, self.k_of], axis=1) * self.h

    def nid(self, i, j, k):
        return i + self.n * (j + self.n * k)

    # ---- node sets -------------------------------------------------------
    def in_box(self, lo, hi):
        return ((self.i_of >= lo) & (self.i_of <= hi) & (self.j_of >= lo)
                & (self.j_of <= hi) & (self.k_of >= lo) & (self.k_of <= hi))

    @property
    def fem_rows(self):
        """Nodes updated by FEM rows: strictly inside the FEM cube."""
        return self.in_box(self.a + 1, self.b - 1)

    @property
    def free_nodes(self):
        """Global ids of the free (coefficient) nodes, x fastest."""
        return np.nonzero(self.in_box(self.f0, self.f1))[0]

    def face_nodes(self, face: str):
        """Boolean mask of the nodes on one face of the domain."""
        n1 = self.n - 1
        sel = {
            "x0": self.i_of == 0, "x1": self.i_of == n1,
            "y0": self.j_of == 0, "y1": self.j_of == n1,
            "bottom": self.k_of == 0, "top": self.k_of == n1,
        }
        return sel[face]

    # ---- Kuhn tetrahedra of the FEM cube -----------------------------------
    def kuhn_tets(self):
        """(T, 4) global node ids of the six Kuhn tetrahedra of each cube in
        the FEM box."""
        cells = np.arange(self.a, self.b)
        K, J, I = np.meshgrid(cells, cells, cells, indexing="ij")
        base = np.stack([I.ravel(), J.ravel(), K.ravel()], axis=1)
        tets = []
        for p in permutations(range(3)):
            v = [base.copy()]
            for ax in p:
                w = v[-1].copy()
                w[:, ax] += 1
                v.append(w)
            tets.append(np.stack([self.nid(x[:, 0], x[:, 1], x[:, 2]) for x in v], axis=1))
        return np.concatenate(tets, axis=0)


class RefinedGrid(Grid):
    """The same grid with an explicit, locally refined FEM mesh (given as
    input geometry: new nodes as midpoints of two parent nodes, and the
    tetrahedra replacing the Kuhn split of the FEM cube).

    Node ids: grid nodes as in Grid, new node e is n^3 + e.  Every new node is
    a FEM row and a free (coefficient) node; the free-node order is the grid's
    free nodes, then the new nodes in order.  FD rows and the domain faces are
    those of the grid nodes."""

    def __init__(self, n: int, fem_n: int, parents, tets):
        super().__init__(n, fem_n)
        parents = np.asarray(parents, dtype=np.int64).reshape(-1, 2)
        self.n_grid = n ** 3
        self.n_extra = parents.shape[0]
        self.nn = self.n_grid + self.n_extra
        X = np.zeros((self.nn, 3))
        X[:self.n_grid] = self.coords
        for e, (p, q) in enumerate(parents):
            if p >= self.n_grid + e or q >= self.n_grid + e:
                raise ValueError("a new node's parents must precede it")
            X[self.n_grid + e] = 0.5 * (X[p] + X[q])
        self.coords = X
        pad = -np.ones(self.n_extra, dtype=self.i_of.dtype)
        self.i_of = np.concatenate([self.i_of, pad])
        self.j_of = np.concatenate([self.j_of, pad])
        self.k_of = np.concatenate([self.k_of, pad])
        self.parents = parents
        self._tets = np.asarray(tets, dtype=np.int64).reshape(-1, 4)

    @property
    def fem_rows(self):
        m = self.in_box(self.a + 1, self.b - 1)
        m[self.n_grid:] = True
        return m

    @property
    def free_nodes(self):
        grid_free = np.nonzero(self.in_box(self.f0, self.f1))[0]
        return np.concatenate([grid_free, np.arange(self.n_grid, self.nn)])

    def kuhn_tets(self):
        return self._tets
