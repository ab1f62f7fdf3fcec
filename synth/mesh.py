"""Locally refined tetrahedral meshes of the FEM cube (input geometry).

The FEM cube [a, b]^3 starts as the six Kuhn tetrahedra of every grid cube,
vertex order (v0, v0 + e_p0, v0 + e_p0 + e_p1, v0 + (1,1,1)) for each axis
permutation p.  Elements are marked by the rule of Sec. 4 (eq. meshref):
K is refined where |h eps_h| >= beta_eps max |h eps_h| and
|h sigma_h| >= beta_sig max |h sigma_h|, with h the element diameter and the
element value the largest of its vertex values.  Marked elements are refined
by conforming newest-vertex bisection in Maubach's form: an element
(x0, x1, x2, x3) with tag k is cut at the midpoint z of its refinement edge
(x0, xk) into (x0, .., x_{k-1}, z, x_{k+1}, .., x3) and (x1, .., xk, z, x_{k+1}, .., x3),
both with tag k-1 (3 after 1); before an edge is cut, every element that
contains it is first refined until the edge is its refinement edge, so no
hanging node remains.  Three bisections halve the element size: one level of
refinement.

This module lays out geometry only (no operator, no time stepping): both the
CPU oracle and the CUDA path take its output as explicit (nodes, tets).
Node ids: grid node i + n (j + n k); new node e has id n^3 + e and is the
midpoint of its two parent nodes (ids of grid or earlier new nodes).
"""
from __future__ import annotations

from itertools import permutations

import numpy as np


def kuhn_cube(n: int, fem_n: int):
    """(T, 4) node ids of the Kuhn tetrahedra of the FEM cube, Maubach order."""
    a = (n - fem_n) // 2
    b = a + fem_n - 1
    cells = np.arange(a, b)
    K, J, I = np.meshgrid(cells, cells, cells, indexing="ij")
    base = np.stack([I.ravel(), J.ravel(), K.ravel()], axis=1)
    out = []
    for p in permutations(range(3)):
        v = [base.copy()]
        for ax in p:
            w = v[-1].copy()
            w[:, ax] += 1
            v.append(w)
        out.append(np.stack([x[:, 0] + n * (x[:, 1] + n * x[:, 2]) for x in v], axis=1))
    return np.concatenate(out, axis=0)


class RefinedMesh:
    """Conforming bisection refinement of the Kuhn mesh of the FEM cube.

    active: optional node box (lo, hi) (grid indices); only the Kuhn elements
    inside it take part in the refinement bookkeeping, the others are kept
    as they are (an error is raised if the conformity closure reaches them)."""

    def __init__(self, n: int, fem_n: int, active=None):
        self.n = n
        self.h = 1.0 / (n - 1)
        self.n3 = n ** 3
        t = kuhn_cube(n, fem_n)
        if active is not None:
            lo, hi = active
            ijk = np.stack([t % n, (t // n) % n, t // (n * n)], axis=2)
            inside = np.all((ijk >= lo) & (ijk <= hi), axis=(1, 2))
            self.static = t[~inside]
            t = t[inside]
            # nodes shared with static elements: edges between two such nodes
            # may not be cut
            self.frozen = set(map(int, np.unique(self.static)))
        else:
            self.static = np.zeros((0, 4), dtype=np.int64)
            self.frozen = set()
        self.tets = [list(map(int, r)) for r in t]
        self.tag = [3] * len(self.tets)
        self.gen = [0] * len(self.tets)
        self.alive = [True] * len(self.tets)
        self.parents = []                  # new node e: (parent, parent)
        self.coords = {}                   # new node id -> coordinates
        self.mid = {}                      # sorted edge -> new node id
        self.edges = {}                    # sorted edge -> set of alive tets
        self.kids = {}                     # cut element -> its two children
        for ti in range(len(self.tets)):
            self._add_edges(ti)

    # ---- geometry -------------------------------------------------------------
    def xyz(self, v: int) -> np.ndarray:
        if v < self.n3:
            n = self.n
            return np.array([v % n, (v // n) % n, v // (n * n)], dtype=np.float64) * self.h
        return self.coords[v]

    def _edge_list(self, ti):
        t = self.tets[ti]
        return [(min(t[i], t[j]), max(t[i], t[j])) for i in range(4) for j in range(i + 1, 4)]

    def _add_edges(self, ti):
        for e in self._edge_list(ti):
            self.edges.setdefault(e, set()).add(ti)

    def _drop_edges(self, ti):
        for e in self._edge_list(ti):
            s = self.edges[e]
            s.discard(ti)
            if not s:
                del self.edges[e]

    def ref_edge(self, ti):
        t, k = self.tets[ti], self.tag[ti]
        return (min(t[0], t[k]), max(t[0], t[k]))

    # ---- bisection ------------------------------------------------------------
    def _midpoint(self, e):
        if e[0] in self.frozen and e[1] in self.frozen:
            raise RuntimeError("refinement closure reached the inactive part of the mesh")
        if e not in self.mid:
            v = self.n3 + len(self.parents)
            self.parents.append(e)
            self.coords[v] = 0.5 * (self.xyz(e[0]) + self.xyz(e[1]))
            self.mid[e] = v
        return self.mid[e]

    def _bisect(self, ti):
        t, k = self.tets[ti], self.tag[ti]
        z = self._midpoint((min(t[0], t[k]), max(t[0], t[k])))
        c1 = t[:k] + [z] + t[k + 1:]
        c2 = t[1:k + 1] + [z] + t[k + 1:]
        nk = k - 1 if k > 1 else 3
        self._drop_edges(ti)
        self.alive[ti] = False
        kids = []
        for c in (c1, c2):
            self.tets.append(c)
            self.tag.append(nk)
            self.gen.append(self.gen[ti] + 1)
            self.alive.append(True)
            self._add_edges(len(self.tets) - 1)
            kids.append(len(self.tets) - 1)
        self.kids[ti] = kids
        return kids

    def refine(self, ti):
        """Bisect element ti and, first, whatever conformity requires."""
        if not self.alive[ti]:
            return
        e = self.ref_edge(ti)
        while True:
            patch = list(self.edges.get(e, ()))
            other = [s for s in patch if self.ref_edge(s) != e]
            if not other:
                break
            self.refine(other[0])
        for s in list(self.edges.get(e, ())):
            self._bisect(s)

    # ---- marking and levels -------------------------------------------------------
    def diameter(self, ti):
        X = np.array([self.xyz(v) for v in self.tets[ti]])
        d = X[:, None, :] - X[None, :, :]
        return float(np.sqrt((d * d).sum(axis=2).max()))

    def refine_marked(self, marked, levels: int = 1):
        """Refine the marked elements (ids of alive elements) `levels` times."""
        target = {ti: self.gen[ti] + 3 * levels for ti in marked}
        work = list(target.items())
        while work:
            ti, tg = work.pop()
            if self.alive[ti]:
                if self.gen[ti] >= tg:
                    continue
                self.refine(ti)
            # the element was cut (by this call or by a neighbour's closure):
            # continue with its alive descendants
            for d in self._alive_descendants(ti):
                if self.gen[d] < tg:
                    work.append((d, tg))

    def _alive_descendants(self, ti):
        out, stack = [], list(self.kids.get(ti, ()))
        while stack:
            u = stack.pop()
            if self.alive[u]:
                out.append(u)
            else:
                stack.extend(self.kids.get(u, ()))
        return out

    def result(self):
        tets = np.array([t for t, al in zip(self.tets, self.alive) if al], dtype=np.int64).reshape(-1, 4)
        par = np.array(self.parents, dtype=np.int64).reshape(-1, 2)
        return par, np.concatenate([self.static, tets])


def mark_elements(mesh: RefinedMesh, node_eps, node_sig, beta_eps: float, beta_sig: float):
    """Alive elements with |h eps_h| >= beta_eps max and |h sig_h| >= beta_sig max
    (eq. meshref); node_eps(v), node_sig(v) give nodal values.  Element value:
    the largest of its vertex values times its diameter."""
    ids = [ti for ti, al in enumerate(mesh.alive) if al]
    he = np.array([mesh.diameter(ti) * max(abs(node_eps(v)) for v in mesh.tets[ti]) for ti in ids])
    hs = np.array([mesh.diameter(ti) * max(abs(node_sig(v)) for v in mesh.tets[ti]) for ti in ids])
    keep = (he >= beta_eps * he.max()) & (hs >= beta_sig * hs.max())
    return [ti for ti, k in zip(ids, keep) if k]


def refined_fem_mesh(n: int, fem_n: int, eps_free, sig_free, beta_eps: float = 0.8, beta_sig: float = 0.8,
                     levels: int = 1, region=None):
    """The FEM cube's Kuhn mesh refined `levels` times where eq. meshref marks
    it, for nodal coefficients given on the free nodes [a+2, b-2]^3 (x fastest;
    eps = 1, sigma = 0 elsewhere).  Marking only looks at elements whose nodes
    all lie in [a+3, b-3]^3 (and in region = (lo, hi), node indices, if given),
    so that the closure stays inside the free box.  Returns (parents (E, 2), tets (T, 4)) as described in the module header."""
    a = (n - fem_n) // 2
    b = a + fem_n - 1
    f0, f1 = a + 2, b - 2
    nf = f1 - f0 + 1
    E = np.asarray(eps_free, dtype=np.float64).reshape(nf, nf, nf)
    S = np.asarray(sig_free, dtype=np.float64).reshape(nf, nf, nf)
    # refinement bookkeeping only around the marked candidates (the
    # closure of newest-vertex bisection on a Kuhn mesh stays within a few
    # cells of them)
    cand = (E >= beta_eps * E.max()) & (S >= beta_sig * S.max()) if beta_eps > 0 or beta_sig > 0 else None
    rlo, rhi = (a + 3, b - 3) if region is None else (max(a + 3, region[0]), min(b - 3, region[1]))
    if cand is not None:
        K, J, I = np.meshgrid(*(np.arange(f0, f1 + 1),) * 3, indexing="ij")
        cand &= (I >= rlo) & (I <= rhi) & (J >= rlo) & (J <= rhi) & (K >= rlo) & (K <= rhi)
    active = None
    if cand is not None and cand.any():
        idx = np.argwhere(cand)  # (k, j, i) of free nodes
        lo = max(a, int(idx.min()) + f0 - 4)
        hi = min(b, int(idx.max()) + f0 + 4)
        active = (lo, hi)
    mesh = RefinedMesh(n, fem_n, active)

    def ijk(v):
        return v % n, (v // n) % n, v // (n * n)

    def val(arr, vac):
        def f(v):
            i, j, k = ijk(v)
            if f0 <= i <= f1 and f0 <= j <= f1 and f0 <= k <= f1:
                return arr[k - f0, j - f0, i - f0]
            return vac
        return f

    inner = [ti for ti in range(len(mesh.tets))  # marking restricted to these
             if all(rlo <= c <= rhi for v in mesh.tets[ti] for c in ijk(v))]
    marked_all = mark_elements(mesh, val(E, 1.0), val(S, 0.0), beta_eps, beta_sig)
    inner_set = set(inner)
    marked = [ti for ti in marked_all if ti in inner_set]
    mesh.refine_marked(marked, levels)
    return mesh.result()


def extend_to_new_nodes(n: int, fem_n: int, parents, eps_free, sig_free):
    """Coefficients on the free nodes of a refined mesh: the grid's free nodes
    (x fastest) followed by the new nodes, each the mean of its parents (the
    P1 interpolant at an edge midpoint, the interpolation onto the refined
    mesh of Sec. 4)."""
    a = (n - fem_n) // 2
    f0, f1 = a + 2, a + fem_n - 3
    nf = f1 - f0 + 1
    n3 = n ** 3
    E = np.asarray(eps_free, dtype=np.float64).reshape(nf, nf, nf)
    S = np.asarray(sig_free, dtype=np.float64).reshape(nf, nf, nf)
    parents = np.asarray(parents, dtype=np.int64).reshape(-1, 2)
    ne = np.empty(parents.shape[0])
    ns = np.empty(parents.shape[0])

    def value(v):
        if v >= n3:
            return ne[v - n3], ns[v - n3]
        i, j, k = v % n, (v // n) % n, v // (n * n)
        if f0 <= i <= f1 and f0 <= j <= f1 and f0 <= k <= f1:
            return E[k - f0, j - f0, i - f0], S[k - f0, j - f0, i - f0]
        return 1.0, 0.0

    for e, (p, q) in enumerate(parents):
        (ep, sp), (eq, sq) = value(p), value(q)
        ne[e] = 0.5 * (ep + eq)
        ns[e] = 0.5 * (sp + sq)
    return (np.concatenate([np.asarray(eps_free, float).ravel(), ne]),
            np.concatenate([np.asarray(sig_free, float).ravel(), ns]))
