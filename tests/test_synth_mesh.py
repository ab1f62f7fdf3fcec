"""The locally refined FEM meshes (synth/mesh.py) are conforming
tetrahedrisations of the FEM cube: volumes add up to the cube, every interior
face is shared by exactly two elements, no split edge survives (no hanging
nodes), new nodes stay in the free box, and one level of refinement halves
the size of the marked elements."""
import itertools

import numpy as np
import pytest

from synth import workload
from synth.mesh import RefinedMesh, kuhn_cube, refined_fem_mesh


def coords(n, par):
    h = 1.0 / (n - 1)
    idx = np.arange(n ** 3)
    X = np.stack([idx % n, (idx // n) % n, idx // (n * n)], axis=1) * h
    out = [X]
    ex = np.zeros((par.shape[0], 3))
    allx = np.concatenate([X, ex])
    for e, (p, q) in enumerate(par):
        allx[n ** 3 + e] = 0.5 * (allx[p] + allx[q])
    return allx


def check_conforming(n, fem_n, par, tets):
    X = coords(n, par)
    P = X[tets]
    vol = np.linalg.det(P[:, 1:] - P[:, :1]) / 6.0
    assert np.all(np.abs(vol) > 0)
    h = 1.0 / (n - 1)
    assert np.abs(vol).sum() == pytest.approx(((fem_n - 1) * h) ** 3, rel=1e-12)
    faces = {}
    for t in tets:
        for f in itertools.combinations(sorted(t), 3):
            faces[f] = faces.get(f, 0) + 1
    a = (n - fem_n) // 2
    b = a + fem_n - 1
    lo, hi = a * h, b * h
    for f, c in faces.items():
        assert c in (1, 2)
        if c == 1:  # boundary face: on the cube's surface
            F = X[list(f)]
            on = [np.allclose(F[:, ax], lo) or np.allclose(F[:, ax], hi) for ax in range(3)]
            assert any(on), f
    edges = set()
    for t in tets:
        for i, j in itertools.combinations(t, 2):
            edges.add((min(i, j), max(i, j)))
    for p, q in par:
        assert (min(p, q), max(p, q)) not in edges  # split everywhere: no hanging node


@pytest.mark.parametrize("beta", [0.9, 0.6])
def test_refined_mesh_is_conforming(beta):
    w = workload("small", n=25, fem_n=17, seed=12)
    eps, sig = w.model()
    par, tets = refined_fem_mesh(w.n, w.fem_n, eps, sig, beta, 0.0)
    assert par.shape[0] > 0
    check_conforming(w.n, w.fem_n, par, tets)
    # new nodes lie inside the free box
    X = coords(w.n, par)[w.n ** 3:]
    h = 1.0 / (w.n - 1)
    a = (w.n - w.fem_n) // 2
    f0, f1 = (a + 2) * h, (a + w.fem_n - 3) * h
    assert np.all(X > f0 - 1e-12) and np.all(X < f1 + 1e-12)


def test_one_level_halves_the_marked_elements():
    n, fem_n = 13, 9
    mesh = RefinedMesh(n, fem_n)
    mid = [ti for ti in range(len(mesh.tets))
           if all(4 <= c <= 7 for v in mesh.tets[ti] for c in (v % n, (v // n) % n, v // (n * n)))][:3]
    d0 = [mesh.diameter(ti) for ti in mid]
    mesh.refine_marked(mid, levels=1)
    for ti, d in zip(mid, d0):
        kids = mesh._alive_descendants(ti)
        assert len(kids) == 8
        assert max(mesh.diameter(k) for k in kids) == pytest.approx(d / 2, rel=1e-12)
    par, tets = mesh.result()
    check_conforming(n, fem_n, par, tets)


def test_unrefined_mesh_is_the_kuhn_split():
    par, tets = RefinedMesh(13, 9).result()
    assert par.shape[0] == 0
    assert np.array_equal(np.sort(tets, axis=1), np.sort(kuhn_cube(13, 9), axis=1))
