"""Pins of the oracle's spatial operators against closed forms.

Each test checks the oracle against something fixed by mathematics, not by the
oracle: the DCT-I spectrum of the Neumann FD Laplacian, exactness of
second-order stencils on quadratic polynomials (including the ghost-node
Neumann closure), P1 exactness on linear fields, mass and area totals, and
the agreement of FEM and FD rows inside the FEM cube.
"""
import numpy as np
import pytest
import scipy.linalg as sla

from oracle.grid import Grid
from oracle.hybrid import HybridOperator


def make_op(n, fem_n, eps=None, sig=None, seed=0):
    g = Grid(n, fem_n)
    nf = g.free_nodes.size
    rng = np.random.default_rng(seed)
    if eps == "random":
        eps = rng.uniform(1.0, 25.0, nf)
    if sig == "random":
        sig = rng.uniform(0.0, 1.0, nf)
    eps = np.ones(nf) if eps is None else eps
    sig = np.zeros(nf) if sig is None else sig
    return g, HybridOperator(g, eps, sig)


def random_quadratic(rng):
    A = rng.standard_normal((3, 3))
    return A + A.T, rng.standard_normal(3), rng.standard_normal()


def test_lumped_masses_sum_to_volume_and_area():
    g, op = make_op(9, 5)
    assert op.m.sum() == pytest.approx(1.0, rel=1e-14)
    h = g.h
    interior = (g.i_of > 0) & (g.i_of < g.n - 1) & (g.j_of > 0) & (g.j_of < g.n - 1) \
        & (g.k_of > 0) & (g.k_of < g.n - 1)
    assert np.allclose(op.m[interior], h ** 3, rtol=1e-14)
    for f, b in op.face_mass.items():
        assert b.sum() == pytest.approx(1.0, rel=1e-14)   # unit face area
        on = g.face_nodes(f)
        # ghost-node closure: surface/volume ratio 2/h on every face node
        assert np.allclose(b[on] / op.m[on], 2.0 / h, rtol=1e-13)


@pytest.mark.parametrize("n", [5, 6, 8])
def test_fd_spectrum_is_dct1(n):
    """Eigenvalues of M^-1 L (FD, Neumann) are sum over axes of
    (4/h^2) sin^2(pi k / (2(n-1))), k = 0..n-1 (the DCT-I spectrum)."""
    from oracle import fdm
    g = _grid_no_fem(n)
    L = fdm.fd_laplacian(g).toarray()
    m = fdm.fd_mass(g)
    lam = sla.eigh(L, np.diag(m), eigvals_only=True)
    h = g.h
    k = np.arange(n)
    l1 = 4.0 / h ** 2 * np.sin(np.pi * k / (2 * (n - 1))) ** 2
    expect = np.sort((l1[:, None, None] + l1[None, :, None] + l1[None, None, :]).ravel())
    assert np.allclose(np.sort(lam), expect, rtol=1e-10, atol=1e-9)


class _grid_no_fem(Grid):
    def __init__(self, n):  # geometry only: FD operators do not look at the FEM box
        self.n = n
        self.h = 1.0 / (n - 1)
        self.nn = n ** 3
        ijk = np.indices((n, n, n))
        self.k_of, self.j_of, self.i_of = (x.ravel() for x in ijk)
        self.coords = np.stack([self.i_of, self.j_of, self.k_of], axis=1) * self.h


def test_hybrid_vacuum_spectrum_equals_fd():
    """With eps = 1 the hybrid operator has the FD spectrum (FE/FD agreement)."""
    g, op = make_op(9, 7)
    lam = sla.eigh(op.L.toarray(), np.diag(op.m), eigvals_only=True)
    h, n = g.h, g.n
    l1 = 4.0 / h ** 2 * np.sin(np.pi * np.arange(n) / (2 * (n - 1))) ** 2
    expect = np.sort((l1[:, None, None] + l1[None, :, None] + l1[None, None, :]).ravel())
    assert np.allclose(np.sort(lam), expect, rtol=1e-10, atol=1e-9)


def test_fem_rows_equal_fd_rows():
    g, op = make_op(13, 9)
    rows = np.nonzero(g.fem_rows)[0]
    d = (op.L_fem[rows] - op.L_fd[rows])
    assert abs(d).max() < 1e-14 * g.h * 10
    assert np.allclose(op.m_fem[rows], op.m_fd[rows], rtol=1e-14)
    # interior FEM row: h * (6, -1 x 6), the 7-point Laplacian
    c = g.nid(6, 6, 6)
    row = op.L_fem[c].toarray().ravel()
    nz = np.nonzero(np.abs(row) > 1e-15)[0]
    expect = {c: 6 * g.h}
    for off in (1, g.n, g.n * g.n):
        expect[c + off] = -g.h
        expect[c - off] = -g.h
    assert set(nz) == set(expect)
    for k, v in expect.items():
        assert row[k] == pytest.approx(v, rel=1e-13)


def test_laplacian_exact_on_quadratics_with_neumann_closure():
    """(M^-1 L f)_i = -Lap f + sum_{faces at i} (2/h) d_n f for quadratic f, at
    every node, corners and edges included."""
    g, op = make_op(11, 7, eps="random", seed=3)
    rng = np.random.default_rng(7)
    X = g.coords
    for _ in range(3):
        A, b, d = random_quadratic(rng)
        f = np.einsum("ni,ij,nj->n", X, A, X) + X @ b + d
        grad = 2.0 * X @ A + b
        expect = np.full(g.nn, -2.0 * np.trace(A))
        for ax, idx in enumerate((g.i_of, g.j_of, g.k_of)):
            expect += np.where(idx == 0, -grad[:, ax], 0.0) * 2.0 / g.h
            expect += np.where(idx == g.n - 1, grad[:, ax], 0.0) * 2.0 / g.h
        got = op.L @ f / op.m
        assert np.abs(got - expect).max() < 1e-12 * np.abs(expect).max()


def test_divdiv_exact_on_quadratics():
    """On the FEM rows, M^-1 D^T D w = -grad div w for quadratic w (the
    stabilising term of eq. forward_prob with eps-1 folded into w)."""
    g, op = make_op(13, 9)
    rng = np.random.default_rng(11)
    X = g.coords
    for _ in range(3):
        parts = [random_quadratic(rng) for _ in range(3)]
        w = np.stack([np.einsum("ni,ij,nj->n", X, A, X) + X @ b + d for A, b, d in parts])
        # div w = sum_c (2 A_c x + b_c)_c  =>  grad div w = 2 sum_c A_c[c, :]
        expect = -2.0 * sum(parts[c][0][c, :] for c in range(3))
        got = (op.D.T @ (op.D @ w.ravel())).reshape(3, -1) / op.m[None, :]
        rows = g.fem_rows
        assert np.abs(got[:, rows] - expect[:, None]).max() < 1e-11 * np.abs(expect).max()


def test_p1_geometry_and_divergence_of_linear_fields():
    g, op = make_op(9, 7)
    G, vol, tets = op.G, op.vol, op.tets
    assert vol.sum() == pytest.approx(((g.fem_n - 1) * g.h) ** 3, rel=1e-13)
    assert np.allclose(vol, g.h ** 3 / 6.0, rtol=1e-13)
    assert np.abs(G.sum(axis=1)).max() < 1e-10 / g.h
    X = g.coords[tets]
    eye = np.einsum("tac,tad->tcd", G, X)          # sum_a g_a x_a^T = I
    assert np.allclose(eye, np.eye(3)[None], atol=1e-12)
    rng = np.random.default_rng(5)
    A = rng.standard_normal((3, 3))
    c = rng.standard_normal(3)
    E = (g.coords @ A.T + c).T                       # E(x) = A x + c, shape (3, nn)
    div = op.D @ E.ravel()
    assert np.allclose(div, np.sqrt(vol) * np.trace(A), rtol=1e-11, atol=1e-13)


def test_divdiv_symmetric_psd_and_kills_constants():
    g, op = make_op(9, 7)
    DtD = (op.D.T @ op.D).toarray()
    assert np.abs(DtD - DtD.T).max() < 1e-15
    w = np.linalg.eigvalsh(DtD)
    assert w.min() > -1e-13
    for c in range(3):
        e = np.zeros((3, g.nn))
        e[c] = 1.0
        assert np.abs(DtD @ e.ravel()).max() < 1e-14


def test_K_transpose_and_adjoint_identity():
    g, op = make_op(11, 7, eps="random", sig="random", seed=2)
    rng = np.random.default_rng(3)
    K = op.sparse_K()
    for _ in range(3):
        x = rng.standard_normal((3, g.nn))
        y = rng.standard_normal((3, g.nn))
        assert np.allclose(op.apply_K(x).ravel(), K @ x.ravel(), rtol=1e-13, atol=1e-14)
        assert np.allclose(op.apply_KT(y).ravel(), K.T @ y.ravel(), rtol=1e-13, atol=1e-14)
        lhs = np.sum(op.apply_K(x) * y)
        rhs = np.sum(x * op.apply_KT(y))
        assert abs(lhs - rhs) <= 1e-13 * abs(lhs)
    # K is not symmetric once eps varies
    assert abs(K - K.T).max() > 1e-3 * abs(K).max()


def test_stabilisation_vanishes_outside_fem_rows():
    g, op = make_op(11, 7, eps="random", seed=4)
    rng = np.random.default_rng(9)
    E = rng.standard_normal((3, g.nn))
    stab = op.apply_K(E) - np.stack([op.L @ E[c] for c in range(3)])
    assert np.abs(stab[:, ~g.fem_rows]).max() == 0.0
