"""Pins of the oracle on a locally refined FEM mesh (conforming bisection of
the Kuhn cube, synth/mesh.py): the P1 operators on the refined elements
(symmetry, constants and linear fields in the kernel of the stiffness and
of the Gauss-law term, lumped masses adding up to the cube), the discrete
energy identity for eps = 1 with conductivity, the space-time adjoint dot
test, and central finite differences of J at every free node, the new nodes
included."""
import numpy as np
import pytest

from oracle import OracleProblem, SourceSpec
from oracle.cfl import lambda_max
from synth import detector_grid
from synth.mesh import refined_fem_mesh

N, FEM_N = 13, 9


def model(seed):
    rng = np.random.default_rng(seed)
    nf = (FEM_N - 4) ** 3
    return rng.uniform(4.0, 12.0, nf), rng.uniform(0.0, 0.5, nf)


@pytest.fixture(scope="module")
def mesh():
    eps, sig = model(0)
    par, tets = refined_fem_mesh(N, FEM_N, eps, sig, beta_eps=0.5, beta_sig=0.0)
    assert par.shape[0] > 0
    return par, tets


def refined_coeffs(par, eps_g, sig_g):
    from oracle.grid import RefinedGrid
    g = RefinedGrid(N, FEM_N, par, np.zeros((0, 4), dtype=np.int64))
    e = np.ones(g.nn)
    s = np.zeros(g.nn)
    free_g = np.nonzero(g.in_box(g.f0, g.f1))[0]
    e[free_g], s[free_g] = eps_g, sig_g
    for k, (p, q) in enumerate(par):
        v = g.n_grid + k
        e[v] = 0.5 * (e[p] + e[q])
        s[v] = 0.5 * (s[p] + s[q])
    free = np.concatenate([free_g, np.arange(g.n_grid, g.nn)])
    return e[free], s[free]


def problem(mesh, eps, sig, Nt=60, cfl=0.2, src=None, **kw):
    return OracleProblem(N, FEM_N, Nt, cfl, eps, sig, detector_grid(N, FEM_N, 2),
                         [src or SourceSpec(freq=4.0, t0=0.15, width=0.06)], mesh=mesh, **kw)


def test_refined_operators(mesh):
    par, tets = mesh
    e, s = refined_coeffs(par, *model(0))
    P = problem(mesh, e, s)
    op, g = P.op, P.g
    fem = g.fem_rows
    Lf = op.L_fem
    assert abs(Lf - Lf.T).max() <= 1e-12 * abs(Lf).max()
    X = g.coords
    h = g.h
    for lin in (X[:, 0], X[:, 1] - 2 * X[:, 2] + 0.3, np.ones(g.nn)):
        assert np.abs((Lf @ lin)[fem]).max() <= 1e-12 / h
    # Gauss-law term: a linear vector field has constant divergence
    V = np.stack([X[:, 0] + 2 * X[:, 1], 3 * X[:, 2] - X[:, 0], X[:, 1]])
    DtD = (op.D.T @ (op.D @ V.ravel())).reshape(3, -1)
    assert np.abs(DtD[:, fem]).max() <= 1e-12 * np.abs(DtD).max() + 1e-12
    # lumped masses: positive on the FEM nodes, adding up to the cube
    assert np.all(op.m_fem[fem] > 0)
    assert op.m_fem.sum() == pytest.approx(((FEM_N - 1) * h) ** 3, rel=1e-12)
    # the new nodes' masses are those of smaller elements
    assert op.m_fem[g.n_grid:].max() < 0.5 * h ** 3
    # one level of bisection puts every new node on the half-spacing lattice,
    # equidistant from its two parents
    Xe = X[g.n_grid:]
    assert np.allclose(Xe * 2 / h, np.round(Xe * 2 / h), atol=1e-9)
    dp = np.linalg.norm(Xe - X[par[:, 0]], axis=1)
    dq = np.linalg.norm(Xe - X[par[:, 1]], axis=1)
    assert np.allclose(dp, dq, rtol=1e-12)


def test_stable_step(mesh):
    par, _ = mesh
    e, s = refined_coeffs(par, *model(0))
    P = problem(mesh, e, s)
    lam = lambda_max(P.op, 800)
    assert P.tau < 2.0 / np.sqrt(lam)


def test_energy_identity_on_refined_mesh(mesh):
    par, _ = mesh
    rng = np.random.default_rng(4)
    nfg = (FEM_N - 4) ** 3
    e, s = refined_coeffs(par, np.ones(nfg), rng.uniform(0, 2.0, nfg))
    src = SourceSpec(freq=3.0, t0=0.3, width=0.1)
    Nt = 120
    P = problem(mesh, e, s, Nt=Nt, src=src)
    f = P.forward(0, keep_fields=range(Nt + 1))
    tau, M = P.tau, P.M
    E = lambda k: f.fields[k] if k >= 0 else np.zeros_like(f.fields[0])

    def energy(k):
        d = E(k + 1) - E(k)
        return 0.5 * np.sum(M * d * d) / tau ** 2 + 0.5 * np.sum(E(k + 1) * P.op.apply_K(E(k)))

    def magnitude(k):
        d = E(k + 1) - E(k)
        return 0.5 * np.sum(M * d * d) / tau ** 2 + 0.5 * np.sum(np.abs(E(k + 1) * P.op.apply_K(E(k))))

    scale = max(magnitude(k) for k in range(Nt))
    assert scale > 0
    for k in range(1, Nt):
        C = P.op.damping(P.absorbing_faces(k, src))
        dE = E(k + 1) - E(k - 1)
        F = P.source_term(k, src)
        lhs = energy(k) - energy(k - 1)
        rhs = -np.sum(C * dE * dE) / (4 * tau) + 0.5 * np.sum(F * dE)
        assert abs(lhs - rhs) <= 1e-12 * scale


def test_dot_test_on_refined_mesh(mesh):
    par, _ = mesh
    e, s = refined_coeffs(par, *model(1))
    P = problem(mesh, e, s, Nt=50, src=SourceSpec(freq=4.0, t0=0.15, width=0.05))
    rng = np.random.default_rng(2)
    Nt, nn = P.n_steps, P.g.nn
    Fs = rng.standard_normal((Nt, 3, nn)) * (rng.random(nn) < 0.3)[None, None, :]
    rs = rng.standard_normal((Nt + 1, P.det_nodes.size, 3))

    def r_src(k):
        j = np.zeros((3, nn))
        for c in range(3):
            np.add.at(j[c], P.det_nodes, rs[k, :, c])
        return j

    f = P.forward(0, source_override=lambda n: Fs[n])
    a = P.adjoint(0, f.trace, f.trace, keep_fields=range(Nt), residual_override=r_src)
    lhs = float(np.sum(rs[1:] * f.trace[1:]))
    rhs = -float(sum(np.sum(a.fields[n] * Fs[n]) for n in range(Nt)))
    assert abs(lhs - rhs) <= 1e-12 * max(abs(lhs), 1e-300)


@pytest.mark.parametrize("which", ["eps", "sig"])
def test_gradient_central_differences_on_refined_mesh(mesh, which):
    par, _ = mesh
    src = SourceSpec(freq=4.0, t0=0.15, width=0.06, direction=(0.3, -0.2, -0.93))
    e, s = refined_coeffs(par, *model(3))
    rng = np.random.default_rng(5)
    kw = dict(gamma_eps=0.02, gamma_sig=0.05, eps0_free=rng.uniform(1, 3, e.size),
              sig0_free=rng.uniform(0, 0.1, e.size))
    base = problem(mesh, e, s, src=src, **kw)
    e2, s2 = refined_coeffs(par, *model(4))
    eobs = problem(mesh, e2, s2, src=src).forward(0).trace * 0.7
    res = base.run([eobs])
    g = res["g_eps"] if which == "eps" else res["g_sig"]
    n_grid_free = (FEM_N - 4) ** 3
    idx = list(range(0, n_grid_free, 7)) + list(range(n_grid_free, e.size))  # every new node
    delta = 1e-5
    for i in idx:
        vals = []
        for sgn in (+1, -1):
            ee, ss = e.copy(), s.copy()
            if which == "eps":
                ee[i] += sgn * delta
            else:
                ss[i] += sgn * delta
            P = problem(mesh, ee, ss, src=src, **kw)
            vals.append(P.functional([P.forward(0).trace], [eobs]))
        fd = (vals[0] - vals[1]) / (2 * delta)
        assert abs(g[i] - fd) <= 1e-6 * np.abs(g).max(), i
