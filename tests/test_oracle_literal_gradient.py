"""Pins of the oracle's paper-literal gradient (eq. gradeps with the
approximation div(eps_bar E) ~ eps_bar div E of Sec. 4):

* brute force: at sampled nodes, the Gauss-law term from an explicit loop over
  the tets around the node, with barycentric gradients and volumes taken from
  the vertex coordinates, equals the assembled form;
* an exact identity: summed over every node, the literal term and the exact
  derivative's term E_i . (D^T D P mu)_i agree, since both equal
  sum_K |K| (div E)_K (div P mu)_K;
* checked against the exact discrete gradient (O6): g_sig is the same, and on a
  25^3 grid g_eps points the same way (cosine > 0.95) while it is no longer
  the derivative of the discrete J (it differs by the dropped
  grad(eps_bar) . E term).
"""
import numpy as np
import pytest

from helpers import oracle_problem
from oracle import OracleProblem, SourceSpec
from synth import detector_grid, workload


def tiny(seed=0):
    n, fem_n = 11, 7
    rng = np.random.default_rng(seed)
    nf = (fem_n - 4) ** 3
    return OracleProblem(n, fem_n, 20, 0.3, rng.uniform(2, 9, nf), rng.uniform(0, 0.5, nf),
                         detector_grid(n, fem_n, 2), [SourceSpec()])


def test_literal_term_matches_a_brute_force_element_loop():
    P = tiny()
    rng = np.random.default_rng(1)
    nn = P.g.nn
    E, mu = rng.standard_normal((3, nn)), rng.standard_normal((3, nn))
    got = P.literal_div_term(E, mu)
    X = P.g.coords
    tets = P.op.tets
    fem = P.op.fem_mask
    for i in P.g.free_nodes[::5]:
        want = 0.0
        for t in np.nonzero((tets == i).any(axis=1))[0]:
            A = np.ones((4, 4))
            A[:, 1:] = X[tets[t]]
            G = np.linalg.inv(A)[1:, :]          # column b: grad of the barycentric function b
            vol = abs(np.linalg.det(A)) / 6.0
            divE = sum(G[:, b] @ E[:, tets[t, b]] for b in range(4))
            divM = sum(G[:, b] @ (fem[tets[t, b]] * mu[:, tets[t, b]]) for b in range(4))
            want += vol / 4.0 * divE * divM
        assert got[i] == pytest.approx(want, rel=1e-12, abs=1e-12 * abs(got).max())


def test_literal_and_exact_terms_agree_summed_over_all_nodes():
    P = tiny(2)
    rng = np.random.default_rng(3)
    E, mu = rng.standard_normal((3, P.g.nn)), rng.standard_normal((3, P.g.nn))
    lit = P.literal_div_term(E, mu)
    exact = np.sum(E * P.op.apply_DtD_masked(mu), axis=0)
    assert lit.sum() == pytest.approx(exact.sum(), rel=1e-12)
    # node by node they differ
    assert np.abs(lit - exact).max() > 1e-3 * np.abs(exact).max()


def test_literal_gradient_checked_against_the_exact_one():
    w = workload("small")
    src = [SourceSpec()]
    eobs = [oracle_problem(w, *w.model(), src).forward(0).trace]
    P = oracle_problem(w, *w.model(inclusions=False), src)
    keep = range(w.n_steps + 1)
    f = P.forward(0, keep_fields=keep)
    a = P.adjoint(0, f.trace, eobs[0], keep_fields=keep)
    ge, gs = P.gradient([f], [a])
    gl, gsl = P.gradient_literal([f], [a])
    assert np.array_equal(gs, gsl)
    cos = ge @ gl / (np.linalg.norm(ge) * np.linalg.norm(gl))
    assert cos > 0.95
    assert np.linalg.norm(gl - ge) > 0.05 * np.linalg.norm(ge)
    with pytest.raises(ValueError):
        P.gradient_literal([P.forward(0)], [a])
