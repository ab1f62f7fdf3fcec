"""Pins of the oracle's conjugate gradient algorithm (Sec. 4, CGA).

A hand-iterated one-node problem (tests/golden/cga_scalar.txt, derivation in
the file) fixes the Fletcher-Reeves directions, the step-size rule, the
gamma schedule, the functional with the current gamma and the stopping rule;
node duplication fixes the mass weighting of the inner products; a low
eps_max fixes the clamp; on the real discrete problem the first CG step is a
descent step of the oracle's functional."""
import math
import os

import numpy as np
import pytest

from oracle.cg import CGParams, cga

GOLD = os.path.join(os.path.dirname(__file__), "golden", "cga_scalar.txt")


def golden():
    out = {}
    for line in open(GOLD):
        line = line.strip()
        if not line or line.startswith("#"):
            continue
        k, v = line.split("=", 1)
        out[k.strip()] = [float(x) for x in v.split(",")]
    return out


def scalar_problem(m=np.array([2.0])):
    def evaluate(eps, sig):
        J = 0.5 * float(np.sum(m * ((eps - 5.0) ** 2 + 2.0 * (sig - 1.0) ** 2)))
        return J, m * (eps - 5.0), m * 2.0 * (sig - 1.0)
    return evaluate


PRM = dict(gamma_eps0=1.0, gamma_sig0=2.0, alpha_eps0=0.25, alpha_sig0=0.125, p=0.5,
           eps_max=1e9, sig_max=1e9)


def test_hand_iterated_sequence():
    g = golden()
    m = np.array([2.0])
    eps, sig, log = cga(scalar_problem(m), np.array([2.0]), np.array([0.0]), m,
                        CGParams(max_iter=3, **PRM))
    assert len(log) == 3 and not any(r["stop"] for r in log)
    assert eps[0] == pytest.approx(g["eps"][3], rel=1e-14)
    assert sig[0] == pytest.approx(g["sig"][3], rel=1e-14)
    for key in ("J", "gnorm_eps", "gnorm_sig", "alpha_eps", "alpha_sig", "beta_eps", "beta_sig",
                "gamma_eps", "gamma_sig"):
        assert [r[key] for r in log] == pytest.approx(g[key], rel=1e-14, abs=1e-15), key
    for key in ("step_eps", "step_sig"):
        assert [r[key] for r in log[:2]] == pytest.approx(g[key], rel=1e-14), key


def test_restart_option():
    g = golden()
    m = np.array([2.0])
    eps, sig, log = cga(scalar_problem(m), np.array([2.0]), np.array([0.0]), m,
                        CGParams(max_iter=3, restart=True, **PRM))
    assert eps[0] == pytest.approx(g["eps3_restart"][0], rel=1e-14)
    assert sig[0] == pytest.approx(g["sig3_restart"][0], rel=1e-14)
    assert [r["beta_eps"] for r in log] == pytest.approx([0.0, 0.25, g["beta2_restart"][0]])
    assert [r["J"] for r in log] == pytest.approx(g["J"], rel=1e-14)


def test_stopping_rule():
    g = golden()
    m = np.array([2.0])
    eps, sig, log = cga(scalar_problem(m), np.array([2.0]), np.array([0.0]), m,
                        CGParams(max_iter=10, eta1_eps=1.2, eta1_sig=1.2, eta2_eps=0.0, eta2_sig=2.5,
                                 **PRM))
    stop_it = int(g["stop_after"][0])
    assert len(log) == stop_it + 1 and log[-1]["stop"] and not any(r["stop"] for r in log[:-1])
    assert eps[0] == pytest.approx(g["eps"][stop_it + 1], rel=1e-14)
    assert sig[0] == pytest.approx(g["sig"][stop_it + 1], rel=1e-14)


def test_inner_products_are_mass_weighted():
    """A node of mass 2 behaves exactly as two nodes of mass 1 with the same data."""
    m1 = np.array([2.0])
    m2 = np.array([1.0, 1.0])
    a = cga(scalar_problem(m1), np.array([2.0]), np.array([0.0]), m1, CGParams(max_iter=4, **PRM))
    b = cga(scalar_problem(m2), np.array([2.0, 2.0]), np.array([0.0, 0.0]), m2, CGParams(max_iter=4, **PRM))
    assert b[0] == pytest.approx([a[0][0]] * 2, rel=1e-14)
    assert b[1] == pytest.approx([a[1][0]] * 2, rel=1e-14)
    for ra, rb in zip(a[2], b[2]):
        for key in ("J", "gnorm_eps", "alpha_eps", "beta_sig", "step_sig"):
            assert rb[key] == pytest.approx(ra[key], rel=1e-13), key


def test_updates_are_clamped_to_the_admissible_set():
    m = np.array([2.0])
    prm = dict(PRM, eps_max=4.5, sig_max=0.9)
    eps, sig, log = cga(scalar_problem(m), np.array([2.0]), np.array([0.0]), m, CGParams(max_iter=2, **prm))
    # unclamped iterate 2 would be (5, 1)
    assert eps[0] == 4.5 and sig[0] == 0.9


def test_first_step_descends_on_the_discrete_problem():
    """The first CG direction is -g: for a small step the oracle's functional
    decreases by about alpha (g, d) (the gradient itself is pinned by finite
    differences elsewhere)."""
    from helpers import oracle_problem, oracle_sources
    from oracle.cg import problem_evaluator
    from synth import workload
    w = workload("tiny", n_steps=120)
    srcs = oracle_sources(w)
    e_lay, s_lay = w.model(inclusions=False)
    P0 = oracle_problem(w, *w.model(), srcs)
    eobs = [P0.forward(0).trace]
    P = oracle_problem(w, e_lay, s_lay, srcs)
    m = P.op.m[P.g.free_nodes]
    evaluate = problem_evaluator(P)(eobs)
    J0, ge, gs = evaluate(e_lay, s_lay)
    alpha = 1e-3 / np.sqrt(np.sum(m * (ge / m) ** 2) + np.sum(m * (gs / m) ** 2))
    eps, sig, log = cga(evaluate, e_lay, s_lay, m,
                        CGParams(max_iter=1, gamma_eps0=0.0, gamma_sig0=0.0, alpha_eps0=alpha, alpha_sig0=alpha))
    J1, _, _ = evaluate(eps, sig)
    pred = -alpha * (np.sum(ge * ge / m) + np.sum(gs * gs / m))
    assert J1 < J0
    assert (J1 - J0) == pytest.approx(pred, rel=2e-2)
