"""Pins of the oracle's adjoint, functional, gradient, CFL bound and source.

* space-time dot test: for any top-face source sequence F and detector
  weights r, sum_k r^k . E^k_det = -sum_n mu^n . F^n, which holds only if the
  backward recursion is the exact transpose of the forward one (including the
  time-shifted damping of the top-face switch);
* central finite differences of J at every free node, for eps and sigma, with
  regularisation, oblique incidence and the z_delta taper;
* J vanishes for Eobs equal to the model's own trace and is quadratic in the
  residual;
* the power-iteration bound against dense eigenvalues and the closed-form
  vacuum maximum 12/h^2; a real spectrum for eps = 1 and a non-real one for
  variable eps (the Gauss-law term is not self-adjoint);
* source flux totals, the integer switch step and z_delta's shape.
"""
import math

import numpy as np
import pytest
import scipy.linalg as sla

from oracle import OracleProblem, SourceSpec
from oracle.cfl import lambda_max
from oracle.source import z_delta
from synth import detector_grid


def tiny_problem(n=9, fem_n=7, Nt=60, seed=0, src=None, gamma=(0.0, 0.0), zfrac=0.1,
                 eps=None, sig=None, det=2):
    rng = np.random.default_rng(seed)
    nf = (fem_n - 4) ** 3
    eps = rng.uniform(4.0, 12.0, nf) if eps is None else eps
    sig = rng.uniform(0.0, 0.5, nf) if sig is None else sig
    return OracleProblem(n, fem_n, Nt, 0.3, eps, sig, detector_grid(n, fem_n, det),
                         [src or SourceSpec(freq=4.0, t0=0.15, width=0.06)],
                         gamma_eps=gamma[0], gamma_sig=gamma[1], z_delta_frac=zfrac,
                         eps0_free=rng.uniform(1.0, 3.0, nf), sig0_free=rng.uniform(0, 0.1, nf))


def test_space_time_dot_test():
    P = tiny_problem(n=11, fem_n=7, Nt=50, seed=1,
                     src=SourceSpec(freq=4.0, t0=0.15, width=0.05))
    n1 = P.sources[0].switch_step(P.tau, P.top_coords)
    assert 5 < n1 < 45           # the top face switches inside the run
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


def _J(P, eobs):
    return P.functional([P.forward(0).trace], [eobs])


@pytest.mark.parametrize("which", ["eps", "sig"])
def test_gradient_matches_central_differences_everywhere(which):
    src = SourceSpec(freq=4.0, t0=0.15, width=0.06, direction=(0.3, -0.2, -0.93))
    base = tiny_problem(seed=3, src=src, gamma=(0.02, 0.05))
    eobs = tiny_problem(seed=4, src=src).forward(0).trace * 0.7
    res = base.run([eobs])
    g = res["g_eps"] if which == "eps" else res["g_sig"]
    eps0 = base.op.eps[base.g.free_nodes].copy()
    sig0 = base.op.sig[base.g.free_nodes].copy()
    delta = 1e-5
    fd = np.empty_like(g)
    for i in range(g.size):
        vals = []
        for s in (+1, -1):
            e, sg = eps0.copy(), sig0.copy()
            if which == "eps":
                e[i] += s * delta
            else:
                sg[i] += s * delta
            P = OracleProblem(base.g.n, base.g.fem_n, base.n_steps, 0.3, e, sg,
                              detector_grid(base.g.n, base.g.fem_n, 2), [src],
                              gamma_eps=base.gamma_eps, gamma_sig=base.gamma_sig,
                              z_delta_frac=base.z_delta_frac,
                              eps0_free=base.eps0, sig0_free=base.sig0)
            vals.append(_J(P, eobs))
        fd[i] = (vals[0] - vals[1]) / (2 * delta)
    assert np.abs(g - fd).max() <= 1e-6 * np.abs(g).max()


def test_functional_zero_at_own_trace_and_quadratic():
    P = tiny_problem(seed=5)
    tr = P.forward(0).trace
    assert P.functional([tr], [tr]) == 0.0
    res = P.run([tr])
    assert np.abs(res["g_eps"]).max() == 0.0 and np.abs(res["g_sig"]).max() == 0.0
    d = np.random.default_rng(6).standard_normal(tr.shape)
    j1 = P.misfit([tr], [tr + d])
    j3 = P.misfit([tr], [tr + 3 * d])
    assert j3 == pytest.approx(9 * j1, rel=1e-13)
    # rectangle rule in time with the z_delta taper, t_1 .. t_Nt
    t = np.arange(P.n_steps + 1) * P.tau
    zz = z_delta(t, P.T, P.z_delta_frac)
    assert j1 == pytest.approx(0.5 * P.tau * np.sum(zz[1:, None, None] * d[1:] ** 2), rel=1e-13)


def test_regularisation_gradient_closed_form():
    """With Eobs = own trace the gradient is exactly gamma m (c - c0)."""
    P = tiny_problem(seed=7, gamma=(0.3, 0.7))
    tr = P.forward(0).trace
    res = P.run([tr])
    m = P.op.m[P.g.free_nodes]
    assert np.allclose(res["g_eps"], 0.3 * m * (P.op.eps[P.g.free_nodes] - P.eps0), rtol=1e-14)
    assert np.allclose(res["g_sig"], 0.7 * m * (P.op.sig[P.g.free_nodes] - P.sig0), rtol=1e-14)


def test_power_iteration_vacuum_closed_form():
    P = tiny_problem(eps=np.ones(27), sig=np.zeros(27))
    lam = lambda_max(P.op, iters=600)
    assert lam == pytest.approx(12.0 / P.g.h ** 2, rel=1e-4)


def test_power_iteration_matches_dense_spectrum():
    P = tiny_problem(seed=8)
    K = P.op.sparse_K().toarray()
    w = sla.eigvals(K / np.tile(P.M, 3)[:, None])
    lam = lambda_max(P.op, iters=1500)
    assert lam == pytest.approx(np.abs(w).max(), rel=1e-3)
    # the workloads' CFL 0.3 is far inside the stability bound
    assert P.tau < 0.8 * 2.0 / math.sqrt(np.abs(w).max())


def test_spectrum_real_for_eps_one_complex_for_variable_eps():
    """The Gauss-law term -grad div((eps - 1) E) of Sec. 2 is not self-adjoint
    once eps varies: with eps = 1 the stepped operator M_eps^-1 K has a real
    spectrum, with eps jumping at the FEM cube (and varying inside it) some
    eigenvalues leave the real axis -- modes that grow at any time step, and
    the reason rough iterates of the CGA can make the forward run overflow."""
    def spectrum(P):
        return sla.eigvals(P.op.sparse_K().toarray() / np.tile(P.M, 3)[:, None])

    vac = spectrum(tiny_problem(eps=np.ones(27), sig=np.zeros(27)))
    assert np.abs(vac.imag).max() <= 1e-9 * np.abs(vac).max()
    var = spectrum(tiny_problem(seed=9, sig=np.zeros(27)))
    assert np.abs(var.imag).max() >= 1e-4 * np.abs(var).max()
    assert var.real.min() >= -1e-9 * np.abs(var).max()


def test_source_flux_total_and_polarisation():
    P = tiny_problem()
    src = P.sources[0]
    for n in (0, 3, 7):
        F = P.source_term(n, SourceSpec())
        total = F.sum(axis=1)
        # unit top face: sum of lumped flux = P(t_n) in the y component only
        assert total[1] == pytest.approx(float(SourceSpec().pulse(n * P.tau)), rel=1e-13, abs=1e-18)
        assert total[0] == 0.0 and total[2] == 0.0
    obl = SourceSpec(direction=(0.4, 0.1, -0.9))
    d = obl.delays(P.top_coords)
    assert d.min() == pytest.approx(0.0, abs=1e-15) and d.min() >= 0.0
    p = obl.polarisation()
    k = np.array(obl.direction) / np.linalg.norm(obl.direction)
    assert abs(p @ k) < 1e-15 and np.linalg.norm(p) == pytest.approx(1.0)
    assert np.allclose(SourceSpec().polarisation(), [0, 1, 0])
    assert np.all(SourceSpec().delays(P.top_coords) == 0.0)
    del src


def test_switch_step_integer_rule():
    src = SourceSpec()                    # t1 = t0 + 3w = 1.5
    top = np.array([[0.5, 0.5, 1.0]])
    assert src.switch_step(0.0015, top) == 1000      # t1 / tau = 1000 exactly
    assert src.switch_step(0.0015000000000000002, top) == 1000
    assert src.switch_step(0.0014999999999999998, top) == 1000
    assert SourceSpec(t1=0.01).switch_step(0.003, top) == 3


def test_z_delta_shape():
    T = 2.0
    t = np.linspace(0, T, 2001)
    z = z_delta(t, T, 0.1)
    assert z[0] == 1.0 and z[-1] == pytest.approx(0.0, abs=1e-15)
    assert np.all(z[t <= 1.8] == 1.0)
    assert np.all(np.diff(z) <= 1e-15)
    assert np.all(z_delta(t, T, 0.0) == 1.0)
