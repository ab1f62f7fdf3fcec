"""Pins of the oracle's forward time stepping.

* vacuum, normal incidence: the 3-D field is laterally invariant and equals a
  separately written 1-D textbook leapfrog (ghost-node Neumann source and
  absorbing ends) of the 1-D model problem, to rounding;
* that 1-D scheme converges at O(h^2) to d'Alembert's solution
  E_y(z, t) = int_0^{t-(1-z)} P(s) ds of the half-space problem;
* the discrete energy identity of the central scheme for eps = 1, sigma >= 0;
* a manufactured solution with variable eps and sigma (forcing built
  symbolically from eq. forward_prob) converges at second order;
* long runs with the layered-inclusion model stay bounded.
"""
import math

import numpy as np
import pytest

from oracle import OracleProblem, SourceSpec
from oracle.solver import ABS_BOTTOM, ABS_TOP
from synth import detector_grid, layered_inclusion_model


def vacuum_problem(n, fem_n, n_steps, src=None, absorbing=ABS_BOTTOM | ABS_TOP, cfl=0.3):
    nf = (fem_n - 4) ** 3
    det = detector_grid(n, fem_n, 2)
    return OracleProblem(n, fem_n, n_steps, cfl, np.ones(nf), np.zeros(nf), det,
                         [src or SourceSpec()], absorbing=absorbing)


def leapfrog_1d(n, n_steps, cfl, src: SourceSpec, n1):
    """Textbook 1-D scheme for E_tt = E_zz on [0,1]: 3-point Laplacian, ghost
    nodes at both ends; top (z=1) flux E_z = P(t) for n <= n1 then
    E_z = -E_t; bottom E_z = E_t (absorbing); E_t by central differences."""
    h = 1.0 / (n - 1)
    tau = cfl * h
    E_prev = np.zeros(n)
    E = np.zeros(n)
    out = [E.copy()]
    r2 = (tau / h) ** 2
    for step in range(n_steps):
        t = step * tau
        new = np.empty(n)
        new[1:-1] = 2 * E[1:-1] - E_prev[1:-1] + r2 * (E[2:] - 2 * E[1:-1] + E[:-2])
        # bottom: ghost E_{-1} = E_1 - 2h E_t, E_t = (new - E_prev)/(2 tau)
        #   new - 2E + E_prev = r2 (2E_1 - 2E_0 - 2h (new - E_prev)/(2 tau))
        a = r2 * h / tau
        new[0] = (2 * E[0] - E_prev[0] + r2 * (2 * E[1] - 2 * E[0]) + a * E_prev[0]) / (1 + a)
        if step <= n1:
            P = float(src.pulse(t))
            new[-1] = 2 * E[-1] - E_prev[-1] + r2 * (2 * E[-2] - 2 * E[-1] + 2 * h * P)
        else:
            new[-1] = (2 * E[-1] - E_prev[-1] + r2 * (2 * E[-2] - 2 * E[-1])
                       + a * E_prev[-1]) / (1 + a)
        E_prev, E = E, new
        out.append(E.copy())
    return np.array(out)


@pytest.mark.parametrize("n,fem_n", [(11, 7), (15, 9)])
def test_vacuum_normal_incidence_is_1d_leapfrog(n, fem_n):
    Nt = 6 * (n - 1)
    src = SourceSpec()
    P = vacuum_problem(n, fem_n, Nt, src)
    n1 = src.switch_step(P.tau, P.top_coords)
    assert 0 < n1 < Nt            # both boundary phases are exercised
    f = P.forward(0, keep_fields=range(Nt + 1))
    ref = leapfrog_1d(n, Nt, 0.3, src, n1)
    g = P.g
    scale = np.abs(ref).max()
    for step in range(Nt + 1):
        E = f.fields[step]
        assert np.abs(E[0]).max() == 0.0 and np.abs(E[2]).max() == 0.0
        Ey = E[1].reshape(n, n, n)                     # [k, j, i]
        assert np.abs(Ey - ref[step][:, None, None]).max() <= 1e-13 * scale


def test_1d_scheme_converges_to_dalembert():
    """E(z, t) = G(t - (1 - z)), G(s) = int_0^s P, at z = 0.5 up to t = 1.4."""
    src = SourceSpec(freq=1.0, t0=1.5, width=0.5)
    errs = []
    for n in (101, 201, 401):
        h = 1.0 / (n - 1)
        tau = 0.3 * h
        Nt = int(round(2.0 / tau))
        n1 = int(math.floor(10.0 / tau))      # source stays on through the window
        sol = leapfrog_1d(n, Nt, 0.3, src, n1)
        k = (n - 1) // 2
        t = np.arange(Nt + 1) * tau
        s = t - 0.5
        # G by fine trapezoid quadrature of the pulse
        sf = np.linspace(0.0, 2.0, 200001)
        Gf = np.concatenate([[0.0], np.cumsum(0.5 * (src.pulse(sf[1:]) + src.pulse(sf[:-1]))
                                              * (sf[1] - sf[0]))])
        exact = np.where(s > 0, np.interp(s, sf, Gf), 0.0)
        errs.append(np.abs(sol[:, k] - exact).max() / np.abs(exact).max())
    r1, r2 = errs[0] / errs[1], errs[1] / errs[2]
    assert errs[2] < 2e-4
    assert 3.3 < r1 < 4.7 and 3.3 < r2 < 4.7, (errs, r1, r2)


def test_oracle_vacuum_close_to_dalembert():
    n, fem_n = 41, 21
    src = SourceSpec(freq=1.0, t0=1.5, width=0.5, t1=10.0)
    P = vacuum_problem(n, fem_n, 200, src)
    f = P.forward(0, keep_fields=[200])
    t = 200 * P.tau
    z = np.arange(n) * P.g.h
    sf = np.linspace(0.0, 2.0, 200001)
    Gf = np.concatenate([[0.0], np.cumsum(0.5 * (src.pulse(sf[1:]) + src.pulse(sf[:-1]))
                                          * (sf[1] - sf[0]))])
    s = t - (1 - z)
    exact = np.where(s > 0, np.interp(s, sf, Gf), 0.0)
    Ey = f.fields[200][1].reshape(n, n, n)[:, n // 2, n // 2]
    assert np.abs(Ey - exact).max() < 0.02 * np.abs(exact).max()


def test_energy_identity_eps1_with_conductivity():
    """E^{n+1/2} - E^{n-1/2} = -|E^{n+1}-E^{n-1}|_C^2/(4 tau)
    + F^n.(E^{n+1}-E^{n-1})/2 for the central scheme with symmetric K,
    E^{n+1/2} = |E^{n+1}-E^n|_M^2/(2 tau^2) + E^{n+1}.K E^n / 2."""
    n, fem_n, Nt = 13, 9, 90
    nf = (fem_n - 4) ** 3
    rng = np.random.default_rng(4)
    src = SourceSpec(freq=3.0, t0=0.3, width=0.1)
    P = OracleProblem(n, fem_n, Nt, 0.3, np.ones(nf), rng.uniform(0, 2.0, nf),
                      detector_grid(n, fem_n, 2), [src])
    n1 = src.switch_step(P.tau, P.top_coords)
    assert 0 < n1 < Nt - 10
    f = P.forward(0, keep_fields=range(Nt + 1))
    tau, M = P.tau, P.M
    E = lambda k: f.fields[k] if k >= 0 else np.zeros_like(f.fields[0])

    def energy(k):  # E^{k+1/2}
        d = E(k + 1) - E(k)
        return 0.5 * np.sum(M * d * d) / tau ** 2 + 0.5 * np.sum(E(k + 1) * P.op.apply_K(E(k)))

    def magnitude(k):  # sum of |terms| of E^{k+1/2}: the rounding scale of the identity
        d = E(k + 1) - E(k)
        return 0.5 * np.sum(M * d * d) / tau ** 2 + 0.5 * np.sum(np.abs(E(k + 1) * P.op.apply_K(E(k))))

    scale = max(magnitude(k) for k in range(Nt))
    for k in range(1, Nt):
        C = P.op.damping(P.absorbing_faces(k, src))
        dE = E(k + 1) - E(k - 1)
        F = P.source_term(k, src)
        lhs = energy(k) - energy(k - 1)
        rhs = -np.sum(C * dE * dE) / (4 * tau) + 0.5 * np.sum(F * dE)
        assert abs(lhs - rhs) <= 1e-12 * scale
    # after the source phase the energy decays
    tail = [energy(k) for k in range(n1 + 2, Nt)]
    assert all(b <= a * (1 + 1e-12) for a, b in zip(tail, tail[1:]))


def _smoothed(n, fem_n, seed, n_incl, width):
    """The layered-inclusion model with C^2-smoothed interfaces (Gaussian
    filter of eps-1 and sigma, vacuum padding), as eq. epsilon_sigma_constraint
    assumes eps, sigma in C^2."""
    from scipy.ndimage import gaussian_filter
    eps, sig = layered_inclusion_model(n, fem_n, seed, n_incl)
    nf = fem_n - 4
    e = np.pad(eps.reshape(nf, nf, nf) - 1.0, 2)
    s = np.pad(sig.reshape(nf, nf, nf), 2)
    e = gaussian_filter(e, width)[2:-2, 2:-2, 2:-2]
    s = gaussian_filter(s, width)[2:-2, 2:-2, 2:-2]
    return 1.0 + e.ravel(), s.ravel()


def _norms(n, fem_n, Nt, eps, sig):
    P = OracleProblem(n, fem_n, Nt, 0.3, eps, sig, detector_grid(n, fem_n, 2),
                      [SourceSpec()])
    f = P.forward(0)
    return np.linalg.norm(f.E_free.reshape(Nt + 2, -1), axis=1), P.tau


@pytest.mark.parametrize("kind", ["jumps", "smooth"])
def test_variable_eps_growth_is_slow(kind):
    """For varying eps the non-symmetric stabilisation gives M^-1 K complex
    eigenvalue pairs, so the field drifts exponentially over very long runs,
    with jump or C^2-smoothed coefficients alike.  The drift must stay slow
    (rate < 0.15 per unit time over 4000 steps, T = 75) so that it is at most
    a few tens of percent over the horizon of the workloads (T <= 4)."""
    n, fem_n, Nt = 17, 13, 4000
    if kind == "jumps":
        eps, sig = layered_inclusion_model(n, fem_n, 5, 2)
    else:
        eps, sig = _smoothed(n, fem_n, 5, 2, 1.5)
    norms, tau = _norms(n, fem_n, Nt, eps, sig)
    assert np.all(np.isfinite(norms))
    a, b = Nt // 2, Nt
    rate = np.log(norms[b] / norms[a]) / ((b - a) * tau)
    assert rate < 0.15
    k4 = int(4.0 / tau)
    assert norms[:k4].max() <= 1.5 * norms[: k4 // 2].max()


def _mms_fields():
    sp = pytest.importorskip("sympy")
    x, y, z, t = sp.symbols("x y z t", real=True)
    X = (x, y, z)
    b = lambda s: (1 - ((s - sp.Rational(1, 2)) / sp.Rational(1, 5)) ** 2) ** 4
    beta = b(x) * b(y) * b(z)
    eps = 1 + 3 * beta
    sig = sp.Rational(1, 2) * beta
    phi = sp.sin(2 * sp.pi * t) * t ** 3
    u = [beta * (1 + x), beta * (1 - 2 * y + x * z), beta * (z + x * y)]
    E = [phi * c for c in u]
    div_w = sum(sp.diff((eps - 1) * E[c], X[c]) for c in range(3))
    f = []
    for c in range(3):
        lap = sum(sp.diff(E[c], v, 2) for v in X)
        f.append(eps * sp.diff(E[c], t, 2) + sig * sp.diff(E[c], t) - lap - sp.diff(div_w, X[c]))
    lam = lambda e: sp.lambdify((x, y, z, t), e, "numpy")
    return lam(eps), lam(sig), [lam(e) for e in E], [lam(e) for e in f]


def test_manufactured_solution_second_order():
    """Variable eps, sigma: forcing f = eps E_tt + sigma E_t - Lap E
    - grad div((eps-1)E) for a smooth E supported inside the free box, fed as
    the lumped load M f; nodal error at T must fall ~4x per halving of h."""
    eps_f, sig_f, E_f, f_f = _mms_fields()
    errs = []
    for n in (21, 41):
        fem_n = n - 4
        h = 1.0 / (n - 1)
        tau = 0.3 * h
        Nt = int(round(0.35 / tau))     # phi(0.35) = 0.81 * 0.35^3, well away from a zero
        from oracle.grid import Grid
        g = Grid(n, fem_n)
        X = g.coords
        inside = np.all(np.abs(X - 0.5) < 0.2, axis=1)
        fx = X[g.free_nodes]
        fin = inside[g.free_nodes]
        eps = np.where(fin, eps_f(fx[:, 0], fx[:, 1], fx[:, 2], 0.0), 1.0)
        sig = np.where(fin, sig_f(fx[:, 0], fx[:, 1], fx[:, 2], 0.0), 0.0)
        assert np.all(~inside[~np.isin(np.arange(g.nn), g.free_nodes)])
        P = OracleProblem(n, fem_n, Nt, 0.3, eps, sig, detector_grid(n, fem_n, 2),
                          [SourceSpec()], absorbing=ABS_BOTTOM)
        m = P.op.m

        def load(step):
            tn = step * tau
            F = np.zeros((3, g.nn))
            for c in range(3):
                F[c, inside] = m[inside] * f_f[c](X[inside, 0], X[inside, 1], X[inside, 2], tn)
            return F

        res = P.forward(0, keep_fields=[Nt], source_override=load)
        T = Nt * tau
        ex = np.zeros((3, g.nn))
        for c in range(3):
            ex[c, inside] = E_f[c](X[inside, 0], X[inside, 1], X[inside, 2], T)
        errs.append(np.abs(res.fields[Nt] - ex).max() / np.abs(ex).max())
    ratio = errs[0] / errs[1]
    assert errs[1] < 0.05, errs
    assert 3.3 < ratio < 5.5, (errs, ratio)
