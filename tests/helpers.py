"""Shared test utilities: run one workload through the CUDA library and
through the oracle on the same seeded inputs, and compare them."""
from __future__ import annotations

import numpy as np

from synth import Workload


def rel_l2(x, y):
    x = np.asarray(x, dtype=np.float64)
    y = np.asarray(y, dtype=np.float64)
    ny = np.linalg.norm(y)
    return float(np.linalg.norm(x - y) / ny) if ny > 0 else float(np.linalg.norm(x))


def capture_steps(nt):
    """E at Nt/4, Nt/2, 3Nt/4, Nt; mu (defined for 0..Nt-1) at 0, Nt/4, Nt/2, 3Nt/4."""
    e = sorted({max(1, nt // 4), max(1, nt // 2), max(1, 3 * nt // 4), nt})
    m = sorted({0, nt // 4, nt // 2, 3 * nt // 4} - {nt})
    return e, m


def oracle_problem(w: Workload, eps, sig, src_specs, **kw):
    from oracle import OracleProblem
    return OracleProblem(w.n, w.fem_n, w.n_steps, w.cfl, eps, sig, w.detectors(), src_specs,
                         z_delta_frac=w.z_delta_frac, gamma_eps=w.gamma_eps,
                         gamma_sig=w.gamma_sig, **kw)


def oracle_sources(w: Workload, **src_kw):
    from oracle import SourceSpec
    return [SourceSpec(direction=tuple(d), **src_kw) for d in w.directions()]


def run_oracle(w: Workload, eobs=None, keep_e=(), keep_mu=(), src_kw=None, absorbing=None,
               eps0=None, sig0=None, obs="half"):
    """Full oracle path.  Without eobs, the observed data is the layers-only
    model's trace (the workloads' observed data) for obs="layers", or half of
    it for obs="half".  The half trace gives a residual E - Eobs of the size
    of E, so J, mu and g are as well conditioned as E: the small code-path
    cases use it, because on their grids and horizons the inclusion's echo
    never reaches the detectors and the true residual is ~1e-6 of E.  The
    result carries kappa = ||trace|| / ||trace - Eobs||, the factor by which
    the residual amplifies the trace's relative rounding."""
    src_kw = src_kw or {}
    srcs = oracle_sources(w, **src_kw)
    extra = {}
    if absorbing is not None:
        extra["absorbing"] = absorbing
    if eobs is None:
        e0, s0 = w.model(inclusions=False)
        P0 = oracle_problem(w, e0, s0, srcs, **extra)
        scale = 0.5 if obs == "half" else 1.0
        eobs = [scale * P0.forward(s).trace for s in range(len(srcs))]
    eps, sig = w.model()
    P = oracle_problem(w, eps, sig, srcs, eps0_free=eps0, sig0_free=sig0, **extra)
    fwds = [P.forward(s, keep_fields=keep_e) for s in range(len(srcs))]
    J = P.functional([f.trace for f in fwds], eobs)
    adjs = [P.adjoint(s, fwds[s].trace, eobs[s], keep_fields=keep_mu) for s in range(len(srcs))]
    ge, gs = P.gradient(fwds, adjs)
    trace = np.stack([f.trace for f in fwds])
    eobs = np.stack(eobs)
    return dict(P=P, eobs=eobs, trace=trace, J=J, g_eps=ge, g_sig=gs, E=fwds[0].fields,
                mu=adjs[0].fields, kappa=conditioning(trace, eobs))


def conditioning(trace, eobs):
    """kappa = ||trace|| / ||trace - eobs||: a relative error e of the trace
    becomes a relative error of at most kappa * e in the residual, and so in
    J, mu and g, which are computed from it."""
    return float(np.linalg.norm(trace) / np.linalg.norm(np.asarray(trace) - eobs))


def gpu_problem(w: Workload, precision=None, src_kw=None, **kw):
    from paper_2508_07780_gb300 import Problem
    src_kw = dict(src_kw or {})
    p = Problem(n=w.n, fem_n=w.fem_n, n_steps=w.n_steps, cfl=w.cfl,
                precision=precision or w.precision, src_dir=w.directions(),
                det_ij=w.detectors(), z_delta_frac=w.z_delta_frac, gamma_eps=w.gamma_eps,
                gamma_sig=w.gamma_sig, **src_kw, **kw)
    return p


def run_gpu(w: Workload, eobs, precision=None, keep_e=(), keep_mu=(), src_kw=None,
            eps0=None, sig0=None, eobs_fn=None, **kw):
    """The library path on the workload's model.  eobs_fn, if given, maps the
    forward trace to the observed data actually passed to the functional and
    the adjoint (to drive the adjoint with a residual of the caller's choice)."""
    from paper_2508_07780_gb300 import Problem  # noqa: F401
    p = gpu_problem(w, precision, src_kw, **kw)
    steps = sorted(set(keep_e) | set(keep_mu))
    if steps:
        p.set_capture(steps)
    eps, sig = w.model()
    p.set_coeffs(eps, sig, eps0, sig0)
    trace = p.forward()
    if eobs_fn is not None:
        eobs = eobs_fn(trace)
    J = p.functional(eobs)
    p.adjoint(eobs)
    ge, gs = p.gradient()
    E = {s: p.get_capture(0, i) for i, s in enumerate(steps) if s in keep_e}
    mu = {s: p.get_capture(1, i) for i, s in enumerate(steps) if s in keep_mu}
    info = p.get_info()
    p.close()
    return dict(trace=trace, J=J, g_eps=ge, g_sig=gs, E=E, mu=mu, info=info)
