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
               eps0=None, sig0=None):
    """Full oracle path.  eobs defaults to half the layers-only model's trace:
    the residual E - Eobs is then of the size of E, so J, mu and g are as well
    conditioned as E and FP64 rounding shows at the 1e-15 level (with Eobs the
    full layers-only trace, the residual of a small inclusion can be 1e-6 of
    E and every adjoint-side quantity inherits the trace's rounding times
    1e6)."""
    src_kw = src_kw or {}
    srcs = oracle_sources(w, **src_kw)
    extra = {}
    if absorbing is not None:
        extra["absorbing"] = absorbing
    if eobs is None:
        e0, s0 = w.model(inclusions=False)
        P0 = oracle_problem(w, e0, s0, srcs, **extra)
        eobs = [0.5 * P0.forward(s).trace for s in range(len(srcs))]
    eps, sig = w.model()
    P = oracle_problem(w, eps, sig, srcs, eps0_free=eps0, sig0_free=sig0, **extra)
    fwds = [P.forward(s, keep_fields=keep_e) for s in range(len(srcs))]
    J = P.functional([f.trace for f in fwds], eobs)
    adjs = [P.adjoint(s, fwds[s].trace, eobs[s], keep_fields=keep_mu) for s in range(len(srcs))]
    ge, gs = P.gradient(fwds, adjs)
    return dict(P=P, eobs=np.stack(eobs), trace=np.stack([f.trace for f in fwds]), J=J,
                g_eps=ge, g_sig=gs, E=fwds[0].fields, mu=adjs[0].fields)


def gpu_problem(w: Workload, precision=None, src_kw=None, **kw):
    from paper_2508_07780_gb300 import Problem
    src_kw = dict(src_kw or {})
    p = Problem(n=w.n, fem_n=w.fem_n, n_steps=w.n_steps, cfl=w.cfl,
                precision=precision or w.precision, src_dir=w.directions(),
                det_ij=w.detectors(), z_delta_frac=w.z_delta_frac, gamma_eps=w.gamma_eps,
                gamma_sig=w.gamma_sig, **src_kw, **kw)
    return p


def run_gpu(w: Workload, eobs, precision=None, keep_e=(), keep_mu=(), src_kw=None,
            eps0=None, sig0=None, **kw):
    from paper_2508_07780_gb300 import Problem  # noqa: F401
    p = gpu_problem(w, precision, src_kw, **kw)
    steps = sorted(set(keep_e) | set(keep_mu))
    if steps:
        p.set_capture(steps)
    eps, sig = w.model()
    p.set_coeffs(eps, sig, eps0, sig0)
    trace = p.forward()
    J = p.functional(eobs)
    p.adjoint(eobs)
    ge, gs = p.gradient()
    E = {s: p.get_capture(0, i) for i, s in enumerate(steps) if s in keep_e}
    mu = {s: p.get_capture(1, i) for i, s in enumerate(steps) if s in keep_mu}
    info = p.get_info()
    p.close()
    return dict(trace=trace, J=J, g_eps=ge, g_sig=gs, E=E, mu=mu, info=info)
