"""The conjugate gradient algorithm (CGA) of Sec. 4 for the reconstruction of
eps and sigma, in plain numpy FP64.

TEST INFRASTRUCTURE ONLY (see the package header).

The algorithm, in the paper's order (iteration m = 0, 1, ...):
  1. E^m, lambda^m and the gradients g_eps^m, g_sig^m at (eps^m, sig^m);
  2. d_eps^m = -g_eps^m + beta_eps^m d_eps^{m-1}, beta_eps^m = ||g_eps^m||^2 / ||g_eps^{m-1}||^2
     (Fletcher-Reeves; d^0 = -g^0), eps^{m+1} = eps^m + alpha_eps^m d_eps^m;
  3. the same for sigma;
  4. alpha^{m+1} = -(g^m, d^m) / (gamma^m (d^m, d^m));
  5. gamma^{m+1} = gamma^0 / (m+1)^p;
  6. stop if (||eps^{m+1} - eps^m|| < eta1_eps or ||sig^{m+1} - sig^m|| < eta1_sig) and
     (||g_eps^m|| < eta2_eps or ||g_sig^m|| < eta2_sig).

Readings (where the paper is silent): the gradients and norms are those of
L2(Omega) with the lumped nodal quadrature, (u, v) = sum_i m_i u_i v_i over
the free nodes, so the gradient function is the Riesz representative
g_i = (dJ/deps_i) / m_i of the derivative of the discrete functional; the
functional at iteration m uses gamma^m with the initial guess as the
regularisation centre (eq. tikhonov_functional names both eps^0); the
"and/or" of the stopping rule groups as written above; after each update eps
is clamped to [1, eps_max] and sigma to [0, sig_max] (the admissible set of
eq. epsilon_sigma_constraint), the directions are not.

Option (not in the paper, off by default): restart, the usual safeguard of
nonlinear conjugate gradients -- when the Fletcher-Reeves direction is not a
descent direction, (g^m, d^m) >= 0, it is replaced by -g^m.
"""
from __future__ import annotations

from dataclasses import dataclass
from typing import Callable, Optional

import numpy as np


@dataclass
class CGParams:
    max_iter: int = 20
    gamma_eps0: float = 1.0
    gamma_sig0: float = 1.0
    alpha_eps0: float = 1.0
    alpha_sig0: float = 1.0
    p: float = 0.5
    eta1_eps: float = 0.0
    eta1_sig: float = 0.0
    eta2_eps: float = 0.0
    eta2_sig: float = 0.0
    eps_max: float = 100.0
    sig_max: float = 100.0
    restart: bool = False


def cga(evaluate: Callable, eps0: np.ndarray, sig0: np.ndarray, m: np.ndarray, prm: CGParams,
        eps_ref: Optional[np.ndarray] = None, sig_ref: Optional[np.ndarray] = None):
    """Run the CGA.  evaluate(eps, sig) -> (J_data, dJ_data/deps_i, dJ_data/dsig_i),
    the data term of the discrete functional and its exact derivative at the free
    nodes; m: their lumped masses.  eps_ref / sig_ref: regularisation centres
    (default: the initial guess).  Returns (eps, sig, log), log one dict per
    iteration."""
    eps = np.array(eps0, dtype=np.float64)
    sig = np.array(sig0, dtype=np.float64)
    ref_e = eps.copy() if eps_ref is None else np.asarray(eps_ref, dtype=np.float64)
    ref_s = sig.copy() if sig_ref is None else np.asarray(sig_ref, dtype=np.float64)

    def ip(u, v):
        return float(np.sum(m * u * v))

    gamma_e, gamma_s = prm.gamma_eps0, prm.gamma_sig0
    alpha_e, alpha_s = prm.alpha_eps0, prm.alpha_sig0
    d_e = d_s = None
    gg_e_prev = gg_s_prev = None
    log = []
    for it in range(prm.max_iter):
        # step 1
        J_data, de_data, ds_data = evaluate(eps, sig)
        g_e = de_data / m + gamma_e * (eps - ref_e)
        g_s = ds_data / m + gamma_s * (sig - ref_s)
        J = J_data + 0.5 * gamma_e * ip(eps - ref_e, eps - ref_e) + 0.5 * gamma_s * ip(sig - ref_s, sig - ref_s)
        gg_e, gg_s = ip(g_e, g_e), ip(g_s, g_s)
        # steps 2 and 3
        if it == 0:
            beta_e = beta_s = 0.0
            d_e, d_s = -g_e, -g_s
        else:
            beta_e = gg_e / gg_e_prev if gg_e_prev > 0 else 0.0
            beta_s = gg_s / gg_s_prev if gg_s_prev > 0 else 0.0
            d_e = -g_e + beta_e * d_e
            d_s = -g_s + beta_s * d_s
            if prm.restart and ip(g_e, d_e) >= 0.0:
                beta_e, d_e = 0.0, -g_e
            if prm.restart and ip(g_s, d_s) >= 0.0:
                beta_s, d_s = 0.0, -g_s
        eps_new = np.clip(eps + alpha_e * d_e, 1.0, prm.eps_max)
        sig_new = np.clip(sig + alpha_s * d_s, 0.0, prm.sig_max)
        # step 4
        dd_e, dd_s = ip(d_e, d_e), ip(d_s, d_s)
        alpha_e_next = -ip(g_e, d_e) / (gamma_e * dd_e) if gamma_e > 0 and dd_e > 0 else alpha_e
        alpha_s_next = -ip(g_s, d_s) / (gamma_s * dd_s) if gamma_s > 0 and dd_s > 0 else alpha_s
        # step 5
        gamma_e_next = prm.gamma_eps0 / (it + 1) ** prm.p
        gamma_s_next = prm.gamma_sig0 / (it + 1) ** prm.p
        # step 6
        step_e = np.sqrt(ip(eps_new - eps, eps_new - eps))
        step_s = np.sqrt(ip(sig_new - sig, sig_new - sig))
        stop = (step_e < prm.eta1_eps or step_s < prm.eta1_sig) and \
               (np.sqrt(gg_e) < prm.eta2_eps or np.sqrt(gg_s) < prm.eta2_sig)
        log.append(dict(iter=it, J=J, J_data=J_data, gnorm_eps=np.sqrt(gg_e), gnorm_sig=np.sqrt(gg_s),
                        alpha_eps=alpha_e, alpha_sig=alpha_s, beta_eps=beta_e, beta_sig=beta_s,
                        gamma_eps=gamma_e, gamma_sig=gamma_s, step_eps=step_e, step_sig=step_s,
                        stop=bool(stop)))
        eps, sig = eps_new, sig_new
        alpha_e, alpha_s = alpha_e_next, alpha_s_next
        gamma_e, gamma_s = gamma_e_next, gamma_s_next
        gg_e_prev, gg_s_prev = gg_e, gg_s
        if stop:
            break
    return eps, sig, log


def problem_evaluator(P):
    """evaluate(eps, sig) for an OracleProblem P with its sources and Eobs, data
    term only (P's own gammas must be zero): rebuilds P's operator at the
    given coefficients."""
    from .hybrid import HybridOperator

    def make(eobs):
        def evaluate(eps, sig):
            P.op = HybridOperator(P.g, eps, sig)
            P.M = P.op.m * P.op.eps
            res = P.run(eobs)
            return res["J"], res["g_eps"], res["g_sig"]
        return evaluate
    return make
