"""Leapfrog stability bound (oracle).

Test infrastructure only (see oracle/__init__.py).

The explicit central scheme for M_eps E'' + K E = 0 is stable when
tau^2 lambda_max < 4, lambda_max the largest eigenvalue of M_eps^{-1} K; the
damping C only adds dissipation.  lambda_max is estimated by power iteration
on M_eps^{-1} K (the Rayleigh-type ratio |A x| / |x| of the last iterate).
"""
from __future__ import annotations

import numpy as np

from .hybrid import HybridOperator


def lambda_max(op: HybridOperator, iters: int = 400, seed: int = 0) -> float:
    rng = np.random.default_rng(seed)
    x = rng.standard_normal((3, op.g.nn))
    minv = 1.0 / (op.m * op.eps)
    lam = 0.0
    for _ in range(iters):
        y = minv[None, :] * op.apply_K(x)
        lam = float(np.linalg.norm(y) / np.linalg.norm(x))
        x = y / np.linalg.norm(y)
    return lam


def max_stable_tau(op: HybridOperator, iters: int = 400) -> float:
    return 2.0 / np.sqrt(lambda_max(op, iters))
