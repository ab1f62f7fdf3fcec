"""Central finite-difference check of the adjoint gradient.

The library's gradient is the exact derivative of the discrete Tikhonov
functional (Sec. 3 eq. tikhonov_functional, Sec. 4 eq. gradeps), so central
differences of J confirm it node by node:

    d_i = (J(c + delta e_i) - J(c - delta e_i)) / (2 delta),   c = eps or sigma,

with J evaluated by FP64 forward runs (an FP32 J cannot resolve delta = 1e-4).
The nodes are drawn uniformly from the free nodes (seeded).  Per node the
check holds the adjoint gradient g_i to

    |g_i - d_i| <= 1e-3 |d_i| + eps_J |J| / delta,

the relative bar of the gradient plus the finite difference's own rounding:
the two J values carry a relative rounding noise of about 5e-16 on these
workloads (measured as the difference between central differences and the
exact FP64 gradient at the nodes with the smallest gradients), and
eps_J = 1e-14 leaves a factor 20 over it.  At nodes whose gradient is tiny
that floor, not the relative bar, decides.  All arithmetic runs in the CUDA
library; this module drives it.

    python -m paper_2508_07780_gb300.fdcheck --workload c4_fp32_301 --nodes 20
"""
from __future__ import annotations

import argparse
import json
import time

import numpy as np

from .binding import Problem

EPS_J = 1e-14


def _problem(w, precision, **kw):
    return Problem(n=w.n, fem_n=w.fem_n, n_steps=w.n_steps, cfl=w.cfl, precision=precision,
                   src_dir=w.directions(), det_ij=w.detectors(), z_delta_frac=w.z_delta_frac, **kw)


def check_gradient(w, n_nodes=20, delta=1e-4, seed=2024, n_snapshots=32, precisions=("fp32", "fp64"),
                   log=None):
    """Runs the check on workload `w` (a synth Workload) with its layers-only
    model's FP64 trace as observed data.  Returns a report dict: per node
    and coefficient the FD value, each precision's adjoint gradient, its bar
    and whether it holds."""
    t0 = time.time()
    eps, sig = w.model()
    e_lay, s_lay = w.model(inclusions=False)
    p64 = _problem(w, "fp64", forward_only=1)
    p64.set_coeffs(e_lay, s_lay)
    eobs = p64.forward()
    grads = {}
    for prec in precisions:
        p = _problem(w, prec, n_snapshots=n_snapshots)
        p.set_coeffs(eps, sig)
        p.forward(want_trace=False)
        p.functional(eobs)
        p.adjoint(eobs)
        grads[prec] = p.gradient()
        p.close()
    p64.set_coeffs(eps, sig)
    p64.forward(want_trace=False)
    J = p64.functional(eobs)
    n_free = eps.size
    rng = np.random.default_rng(seed)
    nodes = sorted(int(i) for i in rng.choice(n_free, size=min(n_nodes, n_free), replace=False))
    fJ = EPS_J * abs(J) / delta
    rows, ok = [], True
    for which, k in (("eps", 0), ("sig", 1)):
        base = (eps, sig)[k]
        for i in nodes:
            vals = []
            for sign in (1.0, -1.0):
                e2, s2 = eps.copy(), sig.copy()
                (e2, s2)[k][i] = base[i] + sign * delta
                p64.set_coeffs(e2, s2)
                p64.forward(want_trace=False)
                vals.append(p64.functional(eobs))
            fd = (vals[0] - vals[1]) / (2.0 * delta)
            row = {"coef": which, "node": i, "fd": fd}
            for prec, g in grads.items():
                gv = g[k]
                bar = 1e-3 * abs(fd) + fJ
                good = abs(gv[i] - fd) <= bar
                ok &= bool(good)
                row[prec] = {"g": float(gv[i]), "err": float(abs(gv[i] - fd)), "bar": float(bar),
                             "rel": float(abs(gv[i] - fd) / abs(fd)) if fd != 0 else None, "ok": bool(good)}
            rows.append(row)
            if log:
                log(json.dumps(row))
    p64.close()
    gnorm = {prec: [float(np.linalg.norm(g[0])), float(np.linalg.norm(g[1]))] for prec, g in grads.items()}
    return {"workload": w.name, "n": w.n, "fem_n": w.fem_n, "n_steps": w.n_steps, "delta": delta,
            "n_snapshots": n_snapshots, "J": J, "f_J": fJ, "gnorm": gnorm, "nodes": nodes, "rows": rows,
            "ok": ok, "seconds": time.time() - t0}


def main():
    from synth import workload
    ap = argparse.ArgumentParser(description=__doc__.splitlines()[0])
    ap.add_argument("--workload", default="c4_fp32_301")
    ap.add_argument("--nodes", type=int, default=20)
    ap.add_argument("--delta", type=float, default=1e-4)
    ap.add_argument("--seed", type=int, default=2024)
    args = ap.parse_args()
    rep = check_gradient(workload(args.workload), args.nodes, args.delta, args.seed, log=print)
    worst = {p: max(r[p]["err"] / r[p]["bar"] for r in rep["rows"]) for p in ("fp32", "fp64")}
    print(json.dumps({k: v for k, v in rep.items() if k != "rows"} | {"worst_err_over_bar": worst}))


if __name__ == "__main__":
    main()
