"""Gradient-based reconstruction of eps and sigma with the conjugate gradient
algorithm of Sec. 4 on the GPU (ddfd_cg_run), on a synthetic workload.

The default workload is 8 incident plane waves (normal incidence and 7
hemisphere directions) on a 241^3 grid with a 61^3 FEM cube and 2400 steps,
FP32 fields.  The observed data come from a forward run on the 2x finer grid
(481^3, FEM cube 121^3, 4800 steps, FP64 by default) of the same physical
model, sampled at the coarse detector nodes and times, with 1% multiplicative
Gaussian noise.  The initial guess is the layers-only model (the known skin
layers); the target is the model with its inclusions.

    python -m paper_2508_07780_gb300.reconstruct [--n 241] [--fem-n 61]
        [--sources 8] [--iters 20] [--fine-precision fp64|fp32] [--out report.json]

Prints one JSON report: per CG variant and iteration J, gradient norms, step
sizes, device time, and the relative L2 errors of eps and sigma on the free
nodes.  Variants: "literal" (the paper's rules) and "restart" (the same with
the Fletcher-Reeves restart safeguard, ddfd_cg_params.restart).
"""
from __future__ import annotations

import argparse
import json
import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--n", type=int, default=241)
    ap.add_argument("--fem-n", type=int, default=61)
    ap.add_argument("--steps", type=int, default=None, help="coarse steps (default: T = 3)")
    ap.add_argument("--sources", type=int, default=8)
    ap.add_argument("--iters", type=int, default=20)
    ap.add_argument("--seed", type=int, default=5)
    ap.add_argument("--incl", type=int, default=1)
    ap.add_argument("--det", type=int, default=32)
    ap.add_argument("--noise", type=float, default=0.01)
    ap.add_argument("--fine-precision", choices=["fp64", "fp32"], default="fp64")
    ap.add_argument("--p", type=float, default=0.5)
    ap.add_argument("--step0", type=float, default=0.5,
                    help="first update's RMS change of eps on the free nodes")
    ap.add_argument("--eps-max", type=float, default=30.0, help="admissible box: eps in [1, eps_max]")
    ap.add_argument("--sig-max", type=float, default=5.0, help="admissible box: sigma in [0, sig_max]")
    ap.add_argument("--variants", default="literal,restart",
                    help="CG variants: literal (the paper's rules) and/or restart (FR restart safeguard)")
    ap.add_argument("--refine", action="store_true",
                    help="refine the FEM cube once where eq. meshref marks the model with its inclusion "
                         "(beta_eps 0.8, marking limited to the central 40%% of the free box)")
    ap.add_argument("--out", default=None)
    a = ap.parse_args(argv)
    if ROOT not in sys.path:
        sys.path.insert(0, ROOT)
    import torch
    from synth import box_bounds, detector_grid, free_box, layered_inclusion_model, shard_directions
    from synth.mesh import extend_to_new_nodes, refined_fem_mesh
    from . import Batch, DDFDError

    n, fem_n = a.n, a.fem_n
    # one level of refinement halves the smallest elements: its vacuum
    # stability bound is tau/h ~ 0.27 (eps >= 1 only raises it)
    cfl = 0.25 if a.refine else 0.3
    h = 1.0 / (n - 1)
    nt = a.steps or int(round(3.0 / (cfl * h)))
    nf_, fem_f, nt_f = 2 * (n - 1) + 1, 2 * (fem_n - 1) + 1, 2 * nt
    dirs = shard_directions(a.sources)
    det = detector_grid(n, fem_n, a.det)
    report = dict(workload=dict(grid=n, fem_n=fem_n, n_steps=nt, sources=a.sources, detectors=int(det.shape[0]),
                                fine_grid=nf_, fine_fem_n=fem_f, fine_steps=nt_f, fine_precision=a.fine_precision,
                                noise=a.noise, seed=a.seed, inclusions=a.incl,
                                fem=("Kuhn cube refined once around the inclusion" if a.refine
                                     else "uniform Kuhn cube (no local refinement)")))
    stream = torch.cuda.current_stream().cuda_stream

    # observed data: the finer forward of the same physical model
    t0 = time.perf_counter()
    ef, sf = layered_inclusion_model(nf_, fem_f, a.seed, a.incl, box=free_box(n, fem_n))
    fine = Batch([dict(n=nf_, fem_n=fem_f, n_steps=nt_f, cfl=cfl, precision=a.fine_precision,
                       src_dir=d[None, :], det_ij=2 * det, forward_only=1, stream=stream) for d in dirs])
    for m in fine.members:
        m.set_coeffs(ef, sf)
    traces = fine.forward()
    fine_info = fine.get_info()
    fine.close()
    rng = np.random.default_rng(a.seed)
    eobs = []
    for tr in traces:
        coarse = tr[:, ::2][:, : nt + 1]                     # t_n = n tau = 2n tau_fine
        eobs.append(np.ascontiguousarray(coarse * (1.0 + a.noise * rng.standard_normal(coarse.shape))))
    report["data"] = dict(seconds=time.perf_counter() - t0, fine_forward_ms=fine_info.forward_loop_ms,
                          fine_device_bytes=int(fine_info.device_bytes))

    # reconstruction
    e_true, s_true = layered_inclusion_model(n, fem_n, a.seed, a.incl)
    e0, s0 = layered_inclusion_model(n, fem_n, a.seed, 0)
    extra = {}
    if a.refine:
        _, _, f0, f1 = box_bounds(n, fem_n)
        nfr = f1 - f0 + 1
        t1 = time.perf_counter()
        par, tets = refined_fem_mesh(n, fem_n, e_true, s_true, beta_eps=0.8, beta_sig=0.0,
                                     region=(f0 + int(0.3 * nfr), f0 + int(0.7 * nfr)))
        report["mesh"] = dict(new_nodes=int(par.shape[0]), tets=int(tets.shape[0]),
                              base_tets=6 * (fem_n - 1) ** 3, seconds=time.perf_counter() - t1)
        # the truth at the new nodes is the physical model there: they sit on
        # the finer grid, which carries the same model
        _, _, F0, F1 = box_bounds(nf_, fem_f)
        NF = F1 - F0 + 1
        EF, SF = ef.reshape(NF, NF, NF), sf.reshape(NF, NF, NF)
        X = np.zeros((par.shape[0], 3), dtype=np.int64)   # fine-grid indices of the new nodes
        n3 = n ** 3
        for e, (p, q) in enumerate(par):
            pts = []
            for v in (p, q):
                pts.append(X[v - n3] if v >= n3 else 2 * np.array([v % n, (v // n) % n, v // (n * n)]))
            X[e] = (pts[0] + pts[1]) // 2
        li = X - F0
        e_new, s_new = EF[li[:, 2], li[:, 1], li[:, 0]], SF[li[:, 2], li[:, 1], li[:, 0]]
        e_true = np.concatenate([e_true, e_new])
        s_true = np.concatenate([s_true, s_new])
        e0, s0 = extend_to_new_nodes(n, fem_n, par, e0, s0)
        extra = dict(mesh=(par, tets))
    b = Batch([dict(n=n, fem_n=fem_n, n_steps=nt, cfl=cfl, precision="fp32", src_dir=d[None, :], det_ij=det,
                    eps_max=max(100.0, a.eps_max), sig_max=max(100.0, a.sig_max), stream=stream, **extra)
               for d in dirs])
    kz = b.autotune(steps=4)
    # step sizes: the first update moves eps by step0 (RMS over the free box);
    # gamma^0 = 1/alpha^0 keeps the step rule's alpha^1 at the same scale
    _, _, probe = b.cg_run(eobs, e0, s0, max_iter=1, gamma_eps0=1.0, gamma_sig0=1.0, alpha_eps0=0.0,
                           alpha_sig0=0.0)
    _, _, f0, f1 = box_bounds(n, fem_n)
    vol = ((f1 - f0) * h) ** 3
    ge0, gs0 = probe[0]["gnorm_eps"], probe[0]["gnorm_sig"]
    alpha_e = a.step0 * np.sqrt(vol) / ge0
    alpha_s = 0.1 * a.step0 * np.sqrt(vol) / gs0
    ne, ns = np.linalg.norm(e_true), np.linalg.norm(s_true)
    report["initial_eps_rel_err"] = float(np.linalg.norm(e0 - e_true) / ne)
    report["initial_sig_rel_err"] = float(np.linalg.norm(s0 - s_true) / ns)
    report["tile_kz"] = kz
    report["updates_per_iteration"] = 2 * n ** 3 * nt * a.sources
    for variant in a.variants.split(","):
        prm = dict(max_iter=a.iters, gamma_eps0=1.0 / alpha_e, gamma_sig0=1.0 / alpha_s, alpha_eps0=alpha_e,
                   alpha_sig0=alpha_s, p=a.p, eps_max=a.eps_max, sig_max=a.sig_max,
                   restart=int(variant == "restart"))
        err = None
        try:
            eps, sig, log = b.cg_run(eobs, e0, s0, iterates=True, **prm)
        except DDFDError as exc:  # recorded with the iterations before it; the other variants still run
            err, eps, sig, log = exc, exc.eps, exc.sig, exc.log
        rows = []
        for r in log:
            rows.append({k: float(v) for k, v in r.items() if k not in ("eps", "sig")})
            rows[-1]["eps_rel_err"] = float(np.linalg.norm(r["eps"] - e_true) / ne)
            rows[-1]["sig_rel_err"] = float(np.linalg.norm(r["sig"] - s_true) / ns)
        out = dict(params=prm, iterations=rows)
        if log:
            ms = float(np.mean([r["ms"] for r in log]))
            out.update(ms_per_iteration=ms, updates_per_s=report["updates_per_iteration"] / (ms / 1e3))
        if err is not None:
            out.update(error=str(err), failed_iteration=len(log),
                       failed_iterate=dict(eps_min=float(eps.min()), eps_max=float(eps.max()),
                                           sig_max=float(sig.max())))
        report["cg_" + variant] = out
    report["device_bytes"] = int(b.get_info().device_bytes)
    b.close()
    txt = json.dumps(report)
    if a.out:
        with open(a.out, "w") as f:
            f.write(txt + "\n")
    print(txt, flush=True)


if __name__ == "__main__":
    main()
