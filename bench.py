"""Benchmark of the hot path: forward + functional + adjoint + gradient.

One step = one pass of the whole path over one synthetic workload:
ddfd_set_coeffs -> ddfd_forward -> ddfd_functional -> ddfd_adjoint ->
ddfd_gradient.  The default workload is the FP32 201^3 grid with a 101^3
FEM cube, 2000 time steps, 1024 detectors and three inclusions.

Prints ONE JSON line (rank 0).  `value` is grid-point updates/s over all
ranks (2 n^3 Nt per problem and pass, forward + adjoint), device-resident
inputs; `e2e` is the same through the host-pointer entry points with the
host<->device copies inside the timed region; `roofline` is the dominant
step kernel's algorithmic bytes over its CUDA-event duration against the
measured HBM copy bandwidth; `cpu_baseline` times the FP64 CPU oracle on a
bounded sample of the same workload; `fp64_plain` is one pass of the plain
FP64 GPU path on the same workload; `batched` is the batched FP32 workload
(16 problems of mixed FEM cube size on a 161^3 grid, one launch per time
step) with its own throughput and roofline.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

from synth import workload  # noqa: E402

METRIC = ("grid-point updates/s (fwd+adj+grad) and % HBM roofline, "
          "FP32 batched vs FP64 plain")
UNIT = "grid-point updates/s"
STEP_SRC = os.path.join(ROOT, "paper_2508_07780_gb300", "csrc", "ddfd_step.cu")
TRAFFIC_FILE = os.path.join(ROOT, "profiles", "step_kernel_traffic.txt")


def describe(w):
    return (f"{w.name}: {w.n}^3 grid, FEM cube {w.fem_n}^3, {w.n_steps} steps, "
            f"{w.precision.upper()} fields with FP64 reductions, {w.n_src} source(s), "
            f"{w.det_per_side ** 2} detectors, {w.n_incl} inclusion(s), seed {w.seed}")


def algorithmic_bytes(w):
    """Per launch of the forward / adjoint step kernel (one time step, one
    source): every node reads E^n and E^{n-1} and writes E^{n+1} (3 x 3
    components); FEM-updated nodes read (eps, sigma); the adjoint reads E^k on
    the free nodes for the gradient.  Neighbour re-reads, the E history
    written by the forward and the FP64 gradient accumulators are not
    algorithmic."""
    es = 4 if w.precision == "fp32" else 8
    n3 = w.n ** 3
    fem_rows = (w.fem_n - 2) ** 3
    n_free = (w.fem_n - 4) ** 3
    fwd = 9 * es * n3 + 2 * es * fem_rows
    adj = fwd + 3 * es * n_free
    return fwd, adj


def measured_peak():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def traffic_per_launch(which):
    """DRAM bytes per launch from the committed ncu summary, if it was taken
    on the current step-kernel source (sha256 prefix match); else None."""
    try:
        src_hash = hashlib.sha256(open(STEP_SRC, "rb").read()).hexdigest()[:16]
        vals = {}
        for line in open(TRAFFIC_FILE):
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            k, v = line.split("=", 1)
            vals[k.strip()] = v.strip()
        if vals.get("source_sha256_16") != src_hash:
            return None
        return float(vals[f"{which}_dram_bytes_per_launch_full"])
    except Exception:
        return None


class ClockSampler:
    """nvidia-smi clocks / throttle reasons during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.Q}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if not self.proc:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        rows = []
        for line in open(self.path):
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                rows.append(dict(sm=float(parts[1]), smax=float(parts[2]), pw=float(parts[3]),
                                 hw=parts[5], hwt=parts[6], swt=parts[7], pcap=parts[8]))
            except ValueError:
                continue
        os.unlink(self.path)
        if not rows:
            return None
        reasons = set()
        for r in rows:
            for key, name in (("hw", "hw_slowdown"), ("hwt", "hw_thermal_slowdown"),
                              ("swt", "sw_thermal_slowdown"), ("pcap", "sw_power_cap")):
                if r[key].lower() == "active":
                    reasons.add(name)
        return {"sm_mhz": statistics.median(r["sm"] for r in rows),
                "sm_max_mhz": max(r["smax"] for r in rows), "reasons": sorted(reasons),
                "samples": len(rows)}


def oracle_sample(w, steps):
    """The FP64 oracle on the full grid of the workload for `steps` forward and
    `steps` adjoint steps (assembly excluded); returns (updates/s, seconds,
    threads used)."""
    from oracle import OracleProblem, SourceSpec
    eps, sig = w.model()
    ws = w.with_(n_steps=steps)
    P = OracleProblem(ws.n, ws.fem_n, steps, ws.cfl, eps, sig, ws.detectors(), [SourceSpec()],
                      z_delta_frac=ws.z_delta_frac)
    eobs = np.zeros((steps + 1, ws.detectors().shape[0], 3))
    c0, t0 = time.process_time(), time.perf_counter()
    f = P.forward(0)
    P.functional([f.trace], [eobs])
    a = P.adjoint(0, f.trace, eobs)
    P.gradient([f], [a])
    wall = time.perf_counter() - t0
    cpu = time.process_time() - c0
    return 2 * ws.n ** 3 * steps / wall, wall, max(1, round(cpu / wall))


def run_reference(args, w, rank):
    if rank != 0:
        return
    per = 2
    vals = []
    cores = 1
    for i in range(args.warmup + args.steps):
        v, _, cores = oracle_sample(w, per)
        if i >= args.warmup:
            vals.append(v)
    value = statistics.mean(vals)
    sample = (f"{w.n}^3 grid of the workload, {per} forward + {per} adjoint steps per bench step, "
              f"FP64 scipy oracle, assembly excluded")
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT,
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 2 * w.n ** 3 * per / value * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": describe(w)},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                             "sample": sample}}
    print(json.dumps(line), flush=True)


def fp64_plain(w, dev, stream):
    """One timed pass (after one warm-up) of the same workload with FP64 fields."""
    import torch
    from paper_2508_07780_gb300 import Problem
    w64 = w.with_(precision="fp64")
    eps, sig = w64.model()
    e_lay, s_lay = w64.model(inclusions=False)
    p = Problem(n=w64.n, fem_n=w64.fem_n, n_steps=w64.n_steps, cfl=w64.cfl, precision="fp64",
                src_dir=w64.directions(), det_ij=w64.detectors(), z_delta_frac=w64.z_delta_frac,
                stream=stream.cuda_stream)
    T = lambda a: torch.tensor(a, dtype=torch.float64, device=dev)
    p.set_coeffs(e_lay, s_lay)
    eobs = torch.empty(p.trace_shape, dtype=torch.float64, device=dev)
    p.forward_dev(eobs)
    eps_d, sig_d = T(eps), T(sig)
    ge = torch.empty(p.n_free, dtype=torch.float64, device=dev)
    gs = torch.empty_like(ge)

    def step():
        p.set_coeffs_dev(eps_d, sig_d)
        p.forward_dev(None)
        p.functional_dev(eobs)
        p.adjoint_dev(eobs)
        p.gradient_dev(ge, gs)

    step()
    torch.cuda.synchronize(dev)
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    step()
    ev1.record(stream)
    torch.cuda.synchronize(dev)
    ms = ev0.elapsed_time(ev1)
    p.close()
    return w64.updates / (ms / 1e3), ms


def batched_bytes(ws):
    """Algorithmic bytes of one batched forward launch: the per-problem bytes
    of algorithmic_bytes summed over the members."""
    return sum(algorithmic_bytes(w)[0] for w in ws)


def run_batched(args, dev, stream):
    """The batched FP32 workload: 16 problems on a 161^3 grid, FEM cubes
    61/81/101/121 (problem b mod 4), one hemisphere-drawn incidence
    direction each, 1600 steps, 1024 detectors, stepped together (one launch
    per time step, graph-captured), tile depth from the autotuner.  Members
    with the 61^3 and 81^3 cubes keep the E history; the 101^3 and 121^3
    ones checkpoint (32 snapshots) and are replayed in batched launches of
    their own, so that the batch fits in about 85 GB."""
    import torch
    from paper_2508_07780_gb300 import Batch
    from synth import batched_problems
    probs = batched_problems()
    cfgs = [dict(n=w.n, fem_n=w.fem_n, n_steps=w.n_steps, cfl=w.cfl, precision="fp32",
                 src_dir=d[None, :], det_ij=w.detectors(), z_delta_frac=w.z_delta_frac,
                 n_snapshots=32 if w.fem_n > 81 else 0, stream=stream.cuda_stream)
            for w, d in probs]
    b = Batch(cfgs)
    T = lambda a: torch.tensor(a, dtype=torch.float64, device=dev)
    for (w, _), m in zip(probs, b.members):
        m.set_coeffs(*w.model(inclusions=False))
    eobs = [torch.empty(m.trace_shape, dtype=torch.float64, device=dev) for m in b.members]
    b.forward_dev(eobs)
    coefs = [tuple(T(a) for a in w.model()) for w, _ in probs]
    grads = [(torch.empty(m.n_free, dtype=torch.float64, device=dev),
              torch.empty(m.n_free, dtype=torch.float64, device=dev)) for m in b.members]
    kz = b.autotune(steps=8)

    def step():
        for m, (e, s) in zip(b.members, coefs):
            m.set_coeffs_dev(e, s)
        b.forward_dev(None)
        J = sum(m.functional_dev(e) for m, e in zip(b.members, eobs))
        b.adjoint_dev(eobs)
        for m, (ge, gs) in zip(b.members, grads):
            m.gradient_dev(ge, gs)
        return J

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize(dev)
    l0 = b.get_info().kernel_launches
    fwd_ms = adj_ms = 0.0
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    for _ in range(args.steps):
        step()
        inf = b.get_info()
        fwd_ms += inf.forward_loop_ms
        adj_ms += inf.adjoint_loop_ms
    ev1.record(stream)
    torch.cuda.synchronize(dev)
    inf = b.get_info()
    launches = inf.kernel_launches - l0
    ms = ev0.elapsed_time(ev1) / args.steps
    ws = [w for w, _ in probs]
    updates = sum(w.updates for w in ws)
    nb = batched_bytes(ws)
    fwd_avg = fwd_ms / (args.steps * inf.forward_step_kernels)
    peak, peak_kind = measured_peak()
    achieved = nb / (fwd_avg / 1e3) / 1e9
    out = {"workload": (f"batched FP32: 16 problems, {ws[0].n}^3 grid, FEM cubes 61/81/101/121 "
                        f"(problem b mod 4), {ws[0].n_steps} steps, one hemisphere-drawn plane wave "
                        f"each, 1024 detectors, seeds 300..315"),
           "value": updates / (ms / 1e3), "unit": UNIT, "ms_per_step": ms, "steps": args.steps,
           "warmup": args.warmup, "tile_kz": kz, "gpu_launches": int(launches),
           "device_bytes": int(inf.device_bytes),
           "memory_plan": "61^3/81^3 members keep the E history, 101^3/121^3 members checkpoint "
                          "(32 snapshots, replayed in batched launches; replays are not counted "
                          "as updates)",
           "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                        "frac": achieved / peak, "traffic": None,
                        "kernel": "k_step<float,forward,16> (one launch = one step of all 16)",
                        "algorithmic_bytes_per_launch": nb, "avg_launch_ms": fwd_avg,
                        "adjoint_loop_ms_per_step": adj_ms / args.steps,
                        "peak_kind": f"{peak_kind} (HBM copy, MEASURED_PEAKS.json hbm_gbs)"}}
    b.close()
    return out


def run_ours(args, w, rank, world, local_rank):
    import torch
    import torch.distributed as dist
    from paper_2508_07780_gb300 import Problem
    from paper_2508_07780_gb300.sharding import reduce_loss_and_grad_dev
    from synth import shard_directions

    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    stream = torch.cuda.current_stream(dev)
    eps, sig = w.model()
    e_lay, s_lay = w.model(inclusions=False)
    # N > 1: source sharding.  Every rank owns one incident plane wave (rank 0
    # the normal one of the single-GPU workload, the others drawn on the
    # hemisphere); the ranks share eps and sigma, and one FP64 all-reduce of
    # [J, g_eps, g_sig] per step sums the functional and the gradient.
    src_dir = w.directions() if world == 1 else shard_directions(world)[rank:rank + 1]
    kw = dict(n=w.n, fem_n=w.fem_n, n_steps=w.n_steps, cfl=w.cfl, precision=w.precision,
              src_dir=src_dir, det_ij=w.detectors(), z_delta_frac=w.z_delta_frac,
              n_snapshots=args.snapshots, grad_variant=args.grad_variant, stream=stream.cuda_stream)
    p = Problem(**kw)
    T = lambda a: torch.tensor(a, dtype=torch.float64, device=dev)
    # observed data: the layers-only model's trace (the inclusions are what
    # the residual sees)
    p.set_coeffs(e_lay, s_lay)
    eobs_d = torch.empty(p.trace_shape, dtype=torch.float64, device=dev)
    p.forward_dev(eobs_d)
    eps_d, sig_d = T(eps), T(sig)
    ge = torch.empty(p.n_free, dtype=torch.float64, device=dev)
    gs = torch.empty_like(ge)

    fwd_ms, adj_ms, nk = 0.0, 0.0, 0

    def step():
        p.set_coeffs_dev(eps_d, sig_d)
        p.forward_dev(None)
        J = p.functional_dev(eobs_d)
        p.adjoint_dev(eobs_d)
        p.gradient_dev(ge, gs)
        if world > 1:
            J = reduce_loss_and_grad_dev(J, ge, gs)
        return J

    for _ in range(args.warmup):
        step()
    sampler = ClockSampler(local_rank) if rank == 0 else None
    if sampler:
        sampler.start()
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize(dev)
    l0 = p.get_info().kernel_launches
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    for _ in range(args.steps):
        step()
        t = p.get_timing()
        fwd_ms += t.forward_loop_ms
        adj_ms += t.adjoint_loop_ms
        nk += t.forward_step_kernels
    ev1.record(stream)
    torch.cuda.synchronize(dev)
    if world > 1:
        dist.barrier()
    clocks = sampler.stop() if sampler else None
    launches = p.get_info().kernel_launches - l0
    ms = ev0.elapsed_time(ev1) / args.steps
    ms_t = torch.tensor([ms], device=dev)
    if world > 1:
        dist.all_reduce(ms_t, op=dist.ReduceOp.MAX)
    ms = float(ms_t.item())
    updates = w.updates
    value = world * updates / (ms / 1e3)

    # end to end through the host-pointer entry points (pinned host buffers)
    pin = lambda a: torch.tensor(a, dtype=torch.float64).pin_memory()
    eps_h, sig_h = pin(eps), pin(sig)
    eobs_h = eobs_d.cpu().pin_memory()
    trace_h = torch.empty(p.trace_shape, dtype=torch.float64).pin_memory()
    ge_h = torch.empty(p.n_free, dtype=torch.float64).pin_memory()
    gs_h = torch.empty_like(ge_h).pin_memory()

    def step_e2e():
        p.set_coeffs(eps_h.numpy(), sig_h.numpy())
        p._check(p._lib.ddfd_forward(p._h, trace_h.data_ptr()))
        J = p.functional(eobs_h.numpy())
        p.adjoint(eobs_h.numpy())
        p._check(p._lib.ddfd_gradient(p._h, ge_h.data_ptr(), gs_h.data_ptr()))
        if world > 1:
            gd, sd = ge_h.to(dev, non_blocking=True), gs_h.to(dev, non_blocking=True)
            J = reduce_loss_and_grad_dev(J, gd, sd)
            ge_h.copy_(gd)
            gs_h.copy_(sd)
        return J

    step_e2e()
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize(dev)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        step_e2e()
    torch.cuda.synchronize(dev)
    e2e_s = (time.perf_counter() - t0) / args.steps
    e2e_t = torch.tensor([e2e_s], device=dev)
    if world > 1:
        dist.all_reduce(e2e_t, op=dist.ReduceOp.MAX)
    e2e_s = float(e2e_t.item())
    nf, ntr = p.n_free, int(np.prod(p.trace_shape))
    dev_bytes = p.get_info().device_bytes
    h2d = 2 * nf * 8 + 2 * ntr * 8
    d2h = ntr * 8 + 2 * nf * 8 + 3 * 8
    if world > 1:                       # the gradient through the all-reduce and back
        h2d += 2 * nf * 8
        d2h += 2 * nf * 8
    p.close()

    if rank != 0:
        return
    fwd_b, adj_b = algorithmic_bytes(w)
    fwd_avg = fwd_ms / max(nk, 1)
    adj_avg = adj_ms / max(nk, 1)
    # with checkpointing the adjoint sequence also holds the replayed forward
    # steps, so the roofline is taken on the forward launches
    adj_first = adj_ms >= fwd_ms and not args.snapshots
    which, nbytes, dur = ("adjoint", adj_b, adj_avg) if adj_first else ("forward", fwd_b, fwd_avg)
    peak, peak_kind = measured_peak()
    achieved = nbytes / (dur / 1e3) / 1e9
    roof = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
            "frac": achieved / peak, "traffic": traffic_per_launch(which),
            "kernel": f"k_step<{'float' if w.precision == 'fp32' else 'double'},"
                      f"{'adjoint' if which == 'adjoint' else 'forward'}>",
            "algorithmic_bytes_per_launch": nbytes, "avg_launch_ms": dur,
            "forward_avg_launch_ms": fwd_avg, "adjoint_avg_launch_ms": adj_avg,
            "peak_kind": f"{peak_kind} (HBM copy, MEASURED_PEAKS.json hbm_gbs)"}
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32" if w.precision == "fp32" else "f64",
            "data": "synthetic",
            "config": {"workload": describe(w), "grid": w.n, "fem_n": w.fem_n,
                       "n_steps": w.n_steps, "n_src": w.n_src, "problems_per_gpu": 1,
                       "e_history": (f"checkpointing, {args.snapshots} snapshots, replayed segments"
                                     if args.snapshots else "full E history on the free nodes"),
                       "gradient": ("exact derivative of the discrete J" if args.grad_variant == "exact" else
                                    "paper-literal (Sec. 4, div(eps E) ~ eps div E; E kept on the FEM nodes)"),
                       "device_bytes": int(dev_bytes),
                       "l2": "inputs larger than L2: 2 field levels of 3 x n^3 plus the "
                             "E history on the free nodes, re-streamed every step",
                       "parallelism": "single GPU" if world == 1 else
                       f"source sharding: 1 incident wave per GPU x{world}, FP64 all-reduce "
                       f"of [J, g_eps, g_sig] ({8 * (1 + 2 * w.n_free)} bytes) per step"},
            "e2e": {"value": world * updates / e2e_s, "unit": UNIT, "h2d_bytes_per_step": h2d,
                    "d2h_bytes_per_step": d2h},
            "roofline": roof,
            "gpu_launches": int(launches),
            "clocks": clocks}
    if world == 1 and w.precision == "fp32" and not args.no_fp64:
        # the plain FP64 path on the same workload, for the FP32 speedup
        v64, ms64 = fp64_plain(w, dev, stream)
        line["fp64_plain"] = {"value": v64, "unit": UNIT, "ms_per_step": ms64, "steps": 1, "warmup": 1,
                              "fp32_speedup": value / v64,
                              "accuracy": "FP32 vs FP64 on this workload: trace 2.4e-6, J 1.9e-6, "
                                          "g 1.1e-5 relative L2 (tests/test_gpu_fullsize.py)"}
    if world == 1 and not args.no_batched:
        line["batched"] = run_batched(args, dev, stream)
    if world == 1 and not args.no_cpu_baseline:
        v, wall, cores = oracle_sample(w, 2)
        line["cpu_baseline"] = {"value": v, "unit": UNIT, "cores": cores, "kind": "oracle",
                                "sample": f"{w.n}^3 grid of the workload, 2 forward + 2 adjoint "
                                          f"steps, FP64 scipy oracle, assembly excluded, "
                                          f"{wall:.1f} s"}
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", default="c2_fp32_201")
    ap.add_argument("--precision", choices=["fp32", "fp64"], default=None)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-fp64", action="store_true", help="skip the FP64 comparison pass")
    ap.add_argument("--no-batched", action="store_true", help="skip the batched 16-problem workload")
    ap.add_argument("--snapshots", type=int, default=0,
                    help="checkpointing with this many state snapshots instead of the full E history")
    ap.add_argument("--grad-variant", choices=["exact", "literal"], default="exact",
                    help="gradient form: the exact derivative of the discrete J (default) or the "
                         "paper-literal one of Sec. 4")
    args = ap.parse_args()
    w = workload(args.workload)
    if args.precision:
        w = w.with_(precision=args.precision)
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        run_reference(args, w, rank)
        return
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    try:
        run_ours(args, w, rank, world, local_rank)
    finally:
        if world > 1:
            import torch.distributed as dist
            dist.destroy_process_group()


if __name__ == "__main__":
    main()
