"""Benchmark of the hot path: forward + functional + adjoint + gradient.

One step = one pass of the whole path over the batched FP32 workload: 16
independent problems on a 161^3 grid (FEM cubes 61/81/101/121 for problem b
mod 4, one hemisphere-drawn incident plane wave each, 1600 time steps, 1024
detectors), stepped together by the batch calls -- per member
ddfd_set_coeffs, then ddfd_batch_forward, ddfd_functional per member,
ddfd_batch_adjoint, ddfd_gradient per member.  Every member keeps its E
history on the free nodes (about 250 GB of HBM in all).

Prints ONE JSON line (rank 0):
  value       grid-point updates/s over all ranks (2 n^3 Nt per problem and
              pass, forward + adjoint), device-resident inputs;
  e2e         the same through the host-pointer entry points, with the
              host<->device copies inside the timed region;
  roofline    the dominant step (the batched adjoint step: its full kernel
              for the tiles with FEM-cube or free nodes and its lean kernel
              for the finite-difference tiles, side by side) against the
              measured HBM copy bandwidth, with the forward step and the
              whole pass beside it;
  fp64_plain  the plain FP64 GPU path on the same 16 problems, solved one at a
              time, its FP64 ALU roofline, and the FP32 speedup;
  accuracy    relative errors of the FP32 batched results (traces, J, g)
              against that FP64 run, measured in this run;
  single_201  the one-source FP32 workload (201^3 grid, FEM cube 101^3, 2000
              steps) with its own roofline and errors against FP64;
  cpu_baseline  the FP64 CPU oracle on the host cores (bounded sample).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import platform
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

from synth import batched_problems, workload  # noqa: E402

METRIC = ("grid-point updates/s (fwd+adj+grad) and % HBM roofline, "
          "FP32 batched vs FP64 plain")
UNIT = "grid-point updates/s"
STEP_SRC = os.path.join(ROOT, "paper_2508_07780_gb300", "csrc", "ddfd_step.cu")
TRAFFIC_FILE = os.path.join(ROOT, "profiles", "step_kernel_traffic.txt")
BATCH_WORKLOAD = ("c3_batched_161: 16 problems on a 161^3 grid, FEM cubes 61/81/101/121 (problem b mod 4), "
                  "1600 steps, FP32 fields with FP64 reductions, one hemisphere-drawn plane wave and 1024 "
                  "detectors each, seeds 300..315, full E history")


def describe(w):
    return (f"{w.name}: {w.n}^3 grid, FEM cube {w.fem_n}^3, {w.n_steps} steps, "
            f"{w.precision.upper()} fields with FP64 reductions, {w.n_src} source(s), "
            f"{w.det_per_side ** 2} detectors, {w.n_incl} inclusion(s), seed {w.seed}")


def algorithmic_bytes(n, fem_n, es):
    """Per launch of the forward / adjoint step kernel (one time step, one
    problem): every node reads E^n and E^{n-1} and writes E^{n+1} (3 x 3
    components); FEM-updated nodes read (eps, sigma); the adjoint reads E^k on
    the free nodes for the gradient.  Neighbour re-reads, the E history
    written by the forward and the gradient accumulators are not
    algorithmic."""
    n3 = n ** 3
    fem_rows = (fem_n - 2) ** 3
    n_free = (fem_n - 4) ** 3
    fwd = 9 * es * n3 + 2 * es * fem_rows
    adj = fwd + 3 * es * n_free
    return fwd, adj


def fp64_flops(n, fem_n):
    """Algorithmic FP64 flops of one forward / adjoint step (FMA = 2), counted
    from the formulas the step kernel evaluates: every node 15 per component
    (the 7-point row: 5 adds and one FMA; the tau^2/h^2 scale; the update
    E + A (E - E_old) + B E - C R: 7); FEM-updated nodes add the forward
    Gauss-law stencil sum_o B_o (s E)_{i+o} (45 products s E, 21 pair sums,
    84 for the integer 3 x 3 blocks, 6 for the 1/6 scale and the add: 156) or
    the adjoint's s_i sum_o B_o mu_{i+o} (21 + 84 + 9 = 114); free nodes add
    the adjoint's gradient terms (30 per node and step, 2 more to accumulate)."""
    n3 = n ** 3
    fem_rows = (fem_n - 2) ** 3
    n_free = (fem_n - 4) ** 3
    fwd = 45 * n3 + 156 * fem_rows
    adj = 45 * n3 + 114 * fem_rows + 32 * n_free
    return fwd, adj


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def traffic_per_launch(*keys):
    """DRAM bytes per launch (the sum over `keys`: the kernels of one step)
    from the committed ncu summary, if it was taken on the current
    step-kernel source (sha256 prefix match); else None."""
    try:
        src_hash = hashlib.sha256(open(STEP_SRC, "rb").read()).hexdigest()[:16]
        vals = {}
        for line in open(TRAFFIC_FILE):
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            k, v = line.split("=", 1)
            vals[k.strip()] = v.split("#", 1)[0].strip()
        if vals.get("source_sha256_16") != src_hash:
            return None
        return float(sum(float(vals[k]) for k in keys))
    except Exception:
        return None


def host_info():
    model = platform.processor() or platform.machine()
    try:
        for line in open("/proc/cpuinfo"):
            low = line.lower()
            if low.startswith("model name") or low.startswith("cpu part") and model in ("", "aarch64"):
                model = line.split(":", 1)[1].strip()
                if low.startswith("model name"):
                    break
    except Exception:
        pass
    try:
        lscpu = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in lscpu.splitlines():
            if line.startswith("Model name:"):
                model = line.split(":", 1)[1].strip()
                break
    except Exception:
        pass
    return {"nproc": os.cpu_count(), "cpu_model": model, "machine": platform.machine()}


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
                "samples": len(rows), "power_w_max": max(r["pw"] for r in rows)}


# --------------------------------------------------------------------------
# CPU oracle (the reference arm and the CPU baseline)
# --------------------------------------------------------------------------

class OracleSample:
    """The FP64 oracle on one problem's full grid, assembled once; run()
    times `steps` forward and `steps` adjoint steps plus the functional and
    the gradient and returns (grid-point updates, seconds, threads used)."""

    def __init__(self, n, fem_n, seed, n_incl, direction, steps):
        from oracle import OracleProblem, SourceSpec
        from synth.models import detector_grid, layered_inclusion_model
        eps, sig = layered_inclusion_model(n, fem_n, seed, n_incl)
        det = detector_grid(n, fem_n, 32)
        self.n, self.steps = n, steps
        self.P = OracleProblem(n, fem_n, steps, 0.3, eps, sig, det, [SourceSpec(direction=tuple(direction))],
                               z_delta_frac=0.1)
        self.eobs = np.zeros((steps + 1, det.shape[0], 3))

    def run(self):
        P = self.P
        c0, t0 = time.process_time(), time.perf_counter()
        f = P.forward(0)
        P.functional([f.trace], [self.eobs])
        a = P.adjoint(0, f.trace, self.eobs)
        P.gradient([f], [a])
        wall = time.perf_counter() - t0
        cpu = time.process_time() - c0
        return 2 * self.n ** 3 * self.steps, wall, max(1, round(cpu / wall))


def oracle_sample(*args):
    """One OracleSample run (a pool worker)."""
    return OracleSample(*args).run()


def oracle_full_run(name):
    """The oracle on a whole workload (forward, functional, adjoint,
    gradient; assembly excluded); returns (updates, seconds)."""
    from oracle import OracleProblem, SourceSpec
    w = workload(name)
    eps, sig = w.model()
    e0, s0 = w.model(inclusions=False)
    P0 = OracleProblem(w.n, w.fem_n, w.n_steps, w.cfl, e0, s0, w.detectors(), [SourceSpec()],
                       z_delta_frac=w.z_delta_frac)
    eobs = P0.forward(0).trace
    P = OracleProblem(w.n, w.fem_n, w.n_steps, w.cfl, eps, sig, w.detectors(), [SourceSpec()],
                      z_delta_frac=w.z_delta_frac)
    t0 = time.perf_counter()
    P.run([eobs])
    return w.updates, time.perf_counter() - t0


SAMPLE_STEPS = 4


def _member_args(b):
    (w, d), = batched_problems(first=b, n_problems=1)
    return (w.n, w.fem_n, w.seed, w.n_incl, d, SAMPLE_STEPS)


def cpu_baseline(workers):
    """The oracle on the host cores: one batch member (161^3 grid) for
    SAMPLE_STEPS forward + SAMPLE_STEPS adjoint steps in one process (single
    core: scipy's sparse products are single-threaded), the same sample on
    `workers` members at once in separate processes (all cores; the members
    are independent problems), and the 41^3 x 300-step plain FP64 workload in
    full.  Processes are started with spawn."""
    import multiprocessing as mp
    info = host_info()
    upd, wall, cores = OracleSample(*_member_args(3)).run()
    single = upd / wall
    out = {"value": single, "unit": UNIT, "cores": cores, "kind": "oracle",
           "sample": (f"one 161^3 member of the batched workload (FEM cube 121^3), {SAMPLE_STEPS} forward + "
                      f"{SAMPLE_STEPS} adjoint steps, functional and gradient, FP64 scipy oracle, assembly "
                      f"excluded, {wall:.1f} s"),
           "host": info}
    mem_gb = None
    try:   # about 5 GB of host memory per oracle process at 161^3; keep half free
        mem_gb = os.sysconf("SC_PHYS_PAGES") * os.sysconf("SC_PAGE_SIZE") / 1e9
        workers = max(1, min(workers, int(mem_gb // 10)))
    except (ValueError, OSError):
        pass
    info["host_memory_gb"] = round(mem_gb, 1) if mem_gb else None
    if workers > 1:
        ctx = mp.get_context("spawn")
        t0 = time.perf_counter()
        with ctx.Pool(workers) as pool:
            res = pool.starmap(oracle_sample, [_member_args(3)] * workers)
        wall_all = time.perf_counter() - t0
        out["all_cores"] = {"value": sum(r[0] / r[1] for r in res), "unit": UNIT, "processes": workers,
                            "sample": f"the same sample in {workers} processes at once (identical assembly, so "
                                      f"the timed parts run concurrently); the value sums their rates; "
                                      f"{wall_all:.1f} s in all"}
    upd1, wall1 = oracle_full_run("c1_fp64_41")
    out["c1_fp64_41_full"] = {"value": upd1 / wall1, "unit": UNIT, "seconds": wall1, "cores": 1,
                              "run": "41^3 grid, FEM 21^3, 300 steps: forward, functional, adjoint, gradient"}
    return out


def run_reference(args, rank):
    """--impl reference: the oracle (this build has no other reference
    implementation) on the same workload, each bench step a bounded sample:
    one batch member for SAMPLE_STEPS forward + adjoint steps."""
    if rank != 0:
        return
    steps = 2
    (w, d), = batched_problems(first=3, n_problems=1)
    sampler = OracleSample(w.n, w.fem_n, w.seed, w.n_incl, d, steps)
    vals, cores = [], 1
    for i in range(args.warmup + args.steps):
        upd, wall, cores = sampler.run()
        if i >= args.warmup:
            vals.append(upd / wall)
    value = statistics.mean(vals)
    sample = (f"problem 3 of the batched workload (161^3 grid, FEM cube 121^3), {steps} forward + {steps} "
              f"adjoint steps, functional and gradient per bench step, FP64 scipy oracle, assembly excluded")
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT,
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 2 * 161 ** 3 * steps / value * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": BATCH_WORKLOAD},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                             "sample": sample, "host": host_info()}}
    print(json.dumps(line), flush=True)


# --------------------------------------------------------------------------
# GPU legs
# --------------------------------------------------------------------------

def rel(a, b):
    a = np.asarray(a, np.float64)
    b = np.asarray(b, np.float64)
    nb = np.linalg.norm(b)
    return float(np.linalg.norm(a - b) / nb) if nb > 0 else float(np.linalg.norm(a))


def fp64_peak_tflops(dev):
    """Measured FP64 rate: cuBLAS DGEMM (torch.matmul float64, 4096^3), best
    of 5, CUDA events.  Used as the FP64 ALU peak of the plain FP64 path."""
    import torch
    a = torch.randn(4096, 4096, dtype=torch.float64, device=dev)
    b = torch.randn(4096, 4096, dtype=torch.float64, device=dev)
    for _ in range(2):
        a @ b
    best = 1e30
    for _ in range(5):
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record()
        a @ b
        e1.record()
        torch.cuda.synchronize(dev)
        best = min(best, e0.elapsed_time(e1))
    return 2 * 4096 ** 3 / (best / 1e3) / 1e12


def run_batched(args, dev, stream, rank, world, peak):
    import torch
    import torch.distributed as dist
    from paper_2508_07780_gb300 import Batch

    probs = batched_problems(first=16 * rank, n_steps=args.batch_steps)
    kzs = {} if args.batch_kz == "auto" else dict(zip(("tile_kz", "tile_kz_lean"),
                                                       (int(v) for v in args.batch_kz.split(","))))
    cfgs = [dict(n=w.n, fem_n=w.fem_n, n_steps=w.n_steps, cfl=w.cfl, precision="fp32",
                 src_dir=d[None, :], det_ij=w.detectors(), z_delta_frac=w.z_delta_frac,
                 stream=stream.cuda_stream, **kzs) for w, d in probs]
    b = Batch(cfgs)
    T = lambda a: torch.tensor(a, dtype=torch.float64, device=dev)
    # observed data: each member's layers-only model trace (FP64 forward of the
    # batch); the inclusions are what the residual sees
    eobs = []
    for (w, d) in probs:
        from paper_2508_07780_gb300 import Problem
        q = Problem(n=w.n, fem_n=w.fem_n, n_steps=w.n_steps, cfl=w.cfl, precision="fp64",
                    src_dir=d[None, :], det_ij=w.detectors(), z_delta_frac=w.z_delta_frac,
                    forward_only=1, stream=stream.cuda_stream)
        q.set_coeffs(*w.model(inclusions=False))
        e = torch.empty(q.trace_shape, dtype=torch.float64, device=dev)
        q.forward_dev(e)
        q.close()
        eobs.append(e)
    coefs = [tuple(T(a) for a in w.model()) for w, _ in probs]
    grads = [(torch.empty(m.n_free, dtype=torch.float64, device=dev),
              torch.empty(m.n_free, dtype=torch.float64, device=dev)) for m in b.members]
    if args.batch_kz == "auto":
        b.autotune(steps=8)
    kz = (b.get_info().tile_kz, b.get_info().tile_kz_lean)

    def mark(parts, name):  # optional per-call wall time (with a device sync), outside the timed steps
        if parts is not None:
            torch.cuda.synchronize(dev)
            now = time.perf_counter()
            parts[name] = round((now - parts.pop("_t", now)) * 1e3, 1)
            parts["_t"] = now

    def step(parts=None):
        mark(parts, "start")
        for m, (e, s) in zip(b.members, coefs):
            m.set_coeffs_dev(e, s)
        mark(parts, "set_coeffs")
        b.forward_dev(None)
        mark(parts, "batch_forward")
        J = sum(m.functional_dev(e) for m, e in zip(b.members, eobs))
        mark(parts, "functional")
        b.adjoint_dev(eobs)
        mark(parts, "batch_adjoint")
        for m, (ge, gs) in zip(b.members, grads):
            m.gradient_dev(ge, gs)
        mark(parts, "gradient")
        return J

    for _ in range(args.warmup):
        step()
    sampler = ClockSampler(dev.index) if rank == 0 else None
    if sampler:
        sampler.start()
    if world > 1:
        dist.barrier()
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
    if world > 1:
        dist.barrier()
    clocks = sampler.stop() if sampler else None
    inf = b.get_info()
    launches = inf.kernel_launches - l0
    ms = ev0.elapsed_time(ev1) / args.steps

    # end to end: host coefficients, host observed data, host gradients and J
    pin = lambda a: torch.tensor(a, dtype=torch.float64).pin_memory()
    coefs_h = [(pin(w.model()[0]), pin(w.model()[1])) for w, _ in probs]
    eobs_h = [e.cpu().pin_memory() for e in eobs]
    grads_h = [(torch.empty(m.n_free, dtype=torch.float64).pin_memory(),
                torch.empty(m.n_free, dtype=torch.float64).pin_memory()) for m in b.members]
    lib = b._lib
    import ctypes

    def step_e2e(parts=None):
        mark(parts, "start")
        for m, (e, s) in zip(b.members, coefs_h):
            m._check(lib.ddfd_set_coeffs(m._h, ctypes.c_void_p(e.data_ptr()), ctypes.c_void_p(s.data_ptr()),
                                         None, None))
        mark(parts, "set_coeffs")
        b._check(lib.ddfd_batch_forward(b._h, None))
        mark(parts, "batch_forward")
        J = 0.0
        for m, e in zip(b.members, eobs_h):
            Jm = ctypes.c_double()
            m._check(lib.ddfd_functional(m._h, ctypes.c_void_p(e.data_ptr()), ctypes.byref(Jm)))
            J += Jm.value
        mark(parts, "functional")
        ptrs = (ctypes.c_void_p * len(eobs_h))(*[e.data_ptr() for e in eobs_h])
        b._check(lib.ddfd_batch_adjoint(b._h, ptrs))
        mark(parts, "batch_adjoint")
        for m, (ge, gs) in zip(b.members, grads_h):
            m._check(lib.ddfd_gradient(m._h, ctypes.c_void_p(ge.data_ptr()), ctypes.c_void_p(gs.data_ptr())))
        mark(parts, "gradient")
        return J

    step_e2e()
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize(dev)
    sampler2 = ClockSampler(dev.index) if rank == 0 else None
    if sampler2:
        sampler2.start()
    e2e_iter = []
    t0 = time.perf_counter()
    for _ in range(args.steps):
        ti = time.perf_counter()
        step_e2e()
        torch.cuda.synchronize(dev)
        e2e_iter.append((time.perf_counter() - ti) * 1e3)
    e2e_s = (time.perf_counter() - t0) / args.steps
    clocks_e2e = sampler2.stop() if sampler2 else None
    # the plain rate of a pinned host -> device copy in this process (torch), beside the calls' copies
    probe_d = torch.empty_like(eobs_h[0], device=dev)
    torch.cuda.synchronize(dev)
    tc = time.perf_counter()
    for e in eobs_h:
        probe_d.copy_(e, non_blocking=True)
    torch.cuda.synchronize(dev)
    host_copy_gbs = sum(e.numel() * 8 for e in eobs_h) / (time.perf_counter() - tc) / 1e9
    del probe_d
    e2e_parts, dev_parts = {}, {}
    step_e2e(e2e_parts)  # one more of each, untimed, with a sync after each call
    step(dev_parts)
    for d in (e2e_parts, dev_parts):
        d.pop("_t", None)
        d.pop("start", None)
    ntr = sum(int(np.prod(m.trace_shape)) for m in b.members)
    nfr = sum(m.n_free for m in b.members)
    h2d = 2 * nfr * 8 + 2 * ntr * 8
    d2h = 2 * nfr * 8 + len(b.members) * 8

    # FP32 results of one more pass, for the accuracy comparison
    out32 = []
    if rank == 0 and not args.no_fp64:
        traces = [torch.empty(m.trace_shape, dtype=torch.float64, device=dev) for m in b.members]
        for m, (e, s) in zip(b.members, coefs):
            m.set_coeffs_dev(e, s)
        b.forward_dev(traces)
        Js = [m.functional_dev(e) for m, e in zip(b.members, eobs)]
        b.adjoint_dev(eobs)
        for i, m in enumerate(b.members):
            ge, gs = grads[i]
            m.gradient_dev(ge, gs)
            out32.append(dict(trace=traces[i].cpu().numpy(), J=Js[i], g_eps=ge.cpu().numpy(),
                              g_sig=gs.cpu().numpy(), eobs=eobs[i].cpu().numpy()))
        del traces
    dev_bytes = inf.device_bytes
    n_groups = (len(b.members) + 15) // 16
    b.close()
    del eobs, coefs, grads
    torch.cuda.empty_cache()

    ws = [w for w, _ in probs]
    fb = sum(algorithmic_bytes(w.n, w.fem_n, 4)[0] for w in ws)
    ab = sum(algorithmic_bytes(w.n, w.fem_n, 4)[1] for w in ws)
    nt = ws[0].n_steps
    fwd_avg = fwd_ms / (args.steps * nt * n_groups)
    adj_avg = adj_ms / (args.steps * nt * n_groups)
    updates = sum(w.updates for w in ws)
    res = dict(ms=ms, updates=updates, e2e_s=e2e_s, e2e_iter=e2e_iter, clocks_e2e=clocks_e2e, e2e_parts=e2e_parts,
               dev_parts=dev_parts, host_copy_gbs=host_copy_gbs,
               h2d=h2d, d2h=d2h,
               launches=launches, clocks=clocks,
               kz=kz, dev_bytes=dev_bytes, out32=out32, probs=probs)
    res["roofline"] = {
        "bound": "hbm", "achieved": ab / (adj_avg / 1e3) / 1e9, "peak": peak[0], "unit": "GB/s",
        "frac": ab / (adj_avg / 1e3) / 1e9 / peak[0],
        "traffic": traffic_per_launch("batched_adjoint_full_dram_bytes", "batched_adjoint_lean_dram_bytes"),
        "kernel": "k_step_pair<adjoint,16>: full kernel (tiles with FEM-cube or free nodes) and lean kernel "
                  "(finite-difference tiles) side by side; one launch = one adjoint step of all 16 problems",
        "algorithmic_bytes_per_launch": ab, "avg_launch_ms": adj_avg,
        "peak_kind": f"{peak[1]} (HBM copy, MEASURED_PEAKS.json hbm_gbs)",
        "forward": {"kernel": "k_step_pair<forward,16>, full and lean kernels side by side",
                    "algorithmic_bytes_per_launch": fb,
                    "avg_launch_ms": fwd_avg, "achieved": fb / (fwd_avg / 1e3) / 1e9,
                    "frac": fb / (fwd_avg / 1e3) / 1e9 / peak[0],
                    "traffic": traffic_per_launch("batched_forward_full_dram_bytes",
                                                  "batched_forward_lean_dram_bytes")},
        "whole_pass": {"algorithmic_bytes": (fb + ab) * nt, "ms": ms,
                       "achieved": (fb + ab) * nt / (ms / 1e3) / 1e9,
                       "frac": (fb + ab) * nt / (ms / 1e3) / 1e9 / peak[0],
                       "note": "forward + adjoint step bytes of every member over the whole pass time "
                               "(set_coeffs, forward, functional, adjoint, gradient)"}}
    return res


def run_fp64_plain(args, dev, stream, probs, out32, fp64_peak):
    """The plain FP64 GPU path on the same problems, one at a time (the FP64
    method without batching), timed pass by pass after one warm-up pass per
    problem; its results are the reference of the accuracy table."""
    import torch
    from paper_2508_07780_gb300 import Problem
    total_ms = 0.0
    upd = 0
    errs = []
    step_ms = []
    for i, (w, d) in enumerate(probs):
        p = Problem(n=w.n, fem_n=w.fem_n, n_steps=w.n_steps, cfl=w.cfl, precision="fp64",
                    src_dir=d[None, :], det_ij=w.detectors(), z_delta_frac=w.z_delta_frac,
                    stream=stream.cuda_stream)
        eps, sig = (torch.tensor(a, dtype=torch.float64, device=dev) for a in w.model())
        eo = torch.tensor(out32[i]["eobs"], dtype=torch.float64, device=dev)
        tr = torch.empty(p.trace_shape, dtype=torch.float64, device=dev)
        ge = torch.empty(p.n_free, dtype=torch.float64, device=dev)
        gs = torch.empty_like(ge)

        def step():
            p.set_coeffs_dev(eps, sig)
            p.forward_dev(tr)
            J = p.functional_dev(eo)
            p.adjoint_dev(eo)
            p.gradient_dev(ge, gs)
            return J

        step()
        torch.cuda.synchronize(dev)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        J = step()
        e1.record(stream)
        torch.cuda.synchronize(dev)
        total_ms += e0.elapsed_time(e1)
        t = p.get_timing()
        step_ms.append((t.forward_loop_ms / t.forward_step_kernels, t.adjoint_loop_ms / t.adjoint_step_kernels))
        upd += w.updates
        a, tr64 = out32[i], tr.cpu().numpy()
        kappa = float(np.linalg.norm(tr64) / np.linalg.norm(tr64 - a["eobs"]))
        errs.append(dict(trace=rel(a["trace"], tr64), J=abs(a["J"] - J) / abs(J),
                         g_eps=rel(a["g_eps"], ge.cpu().numpy()), g_sig=rel(a["g_sig"], gs.cpu().numpy()),
                         kappa=kappa))
        p.close()
        del eps, sig, eo, tr, ge, gs
        torch.cuda.empty_cache()
    # FP64 ALU roofline of the FP64 step kernels (problem 3, the 121^3 FEM cube)
    w3 = probs[3][0]
    ff, fa = fp64_flops(w3.n, w3.fem_n)
    fwd_ms, adj_ms = step_ms[3]
    ach = max(ff / (fwd_ms / 1e3), fa / (adj_ms / 1e3)) / 1e12
    roof = {"bound": "alu", "achieved": ach, "peak": fp64_peak, "unit": "TFLOP/s", "frac": ach / fp64_peak,
            "kernel": "k_step<double> (forward and adjoint, problem 3: FEM cube 121^3)",
            "algorithmic_flops_per_launch": {"forward": ff, "adjoint": fa},
            "avg_launch_ms": {"forward": fwd_ms, "adjoint": adj_ms},
            "peak_kind": "measured in this run: cuBLAS DGEMM 4096^3 (torch.matmul float64), best of 5"}
    worst = {k: max(e[k] for e in errs) for k in ("trace", "J", "g_eps", "g_sig")}
    return dict(value=upd / (total_ms / 1e3), ms=total_ms, errs=errs, worst=worst, roofline=roof)


def run_single_201(args, dev, stream, peak):
    """One single-source FP32 workload (`--workload`, by default the 201^3 grid
    with its 101^3 FEM cube and 2000 steps) with its FP64 counterpart:
    throughput, step rooflines and the FP32 errors against FP64, measured
    here.  `--snapshots K` checkpoints the FP32 run (K state snapshots, each
    segment replayed) instead of keeping the E history; `--no-fp64` skips the
    FP64 pass (its observed data still comes from an FP64 forward run)."""
    import torch
    from paper_2508_07780_gb300 import Problem
    w = workload(args.workload)
    if args.single_steps:
        w = w.with_(n_steps=args.single_steps)
    eps, sig = w.model()
    e_lay, s_lay = w.model(inclusions=False)
    T = lambda a: torch.tensor(a, dtype=torch.float64, device=dev)
    kw = dict(n=w.n, fem_n=w.fem_n, n_steps=w.n_steps, cfl=w.cfl, src_dir=w.directions(), det_ij=w.detectors(),
              z_delta_frac=w.z_delta_frac, grad_variant=args.grad_variant, stream=stream.cuda_stream)
    # observed data: the layers-only model's FP64 trace
    q = Problem(precision="fp64", forward_only=1, **dict(kw, grad_variant="exact"))
    q.set_coeffs(e_lay, s_lay)
    eobs = torch.empty(q.trace_shape, dtype=torch.float64, device=dev)
    q.forward_dev(eobs)
    q.close()
    out = {}
    for prec in ("fp32",) if args.no_fp64 else ("fp64", "fp32"):
        extra = {"n_snapshots": args.snapshots} if prec == "fp32" and args.snapshots else {}
        p = Problem(precision=prec, **kw, **extra)
        eps_d, sig_d = T(eps), T(sig)
        tr = torch.empty(p.trace_shape, dtype=torch.float64, device=dev)
        ge = torch.empty(p.n_free, dtype=torch.float64, device=dev)
        gs = torch.empty_like(ge)

        def step():
            p.set_coeffs_dev(eps_d, sig_d)
            p.forward_dev(tr)
            J = p.functional_dev(eobs)
            p.adjoint_dev(eobs)
            p.gradient_dev(ge, gs)
            return J

        reps = 1 if prec == "fp64" else max(args.steps, 3)
        for _ in range(1 if prec == "fp64" else max(args.warmup, 1)):
            step()
        torch.cuda.synchronize(dev)
        fwd = adj = nk = 0.0
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(reps):
            J = step()
            t = p.get_timing()
            fwd += t.forward_loop_ms
            adj += t.adjoint_loop_ms
            nk += t.forward_step_kernels
        e1.record(stream)
        torch.cuda.synchronize(dev)
        ms = e0.elapsed_time(e1) / reps
        # per forward step; the adjoint sequence per adjoint step (with a
        # replayed forward step in each when checkpointing)
        out[prec] = dict(ms=ms, fwd=fwd / nk, adj=adj / nk, trace=tr.cpu().numpy(), J=J,
                         g_eps=ge.cpu().numpy(), g_sig=gs.cpu().numpy(), bytes=p.get_info().device_bytes)
        p.close()
        del eps_d, sig_d, tr, ge, gs
    eo = eobs.cpu().numpy()
    del eobs
    torch.cuda.empty_cache()
    a = out["fp32"]
    fb, ab = algorithmic_bytes(w.n, w.fem_n, 4)
    kernel_note = "full and lean kernels side by side"
    res = {"workload": describe(w), "gradient": args.grad_variant, "value": w.updates / (a["ms"] / 1e3),
           "unit": UNIT, "ms_per_step": a["ms"], "device_bytes": int(a["bytes"]),
           "e_history": (f"checkpointed: {args.snapshots} state snapshots, each segment replayed"
                         if args.snapshots else "kept in HBM for every step"),
           "roofline": {"bound": "hbm", "peak": peak[0], "unit": "GB/s",
                        "forward": {"kernel": f"k_step_pair<forward,1>, {kernel_note}", "avg_launch_ms": a["fwd"],
                                    "algorithmic_bytes_per_launch": fb,
                                    "frac": fb / (a["fwd"] / 1e3) / 1e9 / peak[0]}}}
    if args.workload == "c2_fp32_201" and not args.snapshots:
        res["roofline"]["forward"]["traffic"] = traffic_per_launch("single_forward_full_dram_bytes",
                                                                   "single_forward_lean_dram_bytes")
    if not args.snapshots:
        res["roofline"]["adjoint"] = {"kernel": f"k_step_pair<adjoint,1>, {kernel_note}", "avg_launch_ms": a["adj"],
                                      "algorithmic_bytes_per_launch": ab,
                                      "frac": ab / (a["adj"] / 1e3) / 1e9 / peak[0]}
        if args.workload == "c2_fp32_201":
            res["roofline"]["adjoint"]["traffic"] = traffic_per_launch("single_adjoint_full_dram_bytes",
                                                                       "single_adjoint_lean_dram_bytes")
    else:
        res["adjoint_sequence_ms_per_step"] = a["adj"]
    if "fp64" in out:
        b = out["fp64"]
        rn = float(np.linalg.norm(b["trace"] - eo))
        kappa = float(np.linalg.norm(b["trace"]) / rn) if rn > 0 else None
        res["fp64_plain"] = {"value": w.updates / (b["ms"] / 1e3), "ms_per_step": b["ms"],
                             "fp32_speedup": b["ms"] / a["ms"]}
        res["accuracy_vs_fp64"] = {"trace": rel(a["trace"], b["trace"]),
                                   "J": abs(a["J"] - b["J"]) / abs(b["J"]) if b["J"] != 0 else None,
                                   "g_eps": rel(a["g_eps"], b["g_eps"]), "g_sig": rel(a["g_sig"], b["g_sig"]),
                                   "kappa": kappa,
                                   "observed_data": "the layers-only model's FP64 trace (unmodified)"}
    return res


def run_ebe(args, dev, stream, peak):
    """The element-by-element FEM apply: the 201^3 workload with its 101^3
    FEM cube gathered over the explicit Kuhn tetrahedra (fem_kind
    DDFD_FEM_EBE), and a 241^3 grid whose 61^3 FEM cube is refined once
    around the inclusion (fem_kind DDFD_FEM_MESH: gathered rows next to
    refined elements and the new nodes, the untouched Kuhn rows on the block
    stencil).  One source each, FP32, a forward + adjoint pass after a warm-up
    pass; the gather's roofline from ddfd_time_gather (CUDA events, 20
    launches each way).  The observed data is the same handle's trace of the
    layers-only model: these legs measure speed (accuracy: the tests)."""
    import torch
    from paper_2508_07780_gb300 import Problem
    from synth import box_bounds, detector_grid, layered_inclusion_model
    from synth.mesh import extend_to_new_nodes, refined_fem_mesh
    out = {}
    legs = [("ebe_201", 201, 101, 2000, 0.3, None)]
    if not args.no_refined:
        legs.append(("refined_241", 241, 61, 2880, 0.25, "refine"))
    for name, n, fem_n, nt, cfl, kind in legs:
        t0 = time.perf_counter()
        eps, sig = layered_inclusion_model(n, fem_n, 2 if n == 201 else 5, 3 if n == 201 else 1)
        e0, s0 = layered_inclusion_model(n, fem_n, 2 if n == 201 else 5, 0)
        kw = dict(n=n, fem_n=fem_n, n_steps=nt, cfl=cfl, precision="fp32", det_ij=detector_grid(n, fem_n, 32),
                  stream=stream.cuda_stream)
        extra = {}
        if kind == "refine":
            _, _, f0, f1 = box_bounds(n, fem_n)
            nfr = f1 - f0 + 1
            par, tets = refined_fem_mesh(n, fem_n, eps, sig, beta_eps=0.8, beta_sig=0.0,
                                         region=(f0 + int(0.3 * nfr), f0 + int(0.7 * nfr)))
            eps, sig = extend_to_new_nodes(n, fem_n, par, eps, sig)
            e0, s0 = extend_to_new_nodes(n, fem_n, par, e0, s0)
            p = Problem(fem_kind=2, mesh=(par, tets), **kw)
            extra = {"new_nodes": int(par.shape[0]), "tets": int(tets.shape[0])}
        else:
            p = Problem(fem_kind=1, **kw)
            extra = {"tets": 6 * (fem_n - 1) ** 3}
        setup_s = time.perf_counter() - t0
        p.set_coeffs(e0, s0)
        eobs = torch.empty(p.trace_shape, dtype=torch.float64, device=dev)
        p.forward_dev(eobs)
        T = lambda a: torch.tensor(a, dtype=torch.float64, device=dev)
        e_d, s_d = T(eps), T(sig)
        ge = torch.empty(p.n_free, dtype=torch.float64, device=dev)
        gs = torch.empty_like(ge)

        def step():
            p.set_coeffs_dev(e_d, s_d)
            p.forward_dev(None)
            p.functional_dev(eobs)
            p.adjoint_dev(eobs)
            p.gradient_dev(ge, gs)

        step()
        torch.cuda.synchronize(dev)
        e0_ = torch.cuda.Event(enable_timing=True)
        e1_ = torch.cuda.Event(enable_timing=True)
        e0_.record(stream)
        for _ in range(2):
            step()
        e1_.record(stream)
        torch.cuda.synchronize(dev)
        ms = e0_.elapsed_time(e1_) / 2
        fms, ams, fb, ab = p.time_gather(20)
        p.close()
        del eobs, e_d, s_d, ge, gs
        torch.cuda.empty_cache()
        updates = 2 * n ** 3 * nt
        out[name] = {"workload": f"{n}^3 grid, FEM cube {fem_n}^3" + (" refined once around the inclusion"
                                                                       if kind else " as explicit Kuhn tets")
                     + f", {nt} steps, FP32, one source", **extra,
                     "value": updates / (ms / 1e3), "unit": UNIT, "ms_per_step": ms, "setup_s": setup_s,
                     "gather_roofline": {
                         "bound": "hbm", "peak": peak[0], "unit": "GB/s",
                         "kernels": "k_ebe" + (" + k_kuhn_rows" if kind else ""),
                         "forward": {"ms": fms, "algorithmic_bytes": fb, "achieved": fb / (fms / 1e3) / 1e9,
                                     "frac": fb / (fms / 1e3) / 1e9 / peak[0]},
                         "adjoint": {"ms": ams, "algorithmic_bytes": ab, "achieved": ab / (ams / 1e3) / 1e9,
                                     "frac": ab / (ams / 1e3) / 1e9 / peak[0]}}}
    return out


def run_ours(args, rank, world, local_rank):
    import torch
    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    stream = torch.cuda.current_stream(dev)
    peak = measured_peaks()
    single = None
    if world == 1 and (not args.no_single or args.no_batched):
        single = run_single_201(args, dev, stream, peak)
    if args.no_batched:
        # an auxiliary run of the single-source leg alone (not the headline workload)
        if rank == 0:
            line = {"metric": METRIC, "value": single["value"], "unit": UNIT, "n_gpus": 1, "steps": args.steps,
                    "warmup": args.warmup, "ms_per_step": single["ms_per_step"], "higher_is_better": True,
                    "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
                    "config": {"workload": single["workload"], "leg": "single source only (--no-batched)"},
                    "single": single}
            print(json.dumps(line), flush=True)
        return
    bat = run_batched(args, dev, stream, rank, world, peak)
    ms_t = torch.tensor([bat["ms"], bat["e2e_s"]], device=dev)
    if world > 1:
        import torch.distributed as dist
        dist.all_reduce(ms_t, op=dist.ReduceOp.MAX)
    ms, e2e_s = float(ms_t[0].item()), float(ms_t[1].item())
    if rank != 0:
        return
    value = world * bat["updates"] / (ms / 1e3)
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": BATCH_WORKLOAD if args.batch_steps == 1600 else
                       BATCH_WORKLOAD.replace("1600 steps", f"{args.batch_steps} steps (profiling run)"),
                       "grid": 161, "problems_per_gpu": 16, "n_steps": args.batch_steps,
                       "fem_n": [61, 81, 101, 121], "tile_kz": bat["kz"], "device_bytes": int(bat["dev_bytes"]),
                       "l2": "inputs larger than L2: 16 problems x 2 field levels of 3 x 161^3 FP32 plus "
                             "the E history, re-streamed every step",
                       "parallelism": "single GPU" if world == 1 else
                       f"{world} GPUs, 16 independent problems each (problems 16 r .. 16 r + 15 on rank r), "
                       f"no data-path collective"},
            "e2e": {"value": world * bat["updates"] / e2e_s, "unit": UNIT, "h2d_bytes_per_step": bat["h2d"],
                    "d2h_bytes_per_step": bat["d2h"], "ms_per_step": e2e_s * 1e3,
                    "ms_each_step": [round(v, 1) for v in bat["e2e_iter"]], "clocks": bat["clocks_e2e"],
                    "ms_by_call_one_more_step": bat["e2e_parts"],
                    "device_resident_ms_by_call_one_more_step": bat["dev_parts"],
                    "torch_pinned_h2d_gbs": bat["host_copy_gbs"]},
            "roofline": bat["roofline"],
            "gpu_launches": int(bat["launches"]),
            "clocks": bat["clocks"]}
    if world == 1 and not args.no_fp64:
        fp = run_fp64_plain(args, dev, stream, bat["probs"], bat["out32"], fp64_peak_tflops(dev))
        line["fp64_plain"] = {"value": fp["value"], "unit": UNIT, "ms_per_step": fp["ms"],
                              "how": "the same 16 problems solved one at a time in FP64 (plain, unbatched)",
                              "fp32_batched_speedup": value / fp["value"], "roofline": fp["roofline"]}
        line["accuracy"] = {"reference": "FP64 plain path on the same problems and observed data",
                            "worst_over_problems": fp["worst"],
                            "north_star_bars": {"trace": 1e-4, "J": 1e-4, "g": 1e-3},
                            "kappa_range": [min(e["kappa"] for e in fp["errs"]), max(e["kappa"] for e in fp["errs"])],
                            "per_problem": fp["errs"]}
    if single is not None:
        line["single_201"] = single
    if world == 1 and not args.no_ebe:
        line["element_gather"] = run_ebe(args, dev, stream, peak)
    if world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(args.cpu_workers)
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-fp64", action="store_true", help="skip the FP64 comparison passes")
    ap.add_argument("--no-single", action="store_true", help="skip the single-source 201^3 workload")
    ap.add_argument("--no-ebe", action="store_true", help="skip the element-gather legs")
    ap.add_argument("--grad-variant", choices=["exact", "literal"], default="exact",
                    help="gradient form of the single-source leg: the exact derivative of the discrete J "
                         "(default) or the paper-literal one of Sec. 4")
    ap.add_argument("--no-refined", action="store_true", help="skip the refined-mesh element-gather leg")
    ap.add_argument("--cpu-workers", type=int, default=min(8, os.cpu_count() or 1))
    ap.add_argument("--no-batched", action="store_true",
                    help="run only the single-source leg (an auxiliary measurement, not the headline)")
    ap.add_argument("--workload", default="c2_fp32_201", help="the single-source leg's workload (synth)")
    ap.add_argument("--snapshots", type=int, default=0,
                    help="the single-source FP32 run checkpoints with this many state snapshots")
    ap.add_argument("--batch-kz", default="auto",
                    help="z depths 'FULL,LEAN' of the batched step kernels, or 'auto' (autotuned)")
    ap.add_argument("--single-steps", type=int, default=0,
                    help="time steps of the single-source workload (0: its own, 2000 for the 201^3 one; "
                         "fewer only for profiler captures)")
    ap.add_argument("--batch-steps", type=int, default=1600,
                    help="time steps of the batched workload (1600; fewer only for profiler captures: "
                         "every step launch does the same work at any step count)")
    args = ap.parse_args()
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        run_reference(args, rank)
        return
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    try:
        run_ours(args, rank, world, local_rank)
    finally:
        if world > 1:
            import torch.distributed as dist
            dist.destroy_process_group()


if __name__ == "__main__":
    main()
