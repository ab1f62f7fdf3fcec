"""Multi-GPU by source sharding.

The incident plane waves are independent forward/adjoint problems that share
eps and sigma: J and the gradient are sums over sources (Sec. 3,
eq. tikhonov_functional summed over the measurements of every source).  Each
rank owns a round-robin subset of the sources, runs the whole path for them on
its own GPU, and one FP64 all-reduce of [J, g_eps, g_sig] (1 + 2 n_free
doubles) makes the result identical on every rank.  The regularisation term
is counted once (by rank 0).  There is no other communication.

The per-rank solver is any object with the Problem methods set_coeffs,
forward, functional, adjoint and gradient; by default a ddfd Problem on the
rank's GPU.
"""
from __future__ import annotations

from typing import Callable, Sequence

import numpy as np


def partition_sources(n_src: int, world: int):
    """Round-robin: rank r owns sources r, r + world, ..."""
    return [list(range(r, n_src, world)) for r in range(world)]


class SourceShard:
    """One rank's share of a multi-source problem.

    make_problem(src_dir, gamma_eps, gamma_sig) -> solver for the given
    [k][3] directions (None when the rank owns no source)."""

    def __init__(self, make_problem: Callable, src_dirs: np.ndarray, rank: int, world: int,
                 gamma_eps: float = 0.0, gamma_sig: float = 0.0, group=None):
        self.rank, self.world, self.group = rank, world, group
        self.src_dirs = np.asarray(src_dirs, dtype=np.float64).reshape(-1, 3)
        self.mine = partition_sources(self.src_dirs.shape[0], world)[rank]
        ge, gs = (gamma_eps, gamma_sig) if rank == 0 else (0.0, 0.0)
        self.problem = make_problem(self.src_dirs[self.mine], ge, gs) if self.mine else None
        if not self.mine and rank == 0:
            raise ValueError("rank 0 must own a source (it carries the regularisation)")

    def loss_and_grad(self, eps, sig, eobs_all: Sequence[np.ndarray], n_free: int,
                      eps0=None, sig0=None):
        """J and (g_eps, g_sig) summed over every source of every rank.
        eobs_all: the observed traces of all sources, [n_src][Nt+1][n_det][3]."""
        local = np.zeros(1 + 2 * n_free)
        if self.problem is not None:
            p = self.problem
            eobs = np.ascontiguousarray(np.asarray(eobs_all)[self.mine])
            p.set_coeffs(eps, sig, eps0, sig0)
            p.forward()
            local[0] = p.functional(eobs)
            p.adjoint(eobs)
            ge, gs = p.gradient()
            local[1:1 + n_free] = ge
            local[1 + n_free:] = gs
        total = self.allreduce(local)
        return float(total[0]), total[1:1 + n_free], total[1 + n_free:]

    def allreduce(self, x: np.ndarray) -> np.ndarray:
        if self.world == 1:
            return x
        import torch
        import torch.distributed as dist
        backend = dist.get_backend(self.group)
        dev = torch.device("cuda", torch.cuda.current_device()) if backend == "nccl" else torch.device("cpu")
        t = torch.from_numpy(x).to(dev)
        dist.all_reduce(t, op=dist.ReduceOp.SUM, group=self.group)
        return t.cpu().numpy()


def ddfd_problem_factory(**config) -> Callable:
    """make_problem for SourceShard backed by a ddfd Problem (this rank's GPU)."""
    from .binding import Problem

    def make(src_dir, gamma_eps, gamma_sig):
        return Problem(src_dir=src_dir, gamma_eps=gamma_eps, gamma_sig=gamma_sig, **config)

    return make


def reduce_loss_and_grad_dev(J: float, g_eps, g_sig, group=None):
    """Device-side form of the one collective: [J, g_eps, g_sig] summed over
    ranks in FP64 (g_eps and g_sig are CUDA float64 tensors, updated in place).
    Returns the summed J."""
    import torch
    import torch.distributed as dist
    n = g_eps.numel()
    buf = torch.empty(1 + 2 * n, dtype=torch.float64, device=g_eps.device)
    buf[0] = J
    buf[1:1 + n].copy_(g_eps)
    buf[1 + n:].copy_(g_sig)
    dist.all_reduce(buf, op=dist.ReduceOp.SUM, group=group)
    g_eps.copy_(buf[1:1 + n])
    g_sig.copy_(buf[1 + n:])
    return buf[0]

