"""Source sharding across ranks (world size 2, gloo, CPU).

The per-rank solver is the FP64 oracle behind the Problem interface, so the
host-side logic -- partition, regularisation counted once, the FP64
all-reduce -- is checked against one process running every source."""
import os
import socket

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


class OracleSolver:
    """The oracle with the Problem methods the sharding layer calls."""

    def __init__(self, w, src_dirs, gamma_eps, gamma_sig):
        from oracle import OracleProblem, SourceSpec
        eps, sig = w.model()
        self.w = w
        self.args = (w.n, w.fem_n, w.n_steps, w.cfl)
        self.kw = dict(z_delta_frac=w.z_delta_frac, gamma_eps=gamma_eps, gamma_sig=gamma_sig)
        self.srcs = [SourceSpec(direction=tuple(d)) for d in src_dirs]
        self.det = w.detectors()
        self.P = None

    def set_coeffs(self, eps, sig, eps0=None, sig0=None):
        from oracle import OracleProblem
        self.P = OracleProblem(*self.args, eps, sig, self.det, self.srcs, eps0_free=eps0,
                               sig0_free=sig0, **self.kw)

    def forward(self):
        self.fw = [self.P.forward(s) for s in range(len(self.srcs))]
        return np.stack([f.trace for f in self.fw])

    def functional(self, eobs):
        return self.P.functional([f.trace for f in self.fw], list(eobs))

    def adjoint(self, eobs):
        self.ad = [self.P.adjoint(s, self.fw[s].trace, eobs[s]) for s in range(len(self.srcs))]

    def gradient(self):
        return self.P.gradient(self.fw, self.ad)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out_path):
    import sys
    sys.path.insert(0, ROOT)
    sys.path.insert(0, os.path.join(ROOT, "tests"))
    import torch.distributed as dist
    from paper_2508_07780_gb300.sharding import SourceShard
    from synth import workload
    from test_sharding import OracleSolver
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    w = workload("tiny", n_src=3, dir_seed=21, n_steps=30, gamma_eps=0.3, gamma_sig=0.1)
    eps, sig = w.model()
    eobs = 0.01 * np.random.default_rng(0).standard_normal((3, w.n_steps + 1, w.det_per_side ** 2, 3))
    shard = SourceShard(lambda d, ge, gs: OracleSolver(w, d, ge, gs), w.directions(), rank, world,
                        gamma_eps=w.gamma_eps, gamma_sig=w.gamma_sig)
    J, ge, gs = shard.loss_and_grad(eps, sig, eobs, w.n_free)
    np.savez(f"{out_path}.{rank}.npz", J=J, ge=ge, gs=gs, mine=np.array(shard.mine))
    dist.destroy_process_group()


def test_partition_is_round_robin_and_complete():
    from paper_2508_07780_gb300.sharding import partition_sources
    parts = partition_sources(7, 3)
    assert parts == [[0, 3, 6], [1, 4], [2, 5]]
    assert sorted(sum(parts, [])) == list(range(7))


def test_two_gloo_ranks_equal_one_process(tmp_path):
    import torch.multiprocessing as mp
    from synth import workload
    port = _free_port()
    out = str(tmp_path / "res")
    mp.spawn(_worker, args=(2, port, out), nprocs=2, join=True)
    r0, r1 = np.load(f"{out}.0.npz"), np.load(f"{out}.1.npz")
    assert list(r0["mine"]) == [0, 2] and list(r1["mine"]) == [1]
    # every rank holds the same reduced result
    assert r0["J"] == r1["J"]
    assert np.array_equal(r0["ge"], r1["ge"]) and np.array_equal(r0["gs"], r1["gs"])
    # and it is the single-process result over all sources
    w = workload("tiny", n_src=3, dir_seed=21, n_steps=30, gamma_eps=0.3, gamma_sig=0.1)
    eps, sig = w.model()
    eobs = 0.01 * np.random.default_rng(0).standard_normal((3, w.n_steps + 1, w.det_per_side ** 2, 3))
    one = OracleSolver(w, w.directions(), w.gamma_eps, w.gamma_sig)
    one.set_coeffs(eps, sig)
    one.forward()
    J = one.functional(eobs)
    one.adjoint(eobs)
    ge, gs = one.gradient()
    assert r0["J"] == pytest.approx(J, rel=1e-13)
    assert np.allclose(r0["ge"], ge, rtol=1e-12, atol=1e-14 * np.abs(ge).max())
    assert np.allclose(r0["gs"], gs, rtol=1e-12, atol=1e-14 * np.abs(gs).max())
