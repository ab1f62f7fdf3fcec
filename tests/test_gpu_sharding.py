"""Source sharding on the CUDA path: what two ranks would compute, one source
each (the regulariser on rank 0 only), summed, equals one ddfd handle that
runs both sources -- and the oracle."""
import numpy as np
import pytest

from helpers import rel_l2
from synth import shard_directions, workload

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="session", autouse=True)
def _built():
    from paper_2508_07780_gb300 import build
    build.build()


def _loss_grad(p, eps, sig, eobs):
    p.set_coeffs(eps, sig)
    p.forward()
    J = p.functional(eobs)
    p.adjoint(eobs)
    ge, gs = p.gradient()
    return J, ge, gs


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_per_source_shards_sum_to_the_joint_problem(prec):
    from paper_2508_07780_gb300 import Problem
    from paper_2508_07780_gb300.sharding import SourceShard, ddfd_problem_factory
    w = workload("small", n_src=2, gamma_eps=0.05, gamma_sig=0.2)
    dirs = shard_directions(2)
    eps, sig = w.model()
    cfg = dict(n=w.n, fem_n=w.fem_n, n_steps=w.n_steps, cfl=w.cfl, precision=prec,
               det_ij=w.detectors(), z_delta_frac=w.z_delta_frac)
    rng = np.random.default_rng(4)
    eobs = 0.01 * rng.standard_normal((2, w.n_steps + 1, w.detectors().shape[0], 3))
    joint = Problem(src_dir=dirs, gamma_eps=w.gamma_eps, gamma_sig=w.gamma_sig, **cfg)
    J, ge, gs = _loss_grad(joint, eps, sig, eobs)
    joint.close()
    parts = [SourceShard(ddfd_problem_factory(**cfg), dirs, r, 2, w.gamma_eps, w.gamma_sig)
             for r in range(2)]
    acc = np.zeros(1 + 2 * w.n_free)
    for sh in parts:
        p = sh.problem
        j, a, b = _loss_grad(p, eps, sig, np.ascontiguousarray(eobs[sh.mine]))
        acc += np.concatenate([[j], a, b])
        p.close()
    tol = 1e-12 if prec == "fp64" else 1e-5
    assert abs(acc[0] - J) <= tol * abs(J)
    assert rel_l2(acc[1:1 + w.n_free], ge) <= tol
    assert rel_l2(acc[1 + w.n_free:], gs) <= tol
