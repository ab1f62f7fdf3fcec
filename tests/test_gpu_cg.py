"""ddfd_cg_run (the CGA of Sec. 4 on the GPU) against the oracle's CGA on the
same problem: two incident waves on the 13^3 grid, observed data from the
model with its inclusion, initial guess the layers-only model."""
import numpy as np
import pytest

from helpers import oracle_problem, rel_l2
from synth import shard_directions, workload

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="session", autouse=True)
def _built():
    from paper_2508_07780_gb300 import build
    build.build()


W = workload("tiny", n_steps=120, n_src=2)
DIRS = shard_directions(2)
PRM = dict(gamma_eps0=1e-3, gamma_sig0=1e-3, alpha_eps0=1038.793635, alpha_sig0=744.154304, p=0.5,
           eps_max=30.0, sig_max=5.0)


@pytest.fixture(scope="module")
def oracle_run():
    from oracle import SourceSpec
    from oracle.cg import CGParams, cga, problem_evaluator
    srcs = [SourceSpec(direction=tuple(d)) for d in DIRS]
    P0 = oracle_problem(W, *W.model(), srcs)
    eobs = [P0.forward(s).trace for s in range(2)]
    e0, s0 = W.model(inclusions=False)
    P = oracle_problem(W, e0, s0, srcs)
    m = P.op.m[P.g.free_nodes]
    ev = problem_evaluator(P)(eobs)
    eps, sig, log = cga(ev, e0, s0, m, CGParams(max_iter=3, **PRM))
    return dict(eobs=eobs, e0=e0, s0=s0, eps=eps, sig=sig, log=log, ev=ev, m=m)


def make_batch(prec, **kw):
    from paper_2508_07780_gb300 import Batch
    cfg = dict(n=W.n, fem_n=W.fem_n, n_steps=W.n_steps, cfl=W.cfl, precision=prec, det_ij=W.detectors(),
               z_delta_frac=W.z_delta_frac, eps_max=30.0, sig_max=5.0)
    cfg.update(kw)
    return Batch([dict(cfg, src_dir=d[None, :]) for d in DIRS])


KEYS = ("J", "J_data", "gnorm_eps", "gnorm_sig", "alpha_eps", "alpha_sig", "beta_eps", "beta_sig",
        "gamma_eps", "gamma_sig", "step_eps", "step_sig")


def test_cg_fp64_matches_the_oracle(oracle_run):
    o = oracle_run
    b = make_batch("fp64")
    eps, sig, log = b.cg_run(o["eobs"], o["e0"], o["s0"], max_iter=3, **PRM)
    b.close()
    assert len(log) == len(o["log"]) == 3
    for g, r in zip(log, o["log"]):
        for k in KEYS:
            assert g[k] == pytest.approx(r[k], rel=1e-8, abs=1e-30), (g["iter"], k)
        assert g["ms"] > 0
    assert rel_l2(eps - o["e0"], o["eps"] - o["e0"]) <= 1e-8
    assert rel_l2(sig - o["s0"], o["sig"] - o["s0"]) <= 1e-8


def test_cg_fp32_matches_the_oracle(oracle_run):
    o = oracle_run
    b = make_batch("fp32")
    eps, sig, log = b.cg_run(o["eobs"], o["e0"], o["s0"], max_iter=2, **PRM)
    b.close()
    for g, r in zip(log, o["log"][:2]):
        for k in ("J", "J_data", "gnorm_eps", "gnorm_sig"):
            assert g[k] == pytest.approx(r[k], rel=1e-3), (g["iter"], k)
    # the oracle's iterate after two updates
    from oracle.cg import CGParams, cga
    e2, s2, _ = cga(o["ev"], o["e0"], o["s0"], o["m"], CGParams(max_iter=2, **PRM))
    assert rel_l2(eps - o["e0"], e2 - o["e0"]) <= 1e-2
    assert rel_l2(sig - o["s0"], s2 - o["s0"]) <= 1e-2


def test_cg_restart_option_matches_the_oracle(oracle_run):
    from oracle.cg import CGParams, cga
    o = oracle_run
    eo, so, lo = cga(o["ev"], o["e0"], o["s0"], o["m"], CGParams(max_iter=4, restart=True, **PRM))
    assert any(r["beta_eps"] == 0.0 for r in lo[1:]) or any(r["beta_sig"] == 0.0 for r in lo[1:])
    b = make_batch("fp64")
    eps, sig, log = b.cg_run(o["eobs"], o["e0"], o["s0"], max_iter=4, restart=1, **PRM)
    b.close()
    for g, r in zip(log, lo):
        for k in KEYS:
            assert g[k] == pytest.approx(r[k], rel=1e-8, abs=1e-30), (g["iter"], k)
    assert rel_l2(eps - o["e0"], eo - o["e0"]) <= 1e-8


def test_cg_stopping_rule_matches(oracle_run):
    from oracle.cg import CGParams, cga
    o = oracle_run
    r0, r1 = o["log"][0], o["log"][1]
    # stop after iteration 1: its eps step and sigma gradient below the tolerances
    eta = dict(eta1_eps=r1["step_eps"] * 1.01, eta1_sig=0.0, eta2_eps=0.0, eta2_sig=r1["gnorm_sig"] * 1.01)
    assert not (r0["step_eps"] < eta["eta1_eps"] and r0["gnorm_sig"] < eta["eta2_sig"])
    eo, so, lo = cga(o["ev"], o["e0"], o["s0"], o["m"], CGParams(max_iter=5, **PRM, **eta))
    b = make_batch("fp64")
    eps, sig, log = b.cg_run(o["eobs"], o["e0"], o["s0"], max_iter=5, **PRM, **eta)
    b.close()
    assert len(log) == len(lo) == 2 and log[-1]["stop"] == 1 and lo[-1]["stop"]
    assert rel_l2(eps - o["e0"], eo - o["e0"]) <= 1e-8


def test_cg_rejects_regularised_members_and_mixed_cubes(oracle_run):
    from paper_2508_07780_gb300 import Batch, DDFDError
    o = oracle_run
    b = make_batch("fp64", gamma_eps=0.5)
    with pytest.raises(DDFDError) as e:
        b.cg_run(o["eobs"], o["e0"], o["s0"], max_iter=1, **PRM)
    assert e.value.code == -1 and "gamma" in str(e.value)
    b.close()
    cfg = dict(n=W.n, n_steps=W.n_steps, det_ij=W.detectors())
    b = Batch([dict(cfg, fem_n=9), dict(cfg, fem_n=11)])
    with pytest.raises(DDFDError) as e:
        b.cg_run(o["eobs"], o["e0"], o["s0"], max_iter=1, **PRM)
    assert e.value.code == -1 and "fem_n" in str(e.value)
    b.close()


def test_forward_only_handles():
    from paper_2508_07780_gb300 import DDFDError, Problem
    from helpers import run_gpu
    w = workload("small")
    eps, sig = w.model()
    full = run_gpu(w, np.zeros((1, w.n_steps + 1, w.det_per_side ** 2, 3)), precision="fp64")
    p = Problem(n=w.n, fem_n=w.fem_n, n_steps=w.n_steps, cfl=w.cfl, precision="fp64", det_ij=w.detectors(),
                z_delta_frac=w.z_delta_frac, forward_only=1)
    p.set_coeffs(eps, sig)
    tr = p.forward()
    assert np.array_equal(tr, full["trace"])
    assert p.get_info().device_bytes < 0.8 * full["info"].device_bytes
    with pytest.raises(DDFDError) as e:
        p.adjoint(np.zeros(p.trace_shape))
    assert e.value.code == -3
    p.close()


def test_failed_iteration_keeps_log_and_iterate(oracle_run):
    """An iteration that fails hands back what came before it: here the
    functional of iteration 0 overflows (observations of 1e300), so no record
    is kept and the iterate returned is the initial guess; the handle stays
    usable."""
    from paper_2508_07780_gb300 import DDFDError
    o = oracle_run
    b = make_batch("fp64")
    huge = [np.full_like(e, 1e300) for e in o["eobs"]]
    with pytest.raises(DDFDError) as e:
        b.cg_run(huge, o["e0"], o["s0"], max_iter=3, iterates=True, **PRM)
    assert e.value.code == -6 and "functional" in str(e.value)
    assert e.value.log == []
    assert np.array_equal(e.value.eps, o["e0"]) and np.array_equal(e.value.sig, o["s0"])
    eps, sig, log = b.cg_run(o["eobs"], o["e0"], o["s0"], max_iter=1, **PRM)
    b.close()
    assert log[0]["J"] == pytest.approx(o["log"][0]["J"], rel=1e-8)
