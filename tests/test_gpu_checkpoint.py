"""Checkpointing (state snapshots + replayed segments) and the autograd
wrapper.

* checkpointed runs give bitwise the results of the full-history run (the
  kernels are deterministic and the replay recomputes the same E), for even
  and uneven segments, one-step segments and several sources;
* torch.autograd through DDFDFunction returns the oracle's gradient;
* the differentiable 301^3 / 4000-step workload with 32 snapshots: the FP32
  checkpointed adjoint gradient against central finite differences of J in
  FP64 (delta = 1e-4) at seeded free nodes, with far less device memory than
  the full history would take.
"""
import numpy as np
import pytest

from helpers import gpu_problem, rel_l2, run_oracle
from synth import workload

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2508_07780_gb300 import build
    build.build()


def _run(w, prec, nsnap, eobs, keep):
    p = gpu_problem(w, prec, n_snapshots=nsnap)
    p.set_capture(keep)
    eps, sig = w.model()
    p.set_coeffs(eps, sig)
    tr = p.forward()
    J = p.functional(eobs)
    p.adjoint(eobs)
    ge, gs = p.gradient()
    mu = [p.get_capture(1, i) for i in range(len(keep))]
    info = p.get_info()
    p.close()
    return tr, J, ge, gs, mu, info


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
@pytest.mark.parametrize("nsnap", [1, 7, 120])
def test_checkpointing_is_bitwise_the_full_history(prec, nsnap):
    w = workload("small", n_src=2, dir_seed=9)          # 25^3, 120 steps, 2 sources
    rng = np.random.default_rng(1)
    eobs = 1e-3 * rng.standard_normal((2, w.n_steps + 1, w.det_per_side ** 2, 3))
    keep = [0, 17, 60, 119]
    full = _run(w, prec, 0, eobs, keep)
    ck = _run(w, prec, nsnap, eobs, keep)
    assert np.array_equal(full[0], ck[0])
    assert full[1] == ck[1]
    assert np.array_equal(full[2], ck[2]) and np.array_equal(full[3], ck[3])
    for a, b in zip(full[4], ck[4]):
        assert np.array_equal(a, b)
    assert ck[5].forward_steps == 2 * 2 * w.n_steps      # one replay sweep per source
    assert full[5].forward_steps == 2 * w.n_steps


def test_autograd_returns_the_oracle_gradient():
    torch = pytest.importorskip("torch")
    from paper_2508_07780_gb300.autograd import ddfd_loss
    w = workload("tiny", gamma_eps=0.1, gamma_sig=0.2)
    ref = run_oracle(w)
    dev = torch.device("cuda")
    stream = torch.cuda.current_stream(dev)
    p = gpu_problem(w, "fp64", stream=stream.cuda_stream)
    eps, sig = w.model()
    e = torch.tensor(eps, dtype=torch.float64, device=dev, requires_grad=True)
    s = torch.tensor(sig, dtype=torch.float64, device=dev, requires_grad=True)
    eobs = torch.tensor(ref["eobs"], dtype=torch.float64, device=dev)
    loss = ddfd_loss(e, s, p, eobs)
    (2.0 * loss).backward()
    torch.cuda.synchronize()
    assert abs(loss.item() - ref["J"]) <= 1e-12 * abs(ref["J"])
    assert rel_l2(e.grad.cpu().numpy(), 2.0 * ref["g_eps"]) <= 1e-12
    assert rel_l2(s.grad.cpu().numpy(), 2.0 * ref["g_sig"]) <= 1e-12
    p.close()


def test_autograd_two_losses_on_one_handle_keep_their_own_gradients():
    """A second loss on the same handle before the first one's backward: the
    first backward must still return the gradient at its own coefficients
    (the handle's generation counter tells it to restore its forward state)."""
    torch = pytest.importorskip("torch")
    from paper_2508_07780_gb300.autograd import ddfd_loss
    w = workload("tiny")
    dev = torch.device("cuda")
    stream = torch.cuda.current_stream(dev)
    eps, sig = w.model()
    e_lay, s_lay = w.model(inclusions=False)
    rng = np.random.default_rng(3)
    eobs = torch.tensor(1e-3 * rng.standard_normal((1, w.n_steps + 1, w.det_per_side ** 2, 3)),
                        dtype=torch.float64, device=dev)
    want = []
    for e_np, s_np in ((eps, sig), (e_lay, s_lay)):        # each loss alone, fresh handle
        q = gpu_problem(w, "fp64", stream=stream.cuda_stream)
        e = torch.tensor(e_np, dtype=torch.float64, device=dev, requires_grad=True)
        s = torch.tensor(s_np, dtype=torch.float64, device=dev, requires_grad=True)
        ddfd_loss(e, s, q, eobs).backward()
        want.append((e.grad.cpu().numpy(), s.grad.cpu().numpy()))
        q.close()
    p = gpu_problem(w, "fp64", stream=stream.cuda_stream)
    e1 = torch.tensor(eps, dtype=torch.float64, device=dev, requires_grad=True)
    s1 = torch.tensor(sig, dtype=torch.float64, device=dev, requires_grad=True)
    e2 = torch.tensor(e_lay, dtype=torch.float64, device=dev, requires_grad=True)
    s2 = torch.tensor(s_lay, dtype=torch.float64, device=dev, requires_grad=True)
    loss1 = ddfd_loss(e1, s1, p, eobs)
    loss2 = ddfd_loss(e2, s2, p, eobs)       # overwrites the handle's forward state
    loss1.backward()
    loss2.backward()
    torch.cuda.synchronize()
    for got, ref in (((e1, s1), want[0]), ((e2, s2), want[1])):
        assert np.array_equal(got[0].grad.cpu().numpy(), ref[0])
        assert np.array_equal(got[1].grad.cpu().numpy(), ref[1])
    assert not np.array_equal(want[0][0], want[1][0])   # the two gradients do differ
    assert rel_l2(want[0][0], want[1][0]) > 1e-5
    p.close()


def test_differentiable_301_checkpointed_gradient_vs_finite_differences():
    """The differentiable 301^3 / 4000-step workload with 32 snapshots: the
    FP32 and FP64 checkpointed adjoint gradients against central differences
    of the FP64 functional (delta = 1e-4) at free nodes drawn uniformly
    (seeded), for eps and sigma, with the per-node bars of
    paper_2508_07780_gb300.fdcheck; observed data: the layers-only model's
    trace.  Two nodes per coefficient here (each costs four FP64 forward
    runs of 4000 steps); `python -m paper_2508_07780_gb300.fdcheck` runs the
    same check at 20 nodes."""
    from paper_2508_07780_gb300.fdcheck import check_gradient
    w = workload("c4_fp32_301")
    p32 = gpu_problem(w, "fp32", n_snapshots=32)
    p32.set_coeffs(*w.model())
    p32.forward(want_trace=False)
    info = p32.get_info()
    full_history = (w.n_steps + 1) * 3 * w.n_free * 4
    assert info.device_bytes < 0.3 * full_history       # snapshots instead of all time levels
    p32.close()
    rep = check_gradient(w, n_nodes=2, seed=4)
    for r in rep["rows"]:
        print(f"301^3 {r['coef']}[{r['node']}]: FD {r['fd']:.6e}  FP32 {r['fp32']['g']:.6e} "
              f"({r['fp32']['err'] / r['fp32']['bar']:.2f} of bar)  FP64 {r['fp64']['g']:.6e} "
              f"({r['fp64']['err'] / r['fp64']['bar']:.2f} of bar)")
    assert rep["ok"], rep["rows"]
