"""Failure detection without a GPU fault: a bounded wait that runs out.

ddfd_test_gather_timeout makes the element gather's first thread block wait
on an mbarrier that nothing completes (its bulk copy is never started).  The
wait gives up after a small number of polls, the kernel records the timeout
and returns, and the forward call reports DDFD_E_TIMEOUT.  The failed run
has partly overwritten the trace and the E history, so the calls that read
them (functional, adjoint, gradient) must then be refused with
DDFD_E_STATE, even though an earlier run had completed.  The handle must
still work: with the hook cleared the forward trace is bitwise the one of a
clean run."""
import numpy as np
import pytest

from synth import workload

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="session", autouse=True)
def _built():
    from paper_2508_07780_gb300 import build
    build.build()


@pytest.mark.parametrize("prec", ["fp32", "fp64"])
def test_gather_timeout_is_reported_and_the_handle_recovers(prec):
    from paper_2508_07780_gb300 import DDFDError, Problem
    w = workload("small", n=25, fem_n=13, n_steps=20, seed=12)
    p = Problem(n=w.n, fem_n=w.fem_n, n_steps=w.n_steps, cfl=w.cfl, precision=prec, det_ij=w.detectors(),
                z_delta_frac=w.z_delta_frac, fem_kind=1)
    p.set_coeffs(*w.model())
    clean = p.forward()
    eobs = 0.5 * clean
    p.adjoint(eobs)                       # a complete forward + adjoint state ...
    p.test_gather_timeout(1, 1 << 10)
    with pytest.raises(DDFDError) as e:
        p.forward()
    assert e.value.code == -7 and "bounded wait" in str(e.value)
    # ... that the failed forward invalidated
    for call in (lambda: p.functional(eobs), lambda: p.adjoint(eobs), lambda: p.gradient()):
        with pytest.raises(DDFDError) as e:
            call()
        assert e.value.code == -3
    p.test_gather_timeout(0)
    again = p.forward()
    assert np.array_equal(again, clean)
    p.close()


def test_timeout_hook_needs_an_element_gather():
    from paper_2508_07780_gb300 import DDFDError, Problem
    w = workload("tiny")
    p = Problem(n=w.n, fem_n=w.fem_n, n_steps=w.n_steps, det_ij=w.detectors())
    with pytest.raises(DDFDError) as e:
        p.test_gather_timeout(1)
    assert e.value.code == -1
    p.close()
