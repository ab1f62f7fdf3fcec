"""The allocation-free misfit entry point (ddfd_misfit_noalloc).

It serves callers that cannot allocate device memory (and so cannot create a
handle): it reduces a caller-owned device trace against caller-owned observed
data into a caller-owned device scalar, using only a fixed scratch array in
the library image.  Checked against ddfd_functional (regularisation off) on
two calls in a row with different observed data, which also shows that the
shared scratch left by the first call does not leak into the second.  This
file is collected last on purpose.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def test_misfit_noalloc_matches_functional_on_two_calls():
    torch = pytest.importorskip("torch")
    from paper_2508_07780_gb300 import build
    build.build()
    from paper_2508_07780_gb300 import DDFDError, Problem, misfit_noalloc
    from synth import workload

    w = workload("small", n_src=2, dir_seed=5)
    eps, sig = w.model()
    p = Problem(n=w.n, fem_n=w.fem_n, n_steps=w.n_steps, src_dir=w.directions(),
                det_ij=w.detectors(), z_delta_frac=0.2)
    p.set_coeffs(eps, sig)
    trace = p.forward()
    info = p.get_info()
    dev = torch.device("cuda")
    stream = torch.cuda.current_stream(dev)
    tr_d = torch.tensor(trace, dtype=torch.float64, device=dev)
    J_d = torch.full((1,), -1.0, dtype=torch.float64, device=dev)
    rng = np.random.default_rng(0)
    for call in range(2):
        eobs = (0.4 + 0.3 * call) * trace + 1e-3 * rng.standard_normal(trace.shape)
        J_ref = p.functional(eobs)
        eo_d = torch.tensor(eobs, dtype=torch.float64, device=dev)
        misfit_noalloc(tr_d, eo_d, info.n_src, info.n_steps, info.n_det, info.tau, 0.2, J_d,
                       stream=stream.cuda_stream)
        stream.synchronize()
        assert abs(J_d.item() - J_ref) <= 1e-12 * abs(J_ref), (call, J_d.item(), J_ref)
    p.close()
    # more rows than the fixed scratch holds: rejected before any launch
    with pytest.raises(DDFDError) as e:
        misfit_noalloc(tr_d, tr_d, 40, 2000, info.n_det, info.tau, 0.2, J_d)
    assert e.value.code == -1 and "scratch" in str(e.value)
