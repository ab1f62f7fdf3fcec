"""Full-size checks on the 201^3 / 2000-step workload, in the launch
configuration the benchmark times, where the oracle cannot run in full:

* vacuum, normal incidence: the FP32 3-D field equals the separately written
  1-D FP64 textbook scheme (laterally invariant, E_x = E_z = 0), a property
  that holds at any size;
* the FP32 path against the FP64 path (which matches the oracle to 1e-12 at
  the sizes the oracle runs) on traces, J, mu and g;
* the FP64 adjoint gradient against central finite differences of J
  (delta = 1e-4) at seeded free nodes, and the FP32 gradient at the same
  nodes.
"""
import numpy as np
import pytest

from helpers import gpu_problem, rel_l2
from synth import workload

pytestmark = pytest.mark.gpu

W = workload("c2_fp32_201")


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2508_07780_gb300 import build
    build.build()


def test_vacuum_201_fp32_equals_1d_scheme():
    from oracle import SourceSpec
    from test_oracle_forward import leapfrog_1d
    n, Nt = W.n, W.n_steps
    p = gpu_problem(W, "fp32")          # vacuum coefficients until set_coeffs
    steps = [Nt // 4, Nt // 2, 3 * Nt // 4, Nt]
    p.set_capture(steps)
    tr = p.forward()
    info = p.get_info()
    ref = leapfrog_1d(n, Nt, W.cfl, SourceSpec(), info.switch_step)
    top = ref[:, -1]
    assert rel_l2(tr[0, :, :, 1], np.repeat(top[:, None], tr.shape[2], axis=1)) <= 1e-4
    assert np.abs(tr[0, :, :, 0]).max() == 0.0 and np.abs(tr[0, :, :, 2]).max() == 0.0
    # Errors are measured against the run's peak field: once the pulse has
    # left through the absorbing faces (t = 3) the remaining field is ~1e-3 of
    # the peak and a relative norm of it would only measure FP32 round-off.
    peak = np.abs(ref).max()
    norms = {s: np.linalg.norm(ref[s]) for s in steps}
    for i, s in enumerate(steps):
        E = p.get_capture(0, i)
        Ey = E[1].reshape(n, n, n)
        want = np.broadcast_to(ref[s][:, None, None], Ey.shape)
        assert np.abs(Ey - want).max() <= 1e-4 * peak, (s, np.abs(Ey - want).max() / peak)
        if norms[s] >= 0.1 * max(norms.values()):
            assert rel_l2(Ey, want) <= 1e-4, (s, rel_l2(Ey, want))
        assert np.abs(Ey - Ey[:, :1, :1]).max() <= 1e-6 * peak
        assert np.abs(E[0]).max() == 0.0 and np.abs(E[2]).max() == 0.0
    p.close()


def _path(prec, eobs, keep):
    p = gpu_problem(W, prec)
    p.set_capture(keep)
    eps, sig = W.model()
    p.set_coeffs(eps, sig)
    tr = p.forward()
    J = p.functional(eobs)
    p.adjoint(eobs)
    ge, gs = p.gradient()
    mu = {s: p.get_capture(1, i) for i, s in enumerate(keep)}
    p.close()
    return tr, J, ge, gs, mu


@pytest.fixture(scope="module")
def eobs_201():
    """Half the layers-only model's FP64 trace: a residual of the size of E."""
    p = gpu_problem(W, "fp64")
    e0, s0 = W.model(inclusions=False)
    p.set_coeffs(e0, s0)
    tr = p.forward()
    p.close()
    return 0.5 * tr


def test_fp32_matches_fp64_at_full_size(eobs_201):
    keep = [0, W.n_steps // 2]
    t64, J64, ge64, gs64, mu64 = _path("fp64", eobs_201, keep)
    t32, J32, ge32, gs32, mu32 = _path("fp32", eobs_201, keep)
    errs = {"trace": rel_l2(t32, t64), "J": abs(J32 - J64) / abs(J64),
            "g_eps": rel_l2(ge32, ge64), "g_sig": rel_l2(gs32, gs64)}
    for s in keep:
        errs[f"mu{s}"] = rel_l2(mu32[s], mu64[s])
    print("FP32 vs FP64 at 201^3:", errs)
    assert errs["trace"] <= 1e-4 and errs["J"] <= 1e-4
    assert all(errs[f"mu{s}"] <= 1e-4 for s in keep)
    assert errs["g_eps"] <= 1e-3 and errs["g_sig"] <= 1e-3


def test_gradient_matches_central_differences_at_full_size(eobs_201):
    eps, sig = W.model()
    rng = np.random.default_rng(2024)
    p64 = gpu_problem(W, "fp64")
    p64.set_coeffs(eps, sig)
    p64.forward()
    p64.functional(eobs_201)
    p64.adjoint(eobs_201)
    ge, gs = p64.gradient()
    p32 = gpu_problem(W, "fp32")
    p32.set_coeffs(eps, sig)
    p32.forward()
    p32.adjoint(eobs_201)
    ge32, gs32 = p32.gradient()
    p32.close()
    delta = 1e-4

    def J_at(e, s):
        p64.set_coeffs(e, s)
        p64.forward(want_trace=False)
        return p64.functional(eobs_201)

    for which, g, g32 in (("eps", ge, ge32), ("sig", gs, gs32)):
        scale = np.abs(g).max()
        # seeded nodes whose gradient is well above J's rounding / delta
        strong = np.nonzero(np.abs(g) > 0.1 * scale)[0]
        for i in rng.choice(strong, size=min(3, strong.size), replace=False):
            base = (eps if which == "eps" else sig)[i]
            vals = []
            for sign in (+1, -1):
                e2, s2 = eps.copy(), sig.copy()
                if which == "eps":
                    e2[i] = base + sign * delta
                else:
                    s2[i] = base + sign * delta
                vals.append(J_at(e2, s2))
            fd = (vals[0] - vals[1]) / (2 * delta)
            assert abs(g[i] - fd) <= 1e-5 * scale, (which, i, g[i], fd)
            assert abs(g32[i] - fd) <= 1e-3 * scale, (which, i, g32[i], fd)
    p64.close()


def test_element_by_element_matches_stencil_at_full_size(eobs_201):
    """The two FEM implementations (block stencil, element gather) on the
    201^3 workload in FP32."""
    out = {}
    for kind in (0, 1):
        p = gpu_problem(W, "fp32", fem_kind=kind)
        eps, sig = W.model()
        p.set_coeffs(eps, sig)
        tr = p.forward()
        J = p.functional(eobs_201)
        p.adjoint(eobs_201)
        ge, gs = p.gradient()
        out[kind] = (tr, J, ge, gs, p.get_timing())
        p.close()
    a, b = out[0], out[1]
    print("EBE vs stencil at 201^3:", rel_l2(b[0], a[0]), abs(b[1] - a[1]) / abs(a[1]),
          rel_l2(b[2], a[2]), rel_l2(b[3], a[3]),
          "step ms fwd %.4f/%.4f adj %.4f/%.4f" % (a[4].forward_loop_ms / a[4].forward_step_kernels,
                                                  b[4].forward_loop_ms / b[4].forward_step_kernels,
                                                  a[4].adjoint_loop_ms / a[4].adjoint_step_kernels,
                                                  b[4].adjoint_loop_ms / b[4].adjoint_step_kernels))
    assert rel_l2(b[0], a[0]) <= 1e-5 and abs(b[1] - a[1]) <= 1e-5 * abs(a[1])
    assert rel_l2(b[2], a[2]) <= 1e-4 and rel_l2(b[3], a[3]) <= 1e-4
