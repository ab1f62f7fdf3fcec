"""fem_kind = DDFD_FEM_MESH: the FEM cube on an explicit, locally refined
mesh (conforming bisection where eq. meshref marks it, synth/mesh.py),
against the oracle on the same mesh and coefficients: traces, fields at the
grid nodes, J and the gradient at every free node, the new nodes included.
Bars: FP64 1e-12, FP32 1e-4 (traces, fields, J) and 1e-3 (g)."""
import numpy as np
import pytest

from helpers import rel_l2
from synth import detector_grid, workload
from synth.mesh import extend_to_new_nodes, kuhn_cube, refined_fem_mesh

pytestmark = pytest.mark.gpu

TOL = {"fp64": dict(E=1e-12, J=1e-12, g=1e-12), "fp32": dict(E=1e-4, J=1e-4, g=1e-3)}
CFL = 0.2


@pytest.fixture(scope="session", autouse=True)
def _built():
    from paper_2508_07780_gb300 import build
    build.build()


def case(name):
    if name == "n13":
        w = workload("tiny", n=13, fem_n=9, n_steps=80, seed=21, det_per_side=3)
        beta = 0.5
    else:
        w = workload("small", n=25, fem_n=17, n_steps=100, seed=12, dir_seed=5, det_per_side=4)
        beta = 0.8
    eps, sig = w.model()
    par, tets = refined_fem_mesh(w.n, w.fem_n, eps, sig, beta_eps=beta, beta_sig=0.0)
    e, s = extend_to_new_nodes(w.n, w.fem_n, par, eps, sig)
    e0, s0 = w.model(inclusions=False)
    el, sl = extend_to_new_nodes(w.n, w.fem_n, par, e0, s0)
    return w, (par, tets), (e, s), (el, sl)


_oracle = {}


def oracle_of(name):
    if name in _oracle:
        return _oracle[name]
    from oracle import OracleProblem, SourceSpec
    w, mesh, (e, s), (el, sl) = case(name)
    srcs = [SourceSpec(direction=tuple(d)) for d in w.directions()]
    mk = lambda ee, ss: OracleProblem(w.n, w.fem_n, w.n_steps, CFL, ee, ss, w.detectors(), srcs,
                                      z_delta_frac=w.z_delta_frac, mesh=mesh)
    P0 = mk(el, sl)
    eobs = [0.5 * P0.forward(k).trace for k in range(len(srcs))]
    P = mk(e, s)
    keep = sorted({w.n_steps // 2, w.n_steps})
    fw = [P.forward(k, keep_fields=keep) for k in range(len(srcs))]
    J = P.functional([f.trace for f in fw], eobs)
    ad = [P.adjoint(k, fw[k].trace, eobs[k]) for k in range(len(srcs))]
    ge, gs = P.gradient(fw, ad)
    _oracle[name] = dict(eobs=np.stack(eobs), trace=np.stack([f.trace for f in fw]), J=J, g_eps=ge, g_sig=gs,
                         E=fw[0].fields, keep=keep, n_grid=w.n ** 3)
    return _oracle[name]


def gpu_run(name, prec, mesh=None):
    from paper_2508_07780_gb300 import Problem
    w, m, (e, s), _ = case(name)
    ref = oracle_of(name)
    p = Problem(n=w.n, fem_n=w.fem_n, n_steps=w.n_steps, cfl=CFL, precision=prec, src_dir=w.directions(),
                det_ij=w.detectors(), z_delta_frac=w.z_delta_frac, mesh=m if mesh is None else mesh)
    p.set_capture(ref["keep"])
    assert p.n_free == e.size
    p.set_coeffs(e, s)
    tr = p.forward()
    J = p.functional(ref["eobs"])
    p.adjoint(ref["eobs"])
    ge, gs = p.gradient()
    E = {k: p.get_capture(0, i) for i, k in enumerate(ref["keep"])}
    p.close()
    return dict(trace=tr, J=J, g_eps=ge, g_sig=gs, E=E)


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
@pytest.mark.parametrize("name", ["n13", "n25_oblique"])
def test_refined_mesh_matches_the_oracle(name, prec):
    ref = oracle_of(name)
    out = gpu_run(name, prec)
    tol = TOL[prec]
    assert rel_l2(out["trace"], ref["trace"]) <= tol["E"]
    for k in ref["keep"]:
        assert rel_l2(out["E"][k], ref["E"][k][:, :ref["n_grid"]]) <= tol["E"], k
    assert abs(out["J"] - ref["J"]) <= tol["J"] * abs(ref["J"])
    assert rel_l2(out["g_eps"], ref["g_eps"]) <= tol["g"]
    assert rel_l2(out["g_sig"], ref["g_sig"]) <= tol["g"]
    # the new nodes' own gradient entries, separately
    w, (par, _), _, _ = case(name)
    nfg = (w.fem_n - 4) ** 3
    assert rel_l2(out["g_eps"][nfg:], ref["g_eps"][nfg:]) <= 10 * tol["g"]


def test_unrefined_explicit_mesh_equals_the_element_path():
    """The Kuhn split given as an explicit mesh (no new nodes) is the
    element-by-element path of fem_kind = DDFD_FEM_EBE."""
    from paper_2508_07780_gb300 import Problem
    w = workload("small", n=25, fem_n=13, n_steps=60, seed=12)
    eps, sig = w.model()
    eobs = 0.01 * np.random.default_rng(0).standard_normal((1, 61, w.detectors().shape[0], 3))
    res = []
    for kw in (dict(fem_kind=1), dict(mesh=(np.zeros((0, 2), np.int32), kuhn_cube(w.n, w.fem_n)))):
        p = Problem(n=w.n, fem_n=w.fem_n, n_steps=w.n_steps, cfl=w.cfl, precision="fp64",
                    det_ij=w.detectors(), z_delta_frac=w.z_delta_frac, **kw)
        p.set_coeffs(eps, sig)
        tr = p.forward()
        J = p.functional(eobs)
        p.adjoint(eobs)
        res.append((tr, J) + p.gradient())
        p.close()
    (t0, J0, ge0, gs0), (t1, J1, ge1, gs1) = res
    assert rel_l2(t1, t0) <= 1e-13 and abs(J1 - J0) <= 1e-13 * abs(J0)
    assert rel_l2(ge1, ge0) <= 1e-12 and rel_l2(gs1, gs0) <= 1e-12


def test_batch_of_refined_members_equals_single_runs():
    """Batch members on a refined mesh (their gather and new-node launches
    around the batched step) give bitwise the single-problem results."""
    from paper_2508_07780_gb300 import Batch, Problem
    from synth import shard_directions
    w, m, (e, s), _ = case("n13")
    dirs = shard_directions(2)
    cfg = dict(n=w.n, fem_n=w.fem_n, n_steps=w.n_steps, cfl=CFL, precision="fp32", det_ij=w.detectors(),
               z_delta_frac=w.z_delta_frac, mesh=m)
    eobs = [0.01 * np.random.default_rng(i).standard_normal((1, w.n_steps + 1, w.detectors().shape[0], 3))
            for i in range(2)]
    b = Batch([dict(cfg, src_dir=d[None, :]) for d in dirs])
    for mem in b.members:
        mem.set_coeffs(e, s)
    traces = b.forward()
    b.adjoint(eobs)
    got = [(tr, mem.functional(eo)) + mem.gradient() for tr, mem, eo in zip(traces, b.members, eobs)]
    b.close()
    for d, eo, (tr, J, ge, gs) in zip(dirs, eobs, got):
        p = Problem(src_dir=d[None, :], **cfg)
        p.set_coeffs(e, s)
        t1 = p.forward()
        J1 = p.functional(eo)
        p.adjoint(eo)
        ge1, gs1 = p.gradient()
        p.close()
        assert np.array_equal(tr, t1) and J == J1
        assert np.array_equal(ge, ge1) and np.array_equal(gs, gs1)


def test_cg_on_refined_mesh_matches_the_oracle():
    """ddfd_cg_run with per-node lumped masses in its inner products."""
    from oracle import OracleProblem, SourceSpec
    from oracle.cg import CGParams, cga, problem_evaluator
    from paper_2508_07780_gb300 import Batch
    from synth import shard_directions
    w, mesh, (e, s), (el, sl) = case("n13")
    dirs = shard_directions(2)
    srcs = [SourceSpec(direction=tuple(d)) for d in dirs]
    mk = lambda ee, ss: OracleProblem(w.n, w.fem_n, w.n_steps, CFL, ee, ss, w.detectors(), srcs,
                                      z_delta_frac=w.z_delta_frac, mesh=mesh)
    P0 = mk(e, s)
    eobs = [P0.forward(k).trace for k in range(2)]
    P = mk(el, sl)
    mass = P.op.m[P.g.free_nodes]
    ev = problem_evaluator(P)(eobs)
    J0, ge0, gs0 = ev(el, sl)
    g0 = np.sqrt(np.sum(mass * (ge0 / mass) ** 2))
    prm = dict(gamma_eps0=1e-3, gamma_sig0=1e-3, alpha_eps0=0.05 / g0, alpha_sig0=0.01 / g0, p=0.5,
               eps_max=30.0, sig_max=5.0)
    eo, so, lo = cga(ev, el, sl, mass, CGParams(max_iter=3, **prm))
    b = Batch([dict(n=w.n, fem_n=w.fem_n, n_steps=w.n_steps, cfl=CFL, precision="fp64", det_ij=w.detectors(),
                    z_delta_frac=w.z_delta_frac, eps_max=30.0, sig_max=5.0, mesh=mesh, src_dir=d[None, :])
               for d in dirs])
    eps, sig, log = b.cg_run(eobs, el, sl, max_iter=3, **prm)
    b.close()
    for g, r in zip(log, lo):
        for k in ("J", "J_data", "gnorm_eps", "gnorm_sig", "alpha_eps", "beta_eps", "step_eps", "step_sig"):
            assert g[k] == pytest.approx(r[k], rel=1e-8, abs=1e-30), (g["iter"], k)
    assert rel_l2(eps - el, eo - el) <= 1e-8 and rel_l2(sig - sl, so - sl) <= 1e-8


def test_time_gather_reports_times_and_bytes_and_keeps_the_state():
    """ddfd_time_gather on an element-gather handle: positive times and the
    algorithmic bytes of the launches; the forward state survives it (the
    adjoint afterwards gives the gradient of a run without it); a stencil
    handle is refused."""
    from paper_2508_07780_gb300 import DDFDError, Problem
    w = workload("small", n=25, fem_n=13, n_steps=40, seed=12)
    eps, sig = w.model()
    kw = dict(n=w.n, fem_n=w.fem_n, n_steps=w.n_steps, cfl=w.cfl, precision="fp32", det_ij=w.detectors(),
              z_delta_frac=w.z_delta_frac, fem_kind=1)
    res = []
    for timed in (False, True):
        p = Problem(**kw)
        p.set_coeffs(eps, sig)
        tr = p.forward()
        if timed:
            fms, ams, fb, ab = p.time_gather(5)
            assert fms > 0 and ams > 0
            # 10,164 of the 10,368 Kuhn tets of the 12^3 cubes touch a FEM row (the
            # others have every vertex on the cube's faces): ids and gradients at least
            assert fb >= 10164 * (16 + 48) and ab > fb
        p.adjoint(0.5 * tr)
        res.append(p.gradient())
        p.close()
    assert np.array_equal(res[0][0], res[1][0]) and np.array_equal(res[0][1], res[1][1])
    q = Problem(n=13, fem_n=9, n_steps=3)
    with pytest.raises(DDFDError) as e:
        q.time_gather(2)
    assert e.value.code == -1
    q.close()
