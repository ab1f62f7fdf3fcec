"""Batched heterogeneous problems (ddfd_create_batch): members with their own
FEM cube size, model, incidence direction, detectors, boundary set and
regularisation, stepped together in one launch per time step.

Each member must match the oracle within the parity bars, and be bitwise
equal to the same problem run alone (the batched kernel does the same
arithmetic per node); the autotuned tile depth changes no bit either."""
import numpy as np
import pytest

from helpers import rel_l2, run_oracle
from synth import workload

pytestmark = pytest.mark.gpu

TOL = {"fp64": dict(E=1e-12, J=1e-12, g=1e-12), "fp32": dict(E=1e-4, J=1e-4, g=1e-3)}


@pytest.fixture(scope="session", autouse=True)
def _built():
    from paper_2508_07780_gb300 import build
    build.build()


def members(n=25, n_steps=120):
    """(workload, extra Problem kwargs) of five different problems on one grid."""
    out = []
    specs = [  # fem_n, seed, dir_seed, det_per_side, gammas, absorbing sides
        (13, 31, None, 4, (0.0, 0.0), 0),
        (9, 32, 5, 3, (0.1, 0.0), 0),
        (17, 33, 6, 5, (0.0, 0.3), 4 | 32),
        (21, 34, 7, 6, (0.0, 0.0), 0),
        (13, 35, 8, 2, (0.2, 0.2), 8 | 16),
    ]
    for fem_n, seed, ds, d, (ge, gs), sides in specs:
        w = workload("small", n=n, fem_n=fem_n, n_steps=n_steps, seed=seed, dir_seed=ds,
                     det_per_side=d, gamma_eps=ge, gamma_sig=gs)
        out.append((w, sides))
    return out


def problem_kwargs(w, precision, sides, **kw):
    return dict(n=w.n, fem_n=w.fem_n, n_steps=w.n_steps, cfl=w.cfl, precision=precision,
                src_dir=w.directions(), det_ij=w.detectors(), z_delta_frac=w.z_delta_frac,
                gamma_eps=w.gamma_eps, gamma_sig=w.gamma_sig, absorbing_faces=1 | 2 | sides, **kw)


_oracle = {}


def oracle_of(w, sides):
    key = (repr(w), sides)
    if key not in _oracle:
        _oracle[key] = run_oracle(w, absorbing=1 | 2 | sides)
    return _oracle[key]


def run_alone(w, precision, sides, eobs, **kw):
    from paper_2508_07780_gb300 import Problem
    p = Problem(**problem_kwargs(w, precision, sides, **kw))
    eps, sig = w.model()
    p.set_coeffs(eps, sig)
    tr = p.forward()
    J = p.functional(eobs)
    p.adjoint(eobs)
    ge, gs = p.gradient()
    p.close()
    return tr, J, ge, gs


def run_batch(b, ms, eobs):
    for (w, _), m in zip(ms, b.members):
        eps, sig = w.model()
        m.set_coeffs(eps, sig)
    traces = b.forward()
    b.adjoint(eobs)
    out = []
    for m, tr, e in zip(b.members, traces, eobs):
        J = m.functional(e)
        ge, gs = m.gradient()
        out.append((tr, J, ge, gs))
    return out


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_batch_matches_oracle_and_single_runs(prec):
    from paper_2508_07780_gb300 import Batch
    ms = members()
    refs = [oracle_of(w, sides) for w, sides in ms]
    eobs = [r["eobs"] for r in refs]
    b = Batch([problem_kwargs(w, prec, sides) for w, sides in ms])
    got = run_batch(b, ms, eobs)
    info = b.get_info()
    assert info.count == len(ms)
    assert info.forward_step_kernels == ms[0][0].n_steps      # one launch per step
    assert info.adjoint_step_kernels == ms[0][0].n_steps
    b.close()
    tol = TOL[prec]
    for (w, sides), ref, e, (tr, J, ge, gs) in zip(ms, refs, eobs, got):
        assert rel_l2(tr, ref["trace"]) <= tol["E"], w
        assert abs(J - ref["J"]) <= tol["J"] * abs(ref["J"]), w
        assert rel_l2(ge, ref["g_eps"]) <= tol["g"], w
        assert rel_l2(gs, ref["g_sig"]) <= tol["g"], w
        tr1, J1, ge1, gs1 = run_alone(w, prec, sides, e)
        assert np.array_equal(tr, tr1) and J == J1
        assert np.array_equal(ge, ge1) and np.array_equal(gs, gs1)


def test_checkpointing_and_history_members_mixed():
    """Members that checkpoint (replayed in batched launches of their own)
    next to members that keep the history: bitwise the full-history runs."""
    from paper_2508_07780_gb300 import Batch
    ms = members(n_steps=90)
    eobs = [0.01 * np.random.default_rng(i).standard_normal((1, 91, w.detectors().shape[0], 3))
            for i, (w, _) in enumerate(ms)]
    snaps = [0, 7, 0, 7, 7]                   # segment length 13 for the checkpointing ones
    b = Batch([problem_kwargs(w, "fp32", sides, n_snapshots=k) for (w, sides), k in zip(ms, snaps)])
    got = run_batch(b, ms, eobs)
    info = b.get_info()
    assert info.adjoint_step_kernels == 2 * 90  # adjoint launches + the replay launches
    b.close()
    for (w, sides), e, (tr, J, ge, gs) in zip(ms, eobs, got):
        tr1, J1, ge1, gs1 = run_alone(w, "fp32", sides, e)
        assert np.array_equal(tr, tr1) and J == J1
        assert np.array_equal(ge, ge1) and np.array_equal(gs, gs1)


def test_more_members_than_one_launch_holds():
    """18 members: two launches per step (16 + 2)."""
    from paper_2508_07780_gb300 import Batch
    base = workload("tiny", n_steps=30)
    ms = [(base.with_(seed=100 + i, fem_n=(9, 11)[i % 2], dir_seed=200 + i), 0) for i in range(18)]
    eobs = [0.01 * np.random.default_rng(i).standard_normal((1, 31, w.detectors().shape[0], 3))
            for i, (w, _) in enumerate(ms)]
    b = Batch([problem_kwargs(w, "fp64", s) for w, s in ms])
    got = run_batch(b, ms, eobs)
    assert b.get_info().forward_step_kernels == 2 * 30
    b.close()
    for (w, s), e, (tr, J, ge, gs) in zip(ms, eobs, got):
        tr1, J1, ge1, gs1 = run_alone(w, "fp64", s, e)
        assert np.array_equal(tr, tr1) and J == J1
        assert np.array_equal(ge, ge1) and np.array_equal(gs, gs1)


@pytest.mark.parametrize("prec", ["fp32", "fp64"])
def test_autotune_picks_a_candidate_and_changes_no_bit(prec):
    from paper_2508_07780_gb300 import Batch
    ms = members(n=41, n_steps=40)
    eobs = [0.01 * np.random.default_rng(i).standard_normal((1, 41, w.detectors().shape[0], 3))
            for i, (w, _) in enumerate(ms)]
    b = Batch([problem_kwargs(w, prec, s, tile_kz=8) for w, s in ms])
    before = run_batch(b, ms, eobs)
    kz = b.autotune(steps=6)
    assert kz in (4, 6, 8, 12, 16, 24, 32) and b.get_info().tile_kz == kz
    with pytest.raises(Exception):          # the trial steps invalidated the state
        b.members[0].gradient()
    after = run_batch(b, ms, eobs)
    b.close()
    for x, y in zip(before, after):
        assert np.array_equal(x[0], y[0]) and x[1] == y[1]
        assert np.array_equal(x[2], y[2]) and np.array_equal(x[3], y[3])


def test_single_problem_autotune_and_member_alone():
    from paper_2508_07780_gb300 import Batch, Problem
    w, s = members(n=41, n_steps=40)[2]
    e = 0.01 * np.random.default_rng(3).standard_normal((1, 41, w.detectors().shape[0], 3))
    p = Problem(**problem_kwargs(w, "fp32", s))
    eps, sig = w.model()
    p.set_coeffs(eps, sig)
    t0 = p.forward()
    kz = p.autotune(steps=5)
    assert kz in (4, 6, 8, 12, 16, 24, 32)
    t1 = p.forward()
    assert np.array_equal(t0, t1)
    p.close()
    # a batch member run alone through the single-problem entry points
    b = Batch([problem_kwargs(w, "fp32", s), problem_kwargs(w.with_(seed=77), "fp32", s)])
    m = b.members[0]
    m.set_coeffs(eps, sig)
    assert np.array_equal(m.forward(), t0)
    J = m.functional(e)
    m.adjoint(e)
    g = m.gradient()
    b.members[1].set_coeffs(*w.with_(seed=77).model())
    tb = b.forward()
    b.adjoint([e, e])
    assert np.array_equal(tb[0], t0) and m.functional(e) == J
    gb = m.gradient()
    assert np.array_equal(g[0], gb[0]) and np.array_equal(g[1], gb[1])
    b.close()


def test_batch_state_errors():
    from paper_2508_07780_gb300 import Batch, DDFDError
    w = workload("tiny")
    b = Batch([problem_kwargs(w, "fp64", 0), problem_kwargs(w.with_(fem_n=11), "fp64", 0)])
    with pytest.raises(DDFDError) as e:
        b.adjoint([np.zeros((1, w.n_steps + 1, 9, 3))] * 2)
    assert e.value.code == -3
    b.close()


@pytest.mark.parametrize("batched", [False, True])
def test_lean_kernel_matches_the_full_kernel_bitwise(batched):
    """FP32 steps split into the full kernel (FEM-cube and free tiles) and the
    lean kernel (finite-difference tiles).  A tile depth beyond the dispatch
    item packing (65 > 64 planes) runs every tile on the full kernel over the
    3-D grid; the finite-difference nodes must come out bitwise the same."""
    from paper_2508_07780_gb300 import Batch, Problem
    ms = [(w.with_(n=65, n_steps=40, fem_n=f), s) for (w, s), f in zip(members(n=65, n_steps=40)[:3], (21, 33, 15))]
    eobs = [0.01 * np.random.default_rng(i).standard_normal((1, 41, w.detectors().shape[0], 3))
            for i, (w, _) in enumerate(ms)]
    out = {}
    for kz in (16, 65):
        if batched:
            b = Batch([problem_kwargs(w, "fp32", s, tile_kz=kz) for w, s in ms])
            out[kz] = run_batch(b, ms, eobs)
            b.close()
        else:
            out[kz] = [run_alone(w, "fp32", s, e, tile_kz=kz) for (w, s), e in zip(ms, eobs)]
    for x, y in zip(out[16], out[65]):
        assert np.array_equal(x[0], y[0]) and x[1] == y[1]
        assert np.array_equal(x[2], y[2]) and np.array_equal(x[3], y[3])


@pytest.mark.parametrize("batched", [False, True])
def test_odd_tile_depths_change_no_bit(batched):
    """Dispatch items of odd depths (5 planes on the full kernel, 3 on the lean
    one) cut the FEM columns' z ranges and the other columns at other planes;
    every node must still come out bitwise as with the default depths."""
    from paper_2508_07780_gb300 import Batch
    ms = [(w.with_(n_steps=30), s) for w, s in members(n=33, n_steps=30)[:3]]
    eobs = [0.01 * np.random.default_rng(7 + i).standard_normal((1, 31, w.detectors().shape[0], 3))
            for i, (w, _) in enumerate(ms)]
    out = {}
    for kz in ((0, 0), (5, 3)):
        kw = dict(tile_kz=kz[0], tile_kz_lean=kz[1])
        if batched:
            b = Batch([problem_kwargs(w, "fp32", s, **kw) for w, s in ms])
            out[kz] = run_batch(b, ms, eobs)
            b.close()
        else:
            out[kz] = [run_alone(w, "fp32", s, e, **kw) for (w, s), e in zip(ms, eobs)]
    for x, y in zip(out[(0, 0)], out[(5, 3)]):
        assert np.array_equal(x[0], y[0]) and x[1] == y[1]
        assert np.array_equal(x[2], y[2]) and np.array_equal(x[3], y[3])
