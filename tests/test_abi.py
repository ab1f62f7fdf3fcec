"""The C ABI library: builds, loads, exports every entry point of
include/ddfd.h, and rejects bad configurations before touching a GPU."""
import os
import re

import numpy as np

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def header_functions():
    src = open(os.path.join(ROOT, "include", "ddfd.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(ddfd_[a-z0-9_]+)\s*\(", src)))


@pytest.fixture(scope="module")
def lib():
    from paper_2508_07780_gb300 import build
    build.build()
    import paper_2508_07780_gb300 as pkg
    return pkg.load_library()


def test_header_declares_the_binding_symbols():
    import paper_2508_07780_gb300 as pkg
    assert header_functions() == sorted(pkg.ABI_SYMBOLS)


def test_library_exports_every_header_symbol(lib):
    missing = [f for f in header_functions() if not hasattr(lib, f)]
    assert not missing, missing


def _cpu_only():
    try:
        import torch
        return not torch.cuda.is_available()
    except Exception:
        return True


@pytest.mark.parametrize("kw,what", [
    (dict(n=5, fem_n=5, n_steps=3), "n must be"),
    (dict(n=21, fem_n=20, n_steps=3), "fem_n"),
    (dict(n=21, fem_n=11, n_steps=0), "n_steps"),
    (dict(n=21, fem_n=11, n_steps=3, cfl=0.0), "cfl"),
    (dict(n=21, fem_n=11, n_steps=3, det_ij=[[0, 21]]), "detector"),
    (dict(n=21, fem_n=11, n_steps=3, src_dir=[[0.0, 0.3, 0.2]]), "k_z < 0"),
    (dict(n=21, fem_n=11, n_steps=3, z_delta_frac=1.0), "z_delta_frac"),
    (dict(n=21, fem_n=11, n_steps=3, absorbing_faces=64), "absorbing"),
    (dict(n=21, fem_n=11, n_steps=3, precision=7), "precision"),
])
def test_create_rejects_bad_configurations(lib, kw, what):
    from paper_2508_07780_gb300 import DDFDError, Problem
    with pytest.raises(DDFDError) as e:
        Problem(**kw)
    assert e.value.code == -1 and what in str(e.value)


@pytest.mark.skipif(not _cpu_only(), reason="this machine has a GPU")
def test_no_gpu_fails_loudly(lib):
    from paper_2508_07780_gb300 import DDFDError, Problem
    with pytest.raises(DDFDError) as e:
        Problem(n=13, fem_n=9, n_steps=4)
    assert e.value.code == -4


@pytest.mark.parametrize("cfgs,what", [
    ([dict(n=21, fem_n=11, n_steps=3), dict(n=25, fem_n=11, n_steps=3)], "must match member 0"),
    ([dict(n=21, fem_n=11, n_steps=3), dict(n=21, fem_n=11, n_steps=4)], "must match member 0"),
    ([dict(n=21, fem_n=11, n_steps=3, precision="fp32"), dict(n=21, fem_n=11, n_steps=3)],
     "must match member 0"),
    ([dict(n=21, fem_n=11, n_steps=3, src_dir=[[0, 0, -1.0], [0, 0.1, -1.0]])], "one source"),
    ([dict(n=21, fem_n=11, n_steps=30, n_snapshots=3), dict(n=21, fem_n=9, n_steps=30, n_snapshots=5)],
     "segment length"),
    ([dict(n=21, fem_n=11, n_steps=3), dict(n=21, fem_n=30, n_steps=3)], "member 1: fem_n"),
    ([], "1..256"),
])
def test_create_batch_rejects_mismatched_members(lib, cfgs, what):
    from paper_2508_07780_gb300 import Batch, DDFDError
    with pytest.raises(DDFDError) as e:
        Batch(cfgs)
    assert e.value.code == -1 and what in str(e.value), str(e.value)


@pytest.mark.parametrize("mesh_kw,what", [
    (dict(fem_kind=2), "needs mesh_tets"),
    (dict(mesh=(np.array([[0, 7]]), np.zeros((6, 4), int)), n_snapshots=2), "n_snapshots"),
    (dict(mesh=(np.array([[5, 3000]]), np.zeros((6, 4), int))), "parent"),
    (dict(mesh=(np.zeros((0, 2), int), np.full((6, 4), 99999))), "out of range"),
])
def test_create_rejects_bad_refined_meshes(lib, mesh_kw, what):
    from paper_2508_07780_gb300 import DDFDError, Problem
    with pytest.raises(DDFDError) as e:
        Problem(n=13, fem_n=9, n_steps=3, **mesh_kw)
    assert e.value.code == -1 and what in str(e.value), str(e.value)


@pytest.mark.parametrize("kw,what", [
    (dict(grad_variant=2), "bad grad_variant"),
    (dict(grad_variant="literal", n_snapshots=2), "full history"),
    (dict(grad_variant="literal", fem_kind=1), "stencil FEM"),
    (dict(grad_variant="literal", forward_only=1), "adjoint"),
])
def test_create_rejects_unsupported_literal_gradients(lib, kw, what):
    from paper_2508_07780_gb300 import DDFDError, Problem
    with pytest.raises(DDFDError) as e:
        Problem(n=13, fem_n=9, n_steps=3, **kw)
    assert e.value.code == -1 and what in str(e.value), str(e.value)


def test_create_batch_rejects_literal_gradients(lib):
    from paper_2508_07780_gb300 import Batch, DDFDError
    with pytest.raises(DDFDError) as e:
        Batch([dict(n=21, fem_n=11, n_steps=3), dict(n=21, fem_n=11, n_steps=3, grad_variant="literal")])
    assert e.value.code == -1 and "exact gradient only" in str(e.value), str(e.value)


@pytest.mark.parametrize("n_src,n_steps", [(1, 2 ** 31 - 1), (65536, 1), (40, 2000)])
def test_misfit_noalloc_rejects_oversized_traces_before_any_gpu_work(lib, n_src, n_steps):
    """The row count n_src * (n_steps + 1) is formed in 64 bits (n_steps =
    INT32_MAX must not wrap to a negative count that passes the size check);
    anything beyond the fixed scratch is refused with DDFD_E_ARG before the
    call touches a device, so this runs without a GPU.  The pointers are
    placeholders that the call never dereferences."""
    fake = 4096
    st = lib.ddfd_misfit_noalloc(fake, fake, n_src, n_steps, 4, 1e-3, 0.1, fake, None)
    assert st == -1
    assert b"exceeds the fixed scratch" in lib.ddfd_create_error()
