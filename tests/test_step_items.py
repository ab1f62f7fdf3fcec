"""Dispatch order of the step launches (host logic, no GPU).

One step launch must update every grid node of every problem exactly once,
and every node strictly inside the FEM cube or in the free box must fall on
the full FP32 kernel (the lean kernel has neither the block stencil nor the
gradient).  The item list comes from the library itself
(ddfd_test_step_items); this test rebuilds the node coverage from the item
fields alone: tile x of 32 nodes, tile y of 16 rows (FP32) or 8 (FP64), and
on FP32 grids of n = 32 m + 1 nodes the last x tile also owns column n - 1.
"""
import numpy as np
import pytest

from paper_2508_07780_gb300.binding import DDFDError, step_items


def unpack(it):
    it = it.astype(np.int64)
    return (it & 31, (it >> 5) & 127, (it >> 12) & 1023, ((it >> 22) & 63) + 1, (it >> 28) & 15)


def cube_box(n, fem):
    a = (n - fem) // 2
    return (a, a + fem - 1, a + 2, fem - 4)


def check(n, prec, boxes, kz, kz_lean):
    items, n_full = step_items(n, prec, boxes, kz, kz_lean)
    assert 0 <= n_full <= len(items)
    tx, ty, z0, nz, pr = unpack(items)
    rows = 16 if prec == "fp32" else 8
    gx = n // 32 if (prec == "fp32" and n % 32 == 1) else (n + 31) // 32
    depth = np.where(np.arange(len(items)) < n_full, kz, kz_lean)
    assert (nz <= depth).all() and (z0 < n).all() and (pr < len(boxes)).all()
    for q, (a, b, f0, nf) in enumerate(boxes):
        cov = np.zeros((n, n, n), np.int32)      # [z, y, x]
        full = np.zeros((n, n, n), bool)
        for m in np.nonzero(pr == q)[0]:
            tail = prec == "fp32" and n % 32 == 1 and tx[m] == gx - 1  # owns column n - 1 too
            x1 = n if tail else min(32 * tx[m] + 32, n)
            sl = (slice(z0[m], min(z0[m] + nz[m], n)), slice(rows * ty[m], min(rows * ty[m] + rows, n)),
                  slice(32 * tx[m], x1))
            cov[sl] += 1
            if m < n_full:
                full[sl] = True
        assert (cov == 1).all(), (n, prec, q, kz, kz_lean, np.argwhere(cov != 1)[:5])
        idx = np.arange(n)
        fem1 = (idx > a) & (idx < b)
        fre1 = (idx >= f0) & (idx < f0 + nf)
        need = (fem1[:, None, None] & fem1[None, :, None] & fem1[None, None, :]) | \
               (fre1[:, None, None] & fre1[None, :, None] & fre1[None, None, :])
        if prec == "fp32":
            assert full[need].all(), (n, q, np.argwhere(need & ~full)[:5])
        else:
            assert n_full == len(items)
    return items, n_full


@pytest.mark.parametrize("prec", ["fp32", "fp64"])
@pytest.mark.parametrize("n,fem", [(9, 5), (13, 7), (33, 11), (41, 21), (65, 31), (97, 45), (129, 61)])
def test_every_node_once_and_fem_nodes_on_the_full_kernel(n, fem, prec):
    for kz, kz_lean in ((4, 16), (8, 8), (16, 24), (32, 4)):
        check(n, prec, [cube_box(n, fem)], kz, kz_lean)


def test_heterogeneous_batch_group():
    n = 65
    boxes = [cube_box(n, f) for f in (15, 25, 35, 45)] * 4  # a full group of 16 problems
    items, n_full = check(n, "fp32", boxes, 24, 16)
    # the FEM z range of each FEM column is on the full kernel, the rest lean
    assert 0 < n_full < len(items)


def test_lean_items_avoid_fem_planes_of_fem_columns():
    # a 161^3 grid with a 121^3 cube: the FEM columns' planes below and above
    # the cube go to the lean kernel, so the full kernel's planes per column
    # are the cube's interior planes only
    n, fem = 161, 121
    a, b, f0, nf = cube_box(n, fem)
    items, n_full = check(n, "fp32", [(a, b, f0, nf)], 32, 16)
    tx, ty, z0, nz, pr = unpack(items[:n_full])
    assert z0.min() == a + 1 and (z0 + nz).max() == b


def test_argument_checks():
    with pytest.raises(DDFDError):
        step_items(5, "fp32", [(1, 3, 2, 0)], 8, 8)        # n < 7
    with pytest.raises(DDFDError):
        step_items(41, "fp32", [(10, 50, 12, 4)], 8, 8)    # cube outside the grid
    with pytest.raises(DDFDError):
        step_items(41, "fp32", [cube_box(41, 11)], 65, 8)  # depth beyond the item packing
