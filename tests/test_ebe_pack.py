"""CPU checks of the element-by-element block packer (csrc/ddfd_ebe_pack.cpp),
compiled here with the host compiler through tests/ebe_pack_shim.cpp.

The gather kernel trusts the packed layout for every shared-memory index, so
these tests check it on the host before any GPU run:
* every FEM row lands in exactly one block, each block within the row count
  and the shared-memory budget, blobs 16-byte aligned;
* every local node id and every incidence's local tet lies inside its block;
* the kernel's arithmetic emulated on the packed blocks (nodes gathered once
  per block, one divergence per tet, rows summed over their incidences)
  reproduces a direct element loop over the mesh, for a uniform Kuhn cube and
  a locally refined one, with 4- and 8-byte gradients.
"""
import ctypes
import os
import shutil
import subprocess

import numpy as np
import pytest

from synth import box_bounds
from synth.mesh import kuhn_cube, refined_fem_mesh

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_2508_07780_gb300", "csrc")


def _cuda_include():
    for d in (os.environ.get("CUDA_HOME", ""), "/usr/local/cuda"):
        if d and os.path.exists(os.path.join(d, "include", "cuda_runtime.h")):
            return os.path.join(d, "include")
    return None


@pytest.fixture(scope="module")
def lib(tmp_path_factory):
    cxx = shutil.which("g++")
    inc = _cuda_include()
    if not cxx or not inc:
        pytest.skip("host compiler or CUDA headers missing")
    out = str(tmp_path_factory.mktemp("pack") / "libpack.so")
    subprocess.run([cxx, "-O2", "-std=c++17", "-fPIC", "-shared", "-I", os.path.join(ROOT, "include"), "-I", CSRC,
                    "-I", inc, os.path.join(ROOT, "tests", "ebe_pack_shim.cpp"),
                    os.path.join(CSRC, "ddfd_ebe_pack.cpp"), os.path.join(CSRC, "ddfd_kuhn.cpp"), "-o", out],
                   check=True)
    L = ctypes.CDLL(out)
    L.ebe_pack_smem.restype = ctypes.c_longlong
    L.ebe_pack_smem.argtypes = [ctypes.c_longlong, ctypes.c_longlong, ctypes.c_longlong, ctypes.c_int]
    v = (ctypes.c_int * 3)()
    L.ebe_pack_consts(v)
    L.RB, L.BUDGET, L.PAD = v[0], v[1], v[2]
    return L


def mesh_arrays(n, fem_n, parents, tets, px):
    """What the library's mesh builder hands the packer: padded node offsets,
    sqrt|K| times the P1 gradients, each FEM row's incidences and position."""
    a, b, _, _ = box_bounds(n, fem_n)
    n3, cs = n ** 3, px * n * n
    n_new = parents.shape[0]
    gx = np.stack([np.arange(n3) % n, (np.arange(n3) // n) % n, np.arange(n3) // (n * n)], 1).astype(float)
    X = np.zeros((n_new, 3))
    for e, (p, q) in enumerate(parents):       # parents precede their children
        xp = gx[p] if p < n3 else X[p - n3]
        xq = gx[q] if q < n3 else X[q - n3]
        X[e] = 0.5 * (xp + xq)
    coords = lambda v: gx[v] if v < n3 else X[v - n3]
    fm = b - a - 1
    grid_rows = fm ** 3

    def rowof(v):
        if v >= n3:
            return grid_rows + (v - n3)
        i, j, k = v % n, (v // n) % n, v // (n * n)
        if not (a < i < b and a < j < b and a < k < b):
            return -1
        return (i - a - 1) + fm * ((j - a - 1) + fm * (k - a - 1))

    def off(v):
        if v >= n3:
            return cs + (v - n3)
        return int(v % n + px * ((v // n) % n + n * (v // (n * n))))

    T = tets.shape[0]
    rows = grid_rows + n_new
    tnode = np.zeros((T, 4), np.int32)
    tgrad = np.zeros((T, 12))
    inc = [[] for _ in range(rows)]
    for t in range(T):
        A = np.ones((4, 4))
        for q in range(4):
            A[q, 1:] = coords(tets[t, q])
        C = np.linalg.inv(A)
        vol = abs(np.linalg.det(A[1:, 1:] - A[0, 1:])) / 6.0
        for q in range(4):
            tnode[t, q] = off(tets[t, q])
            tgrad[t, 3 * q:3 * q + 3] = np.sqrt(vol) * C[1:, q]
            r = rowof(tets[t, q])
            if r >= 0:
                inc[r].append((t, q))
    rptr = np.zeros(rows + 1, np.int32)
    rptr[1:] = np.cumsum([len(x) for x in inc])
    itet = np.array([t for x in inc for t, _ in x], np.int32)
    iloc = np.array([q for x in inc for _, q in x], np.int32)
    rpos = np.zeros((rows, 3))
    for k in range(a + 1, b):
        for j in range(a + 1, b):
            for i in range(a + 1, b):
                rpos[rowof(i + n * (j + n * k))] = (i, j, k)
    rpos[grid_rows:] = X
    return dict(tnode=tnode, tgrad=tgrad, rptr=rptr, itet=itet, iloc=iloc, rpos=rpos, rows=rows, cs=cs,
                n_new=n_new, grid_rows=grid_rows, tet_ids=np.ascontiguousarray(tets, dtype=np.int32), n=n, px=px)


def pack(lib, m, esz, use=None):
    p = lambda x: x.ctypes.data_as(ctypes.c_void_p)
    sizes = np.zeros(5, np.int64)
    err = ctypes.create_string_buffer(256)
    st = lib.ebe_pack_run(ctypes.c_longlong(m["rows"]), ctypes.c_longlong(m["tnode"].shape[0]), p(m["tnode"]),
                          p(m["tgrad"]), p(m["rptr"]), p(m["itet"]), p(m["iloc"]), p(m["rpos"]), esz, p(sizes),
                          err, 256, None if use is None else p(use))
    assert st == 0, err.value
    nb, nblob, nn, nr, smem = (int(v) for v in sizes)
    blocks = np.zeros((nb, 8), np.int64)
    blob = np.zeros(nblob, np.uint8)
    nodes = np.zeros(nn, np.int32)
    rows = np.zeros(nr, np.int32)
    lib.ebe_pack_fetch(p(blocks), p(blob), p(nodes), p(rows))
    return blocks, blob, nodes, rows, smem


def direct_rows(m, field, s):
    """(K E)_a summed straight over the tets (forward, no mass scaling)."""
    y = np.zeros((m["rows"], 3))
    for r in range(m["rows"]):
        for e in range(m["rptr"][r], m["rptr"][r + 1]):
            t, a = m["itet"][e], m["iloc"][e]
            g = m["tgrad"][t].reshape(4, 3)
            E = np.stack([field(o) for o in m["tnode"][t]])
            sv = np.array([s(o) for o in m["tnode"][t]])
            div = np.sum(sv * np.sum(g * E, 1))
            y[r] += (g[a] @ g.T) @ E + g[a] * div
    return y


def emulate(lib, m, esz, field, s, use=None):
    blocks, blob, nodes, rows, smem = pack(lib, m, esz, use)
    ft = np.float32 if esz == 4 else np.float64
    RB, PAD = lib.RB, lib.PAD
    assert smem <= lib.BUDGET
    seen = np.zeros(m["rows"], np.int64)
    y = np.zeros((m["rows"], 3))
    for blob_off, nbytes, nt, nn, maxinc, nrows, node0, row0 in blocks:
        assert blob_off % 16 == 0 and nbytes % 16 == 0 and blob_off + nbytes <= blob.size
        assert nt % 2 == 0 and 0 < nrows <= RB and nn > 0
        assert lib.ebe_pack_smem(int(nt), int(nn), int(maxinc), esz) <= smem
        raw = blob[blob_off:blob_off + nbytes]
        G = raw[:nt * 12 * esz].view(ft).reshape(nt, 4, 3).astype(np.float64)
        TN = raw[nt * 12 * esz:nt * (12 * esz + 8)].view(np.uint16).reshape(nt, 4).astype(np.int64)
        INC = raw[nt * (12 * esz + 8):nt * (12 * esz + 8) + maxinc * RB * 2].view(np.uint16).reshape(maxinc, RB)
        assert TN.max() < nn
        bn = nodes[node0:node0 + nn]
        assert np.all(np.diff(bn) > 0)                    # sorted, distinct
        sN = np.array([list(field(o)) + [s(o)] for o in bn])
        div = np.einsum("tb,tbc,tbc->t", sN[TN, 3], G, sN[TN, :3])
        for lr in range(RB):
            codes = INC[:, lr]
            if lr >= nrows:
                assert np.all(codes == PAD)
                continue
            live = codes[codes != PAD]
            assert np.all(codes[len(live):] == PAD)      # incidences first, then padding
            r = rows[row0 + lr]
            seen[r] += 1
            assert len(live) == m["rptr"][r + 1] - m["rptr"][r]
            t, a = live.astype(np.int64) >> 2, live.astype(np.int64) & 3
            assert np.all(t < nt)
            ga = G[t, a]
            lap = np.einsum("ic,ibc,ibd->id", ga, G[t], sN[TN[t], :3])
            y[r] = lap.sum(0) + (ga * div[t, None]).sum(0)
    assert np.array_equal(seen, np.ones(m["rows"], np.int64) if use is None else use.astype(np.int64))
    return y, blocks


def fields(m, seed):
    rng = np.random.default_rng(seed)
    cs, n_new = m["cs"], m["n_new"]
    F = rng.standard_normal((3, cs))
    XF = rng.standard_normal((3, max(n_new, 1)))
    S = rng.uniform(0.0, 10.0, cs)
    XS = rng.uniform(0.0, 10.0, max(n_new, 1))
    field = lambda o: F[:, o] if o < cs else XF[:, o - cs]
    s = lambda o: S[o] if o < cs else XS[o - cs]
    return field, s


@pytest.mark.parametrize("esz", [4, 8])
def test_pack_of_a_kuhn_cube_reproduces_the_element_loop(lib, esz):
    n, fem_n = 17, 11
    m = mesh_arrays(n, fem_n, np.zeros((0, 2), np.int64), kuhn_cube(n, fem_n), px=20)
    field, s = fields(m, 1)
    y, blocks = emulate(lib, m, esz, field, s)
    ref = direct_rows(m, field, s)
    tol = 1e-5 if esz == 4 else 1e-13
    assert np.abs(y - ref).max() <= tol * np.abs(ref).max()


@pytest.mark.parametrize("esz", [4, 8])
def test_pack_of_a_refined_mesh_reproduces_the_element_loop(lib, esz):
    n, fem_n = 25, 17
    nf = (fem_n - 4) ** 3
    rng = np.random.default_rng(3)
    eps = np.full(nf, 4.0)
    eps[rng.random(nf) < 0.05] = 20.0
    par, tets = refined_fem_mesh(n, fem_n, eps, np.zeros(nf), beta_eps=0.5, beta_sig=0.0)
    assert par.shape[0] > 0
    m = mesh_arrays(n, fem_n, par, tets, px=28)
    field, s = fields(m, 2)
    y, blocks = emulate(lib, m, esz, field, s)
    ref = direct_rows(m, field, s)
    tol = 1e-5 if esz == 4 else 1e-13
    assert np.abs(y - ref).max() <= tol * np.abs(ref).max()
    # several blocks, and in FP64 the byte budget (not only the row count) cuts them
    assert blocks.shape[0] > m["rows"] // lib.RB


def stencil_rows(lib, m):
    p = lambda x: x.ctypes.data_as(ctypes.c_void_p)
    out = np.zeros(m["grid_rows"], np.uint8)
    lib.ebe_kuhn_rows(ctypes.c_longlong(m["grid_rows"]), m["n"], p(m["rptr"]), p(m["itet"]), p(m["tet_ids"]), p(out))
    return out


def test_pack_of_a_row_subset_covers_exactly_those_rows(lib):
    n, fem_n = 17, 11
    m = mesh_arrays(n, fem_n, np.zeros((0, 2), np.int64), kuhn_cube(n, fem_n), px=20)
    use = (np.random.default_rng(4).random(m["rows"]) < 0.3).astype(np.uint8)
    field, s = fields(m, 5)
    y, _ = emulate(lib, m, 8, field, s, use)
    ref = direct_rows(m, field, s)
    sel = use.astype(bool)
    assert np.abs(y[sel] - ref[sel]).max() <= 1e-13 * np.abs(ref).max()


def test_kuhn_stencil_rows_are_the_untouched_kuhn_rows(lib):
    n, fem_n = 25, 17
    # uniform split: every grid row
    m = mesh_arrays(n, fem_n, np.zeros((0, 2), np.int64), kuhn_cube(n, fem_n), px=28)
    assert stencil_rows(lib, m).all()
    # refined mesh: exactly the rows none of whose tets holds a new node
    nf = (fem_n - 4) ** 3
    rng = np.random.default_rng(3)
    eps = np.full(nf, 4.0)
    eps[rng.random(nf) < 0.05] = 20.0
    par, tets = refined_fem_mesh(n, fem_n, eps, np.zeros(nf), beta_eps=0.5, beta_sig=0.0)
    m = mesh_arrays(n, fem_n, par, tets, px=28)
    got = stencil_rows(lib, m).astype(bool)
    want = np.array([not (tets[m["itet"][m["rptr"][r]:m["rptr"][r + 1]]] >= n ** 3).any()
                     for r in range(m["grid_rows"])])
    assert np.array_equal(got, want) and 0 < got.sum() < m["grid_rows"]
    # a cube split along another diagonal: the rows at its corners are gathered
    a, b, _, _ = box_bounds(n, fem_n)
    T = kuhn_cube(n, fem_n).copy()
    c = (a + 3) + n * ((a + 3) + n * (a + 3))          # cube corner
    i, j, k = T % n, (T // n) % n, T // (n * n)
    inside = ((i >= a + 3) & (i <= a + 4) & (j >= a + 3) & (j <= a + 4) & (k >= a + 3) & (k <= a + 4)).all(axis=1)
    T[inside] = (2 * (a + 3) + 1 - i[inside]) + n * (j[inside] + n * k[inside])   # mirrored in x
    m = mesh_arrays(n, fem_n, np.zeros((0, 2), np.int64), T, px=28)
    got = stencil_rows(lib, m).astype(bool)
    corners = [(a + 3 + dx) + n * ((a + 3 + dy) + n * (a + 3 + dz)) for dx in (0, 1) for dy in (0, 1) for dz in (0, 1)]
    fm = b - a - 1
    rowid = lambda v: (v % n - a - 1) + fm * ((v // n % n - a - 1) + fm * (v // (n * n) - a - 1))
    assert not any(got[rowid(v)] for v in corners)
    assert got.sum() == m["grid_rows"] - 8


def test_kuhn_stencil_rows_reproduce_the_element_loop(lib):
    """The formula of the stencil-row kernel, with the blocks the library
    assembles, on the untouched rows of a refined mesh."""
    p = lambda x: x.ctypes.data_as(ctypes.c_void_p)
    B = np.zeros((8, 9))
    assert lib.ebe_kuhn_blocks(p(B)) == 0
    n, fem_n = 25, 17
    nf = (fem_n - 4) ** 3
    rng = np.random.default_rng(3)
    eps = np.full(nf, 4.0)
    eps[rng.random(nf) < 0.05] = 20.0
    par, tets = refined_fem_mesh(n, fem_n, eps, np.zeros(nf), beta_eps=0.5, beta_sig=0.0)
    m = mesh_arrays(n, fem_n, par, tets, px=28)
    field, s = fields(m, 6)
    ref = direct_rows(m, field, s)
    st = stencil_rows(lib, m)
    px = m["px"]
    sx, sy, sz = 1, px, px * n
    offs = [sx, sy, sz, sx + sy, sx + sz, sy + sz, sx + sy + sz]
    for r in np.nonzero(st)[0]:
        i, j, k = (int(v) for v in m["rpos"][r])
        o = i + px * (j + n * k)
        lap = 6 * field(o) - sum(field(o + d) + field(o - d) for d in (sx, sy, sz))
        g = B[0].reshape(3, 3) @ (s(o) * field(o))
        for b, d in enumerate(offs):
            g += B[b + 1].reshape(3, 3) @ (s(o + d) * field(o + d) + s(o - d) * field(o - d))
        assert np.allclose(lap + g, ref[r], rtol=1e-12, atol=1e-12 * np.abs(ref).max())
