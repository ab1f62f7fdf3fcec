"""CPU check of the enumeration that the paper-literal gradient kernel
(csrc/ddfd_literal.cu, k_grad_literal) uses, against the oracle.

The kernel visits, for each free node, the 8 cubes around it and the 6 Kuhn
path tets of each cube, keeps the 24 that contain the node, and adds
(h / 6) sum (div mu)_K ((div E)_K / 4 - grad phi_i . E_i) with unit-gradient
divergences.  The same loop, written here step for step, must give the
oracle's literal-minus-exact Gauss-law term at every free node, and touch
only FEM-updated nodes (the ones whose E the library keeps)."""
import numpy as np

from oracle import OracleProblem, SourceSpec
from synth import box_bounds, detector_grid


def kernel_loop(E, mu, n, a, b, h):
    nid = lambda x, y, z: x + n * (y + n * z)
    nf = b - a - 3
    out = {}
    for f in range(nf ** 3):
        x, y, z = a + 2 + f % nf, a + 2 + (f // nf) % nf, a + 2 + f // (nf * nf)
        acc, ntet = 0.0, 0
        for corner in range(8):
            r = (corner & 1, (corner >> 1) & 1, (corner >> 2) & 1)
            o = (x - r[0], y - r[1], z - r[2])
            for t in range(6):
                p0 = t >> 1
                q0 = 1 if p0 == 0 else 0
                q1 = 1 if p0 == 2 else 2
                p1, p2 = (q1, q0) if t & 1 else (q0, q1)
                w = [[0, 0, 0], [0, 0, 0], [0, 0, 0], [1, 1, 1]]
                w[1][p0] = 1
                w[2][p0] = 1
                w[2][p1] = 1
                va = [j for j in range(4) if tuple(w[j]) == r]
                if not va:
                    continue
                va, ntet = va[0], ntet + 1
                V = [(o[0] + w[j][0], o[1] + w[j][1], o[2] + w[j][2]) for j in range(4)]
                assert all(a + 1 <= c <= b - 1 for v in V for c in v)     # FEM-updated nodes only
                Ev = [E[:, nid(*v)] for v in V]
                Mv = [mu[:, nid(*v)] for v in V]
                dE = (Ev[1][p0] - Ev[0][p0]) + (Ev[2][p1] - Ev[1][p1]) + (Ev[3][p2] - Ev[2][p2])
                dM = (Mv[1][p0] - Mv[0][p0]) + (Mv[2][p1] - Mv[1][p1]) + (Mv[3][p2] - Mv[2][p2])
                own = [-Ev[0][p0], Ev[1][p0] - Ev[1][p1], Ev[2][p1] - Ev[2][p2], Ev[3][p2]][va]
                acc += dM * (0.25 * dE - own)
        assert ntet == 24
        out[nid(x, y, z)] = h / 6.0 * acc
    return out


def test_kernel_enumeration_gives_the_oracle_difference():
    n, fem_n = 13, 9
    rng = np.random.default_rng(0)
    nf = (fem_n - 4) ** 3
    P = OracleProblem(n, fem_n, 10, 0.3, rng.uniform(2, 9, nf), rng.uniform(0, 0.5, nf),
                      detector_grid(n, fem_n, 2), [SourceSpec()])
    E, mu = rng.standard_normal((3, P.g.nn)), rng.standard_normal((3, P.g.nn))
    want = P.literal_div_term(E, mu) - np.sum(E * P.op.apply_DtD_masked(mu), axis=0)
    a, b, _, _ = box_bounds(n, fem_n)
    got = kernel_loop(E, mu, n, a, b, P.g.h)
    assert len(got) == nf
    scale = np.abs(want).max()
    for i, v in got.items():
        assert abs(v - want[i]) <= 1e-13 * scale
