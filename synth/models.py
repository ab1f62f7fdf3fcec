"""Seeded synthetic workloads: layered skin with ellipsoidal inclusions.

The paper's melanoma model (its Table 1 and Figs. 3-4) is not available, so
these generators stand in for it with the same structure: a homogeneous
immersion margin (epsilon = 1, sigma = 0) around a FEM cube that holds three
planar tissue layers (epidermis, dermis, fat, top to bottom) and one or more
ellipsoidal tumour inclusions of higher permittivity and conductivity.

Geometry conventions (shared by every consumer of these arrays):
  * grid: n^3 nodes on [0,1]^3, spacing h = 1/(n-1), node id i + n*(j + n*k),
    x fastest; k is depth and the top (incident, observed) face is k = n-1.
  * FEM box: node indices [a, b]^3 with a = (n - fem_n)//2, b = a + fem_n - 1.
  * free (coefficient) nodes: [a+2, b-2]^3, listed x fastest.  Coefficients
    are 1 / 0 on every other node.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field, replace
from typing import Optional

import numpy as np

_MASK64 = (1 << 64) - 1


class SplitMix64:
    """SplitMix64 generator (Steele, Lea & Flood, OOPSLA 2014).

    Doubles are drawn as the top 53 bits of the 64-bit output times 2^-53,
    so they lie in [0, 1).
    """

    def __init__(self, seed: int):
        self.state = seed & _MASK64

    def next_u64(self) -> int:
        self.state = (self.state + 0x9E3779B97F4A7C15) & _MASK64
        z = self.state
        z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & _MASK64
        z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & _MASK64
        return z ^ (z >> 31)

    def uniform(self, lo: float = 0.0, hi: float = 1.0) -> float:
        u = (self.next_u64() >> 11) * (1.0 / 9007199254740992.0)
        return lo + (hi - lo) * u


def box_bounds(n: int, fem_n: int):
    """Return (a, b, f0, f1): FEM box [a,b] and free box [f0,f1] node indices."""
    if fem_n < 5 or fem_n > n - 2:
        raise ValueError(f"fem_n={fem_n} must satisfy 5 <= fem_n <= n-2 (n={n})")
    a = (n - fem_n) // 2
    b = a + fem_n - 1
    return a, b, a + 2, b - 2


# Layer fractions of the free-box height, top to bottom: epidermis, dermis, fat.
LAYER_FRACTIONS = (0.10, 0.35, 0.55)
LAYER_EPS = (4.0, 12.0)
LAYER_SIG = (0.0, 0.5)
INCL_EPS = (15.0, 25.0)
INCL_SIG = (0.5, 1.0)
INCL_SEMI_AXIS = (0.1, 0.2)


def layered_inclusion_model(n: int, fem_n: int, seed: int, n_incl: int, box=None):
    """Nodal (eps, sigma) on the free nodes, flattened x fastest.

    Draw order from one SplitMix64 stream: (eps, sigma) for each layer from
    the top, then per inclusion the three semi-axes, the three centre
    coordinates and (eps, sigma).  The layers-only model of the same seed
    (n_incl = 0) is therefore the inclusion model without its inclusions.
    A later inclusion overwrites an earlier one where they overlap.

    box: (lo, hi), the physical extent [lo, hi]^3 the model is defined on
    (default: this grid's free box).  Passing another grid's box samples the
    same physical model on this grid (free nodes outside the box are vacuum,
    eps = 1, sigma = 0): a finer grid then carries the coarse grid's model.
    """
    h = 1.0 / (n - 1)
    _, _, f0, f1 = box_bounds(n, fem_n)
    rng = SplitMix64(seed)
    idx = np.arange(f0, f1 + 1)
    x = idx * h
    X = x[None, None, :]
    Y = x[None, :, None]
    Z = x[:, None, None]
    nf = idx.size
    shape = (nf, nf, nf)
    eps = np.empty(shape)
    sig = np.empty(shape)
    z_lo, z_hi = (x[0], x[-1]) if box is None else (float(box[0]), float(box[1]))
    height = z_hi - z_lo
    cuts = [z_hi - LAYER_FRACTIONS[0] * height,
            z_hi - (LAYER_FRACTIONS[0] + LAYER_FRACTIONS[1]) * height]
    layer_vals = [(rng.uniform(*LAYER_EPS), rng.uniform(*LAYER_SIG)) for _ in range(3)]
    zz = np.broadcast_to(Z, shape)
    top = zz >= cuts[0]
    mid = (zz >= cuts[1]) & ~top
    low = ~(top | mid)
    for mask, (e, s) in zip((top, mid, low), layer_vals):
        eps[mask] = e
        sig[mask] = s
    for _ in range(n_incl):
        r = [rng.uniform(*INCL_SEMI_AXIS) for _ in range(3)]
        c = []
        for ax in range(3):
            lo, hi = z_lo + r[ax], z_hi - r[ax]
            if hi < lo:  # box smaller than the ellipsoid: centre it
                lo = hi = 0.5 * (z_lo + z_hi)
            c.append(rng.uniform(lo, hi))
        e, s = rng.uniform(*INCL_EPS), rng.uniform(*INCL_SIG)
        inside = (((X - c[0]) / r[0]) ** 2 + ((Y - c[1]) / r[1]) ** 2
                  + ((Z - c[2]) / r[2]) ** 2) <= 1.0
        inside = np.broadcast_to(inside, shape)
        eps[inside] = e
        sig[inside] = s
    if box is not None:
        tol = 1e-9 * h
        outside = ((X < z_lo - tol) | (X > z_hi + tol) | (Y < z_lo - tol) | (Y > z_hi + tol)
                   | (Z < z_lo - tol) | (Z > z_hi + tol))
        outside = np.broadcast_to(outside, shape)
        eps[outside] = 1.0
        sig[outside] = 0.0
    return eps.ravel().copy(), sig.ravel().copy()


def free_box(n: int, fem_n: int):
    """Physical extent (lo, hi) of the free box of a grid."""
    _, _, f0, f1 = box_bounds(n, fem_n)
    h = 1.0 / (n - 1)
    return f0 * h, f1 * h


def detector_grid(n: int, fem_n: int, d: int) -> np.ndarray:
    """d x d detectors on the top face over the FEM box, as (i, j) node pairs.

    Index q in 0..d-1 sits at floor(a + (b-a)(q+1/2)/d + 1/2).
    """
    a, b, _, _ = box_bounds(n, fem_n)
    q = np.arange(d)
    pos = np.floor(a + (b - a) * (q + 0.5) / d + 0.5).astype(np.int32)
    jj, ii = np.meshgrid(pos, pos, indexing="ij")
    return np.stack([ii.ravel(), jj.ravel()], axis=1).astype(np.int32)


def hemisphere_directions(n_src: int, seed: int) -> np.ndarray:
    """Incidence directions k = (sin t cos p, sin t sin p, -cos t), uniform on
    the downward hemisphere: cos t ~ U(0,1), p ~ U(0, 2 pi)."""
    rng = SplitMix64(seed)
    out = np.empty((n_src, 3))
    for s in range(n_src):
        ct = rng.uniform(0.0, 1.0)
        ph = rng.uniform(0.0, 2.0 * math.pi)
        st = math.sqrt(max(0.0, 1.0 - ct * ct))
        out[s] = (st * math.cos(ph), st * math.sin(ph), -ct)
    return out


def shard_directions(n_src: int, seed: int = 5) -> np.ndarray:
    """n_src incidence directions for source sharding: normal incidence first,
    then n_src - 1 drawn on the lower hemisphere."""
    d = np.zeros((n_src, 3))
    d[0, 2] = -1.0
    if n_src > 1:
        d[1:] = hemisphere_directions(n_src - 1, seed)
    return d


@dataclass(frozen=True)
class Workload:
    """One problem description, as plain numbers and seeds."""

    name: str
    n: int
    fem_n: int
    n_steps: int
    cfl: float = 0.3
    precision: str = "fp64"        # "fp64" or "fp32"
    seed: int = 1
    n_incl: int = 1
    det_per_side: int = 8
    n_src: int = 1
    dir_seed: Optional[int] = None  # None: normal incidence for every source
    z_delta_frac: float = 0.1
    gamma_eps: float = 0.0
    gamma_sig: float = 0.0
    extra: dict = field(default_factory=dict)

    def with_(self, **kw) -> "Workload":
        return replace(self, **kw)

    def model(self, inclusions: bool = True):
        return layered_inclusion_model(self.n, self.fem_n, self.seed,
                                       self.n_incl if inclusions else 0)

    def detectors(self) -> np.ndarray:
        if "det" in self.extra:
            return np.asarray(self.extra["det"], dtype=np.int32).reshape(-1, 2)
        return detector_grid(self.n, self.fem_n, self.det_per_side)

    def directions(self) -> np.ndarray:
        if self.dir_seed is None:
            d = np.zeros((self.n_src, 3))
            d[:, 2] = -1.0
            return d
        return hemisphere_directions(self.n_src, self.dir_seed)

    @property
    def n_free(self) -> int:
        return (self.fem_n - 4) ** 3

    @property
    def updates(self) -> int:
        """Grid-point updates of one forward + adjoint pass (all sources)."""
        return 2 * self.n ** 3 * self.n_steps * self.n_src


WORKLOADS = {
    # plain FP64 method, 41^3 grid, 21^3 FEM cube, 300 steps, 64 detectors
    "c1_fp64_41": Workload("c1_fp64_41", 41, 21, 300, precision="fp64", seed=1,
                           n_incl=1, det_per_side=8),
    # FP32 fields with FP64 reductions, 201^3 grid, 101^3 FEM cube, 2000 steps,
    # 1 + (seed mod 3) = 3 inclusions, 1024 detectors
    "c2_fp32_201": Workload("c2_fp32_201", 201, 101, 2000, precision="fp32",
                            seed=2, n_incl=3, det_per_side=32),
    # the same grid and kernels for 20 steps: small device footprint for
    # profiler captures
    "c2_profile": Workload("c2_profile", 201, 101, 20, precision="fp32",
                           seed=2, n_incl=3, det_per_side=32),
    # differentiable FP32 run, 301^3 grid, 151^3 FEM cube, 4000 steps
    "c4_fp32_301": Workload("c4_fp32_301", 301, 151, 4000, precision="fp32",
                            seed=4, n_incl=2, det_per_side=32),
    # small cases the oracle finishes in seconds
    "tiny": Workload("tiny", 13, 9, 40, seed=11, n_incl=1, det_per_side=3),
    "small": Workload("small", 25, 13, 120, seed=12, n_incl=1, det_per_side=4),
}


def workload(name: str, **overrides) -> Workload:
    w = WORKLOADS[name]
    return w.with_(**overrides) if overrides else w


def batched_problems(n: int = 161, n_problems: int = 16, n_steps: int = 1600, first: int = 0):
    """The heterogeneous batch: FEM cube 61/81/101/121 for problem b mod 4,
    seed 300 + b, one hemisphere-drawn incidence direction per problem, for
    problems b = first .. first + n_problems - 1 (first = 0: the 16-problem
    workload; a later `first` gives further, independent problems of the
    same kind, e.g. for another GPU)."""
    sizes = (61, 81, 101, 121)
    dirs = hemisphere_directions(first + n_problems, 3000)
    out = []
    for b in range(first, first + n_problems):
        w = Workload(f"batch{b}", n, sizes[b % 4], n_steps, precision="fp32",
                     seed=300 + b, n_incl=1 + (300 + b) % 3, det_per_side=32,
                     n_src=1, dir_seed=None)
        out.append((w, dirs[b]))
    return out
