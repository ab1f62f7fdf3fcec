"""Incident source, source-phase switch and the observation time weight (oracle).

Test infrastructure only (see oracle/__init__.py).

Boundary data of the model problem (Sec. 5, eq. model1): d_n E = P(t) on the
top face while t <= t1, d_n E = -d_t E on the top face afterwards and on the
bottom face always, d_n E = 0 on the four sides.  The paper's P is
(0, P_2, 0) with P_2 one period of sin(omega t) (eq. f).

Readings (the paper leaves omega, t1 and T open):
  * kind "gauss" (default): P(t) = sin(2 pi f (t - t0)) exp(-((t - t0)/w)^2),
    the Gaussian-modulated pulse; its source phase ends at t0 + 3 w.
  * kind "sine": the paper's single period, sin(2 pi f t) on (0, 1/f), else 0;
    its source phase ends at 1/f.
  * oblique incidence: a plane wave with direction k (k_z < 0) reaches top node
    x after the delay d(x) = k.(x - x_c) + Delta, x_c the face centre and Delta
    the largest -k.(x - x_c) over the face, so d >= 0; the flux is
    p P(t - d(x)) with polarisation p = normalise(y - (y.k) k) (= y at normal
    incidence, as in eq. f).  t1 defaults to the end of the phase + Delta.
  * the switch is taken as an integer step: steps n <= n1 = floor(t1/tau +
    1e-9) carry the Neumann source, later steps the absorbing top face; the
    1e-9 guard keeps an exact t1/tau from flipping on rounding.
  * z_delta (the smoothing function in eq. tikhonov_functional): 1 for
    t <= T - delta, then (1 + cos(pi (t - T + delta)/delta))/2, delta =
    frac * T; frac = 0 gives z = 1.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np


@dataclass
class SourceSpec:
    kind: str = "gauss"
    freq: float = 2.0
    t0: float = 0.75
    width: float = 0.25
    t1: float = -1.0
    direction: tuple = field(default=(0.0, 0.0, -1.0))

    def pulse(self, t):
        t = np.asarray(t, dtype=np.float64)
        if self.kind == "gauss":
            s = t - self.t0
            return np.sin(2.0 * math.pi * self.freq * s) * np.exp(-(s / self.width) ** 2)
        if self.kind == "sine":
            on = (t > 0.0) & (t < 1.0 / self.freq)
            return np.where(on, np.sin(2.0 * math.pi * self.freq * t), 0.0)
        raise ValueError(self.kind)

    def phase_end(self) -> float:
        return self.t0 + 3.0 * self.width if self.kind == "gauss" else 1.0 / self.freq

    def polarisation(self) -> np.ndarray:
        k = np.asarray(self.direction, dtype=np.float64)
        k = k / np.linalg.norm(k)
        y = np.array([0.0, 1.0, 0.0])
        p = y - (y @ k) * k
        if np.linalg.norm(p) < 1e-12:
            x = np.array([1.0, 0.0, 0.0])
            p = x - (x @ k) * k
        return p / np.linalg.norm(p)

    def delays(self, top_coords: np.ndarray) -> np.ndarray:
        k = np.asarray(self.direction, dtype=np.float64)
        k = k / np.linalg.norm(k)
        xc = np.array([0.5, 0.5, 1.0])
        proj = (top_coords - xc) @ k
        return proj + np.max(-proj)

    def t1_value(self, top_coords: np.ndarray) -> float:
        if self.t1 >= 0.0:
            return self.t1
        d = self.delays(top_coords)
        return self.phase_end() + float(np.max(d))

    def switch_step(self, tau: float, top_coords: np.ndarray) -> int:
        return int(math.floor(self.t1_value(top_coords) / tau + 1e-9))


def z_delta(t, T: float, frac: float):
    t = np.asarray(t, dtype=np.float64)
    if frac <= 0.0:
        return np.ones_like(t)
    d = frac * T
    return np.where(t <= T - d, 1.0, 0.5 * (1.0 + np.cos(math.pi * (t - T + d) / d)))
