"""Forward, functional, adjoint and gradient (oracle).

Test infrastructure only (see oracle/__init__.py).

Time discretisation (explicit central differences; the paper refines only in
space so that one explicit step serves both regions, Sec. 4): with tau the
time step, t_n = n tau, E^{-1} = E^0 = 0 (zero initial data, eq. model1) and
for n = 0 .. Nt-1

  A+_n E^{n+1} = (2 M_eps / tau^2) E^n - K E^n - A-_n E^{n-1} + F^n,
  A+-_n = M_eps / tau^2 +- C_n / (2 tau),

where C_n holds the faces that are absorbing at step n and F^n = b_top p
P(t_n - d) is the lumped Neumann flux on the top face during the source phase.

Discrete functional (Sec. 3, eq. tikhonov_functional; delta_obs read as point
evaluation at the detector nodes, time integral by the rectangle rule on
t_1..t_Nt):
  J = tau/2 sum_n z(t_n) sum_d |E^n_d - Eobs^n_d|^2
      + gamma_eps/2 sum_i m_i (eps_i - eps0_i)^2 + gamma_sig/2 sum_i m_i (sig_i - sig0_i)^2

Adjoint: the multipliers mu^n of the step equations (the discrete Lagrangian of
eq. lagrangian_weak) solve, for k = Nt .. 1 with mu^Nt = mu^{Nt+1} = 0,

  A+_{k-1} mu^{k-1} = (2 M_eps / tau^2) mu^k - K^T mu^k - A-_{k+1} mu^{k+1} - j^k,
  j^k = tau z(t_k) (E^k - Eobs^k) at the detectors,

the discrete counterpart of eq. adjoint_prob (lambda ~ mu / tau): time runs
backwards, the -sigma d_t lambda and d_n lambda = d_t lambda terms appear as
damping, and the terminal conditions hold by construction.  Reading: the
adjoint boundary pattern is the transpose of the forward one.

Gradient (Sec. 4, eq. gradeps, taken as the exact derivative of the discrete
J so that finite differences confirm it; the paper's simplification
div(eps E) ~ eps div E is not applied):
  g_eps_i = gamma_eps m_i (eps_i - eps0_i)
            + sum_{n=0}^{Nt-1} [ m_i mu^n_i . (E^{n+1} - 2E^n + E^{n-1})_i / tau^2
                                 + E^n_i . (D^T D P mu^n)_i ]
  g_sig_i = gamma_sig m_i (sig_i - sig0_i)
            + sum_{n=0}^{Nt-1} m_i mu^n_i . (E^{n+1} - E^{n-1})_i / (2 tau)
term by term the discrete forms of -int d_t lambda d_t E, int div lambda div E
and int lambda d_t E; f1 = 0 (eq. model1) removes the lambda(0) f1 term.

Paper-literal variant (gradient_literal): eq. gradeps as printed, with the
approximation div(eps_bar E) ~ eps_bar div E made under it.  The time terms
and g_sig are those above; the Gauss-law term becomes the lumped quadrature
of int phi_i div lambda div E over the tets K around node i (P1 divergences
are constant on K, int_K phi_i = |K|/4):
  sum_{n=0}^{Nt-1} sum_{K ni i} |K|/4 (div E^n)_K (div P mu^n)_K
instead of sum_K |K| (grad phi_i . E^n_i) (div P mu^n)_K.  Summed over every
node of the tets, the two agree (both are sum_K |K| (div E)_K (div P mu)_K);
node by node they differ by the dropped grad(eps_bar) . E term.
"""
from __future__ import annotations

from dataclasses import dataclass, field
from typing import Callable, Optional, Sequence

import numpy as np

from .grid import Grid, RefinedGrid
from .hybrid import HybridOperator
from .source import SourceSpec, z_delta

# absorbing-face bits, as in the library's configuration
ABS_BOTTOM, ABS_TOP = 1, 2
ABS_X0, ABS_X1, ABS_Y0, ABS_Y1 = 4, 8, 16, 32


@dataclass
class ForwardResult:
    trace: np.ndarray                       # (Nt+1, n_det, 3)
    E_free: np.ndarray                      # (Nt+2, 3, n_free): E^{-1} .. E^{Nt}
    fields: dict = field(default_factory=dict)   # n -> (3, nn) E^n at requested n


@dataclass
class AdjointResult:
    mu_free: np.ndarray                     # (Nt, 3, n_free): mu^0 .. mu^{Nt-1}
    dtd_free: np.ndarray                    # (Nt, 3, n_free): (D^T D P mu^n) at free nodes
    fields: dict = field(default_factory=dict)   # n -> (3, nn) mu^n at requested n


class OracleProblem:
    def __init__(self, n: int, fem_n: int, n_steps: int, cfl: float,
                 eps_free, sig_free, det_ij, sources: Sequence[SourceSpec],
                 absorbing: int = ABS_BOTTOM | ABS_TOP, z_delta_frac: float = 0.1,
                 gamma_eps: float = 0.0, gamma_sig: float = 0.0,
                 eps0_free=None, sig0_free=None, mesh=None):
        # mesh: None (the Kuhn split of the FEM cube) or an explicit refined
        # FEM mesh (parents, tets) as described in grid.RefinedGrid
        self.g = Grid(n, fem_n) if mesh is None else RefinedGrid(n, fem_n, *mesh)
        self.op = HybridOperator(self.g, eps_free, sig_free)
        self.n_steps = int(n_steps)
        self.tau = cfl * self.g.h
        self.T = self.n_steps * self.tau
        det_ij = np.asarray(det_ij, dtype=np.int64).reshape(-1, 2)
        self.det_nodes = self.g.nid(det_ij[:, 0], det_ij[:, 1], n - 1)
        self.sources = list(sources)
        self.absorbing = absorbing
        self.z_delta_frac = z_delta_frac
        self.gamma_eps, self.gamma_sig = gamma_eps, gamma_sig
        nf = self.g.free_nodes.size
        self.eps0 = np.ones(nf) if eps0_free is None else np.asarray(eps0_free, float)
        self.sig0 = np.zeros(nf) if sig0_free is None else np.asarray(sig0_free, float)
        self.top = np.nonzero(self.g.face_nodes("top"))[0]
        self.top_coords = self.g.coords[self.top]
        self.M = self.op.m * self.op.eps

    # ---- boundary pattern and source ------------------------------------
    def absorbing_faces(self, n: int, src: SourceSpec):
        faces = []
        if self.absorbing & ABS_BOTTOM:
            faces.append("bottom")
        if (self.absorbing & ABS_TOP) and n > src.switch_step(self.tau, self.top_coords):
            faces.append("top")
        for bit, f in ((ABS_X0, "x0"), (ABS_X1, "x1"), (ABS_Y0, "y0"), (ABS_Y1, "y1")):
            if self.absorbing & bit:
                faces.append(f)
        return faces

    def source_term(self, n: int, src: SourceSpec) -> np.ndarray:
        F = np.zeros((3, self.g.nn))
        if n > src.switch_step(self.tau, self.top_coords):
            return F
        t = n * self.tau
        val = src.pulse(t - src.delays(self.top_coords))
        b = self.op.face_mass["top"][self.top]
        p = src.polarisation()
        for c in range(3):
            F[c, self.top] = b * p[c] * val
        return F

    def coeff(self, n: int, src: SourceSpec):
        """(A+_n, A-_n) diagonals; n outside 0..Nt-1 is allowed (pattern only)."""
        C = self.op.damping(self.absorbing_faces(n, src))
        return self.M / self.tau ** 2 + C / (2 * self.tau), self.M / self.tau ** 2 - C / (2 * self.tau)

    # ---- forward (O3) ------------------------------------------------------
    def forward_step(self, n: int, E_prev: np.ndarray, E_cur: np.ndarray, F: np.ndarray,
                     src: SourceSpec) -> np.ndarray:
        """One step of the scheme: E^{n+1} from E^{n-1}, E^n and the flux F^n,
        A+_n E^{n+1} = (2 M_eps / tau^2) E^n - K E^n - A-_n E^{n-1} + F^n."""
        tau = self.tau
        Ap, Am = self.coeff(n, src)
        rhs = (2.0 * self.M / tau ** 2) * E_cur - self.op.apply_K(E_cur) - Am * E_prev + F
        return rhs / Ap

    def forward(self, s: int = 0, keep_fields: Sequence[int] = (),
                source_override: Optional[Callable[[int], np.ndarray]] = None) -> ForwardResult:
        src = self.sources[s]
        nn, Nt, tau = self.g.nn, self.n_steps, self.tau
        free = self.g.free_nodes
        E_prev = np.zeros((3, nn))      # E^{n-1}
        E_cur = np.zeros((3, nn))       # E^n
        trace = np.zeros((Nt + 1, self.det_nodes.size, 3))
        E_free = np.zeros((Nt + 2, 3, free.size))
        fields = {0: E_cur.copy()} if 0 in keep_fields else {}
        for n in range(Nt):
            F = source_override(n) if source_override is not None else self.source_term(n, src)
            E_next = self.forward_step(n, E_prev, E_cur, F, src)
            trace[n + 1] = E_next[:, self.det_nodes].T
            E_free[n + 2] = E_next[:, free]
            if (n + 1) in keep_fields:
                fields[n + 1] = E_next.copy()
            E_prev, E_cur = E_cur, E_next
        return ForwardResult(trace, E_free, fields)

    # ---- functional (O4) ------------------------------------------------------
    def misfit(self, traces: Sequence[np.ndarray], eobs: Sequence[np.ndarray]) -> float:
        t = np.arange(self.n_steps + 1) * self.tau
        z = z_delta(t, self.T, self.z_delta_frac)
        J = 0.0
        for tr, eo in zip(traces, eobs):
            r2 = np.sum((tr - eo) ** 2, axis=(1, 2))
            J += 0.5 * self.tau * float(np.sum(z[1:] * r2[1:]))
        return J

    def regulariser(self) -> float:
        m = self.op.m[self.g.free_nodes]
        e = self.op.eps[self.g.free_nodes] - self.eps0
        s = self.op.sig[self.g.free_nodes] - self.sig0
        return 0.5 * self.gamma_eps * float(np.sum(m * e * e)) + \
            0.5 * self.gamma_sig * float(np.sum(m * s * s))

    def functional(self, traces, eobs) -> float:
        return self.misfit(traces, eobs) + self.regulariser()

    # ---- adjoint (O5) --------------------------------------------------------
    def residual_source(self, k: int, trace: np.ndarray, eobs: np.ndarray) -> np.ndarray:
        j = np.zeros((3, self.g.nn))
        zk = float(z_delta(k * self.tau, self.T, self.z_delta_frac))
        r = self.tau * zk * (trace[k] - eobs[k])            # (n_det, 3)
        for c in range(3):
            np.add.at(j[c], self.det_nodes, r[:, c])
        return j

    def adjoint_step(self, k: int, mu_next: np.ndarray, mu_cur: np.ndarray, j: np.ndarray,
                     src: SourceSpec) -> np.ndarray:
        """One step of the discrete adjoint: mu^{k-1} from mu^{k+1}, mu^k and j^k,
        A+_{k-1} mu^{k-1} = (2 M_eps / tau^2) mu^k - K^T mu^k - A-_{k+1} mu^{k+1} - j^k."""
        tau = self.tau
        Ap_km1, _ = self.coeff(k - 1, src)
        _, Am_kp1 = self.coeff(k + 1, src)
        rhs = (2.0 * self.M / tau ** 2) * mu_cur - self.op.apply_KT(mu_cur) - Am_kp1 * mu_next - j
        return rhs / Ap_km1

    def adjoint(self, s: int, trace: np.ndarray, eobs: np.ndarray,
                keep_fields: Sequence[int] = (),
                residual_override: Optional[Callable[[int], np.ndarray]] = None) -> AdjointResult:
        src = self.sources[s]
        nn, Nt, tau = self.g.nn, self.n_steps, self.tau
        free = self.g.free_nodes
        mu_next = np.zeros((3, nn))     # mu^{k+1}
        mu_cur = np.zeros((3, nn))      # mu^k
        mu_free = np.zeros((Nt, 3, free.size))
        dtd_free = np.zeros((Nt, 3, free.size))
        fields = {}
        for k in range(Nt, 0, -1):
            j = residual_override(k) if residual_override is not None else \
                self.residual_source(k, trace, eobs)
            mu_prev = self.adjoint_step(k, mu_next, mu_cur, j, src)
            mu_free[k - 1] = mu_prev[:, free]
            dtd_free[k - 1] = self.op.apply_DtD_masked(mu_prev)[:, free]
            if (k - 1) in keep_fields:
                fields[k - 1] = mu_prev.copy()
            mu_next, mu_cur = mu_cur, mu_prev
        return AdjointResult(mu_free, dtd_free, fields)

    # ---- gradient (O6) -------------------------------------------------------
    def gradient_terms(self, fwd: ForwardResult, adj: AdjointResult):
        """Time sums of one source (without the regularisation terms)."""
        m = self.op.m[self.g.free_nodes]
        tau = self.tau
        Nt = self.n_steps
        ge = np.zeros(m.size)
        gs = np.zeros(m.size)
        for n in range(Nt):
            Em1, E0, Ep1 = fwd.E_free[n], fwd.E_free[n + 1], fwd.E_free[n + 2]  # E^{n-1}, E^n, E^{n+1}
            mu = adj.mu_free[n]
            ge += m * np.sum(mu * (Ep1 - 2.0 * E0 + Em1), axis=0) / tau ** 2
            ge += np.sum(E0 * adj.dtd_free[n], axis=0)
            gs += m * np.sum(mu * (Ep1 - Em1), axis=0) / (2.0 * tau)
        return ge, gs

    def literal_div_term(self, E: np.ndarray, mu: np.ndarray) -> np.ndarray:
        """sum_{K ni i} |K|/4 (div E)_K (div P mu)_K at every node (paper-literal
        Gauss-law term of eq. gradeps for one time level; E, mu: (3, nn))."""
        op = self.op
        dE = op.D @ E.ravel()                                   # sqrt|K| (div E)_K
        dM = op.D @ (op.fem_mask[None, :] * mu).ravel()         # sqrt|K| (div P mu)_K
        prod = 0.25 * dE * dM
        out = np.zeros(self.g.nn)
        for q in range(4):
            np.add.at(out, op.tets[:, q], prod)
        return out

    def gradient_literal(self, fwds, adjs):
        """The paper-literal gradient (module docstring).  Needs every forward
        level 0..Nt and every adjoint level 0..Nt-1 kept (keep_fields)."""
        free = self.g.free_nodes
        m = self.op.m[free]
        ge = self.gamma_eps * m * (self.op.eps[free] - self.eps0)
        gs = self.gamma_sig * m * (self.op.sig[free] - self.sig0)
        Nt = self.n_steps
        for f, a in zip(fwds, adjs):
            if any(n not in f.fields for n in range(Nt)) or any(n not in a.fields for n in range(Nt)):
                raise ValueError("gradient_literal needs the full forward and adjoint fields (keep_fields)")
            for n in range(Nt):
                Em1, E0, Ep1 = f.E_free[n], f.E_free[n + 1], f.E_free[n + 2]
                mu = a.mu_free[n]
                ge += m * np.sum(mu * (Ep1 - 2.0 * E0 + Em1), axis=0) / self.tau ** 2
                ge += self.literal_div_term(f.fields[n], a.fields[n])[free]
                gs += m * np.sum(mu * (Ep1 - Em1), axis=0) / (2.0 * self.tau)
        return ge, gs

    def gradient(self, fwds, adjs):
        m = self.op.m[self.g.free_nodes]
        ge = self.gamma_eps * m * (self.op.eps[self.g.free_nodes] - self.eps0)
        gs = self.gamma_sig * m * (self.op.sig[self.g.free_nodes] - self.sig0)
        for f, a in zip(fwds, adjs):
            e, s = self.gradient_terms(f, a)
            ge = ge + e
            gs = gs + s
        return ge, gs

    # ---- the whole path ---------------------------------------------------------
    def run(self, eobs: Sequence[np.ndarray], keep_fields: Sequence[int] = ()):
        """Forward for every source, J, adjoint for every source, gradient."""
        fwds = [self.forward(s, keep_fields) for s in range(len(self.sources))]
        traces = [f.trace for f in fwds]
        J = self.functional(traces, eobs)
        adjs = [self.adjoint(s, fwds[s].trace, eobs[s], keep_fields)
                for s in range(len(self.sources))]
        ge, gs = self.gradient(fwds, adjs)
        return dict(J=J, g_eps=ge, g_sig=gs, traces=traces, fwds=fwds, adjs=adjs)
