"""FP64 CPU oracle of the ADDFE/FDM forward / adjoint / gradient path.

TEST INFRASTRUCTURE ONLY.  Nothing in the product (the CUDA library and its
Python binding) imports, calls or links anything here; only the tests, the
smoke check and the CPU-baseline leg of the benchmark do.

What it computes, in plain numpy/scipy, FP64, with no blocking or fusion:
  * the semi-discrete operators of the hybrid FE/FD discretisation of the
    stabilized Maxwell model problem (Sec. 5, eq. model1; Sec. 2,
    eq. forward_prob) by *global sparse assembly* -- finite differences on the
    hexahedral grid everywhere, P1 elements on the Kuhn-split FEM cube
    (grid.py, fdm.py, fem.py, hybrid.py);
  * explicit central time stepping forward in time for E (solver.forward);
  * the Tikhonov functional (Sec. 3, eq. tikhonov_functional; solver.functional);
  * the exact discrete adjoint backward in time for lambda (Sec. 3,
    eq. adjoint_prob, derived from the Lagrangian eq. lagrangian_weak;
    solver.adjoint);
  * the gradient with respect to epsilon and sigma (Sec. 4, eq. gradeps, taken
    as the exact derivative of the discrete functional; solver.gradient), and
    the paper-literal form with div(eps_bar E) ~ eps_bar div E
    (solver.gradient_literal);
  * the leapfrog stability bound by power iteration (cfl.py);
  * the conjugate gradient reconstruction of Sec. 4 (cg.py);
  * all of the above on a locally refined FEM mesh given as explicit
    (new nodes, tetrahedra) (grid.RefinedGrid, OracleProblem(mesh=...)).

It shares no code with the CUDA path.  Seeded inputs come from the separate
``synth`` package, which holds none of the method's arithmetic.

Every part is pinned by tests under tests/test_oracle_*.py to values fixed by
mathematics rather than by this code: closed-form spectra, exactness on
polynomials, a 1-D textbook reduction, d'Alembert's solution, a discrete energy
identity, the space-time adjoint dot test and central finite differences.
"""
from .grid import Grid, RefinedGrid  # noqa: F401
from .hybrid import HybridOperator  # noqa: F401
from .source import SourceSpec  # noqa: F401
from .solver import OracleProblem  # noqa: F401
