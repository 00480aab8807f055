"""Plain FP64 CPU oracle of the projection-method FEM (test infrastructure only).

This package is the independent reference the CUDA path is checked against. It is slow and
written to be read against the paper: the P1 tetrahedral discretisation of the weak forms
(Sections 4 and 5), the BDF2 velocity-correction projection step (Section 3) and the
preconditioned conjugate gradient solves with the preconditioners of the Section 5 remark.

Only the tests, the smoke check and the bench's CPU-baseline leg may import it. It shares no
code with the CUDA library: its one native part, ``ic0.c`` (incomplete Cholesky factor and
triangular sweeps on CSR), is compiled on its own by ``oracle.native.build()``.

``q2q1`` restates the paper's own discretisation of Section 5 (Q2 velocity and Q1 pressure on
bricks, the same projection step) for tests only; the CUDA library discretises with P1 tetrahedra
and has no Q2/Q1 path.

Parity status per function is stated in each module header. The "DIAG + LS CGS OPT" pressure
preconditioner of the Section 5 remark is not defined in the paper: parity unpinned, and not
implemented here.
"""
from . import mesh, fem, pcg, step, q2q1  # noqa: F401
