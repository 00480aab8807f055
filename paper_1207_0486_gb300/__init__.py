"""GB300-native projection-method FEM solver for thin ocean basins.

The hot path -- P1 assembly on a layered Kuhn-tet mesh, PCG solves of the velocity prediction
and pressure increment systems, and the BDF2 velocity-correction step (Besson & Straubhaar,
Sections 3-5) -- runs in hand-written sm_103a CUDA kernels behind the C ABI of include/pm.h.
This package is the thin Python binding (`api`) and the in-tree build (`build`).
"""
from .api import (  # noqa: F401
    Operator, State, Options, SolveStats, PMError, Batch, Server, debug_barrier_timeout,
    assemble_operator, pcg_solve, project_step, operator_bytes, kernel_launch_count, load,
    select_library, set_log, build_flags, PM_BUILD_CHECKED,
    OP_VEL_U1, OP_VEL_U2, OP_VEL_U3, OP_PRESSURE, OP_MASS, OP_VEL1_U1, OP_VEL1_U2, OP_VEL1_U3,
    OP_GRAD_X, OP_GRAD_Y, OP_GRAD_Z, PREC_JACOBI, PREC_IC0, PREC_NONE, PREC_LINE, PREC_DEFAULT, FP64, FP32_REFINE,
    BF16_REFINE, STEP_LUMPED, STEP_CONSISTENT, SLOT_OFFSETS, NBR_OFFSETS,
    FIELD_U1, FIELD_U2, FIELD_U3, FIELD_U1_PREV, FIELD_U2_PREV, FIELD_U3_PREV, FIELD_P, FIELD_Q,
    FIELD_UT1, FIELD_UT2, FIELD_UT3, FIELD_BP, DIAG_NAMES, KERNEL_AUTO, KERNEL_STREAM, KERNEL_RESIDENT,
    PM_OK, PM_EINVAL, PM_ENOMEM, PM_ECUDA, PM_NOT_CONVERGED, PM_BREAKDOWN, PM_TIMEOUT,
    PM_DISCONNECTED, PM_EBUSY, PM_EBOUNDS,
)
