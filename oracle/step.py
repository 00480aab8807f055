"""Oracle BDF2 velocity-correction projection step (Section 3, discretised as in Section 5).

One step k -> k+1 (Eqs. fofa_velo_pred_h, fofa_q_cor_h, fofa_pres_cor_h, fofa_velo_cor_h):
  1. b_c = velocity right-hand side (fem.velocity_rhs), c = 1, 2, 3
  2. solve (alpha M + K_nu) u~_c = b_c with component c's Dirichlet set (PCG, IC0 by default;
     x0 = u^k_c)
  3. b_p = -alpha sum_c G_c u~_c
  4. solve K_I q = b_p for mean-zero q (Lagrange-multiplier reading; PCG, Jacobi = DIAG)
  5. p^{k+1} = p^k + q   (Eq. fofa_pres_cor_h: q and p^k lie in P_h, so the L2 projection is
     the identity)
  6. u_c = u~_c + (1/alpha) M^{-1} G_c q, then u_c = 0 on component c's Dirichlet set
     (lumped M_L = diag(M 1) by default; the consistent M solved by PCG on request)
alpha = 1/dt on the first step (BDF1 start, the paper leaves u^1 unspecified) and 3/(2 dt)
after. Parity of the step as a whole is pinned through its parts (operators, solves) and the
invariant that a basin at rest with no forcing stays at rest.
"""
from __future__ import annotations

from dataclasses import dataclass, field
from typing import Optional

import numpy as np

from . import fem, pcg as pcgm
from .mesh import Mesh


@dataclass
class State:
    u: np.ndarray        # (3, n) u^k
    u_prev: np.ndarray   # (3, n) u^{k-1}
    p: np.ndarray        # (n,) p^k
    q: np.ndarray        # (n,) last pressure increment (warm start)
    step: int = 0


def initial_state(n: int) -> State:
    """u^0 = 0 (Eq. prim_ci), p^0 = 0."""
    return State(u=np.zeros((3, n)), u_prev=np.zeros((3, n)), p=np.zeros(n), q=np.zeros(n))


@dataclass
class StepOptions:
    vel_rtol: float = 1e-8
    pres_rtol: float = 1e-8
    vel_prec: str = "ic0"          # "ic0" (multicolour), "ic0_natural", "jacobi"
    pres_prec: str = "jacobi"      # "jacobi" (DIAG), "ic0"
    lumped_correction: bool = True
    mass_prec: str = "ic0"
    max_iter: int = 200000


@dataclass
class StepReport:
    vel: list = field(default_factory=list)
    pres: Optional[pcgm.SolveResult] = None
    mass: list = field(default_factory=list)
    u_tilde: Optional[np.ndarray] = None
    b_vel: Optional[np.ndarray] = None
    b_p: Optional[np.ndarray] = None


def _precond(A, kind: str, mesh: Mesh):
    if kind == "jacobi":
        return pcgm.jacobi_preconditioner(A)
    if kind == "ic0":
        return pcgm.ic0_preconditioner(A, mesh.colour)[0]
    if kind == "ic0_natural":
        return pcgm.ic0_preconditioner(A, None)[0]
    if kind == "line":
        return pcgm.line_preconditioner(A, mesh.nz)
    raise ValueError(kind)


def project_step(ops: fem.Operators, st: State, opts: StepOptions = StepOptions()) -> StepReport:
    mesh = ops.mesh
    bdf1 = st.step == 0
    a = ops.alpha(bdf1)
    rep = StepReport()
    b = fem.velocity_rhs(ops, st.u, st.u_prev, st.p, bdf1)
    rep.b_vel = b
    ut = np.zeros_like(st.u)
    for c in range(3):
        A = ops.A_u(c, bdf1)
        res = pcgm.pcg(A, b[c], x0=st.u[c], rtol=opts.vel_rtol, max_iter=opts.max_iter,
                       precond=_precond(A, opts.vel_prec, mesh))
        ut[c] = res.x
        rep.vel.append(res)
    rep.u_tilde = ut
    bp = fem.divergence_rhs(ops, ut, bdf1)
    rep.b_p = bp
    K = ops.A_p()
    pres = pcgm.pressure_solve(K, ops.m, bp, x0=st.q, rtol=opts.pres_rtol, max_iter=opts.max_iter,
                               precond=_precond(K, opts.pres_prec, mesh))
    rep.pres = pres
    q = pres.x
    p_new = st.p + q
    u_new = np.zeros_like(ut)
    if opts.lumped_correction:
        ml = ops.m
        for c in range(3):
            u_new[c] = ut[c] + (ops.G[c] @ q) / (a * ml)
    else:
        for c in range(3):
            rhs = ops.M @ ut[c] + (ops.G[c] @ q) / a
            res = pcgm.pcg(ops.M, rhs, x0=ut[c], rtol=opts.vel_rtol, max_iter=opts.max_iter,
                           precond=_precond(ops.M, opts.mass_prec, mesh))
            u_new[c] = res.x
            rep.mass.append(res)
    for c in range(3):
        u_new[c][mesh.dirichlet[c]] = 0.0
    st.u_prev = st.u
    st.u = u_new
    st.p = p_new
    st.q = q
    st.step += 1
    return rep
