"""Oracle BDF2 velocity-correction projection step (Section 3, discretised as in Section 5).

One step k -> k+1 (Eqs. fofa_velo_pred_h, fofa_q_cor_h, fofa_pres_cor_h, fofa_velo_cor_h):
  1. b_c = velocity right-hand side (fem.velocity_rhs), c = 1, 2, 3
  2. solve (alpha M + K_nu) u~_c = b_c with component c's Dirichlet set (PCG, IC0 by default;
     x0 = u^k_c)
  3. b_p = -alpha sum_c G_c u~_c
  4. solve K_I q = b_p for mean-zero q (Lagrange-multiplier reading; PCG, Jacobi = DIAG)
  5. p^{k+1} = p^k + q   (Eq. fofa_pres_cor_h: q and p^k lie in P_h, so the L2 projection is
     the identity)
  6. u_c = u~_c - (1/alpha) M^{-1} G_c q, then u_c = 0 on component c's Dirichlet set
     (lumped M_L = diag(M 1) by default; the consistent M solved by PCG on request)
alpha = 1/dt on the first step (BDF1 start, the paper leaves u^1 unspecified) and 3/(2 dt)
after.

Sign of the correction. Eq. correc_velo_u, (3/(2 dt)) (u^{k+1} - u~^{k+1}) + grad q = 0, gives
u^{k+1} = u~^{k+1} - (2 dt / 3) grad q, and Eq. press_cor (-Lap q = -(3/(2 dt)) div u~) follows
from it and div u^{k+1} = 0 only with that minus sign. The closing formula of Section 3 and
Eq. fofa_velo_cor_h print "+ dt (2/3) grad q"; read literally, the correction would add the
gradient instead of removing it and double the divergence it is meant to cancel. The oracle
takes the minus sign that Eqs. correc_velo_u and press_cor fix.

Pins (tests/test_oracle_step.py): one projection of a pure gradient field grad(phi) with
d phi / dn = 0 on a cube removes it up to the discretisation error (the plus sign would double
it), the corrected velocity of a wind-driven step has a smaller discrete divergence
sum_c G_c u_c than the prediction, and a basin at rest with no forcing stays at rest.
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
    pres_prec: str = "jacobi"      # "jacobi" (DIAG), "ic0", "line"
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


def pressure_increment(ops: fem.Operators, ut: np.ndarray, bdf1: bool, x0: Optional[np.ndarray],
                       opts: StepOptions) -> "tuple[np.ndarray, pcgm.SolveResult]":
    """Steps 3-4: b_p = -alpha sum_c G_c u~_c (Eq. fofa_q_cor_h) and the mean-zero solve of
    K_I q = b_p (Lagrange-multiplier reading). Returns (b_p, result)."""
    bp = fem.divergence_rhs(ops, ut, bdf1)
    K = ops.A_p()
    res = pcgm.pressure_solve(K, ops.m, bp, x0=x0, rtol=opts.pres_rtol, max_iter=opts.max_iter,
                              precond=_precond(K, opts.pres_prec, ops.mesh))
    return bp, res


def correct_velocity(ops: fem.Operators, ut: np.ndarray, q: np.ndarray, a: float,
                     opts: StepOptions) -> "tuple[np.ndarray, list]":
    """Step 6 before the Dirichlet sets: the L2 projection of u~_c - (1/alpha) grad q onto the
    velocity space (Eq. fofa_velo_cor_h with the sign of Eq. correc_velo_u),
        M u_c = M u~_c - (1/alpha) G_c q,
    with the lumped mass M_L = diag(M 1) (opts.lumped_correction) or the consistent M by PCG.
    Returns (u, mass-solve results)."""
    u_new = np.zeros_like(ut)
    mass = []
    if opts.lumped_correction:
        ml = ops.m
        for c in range(3):
            u_new[c] = ut[c] - (ops.G[c] @ q) / (a * ml)
    else:
        for c in range(3):
            rhs = ops.M @ ut[c] - (ops.G[c] @ q) / a
            res = pcgm.pcg(ops.M, rhs, x0=ut[c], rtol=opts.vel_rtol, max_iter=opts.max_iter,
                           precond=_precond(ops.M, opts.mass_prec, ops.mesh))
            u_new[c] = res.x
            mass.append(res)
    return u_new, mass


def discrete_divergence(ops: fem.Operators, u: np.ndarray) -> np.ndarray:
    """sum_c G_c u_c: the integral of div(u) against each basis function."""
    return sum(ops.G[c] @ u[c] for c in range(3))


def diagnostics(ops: fem.Operators, st: State, u_tilde: Optional[np.ndarray] = None) -> dict:
    """Monitors of the time loop (no paper counterpart): kinetic energy (1/2) sum_c u_c' M u_c,
    ||sum_c G_c u_c||_2 for u^k and for the last prediction u~ (the quantity the correction of
    Eq. correc_velo_u reduces), and the mean pressure m'p / 1'm."""
    ut = np.zeros_like(st.u) if u_tilde is None else u_tilde
    return {"kinetic_energy": 0.5 * float(sum(st.u[c] @ (ops.M @ st.u[c]) for c in range(3))),
            "div_u": float(np.linalg.norm(discrete_divergence(ops, st.u))),
            "div_u_tilde": float(np.linalg.norm(discrete_divergence(ops, ut))),
            "p_mean": float(ops.m @ st.p) / float(ops.m.sum())}


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
    bp, pres = pressure_increment(ops, ut, bdf1, st.q, opts)
    rep.b_p = bp
    rep.pres = pres
    q = pres.x
    p_new = st.p + q
    u_new, rep.mass = correct_velocity(ops, ut, q, a, opts)
    for c in range(3):
        u_new[c][mesh.dirichlet[c]] = 0.0
    st.u_prev = st.u
    st.u = u_new
    st.p = p_new
    st.q = q
    st.step += 1
    return rep
