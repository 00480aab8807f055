"""Oracle P1 finite element operators and right-hand sides, in plain FP64 (numpy + scipy.sparse).

Discrete problems (Section 5, Eqs. fofa_velo_pred_h to fofa_velo_cor_h) on P1 tetrahedra:
  velocity prediction  (alpha M + K_nu) u~_c = b_c        (Eq. fofa_velo_pred_h)
  pressure increment   K_I q = -alpha sum_c G_c u~_c       (Eq. fofa_q_cor_h)
  velocity correction  M u_c = M u~_c - (1/alpha) G_c q    (Eq. fofa_velo_cor_h, with the sign of
                                                            Eq. correc_velo_u)
with alpha = 3/(2 dt) for BDF2 (Eq. pred_velo) and alpha = 1/dt for the BDF1 start step.
Element integrals (exact for P1 on a tetrahedron K with barycentric gradients grad phi_i):
  mass       M^K_ij   = |K| (1 + delta_ij) / 20
  stiffness  K^K_ij   = |K| sum_d nu_d d_d phi_i d_d phi_j   (Delta_nu of Section 2; nu = I for K_I)
  gradient   G^K_c,ij = |K| d_c phi_j / 4                    (integral of d_c phi_j phi_i)
  surface    S^F_ij   = |F| (1 + delta_ij) / 12              (wind tension on Gamma_s)
Global matrices are plain sums over elements (scipy COO -> CSR, duplicates summed). Dirichlet
conditions are homogeneous (Eqs. pred_cl_0, pred_cl_1_u, pred_tr_3), imposed by symmetric
elimination: constrained rows and columns zeroed, unit diagonal, zero right-hand side.

Pins (tests/test_oracle_fem.py): reference-tet closed forms, symmetry, K 1 = 0, 1'M1 = |Omega|
(closed-form sigma-mesh volume), G_c 1 = 0, G_c X_d = delta_cd M 1, advection of a linear
field by a constant velocity, and second-order convergence to manufactured solutions.
"""
from __future__ import annotations

from dataclasses import dataclass
from typing import List, Optional

import numpy as np
import scipy.sparse as sp

from .mesh import Mesh, column_field


def tet_geometry(xyz: np.ndarray, tets: np.ndarray):
    """Volumes |K| (T,) and barycentric gradients grad phi (T, 4, 3) of each tetrahedron."""
    X = xyz[tets]                         # (T, 4, 3)
    J = X[:, 1:, :] - X[:, :1, :]         # rows: v_a - v_0, a = 1..3
    vol = np.abs(np.linalg.det(J)) / 6.0
    Jinv = np.linalg.inv(J)
    grads = np.empty((len(tets), 4, 3))
    # lambda = E^{-1} (x - v0) with E = J^T, so grad lambda_a = row a of E^{-1} = column a of J^{-1}
    grads[:, 1:, :] = np.transpose(Jinv, (0, 2, 1))
    grads[:, 0, :] = -grads[:, 1:, :].sum(axis=1)
    return vol, grads


def element_mass(vol):
    e = (np.ones((4, 4)) + np.eye(4)) / 20.0
    return vol[:, None, None] * e[None]


def element_stiffness(vol, grads, nu):
    g = grads * np.asarray(nu, dtype=float)[None, None, :]
    return vol[:, None, None] * np.einsum("tid,tjd->tij", g, grads)


def element_gradient(vol, grads, c):
    # row i (test function phi_i), column j (trial d_c phi_j): |K| d_c phi_j / 4
    return np.broadcast_to((vol / 4.0)[:, None, None] * grads[:, None, :, c], (len(vol), 4, 4))


def assemble_matrix(n: int, tets: np.ndarray, elem: np.ndarray) -> sp.csr_matrix:
    rows = np.broadcast_to(tets[:, :, None], elem.shape).ravel()
    cols = np.broadcast_to(tets[:, None, :], elem.shape).ravel()
    A = sp.coo_matrix((np.ascontiguousarray(elem).ravel(), (rows, cols)), shape=(n, n)).tocsr()
    A.sum_duplicates()
    A.sort_indices()
    return A


def eliminate_dirichlet(A: sp.csr_matrix, mask: np.ndarray) -> sp.csr_matrix:
    """Symmetric elimination of homogeneous Dirichlet nodes, keeping A's sparsity pattern."""
    B = A.copy()
    rows = np.repeat(np.arange(B.shape[0]), np.diff(B.indptr))
    cols = B.indices
    hit = mask[rows] | mask[cols]
    B.data[hit] = 0.0
    B.data[hit & (rows == cols)] = 1.0
    return B


@dataclass
class Operators:
    mesh: Mesh
    nu: tuple
    dt: float
    vol: np.ndarray
    grads: np.ndarray
    M: sp.csr_matrix
    K_nu: sp.csr_matrix
    K_I: sp.csr_matrix
    G: List[sp.csr_matrix]
    S: sp.csr_matrix            # surface mass on Gamma_s
    coriolis: np.ndarray        # (n,) f per node (constant along columns)
    theta: np.ndarray           # (2, n) kinematic wind tension per node (used on Gamma_s)

    @property
    def n(self):
        return self.mesh.n

    @property
    def m(self):
        """m = M 1 (the row sums of the consistent mass, i.e. integral of each basis function)."""
        return np.asarray(self.M.sum(axis=1)).ravel()

    def alpha(self, bdf1: bool) -> float:
        return 1.0 / self.dt if bdf1 else 1.5 / self.dt

    def A_u(self, c: int, bdf1: bool = False) -> sp.csr_matrix:
        """Velocity prediction operator alpha M + K_nu with component c's Dirichlet elimination."""
        A = (self.alpha(bdf1) * self.M + self.K_nu).tocsr()
        A.sort_indices()
        return eliminate_dirichlet(A, self.mesh.dirichlet[c])

    def A_p(self) -> sp.csr_matrix:
        """Pressure increment operator: the pure-Neumann Laplacian K_I."""
        return self.K_I


def assemble(basin, mesh: Optional[Mesh] = None) -> Operators:
    from .mesh import build_mesh
    mesh = build_mesh(basin) if mesh is None else mesh
    vol, grads = tet_geometry(mesh.xyz, mesh.tets)
    n = mesh.n
    M = assemble_matrix(n, mesh.tets, element_mass(vol))
    K_nu = assemble_matrix(n, mesh.tets, element_stiffness(vol, grads, basin.nu))
    K_I = assemble_matrix(n, mesh.tets, element_stiffness(vol, grads, (1.0, 1.0, 1.0)))
    G = [assemble_matrix(n, mesh.tets, element_gradient(vol, grads, c)) for c in range(3)]

    F = mesh.top_faces
    P = mesh.xyz[F]
    area = 0.5 * np.linalg.norm(np.cross(P[:, 1] - P[:, 0], P[:, 2] - P[:, 0]), axis=1)
    se = area[:, None, None] * ((np.ones((3, 3)) + np.eye(3)) / 12.0)[None]
    S = assemble_matrix(n, F, se)

    cor = column_field(mesh, basin.coriolis) if basin.coriolis is not None else np.zeros(n)
    th = np.zeros((2, n))
    if basin.theta is not None:
        th[0] = column_field(mesh, basin.theta[0])
        th[1] = column_field(mesh, basin.theta[1])
    return Operators(mesh=mesh, nu=tuple(basin.nu), dt=float(basin.dt), vol=vol, grads=grads, M=M,
                     K_nu=K_nu, K_I=K_I, G=G, S=S, coriolis=cor, theta=th)


# ----------------------------------------------------------------------------------------------
# Right-hand side of the velocity prediction (Eq. fofa_velo_pred_h), component by component.
# ----------------------------------------------------------------------------------------------

def advection_term(ops: Operators, u: np.ndarray) -> np.ndarray:
    """(3, n): integral over Omega of ((u . grad) u_c) phi_i, exact for P1 fields.

    On each tet grad u_c is constant and u_d is linear, so the integral is
    sum_d (d_d u_c)|_K (M^K u_d)_i.
    """
    tets = ops.mesh.tets
    Me = element_mass(ops.vol)                                   # (T, 4, 4)
    uloc = u[:, tets]                                            # (3, T, 4)
    gu = np.einsum("ctj,tjd->tcd", uloc, ops.grads)              # (T, c, d): d_d u_c on K
    Mu = np.einsum("tij,dtj->tdi", Me, uloc)                     # (T, d, i): (M^K u_d)_i
    loc = np.einsum("tcd,tdi->cti", gu, Mu)                      # (c, T, i)
    out = np.zeros((3, ops.n))
    for c in range(3):
        np.add.at(out[c], tets.ravel(), loc[c].ravel())
    return out


def velocity_rhs(ops: Operators, u_k: np.ndarray, u_km1: np.ndarray, p_k: np.ndarray,
                 bdf1: bool) -> np.ndarray:
    """(3, n) right-hand sides b_c of the velocity prediction, Dirichlet rows zeroed.

    b_c = (1/dt) M (2 u^k_c - u^{k-1}_c / 2)      (BDF2; BDF1 start: (1/dt) M u^k_c)
          - int ((u^k . grad) u^k_c) phi_i         (advection)
          - int (2 omega ^ u^k)_c phi_i            (Coriolis, 2 omega ^ u = f (-u2, u1, 0),
                                                    f taken nodally: f_i (M u)_i)
          + int p^k d_c phi_i = (G_c^T p^k)_i      (pressure)
          + int_{Gamma_s} theta_c phi_i            (wind tension, c = 1, 2; theta P1 on Gamma_s)
    """
    dt = ops.dt
    M = ops.M
    if bdf1:
        b = np.stack([M @ u_k[c] for c in range(3)]) / dt
    else:
        b = np.stack([M @ (2.0 * u_k[c] - 0.5 * u_km1[c]) for c in range(3)]) / dt
    b -= advection_term(ops, u_k)
    f = ops.coriolis
    b[0] += f * (M @ u_k[1])
    b[1] -= f * (M @ u_k[0])
    for c in range(3):
        b[c] += ops.G[c].T @ p_k
    surf = ops.mesh.surface
    for c in range(2):
        b[c] += ops.S @ np.where(surf, ops.theta[c], 0.0)
    for c in range(3):
        b[c][ops.mesh.dirichlet[c]] = 0.0
    return b


def divergence_rhs(ops: Operators, u_tilde: np.ndarray, bdf1: bool) -> np.ndarray:
    """Right-hand side of Eq. fofa_q_cor_h: -alpha int div(u~) phi_i = -alpha sum_c (G_c u~_c)_i."""
    a = ops.alpha(bdf1)
    return -a * sum(ops.G[c] @ u_tilde[c] for c in range(3))
