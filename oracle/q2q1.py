"""Oracle for the paper's own discretisation (Section 5): Q2 velocity / Q1 pressure on bricks.

TEST INFRASTRUCTURE. Only tests/ may use this module. It is a plain, slow restatement of
Section 5 that the P1 hot path does not share: the CUDA library discretises with P1 tetrahedra,
and has no Q2/Q1 path.

Spaces (Section 5). The bricks K are the cells of the layered grid of oracle/mesh.py (active
columns x layers). Each is the image of the unit cube under its trilinear geometry map: x and y
affine, z = -h(x, y) (1 - s), with h bilinear over the cell (its four corner depths) and s the
sigma coordinate, linear in the third reference coordinate. Then
    V_h = {continuous, Q2 on every K}  (27 nodes per brick: corners, edge midpoints, face
                                        centres, centre),
    P_h = {continuous, Q1 on every K}  (the 8 corners: the grid's own nodes).
Q2 nodes are the half-step lattice (I, J, K), I = 0 .. 2(nx-1), J = 0 .. 2(ny-1),
K = 0 .. 2(nz-1), restricted to the closures of active cells; their coordinates are the geometry
map's images of the reference lattice. Numbering: Q2 lattice columns in row-major (J, I) order,
node = column * (2 nz - 1) + K. Q1 nodes are numbered as the P1 mesh's (column * nz + k).

Operators (each an integral over Omega, element by element):
    M2[a, b]   = int phi_a phi_b                  K2[a, b] = int (nu grad phi_a) . grad phi_b
    D_c[i, b]  = int psi_i d_c phi_b   (Q1 test, Q2 trial: int p div v = sum_c (D_c^T p)_b)
    B_c[b, i]  = int phi_b d_c psi_i   (Q2 test, Q1 trial: the gradient of q in Eq. fofa_velo_cor_h)
    K1[i, j]   = int grad psi_i . grad psi_j      M1[i, j] = int psi_i psi_j
    S2[a, b]   = int_{Gamma_s} phi_a phi_b        (the surface z = 0 is flat: area dx dy)
Integrals use 3-point Gauss-Legendre rules per direction. On bricks of constant depth every
integrand above is a polynomial of degree <= 5 per direction and the rule is exact; with a
varying depth the Jacobian determinant is bilinear (the mass is still exact) and the inverse
Jacobian rational, so stiffness and coupling integrals are the rule's values.

Boundary sets (Section 2), node by node as in oracle/mesh.py: Gamma_0 (u = 0) is the sea floor,
coastline columns and no-slip outer walls; Gamma_1 (u . n = 0) the slip outer walls; Gamma_s the
surface, where u3 = 0 and the wind tension acts on u1, u2. A Q2 lattice column is on the coast
when one of the cells whose closure holds it is inactive.

Step (Eqs. fofa_velo_pred_h, fofa_q_cor_h, fofa_pres_cor_h, fofa_velo_cor_h), the same sequence
as oracle/step.py:
  b_c = (1/dt) M2 (2 u^k_c - u^{k-1}_c / 2) - int ((u^k . grad) u^k_c) phi - Coriolis_c
        + (D_c^T p^k) + S2 theta_c (c = 1, 2), zero on component c's Dirichlet set
  (alpha M2 + K2) u~_c = b_c                    (symmetric Dirichlet elimination)
  K1 q = -alpha sum_c D_c u~_c,  m1' q = 0      (Lagrange-multiplier reading, m1 = M1 1)
  p^{k+1} = p^k + q
  M2 u_c = M2 u~_c - (1/alpha) B_c q            (the minus sign of Eq. correc_velo_u, as the P1
                                                 oracle reads Eq. fofa_velo_cor_h)
  u_c = 0 on component c's Dirichlet set.
alpha = 1/dt on a BDF1 start step and 3/(2 dt) after.

Pins (tests/test_oracle_q2q1.py): nodal and polynomial-reproduction properties of the bases,
the exact volume 1'M2 1 = 1'M1 1 of a sigma mesh, exact mass, stiffness and coupling integrals of
quadratic fields on a flat box against closed forms, the integration-by-parts identity linking
D_c and B_c, third-order (Q2) and second-order (Q1) convergence of manufactured solutions, and
the removal of a pure gradient by one projection.
"""
from __future__ import annotations

from dataclasses import dataclass
from typing import List, Optional

import numpy as np
import scipy.sparse as sp

from . import pcg as pcgm
from .mesh import WALL_EAST, WALL_NORTH, WALL_SOUTH, WALL_WEST, Mesh, build_mesh


# ---- reference elements --------------------------------------------------------------------------

def gauss_legendre(nq: int):
    """nq-point Gauss-Legendre points and weights on [0, 1]."""
    x, w = np.polynomial.legendre.leggauss(nq)
    return 0.5 * (x + 1.0), 0.5 * w


def lagrange2(t: np.ndarray):
    """1D quadratic Lagrange basis at nodes 0, 1/2, 1 and its derivative: two (3, len(t)) arrays."""
    t = np.asarray(t, dtype=float)
    val = np.stack([2.0 * (t - 0.5) * (t - 1.0), -4.0 * t * (t - 1.0), 2.0 * t * (t - 0.5)])
    der = np.stack([4.0 * t - 3.0, -8.0 * t + 4.0, 4.0 * t - 1.0])
    return val, der


def lagrange1(t: np.ndarray):
    """1D linear Lagrange basis at nodes 0, 1 and its derivative: two (2, len(t)) arrays."""
    t = np.asarray(t, dtype=float)
    return np.stack([1.0 - t, t]), np.stack([-np.ones_like(t), np.ones_like(t)])


# local node a of a brick: (ax, ay, az) in {0,1,2}^3 (Q2), a = ax + 3 ay + 9 az;
# local node v: (bx, by, bz) in {0,1}^3 (Q1), v = bx + 2 by + 4 bz
Q2_OFF = np.array([(a % 3, (a // 3) % 3, a // 9) for a in range(27)])
Q1_OFF = np.array([(v % 2, (v // 2) % 2, v // 4) for v in range(8)])


def tensor_basis(points: np.ndarray, order: int):
    """Values (P, nb) and reference gradients (P, nb, 3) of the Q_order basis at points (P, 3)."""
    f = lagrange2 if order == 2 else lagrange1
    off = Q2_OFF if order == 2 else Q1_OFF
    vals, ders = [], []
    for d in range(3):
        v, dv = f(points[:, d])
        vals.append(v)
        ders.append(dv)
    nb = len(off)
    phi = np.ones((len(points), nb))
    grad = np.ones((len(points), nb, 3))
    for a in range(nb):
        for d in range(3):
            phi[:, a] *= vals[d][off[a, d]]
            for e in range(3):
                grad[:, a, e] *= (ders[d] if d == e else vals[d])[off[a, d]]
    return phi, grad


def cube_rule(nq: int):
    """Tensor Gauss rule on the unit cube: points (nq^3, 3) and weights (nq^3,)."""
    t, w = gauss_legendre(nq)
    P = np.array([(t[i], t[j], t[k]) for k in range(nq) for j in range(nq) for i in range(nq)])
    W = np.array([w[i] * w[j] * w[k] for k in range(nq) for j in range(nq) for i in range(nq)])
    return P, W


# ---- mesh --------------------------------------------------------------------------------------

@dataclass
class MeshQ2:
    base: Mesh                 # the layered grid: Q1 nodes, cells, boundary classification
    nz2: int                   # 2 nz - 1 lattice levels
    n2: int                    # Q2 nodes
    n1: int                    # Q1 nodes
    col2_i: np.ndarray         # (ncols2,) lattice I of each Q2 column
    col2_j: np.ndarray
    colid2: np.ndarray         # (2ny-1, 2nx-1) Q2 column id or -1
    xyz2: np.ndarray           # (n2, 3)
    cells: np.ndarray          # (E, 3) cell (ci, cj, ck)
    e2: np.ndarray             # (E, 27) Q2 node ids
    e1: np.ndarray             # (E, 8) Q1 node ids
    corners: np.ndarray        # (E, 8, 3) corner coordinates (the geometry map)
    dirichlet: np.ndarray      # (3, n2) bool, Dirichlet set of velocity component c
    surface: np.ndarray        # (n2,) bool
    top_e: np.ndarray          # (F,) elements in the top layer (their faces make Gamma_s)


def build_mesh_q2(basin) -> MeshQ2:
    base = build_mesh(basin)
    nx, ny, nz = basin.nx, basin.ny, basin.nz
    cell = base.cell_active                                   # (ny-1, nx-1)
    nz2 = 2 * nz - 1
    lat = np.zeros((2 * ny - 1, 2 * nx - 1), dtype=bool)
    cj, ci = np.nonzero(cell)
    for dj in range(3):
        for di in range(3):
            lat[2 * cj + dj, 2 * ci + di] = True
    JJ, II = np.nonzero(lat)                                  # row-major (J, I)
    ncols2 = len(II)
    colid2 = -np.ones(lat.shape, dtype=np.int64)
    colid2[JJ, II] = np.arange(ncols2)
    n2 = ncols2 * nz2

    # depth of a lattice column: bilinear interpolation of the corner depths of a cell holding it
    # (the same value from every such cell: on a shared edge it is the edge's linear interpolant)
    d = basin.depth
    i0 = np.minimum(II // 2, nx - 2)
    j0 = np.minimum(JJ // 2, ny - 2)
    tx = (II - 2 * i0) / 2.0
    ty = (JJ - 2 * j0) / 2.0
    h2 = ((1 - tx) * (1 - ty) * d[j0, i0] + tx * (1 - ty) * d[j0, i0 + 1]
          + (1 - tx) * ty * d[j0 + 1, i0] + tx * ty * d[j0 + 1, i0 + 1])
    K = np.arange(nz2)
    node_col = np.repeat(np.arange(ncols2), nz2)
    node_K = np.tile(K, ncols2)
    xyz2 = np.empty((n2, 3))
    xyz2[:, 0] = II[node_col] * 0.5 * basin.dx
    xyz2[:, 1] = JJ[node_col] * 0.5 * basin.dy
    xyz2[:, 2] = -h2[node_col] * (1.0 - node_K / (2.0 * (nz - 1)))

    # elements: active cells x layers
    ck = np.arange(nz - 1)
    E_ci = np.repeat(ci, nz - 1)
    E_cj = np.repeat(cj, nz - 1)
    E_ck = np.tile(ck, len(ci))
    cells = np.stack([E_ci, E_cj, E_ck], axis=1)
    e2 = np.empty((len(E_ci), 27), dtype=np.int64)
    for a, (ax, ay, az) in enumerate(Q2_OFF):
        e2[:, a] = colid2[2 * E_cj + ay, 2 * E_ci + ax] * nz2 + 2 * E_ck + az
    e1 = np.empty((len(E_ci), 8), dtype=np.int64)
    for v, (bx, by, bz) in enumerate(Q1_OFF):
        e1[:, v] = base.colid[E_cj + by, E_ci + bx] * nz + E_ck + bz
    corners = base.xyz[e1]                                    # (E, 8, 3)

    # boundary sets
    def inside_cell(cj_, ci_):
        ok = (ci_ >= 0) & (ci_ < nx - 1) & (cj_ >= 0) & (cj_ < ny - 1)
        act = np.zeros_like(ok)
        act[ok] = cell[cj_[ok], ci_[ok]]
        return ok, act

    coast = np.zeros(ncols2, dtype=bool)
    for dcj in (-1, 0):
        for dci in (-1, 0):
            # cells (ci, cj) with 2 ci <= I <= 2 ci + 2: ci = ceil(I/2) - 1 .. floor(I/2)
            cci = np.where(dci == 0, II // 2, (II + 1) // 2 - 1)
            ccj = np.where(dcj == 0, JJ // 2, (JJ + 1) // 2 - 1)
            ok, act = inside_cell(ccj, cci)
            coast |= ok & ~act
    west, east = II == 0, II == 2 * (nx - 1)
    south, north = JJ == 0, JJ == 2 * (ny - 1)
    sw = basin.slip_walls
    slip = {w: bool(sw & w) for w in (WALL_WEST, WALL_EAST, WALL_SOUTH, WALL_NORTH)}
    noslip_wall = ((west & (not slip[WALL_WEST])) | (east & (not slip[WALL_EAST]))
                   | (south & (not slip[WALL_SOUTH])) | (north & (not slip[WALL_NORTH])))
    g0 = coast | noslip_wall
    g1x = ((west & slip[WALL_WEST]) | (east & slip[WALL_EAST])) & ~g0
    g1y = ((south & slip[WALL_SOUTH]) | (north & slip[WALL_NORTH])) & ~g0
    bottom = node_K == 0
    surface = node_K == nz2 - 1
    gamma0 = g0[node_col] | bottom
    dirichlet = np.zeros((3, n2), dtype=bool)
    dirichlet[0] = gamma0 | g1x[node_col]
    dirichlet[1] = gamma0 | g1y[node_col]
    dirichlet[2] = gamma0 | surface
    top_e = np.nonzero(E_ck == nz - 2)[0]
    return MeshQ2(base=base, nz2=nz2, n2=n2, n1=base.n, col2_i=II, col2_j=JJ, colid2=colid2, xyz2=xyz2,
                  cells=cells, e2=e2, e1=e1, corners=corners, dirichlet=dirichlet, surface=surface,
                  top_e=top_e)


# ---- element integrals ---------------------------------------------------------------------------

@dataclass
class Quadrature:
    W: np.ndarray        # (Q,) reference weights
    phi2: np.ndarray     # (Q, 27)
    phi1: np.ndarray     # (Q, 8)
    dV: np.ndarray       # (E, Q) weight x det J
    g2: np.ndarray       # (E, Q, 27, 3) physical gradients of the Q2 basis
    g1: np.ndarray       # (E, Q, 8, 3)


def element_quadrature(mesh: MeshQ2, nq: int = 3) -> Quadrature:
    """Basis values, physical gradients and weighted Jacobians at the Gauss points of every brick.
    J[i, j] = d X_i / d xi_j of the trilinear map X = sum_v N_v(xi) X_v; grad = J^{-T} grad_xi."""
    P, W = cube_rule(nq)
    phi2, d2 = tensor_basis(P, 2)
    phi1, d1 = tensor_basis(P, 1)
    J = np.einsum("evi,qvj->eqij", mesh.corners, d1)          # (E, Q, 3, 3)
    det = np.linalg.det(J)
    if np.any(det <= 0):
        raise ValueError("a brick's geometry map is not orientation preserving")
    Jinv = np.linalg.inv(J)
    g2 = np.einsum("eqji,qaj->eqai", Jinv, d2)
    g1 = np.einsum("eqji,qaj->eqai", Jinv, d1)
    return Quadrature(W=W, phi2=phi2, phi1=phi1, dV=det * W[None, :], g2=g2, g1=g1)


def assemble(n_rows: int, n_cols: int, rows: np.ndarray, cols: np.ndarray, elem: np.ndarray) -> sp.csr_matrix:
    """Sum element matrices elem (E, r, c) at (rows (E, r), cols (E, c)) into a CSR matrix."""
    R = np.broadcast_to(rows[:, :, None], elem.shape).ravel()
    C = np.broadcast_to(cols[:, None, :], elem.shape).ravel()
    A = sp.coo_matrix((np.ascontiguousarray(elem).ravel(), (R, C)), shape=(n_rows, n_cols)).tocsr()
    A.sum_duplicates()
    A.sort_indices()
    return A


def eliminate_dirichlet(A: sp.csr_matrix, mask: np.ndarray) -> sp.csr_matrix:
    """Symmetric elimination of homogeneous Dirichlet nodes (identity rows, zero columns)."""
    B = A.copy()
    rows = np.repeat(np.arange(B.shape[0]), np.diff(B.indptr))
    hit = mask[rows] | mask[B.indices]
    B.data[hit] = 0.0
    B.data[hit & (rows == B.indices)] = 1.0
    return B


@dataclass
class OperatorsQ2:
    mesh: MeshQ2
    quad: Quadrature
    nu: tuple
    dt: float
    M2: sp.csr_matrix
    K2: sp.csr_matrix
    D: List[sp.csr_matrix]     # (n1, n2) each
    B: List[sp.csr_matrix]     # (n2, n1) each
    K1: sp.csr_matrix
    M1: sp.csr_matrix
    S2: sp.csr_matrix
    coriolis: np.ndarray       # (n2,) f per Q2 node (bilinear in each cell from the grid's f)
    theta: np.ndarray          # (2, n2) kinematic wind tension per Q2 node

    def alpha(self, bdf1: bool) -> float:
        return 1.0 / self.dt if bdf1 else 1.5 / self.dt

    @property
    def m2(self) -> np.ndarray:
        return np.asarray(self.M2.sum(axis=1)).ravel()

    @property
    def m1(self) -> np.ndarray:
        return np.asarray(self.M1.sum(axis=1)).ravel()

    def A_u(self, c: int, bdf1: bool = False) -> sp.csr_matrix:
        A = (self.alpha(bdf1) * self.M2 + self.K2).tocsr()
        A.sort_indices()
        return eliminate_dirichlet(A, self.mesh.dirichlet[c])


def lattice_field(mesh: MeshQ2, grid: np.ndarray) -> np.ndarray:
    """Per-Q2-node values of a (ny, nx) grid field, bilinear over each cell, constant in depth."""
    nx = grid.shape[1]
    ny = grid.shape[0]
    I, J = mesh.col2_i, mesh.col2_j
    i0 = np.minimum(I // 2, nx - 2)
    j0 = np.minimum(J // 2, ny - 2)
    tx = (I - 2 * i0) / 2.0
    ty = (J - 2 * j0) / 2.0
    v = ((1 - tx) * (1 - ty) * grid[j0, i0] + tx * (1 - ty) * grid[j0, i0 + 1]
         + (1 - tx) * ty * grid[j0 + 1, i0] + tx * ty * grid[j0 + 1, i0 + 1])
    return np.repeat(v, mesh.nz2)


def surface_mass(mesh: MeshQ2, dx: float, dy: float, nq: int = 3) -> sp.csr_matrix:
    """int over Gamma_s of phi_a phi_b: the top faces (az = 2) of the top bricks, flat, area dx dy."""
    t, w = gauss_legendre(nq)
    v, _ = lagrange2(t)                                        # (3, nq)
    face = [a for a in range(27) if Q2_OFF[a, 2] == 2]         # 9 nodes of the top face
    phi = np.array([[v[Q2_OFF[a, 0], i] * v[Q2_OFF[a, 1], j] for a in face]
                    for j in range(nq) for i in range(nq)])    # (nq^2, 9)
    W = np.array([w[i] * w[j] for j in range(nq) for i in range(nq)]) * dx * dy
    Se = np.einsum("q,qa,qb->ab", W, phi, phi)
    ids = mesh.e2[mesh.top_e][:, face]
    return assemble(mesh.n2, mesh.n2, ids, ids, np.broadcast_to(Se, (len(ids), 9, 9)))


def assemble_q2q1(basin, nq: int = 3) -> OperatorsQ2:
    mesh = build_mesh_q2(basin)
    q = element_quadrature(mesh, nq)
    e2, e1 = mesh.e2, mesh.e1
    n2, n1 = mesh.n2, mesh.n1
    nu = tuple(basin.nu)
    M2e = np.einsum("eq,qa,qb->eab", q.dV, q.phi2, q.phi2)
    K2e = sum(nu[c] * np.einsum("eq,eqa,eqb->eab", q.dV, q.g2[..., c], q.g2[..., c]) for c in range(3))
    M1e = np.einsum("eq,qa,qb->eab", q.dV, q.phi1, q.phi1)
    K1e = np.einsum("eq,eqac,eqbc->eab", q.dV, q.g1, q.g1)
    D = [assemble(n1, n2, e1, e2, np.einsum("eq,qi,eqb->eib", q.dV, q.phi1, q.g2[..., c])) for c in range(3)]
    B = [assemble(n2, n1, e2, e1, np.einsum("eq,qb,eqi->ebi", q.dV, q.phi2, q.g1[..., c])) for c in range(3)]
    M2 = assemble(n2, n2, e2, e2, M2e)
    K2 = assemble(n2, n2, e2, e2, K2e)
    K1 = assemble(n1, n1, e1, e1, K1e)
    M1 = assemble(n1, n1, e1, e1, M1e)
    S2 = surface_mass(mesh, basin.dx, basin.dy)
    cor = lattice_field(mesh, basin.coriolis) if basin.coriolis is not None else np.zeros(n2)
    th = np.zeros((2, n2))
    if basin.theta is not None:
        th[0] = lattice_field(mesh, basin.theta[0])
        th[1] = lattice_field(mesh, basin.theta[1])
    return OperatorsQ2(mesh=mesh, quad=q, nu=nu, dt=float(basin.dt), M2=M2, K2=K2, D=D, B=B, K1=K1, M1=M1,
                       S2=S2, coriolis=cor, theta=th)


# ---- the projection step -------------------------------------------------------------------------

def advection_term(ops: OperatorsQ2, u: np.ndarray) -> np.ndarray:
    """(3, n2): int ((u . grad) u_c) phi_b by the element rule."""
    q = ops.quad
    e2 = ops.mesh.e2
    uloc = u[:, e2]                                            # (3, E, 27)
    uq = np.einsum("qa,dea->deq", q.phi2, uloc)                # u_d at the points
    gu = np.einsum("eqad,cea->ceqd", q.g2, uloc)               # d_d u_c at the points
    conv = np.einsum("deq,ceqd->ceq", uq, gu)                  # (u . grad) u_c
    loc = np.einsum("eq,ceq,qb->ceb", q.dV, conv, q.phi2)
    out = np.zeros((3, ops.mesh.n2))
    for c in range(3):
        np.add.at(out[c], e2.ravel(), loc[c].ravel())
    return out


def velocity_rhs(ops: OperatorsQ2, u_k, u_km1, p_k, bdf1: bool) -> np.ndarray:
    """(3, n2) right-hand sides of Eq. fofa_velo_pred_h, Dirichlet rows zeroed (see the module
    docstring; Coriolis 2 omega ^ u = f (-u2, u1, 0) with f nodal, as oracle/fem.py)."""
    M = ops.M2
    if bdf1:
        b = np.stack([M @ u_k[c] for c in range(3)]) / ops.dt
    else:
        b = np.stack([M @ (2.0 * u_k[c] - 0.5 * u_km1[c]) for c in range(3)]) / ops.dt
    b -= advection_term(ops, u_k)
    f = ops.coriolis
    b[0] += f * (M @ u_k[1])
    b[1] -= f * (M @ u_k[0])
    for c in range(3):
        b[c] += ops.D[c].T @ p_k
    surf = ops.mesh.surface
    for c in range(2):
        b[c] += ops.S2 @ np.where(surf, ops.theta[c], 0.0)
    for c in range(3):
        b[c][ops.mesh.dirichlet[c]] = 0.0
    return b


@dataclass
class StateQ2:
    u: np.ndarray          # (3, n2)
    u_prev: np.ndarray     # (3, n2)
    p: np.ndarray          # (n1,)
    q: np.ndarray          # (n1,)
    step: int = 0


def initial_state(ops: OperatorsQ2) -> StateQ2:
    n2, n1 = ops.mesh.n2, ops.mesh.n1
    return StateQ2(u=np.zeros((3, n2)), u_prev=np.zeros((3, n2)), p=np.zeros(n1), q=np.zeros(n1))


def pressure_increment(ops: OperatorsQ2, ut: np.ndarray, bdf1: bool, x0=None, rtol: float = 1e-12):
    """Eq. fofa_q_cor_h: K1 q = -alpha sum_c D_c u~_c on the mean-zero subspace (PCG, Jacobi)."""
    bp = -ops.alpha(bdf1) * sum(ops.D[c] @ ut[c] for c in range(3))
    res = pcgm.pressure_solve(ops.K1, ops.m1, bp, x0=x0, rtol=rtol,
                              precond=pcgm.jacobi_preconditioner(ops.K1))
    return bp, res


def correct_velocity(ops: OperatorsQ2, ut: np.ndarray, q: np.ndarray, a: float, lumped: bool = True,
                     rtol: float = 1e-12) -> np.ndarray:
    """Eq. fofa_velo_cor_h with the sign of Eq. correc_velo_u: M2 u_c = M2 u~_c - (1/alpha) B_c q,
    with the row-sum lumped M2 (positive on bricks) or the consistent M2 by PCG."""
    out = np.zeros_like(ut)
    for c in range(3):
        g = ops.B[c] @ q
        if lumped:
            out[c] = ut[c] - g / (a * ops.m2)
        else:
            res = pcgm.pcg(ops.M2, ops.M2 @ ut[c] - g / a, x0=ut[c], rtol=rtol,
                           precond=pcgm.jacobi_preconditioner(ops.M2))
            out[c] = res.x
    return out


def discrete_divergence(ops: OperatorsQ2, u: np.ndarray) -> np.ndarray:
    """sum_c D_c u_c: int div(u) psi_i for every pressure basis function."""
    return sum(ops.D[c] @ u[c] for c in range(3))


def project_step(ops: OperatorsQ2, st: StateQ2, vel_rtol: float = 1e-12, pres_rtol: float = 1e-12,
                 lumped: bool = True) -> dict:
    """One step k -> k+1 (module docstring). Returns the prediction and the solves' results."""
    bdf1 = st.step == 0
    a = ops.alpha(bdf1)
    b = velocity_rhs(ops, st.u, st.u_prev, st.p, bdf1)
    ut = np.zeros_like(st.u)
    vel = []
    for c in range(3):
        A = ops.A_u(c, bdf1)
        res = pcgm.pcg(A, b[c], x0=st.u[c], rtol=vel_rtol, precond=pcgm.jacobi_preconditioner(A))
        ut[c] = res.x
        vel.append(res)
    _, pres = pressure_increment(ops, ut, bdf1, x0=st.q, rtol=pres_rtol)
    q = pres.x
    u_new = correct_velocity(ops, ut, q, a, lumped=lumped, rtol=vel_rtol)
    for c in range(3):
        u_new[c][ops.mesh.dirichlet[c]] = 0.0
    st.u_prev, st.u = st.u, u_new
    st.p = st.p + q
    st.q = q
    st.step += 1
    return {"u_tilde": ut, "vel": vel, "pres": pres, "b": b}
