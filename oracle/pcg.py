"""Oracle preconditioned conjugate gradient and preconditioners (FP64).

PCG (Section 5 remark: the linear systems are solved by preconditioned conjugate gradients), in
the textbook order of Saad's preconditioned CG:
    r0 = b - A x0, z0 = P^{-1} r0, p0 = z0
    for j = 0, 1, ...:
        w = A p_j;  alpha_j = (r_j, z_j) / (w, p_j)
        x_{j+1} = x_j + alpha_j p_j;  r_{j+1} = r_j - alpha_j w
        stop when ||r_{j+1}||_2 <= rtol ||b||_2
        z_{j+1} = P^{-1} r_{j+1};  beta_j = (r_{j+1}, z_{j+1}) / (r_j, z_j)
        p_{j+1} = z_{j+1} + beta_j p_j
At exit the true residual ||b - A x|| / ||b|| is computed; if it exceeds rtol the iteration
restarts from the true residual (at most max_restarts times). b = 0 returns x = 0.
Every true residual r = b - A x (start, restarts, exit) is computed with the compensated dot
product Dot2 of Ogita, Rump and Oishi ("Accurate sum and dot product", SIAM J. Sci. Comput. 26,
2005): each product a_ij x_j is split exactly into p + e (TwoProduct, with Veltkamp-Dekker
splitting), the p are summed by TwoSum and every rounding error is carried, so r is as accurate
as if b - A x were formed in twice the working precision and then rounded. The plain FP64
residual of a nearly converged x is itself wrong by up to u || |A||x| ||, which on the thin
basins' pressure system is of the order of the target.
The paper states no stopping rule. Besides rtol, a solve is accepted when its (exact) true
residual is below the floor that rounding x to FP64 alone can cause,
u || |A||x| + |b| ||_2 / ||b||_2 with u = 2^-53 (backward error at the unit roundoff), and
restarts no longer lower it: a restart that does not halve the true residual, or the last
restart allowed. On the thin ocean basins' pressure system this floor is near 1e-7, above a
1e-8 target.

Preconditioners:
  Jacobi ("DIAG" of the Section 5 remark, and the labelled fallback): P = diag(A).
  IC0 (Section 5 remark, for the velocity and mass systems): incomplete Cholesky with zero
    fill on the pattern of A, in multicolour order (colour = (i&1) | (j&1)<<1 | (k&1)<<2 of the
    node's grid indices; no stencil edge joins two nodes of one colour) or in natural order.
    A non-positive pivot retries with A + s diag(A), s = 1e-3 * 2^m, m = 0..10 (shifted IC).
Pressure (Section 5 remark, zero-mean Lagrange multiplier): the augmented system
  [K_I m; m' 0][q; lambda] = [b; 0] with m = M 1 gives lambda = 1'b / 1'm; CG solves
  K_I q = b - lambda m (now consistent) and q is shifted to m'q = 0.

Pins (tests/test_oracle_pcg.py): dense Cholesky and dense augmented solves on small meshes,
the IC0 defining property (L L^T)_ij = A_ij on the pattern, iteration counts equal to scipy's
cg with the same preconditioner, A-conjugacy of the search directions. tests/test_oracle_exact.py:
TwoSum and TwoProduct are error-free and the compensated residual equals b - A x computed in
exact rational arithmetic (to one rounding), where the plain FP64 residual is wrong; the floor
bounds the exact residual of the correctly rounded solution of small systems.
"""
from __future__ import annotations

from dataclasses import dataclass, field
from typing import Callable, List, Optional

import numpy as np
import scipy.sparse as sp

from . import native


# ---- compensated residual (Ogita, Rump & Oishi 2005: TwoSum, TwoProduct, Dot2) ------------------

_SPLITTER = 134217729.0   # 2^27 + 1: Veltkamp's constant for 53-bit significands


def two_sum(a, b):
    """s = fl(a + b) and the exact error e, a + b = s + e (Knuth's TwoSum, no branch)."""
    s = a + b
    bv = s - a
    return s, (a - (s - bv)) + (b - bv)


def split(a):
    """a = hi + lo exactly, hi and lo with at most 26 significant bits (Veltkamp)."""
    c = _SPLITTER * a
    hi = c - (c - a)
    return hi, a - hi


def two_product(a, b):
    """p = fl(a b) and the exact error e, a b = p + e (Dekker's TwoProduct on split halves)."""
    p = a * b
    ah, al = split(a)
    bh, bl = split(b)
    return p, al * bl - (((p - ah * bh) - al * bh) - ah * bl)


def _padded_rows(A: sp.csr_matrix):
    """A's rows as (width, n) arrays of values and column indices, each row's entries in stored
    order and padded with zeros (a zero term changes neither TwoProduct nor TwoSum). Cached on
    the matrix object."""
    cached = getattr(A, "_dot2_rows", None)
    if cached is not None:
        return cached
    n = A.shape[0]
    cnt = np.diff(A.indptr)
    width = int(cnt.max()) if n else 0
    rows = np.repeat(np.arange(n), cnt)
    pos = np.arange(len(A.indices)) - A.indptr[rows]
    V = np.zeros((width, n))
    J = np.tile(np.arange(n), (width, 1))
    V[pos, rows] = A.data
    J[pos, rows] = A.indices
    A._dot2_rows = (V, J)
    return V, J


def residual_dot2(A: sp.csr_matrix, x: np.ndarray, b: np.ndarray) -> np.ndarray:
    """r = b - A x with Dot2 per row: the sum b_i - sum_j a_ij x_j is formed from the exact
    products (TwoProduct) by TwoSum, and the errors of both are accumulated and added at the
    end. Vectorised over rows, the terms of a row taken in stored (column) order."""
    A = A.tocsr()
    V, J = _padded_rows(A)
    s = np.array(b, dtype=np.float64, copy=True)
    c = np.zeros(len(s))
    for k in range(V.shape[0]):
        p, e = two_product(V[k], x[J[k]])
        s, q = two_sum(s, -p)
        c += q - e
    return s + c


def residual_floor(A: sp.spmatrix, x: np.ndarray, b: np.ndarray) -> float:
    """u || |A||x| + |b| ||_2 / ||b||_2 with u = 2^-53: the relative residual that rounding x (and
    b) to FP64 alone can cause, row by row u (|A||x| + |b|)_i."""
    absA = getattr(A, "_abs", None)
    if absA is None:
        absA = abs(A)
        try:
            A._abs = absA
        except AttributeError:
            pass
    return 2.0 ** -53 * float(np.linalg.norm(absA @ np.abs(x) + np.abs(b))) / float(np.linalg.norm(b))


@dataclass
class SolveResult:
    x: np.ndarray
    iters: int
    restarts: int
    rel_res_true: float
    rel_res_rec: float
    converged: bool
    res_history: List[float] = field(default_factory=list)
    alphas: List[float] = field(default_factory=list)
    betas: List[float] = field(default_factory=list)
    first_pass_iters: int = 0     # iterations until the recursive residual first met rtol
    rel_res_floor: float = 0.0    # u || |A||x| + |b| || / ||b||


def jacobi_preconditioner(A: sp.csr_matrix) -> Callable[[np.ndarray], np.ndarray]:
    d = A.diagonal().copy()
    if np.any(d <= 0):
        raise ValueError("Jacobi needs a positive diagonal")
    inv = 1.0 / d
    return lambda r: inv * r


def identity_preconditioner(A=None):
    return lambda r: r.copy()


def line_blocks(A: sp.csr_matrix, nz: int):
    """The vertical-line blocks of A: for every column of nz nodes, its tridiagonal principal
    submatrix (sub[k] = A[k, k-1], diag[k] = A[k, k], sup[k] = A[k, k+1] inside the column).
    Returns three (ncols, nz) arrays."""
    n = A.shape[0]
    ncols = n // nz
    idx = np.arange(n)
    diag = A.diagonal().reshape(ncols, nz)
    up = np.zeros(n)
    lo = np.zeros(n)
    k = idx % nz
    has_up = k < nz - 1
    up[has_up] = np.asarray(A[idx[has_up], idx[has_up] + 1]).ravel()
    has_lo = k > 0
    lo[has_lo] = np.asarray(A[idx[has_lo], idx[has_lo] - 1]).ravel()
    return lo.reshape(ncols, nz), diag, up.reshape(ncols, nz)


def line_preconditioner(A: sp.csr_matrix, nz: int) -> Callable[[np.ndarray], np.ndarray]:
    """Vertical-line block Jacobi: P = the block diagonal of A made of each column's tridiagonal
    block; z = P^{-1} r by the Thomas algorithm, all columns at once (vectorised over columns,
    sequential in k). A layered-grid reading for the thin-domain pressure system, not the
    paper's undefined DIAG + LS CGS OPT."""
    lo, d, up = line_blocks(A, nz)
    ncols = d.shape[0]
    # forward elimination coefficients (the factorisation does not depend on r)
    w = np.empty_like(d)       # 1 / pivot
    cp = np.empty_like(d)      # modified super-diagonal
    w[:, 0] = 1.0 / d[:, 0]
    cp[:, 0] = up[:, 0] * w[:, 0]
    for k in range(1, nz):
        piv = d[:, k] - lo[:, k] * cp[:, k - 1]
        if np.any(piv <= 0):
            raise ArithmeticError("line preconditioner: non-positive pivot")
        w[:, k] = 1.0 / piv
        cp[:, k] = up[:, k] * w[:, k]

    def apply(r: np.ndarray) -> np.ndarray:
        rr = r.reshape(ncols, nz)
        y = np.empty_like(rr)
        y[:, 0] = rr[:, 0] * w[:, 0]
        for k in range(1, nz):
            y[:, k] = (rr[:, k] - lo[:, k] * y[:, k - 1]) * w[:, k]
        z = np.empty_like(rr)
        z[:, nz - 1] = y[:, nz - 1]
        for k in range(nz - 2, -1, -1):
            z[:, k] = y[:, k] - cp[:, k] * z[:, k + 1]
        return z.reshape(-1)
    return apply


@dataclass
class IC0:
    perm: np.ndarray        # new position -> old index
    indptr: np.ndarray
    indices: np.ndarray
    L: np.ndarray
    shift: float
    lower: sp.csr_matrix    # the (shifted) permuted lower triangle that was factored

    def factor_matrix(self) -> sp.csr_matrix:
        n = len(self.perm)
        return sp.csr_matrix((self.L, self.indices, self.indptr), shape=(n, n))

    def apply(self, r: np.ndarray) -> np.ndarray:
        z_perm = native.ic0_solve(self.indptr, self.indices, self.L, r[self.perm])
        z = np.empty_like(z_perm)
        z[self.perm] = z_perm
        return z


def multicolour_order(colour: np.ndarray) -> np.ndarray:
    """Nodes sorted by colour, ties in natural order (a stable sort)."""
    return np.argsort(colour, kind="stable")


def ic0_factor(A: sp.csr_matrix, perm: Optional[np.ndarray] = None, max_shifts: int = 10) -> IC0:
    n = A.shape[0]
    perm = np.arange(n) if perm is None else np.asarray(perm)
    B = A[perm][:, perm].tocsr()
    B.sort_indices()
    lower = sp.tril(B, format="csr")
    lower.sort_indices()
    diag = B.diagonal()
    shift = 0.0
    for m in range(-1, max_shifts + 1):
        if m >= 0:
            shift = 1e-3 * 2.0 ** m
        Lw = lower.copy()
        if shift:
            Lw = (Lw + sp.diags(shift * diag)).tocsr()
            Lw.sort_indices()
        L, st = native.ic0_factor(Lw.indptr, Lw.indices, Lw.data)
        if st == 0:
            return IC0(perm=perm, indptr=Lw.indptr.astype(np.int64), indices=Lw.indices.astype(np.int32),
                       L=L, shift=shift, lower=Lw)
    raise ArithmeticError("IC0 breakdown after the shift limit")


def ic0_preconditioner(A: sp.csr_matrix, colour: Optional[np.ndarray] = None):
    perm = multicolour_order(colour) if colour is not None else None
    f = ic0_factor(A, perm)
    return f.apply, f


def pcg(A, b: np.ndarray, x0: Optional[np.ndarray] = None, rtol: float = 1e-8, max_iter: int = 100000,
        precond: Optional[Callable] = None, max_restarts: int = 3, record: bool = False) -> SolveResult:
    n = len(b)
    precond = precond or identity_preconditioner()
    bnorm = float(np.sqrt(b @ b))
    if bnorm == 0.0:
        return SolveResult(np.zeros(n), 0, 0, 0.0, 0.0, True)
    x = np.zeros(n) if x0 is None else np.array(x0, dtype=np.float64, copy=True)
    tol = rtol * bnorm
    iters = 0
    restarts = 0
    first_pass = None
    hist, alphas, betas = [], [], []
    prev_true = None
    while True:
        r = residual_dot2(A, x, b)
        rnorm = float(np.sqrt(r @ r))
        converged = rnorm <= tol
        if not converged:
            z = precond(r)
            p = z.copy()
            rz = float(r @ z)
            while iters < max_iter:
                w = A @ p
                pw = float(p @ w)
                alpha = rz / pw
                x += alpha * p
                r -= alpha * w
                iters += 1
                rnorm = float(np.sqrt(r @ r))
                if record:
                    hist.append(rnorm)
                    alphas.append(alpha)
                if rnorm <= tol:
                    converged = True
                    break
                z = precond(r)
                rz_new = float(r @ z)
                beta = rz_new / rz
                if record:
                    betas.append(beta)
                rz = rz_new
                p = z + beta * p
        if first_pass is None:
            first_pass = iters
        true_res = float(np.linalg.norm(residual_dot2(A, x, b))) / bnorm
        floor = residual_floor(A, x, b)
        stalled = prev_true is not None and true_res > 0.5 * prev_true
        last = restarts >= max_restarts or iters >= max_iter
        ok = true_res <= rtol or (true_res <= floor and (stalled or last))
        if ok or last:
            return SolveResult(x, iters, restarts, true_res, rnorm / bnorm, ok,
                               hist, alphas, betas, first_pass, floor)
        prev_true = true_res
        restarts += 1


def pressure_solve(K: sp.csr_matrix, m: np.ndarray, b: np.ndarray, x0: Optional[np.ndarray] = None,
                   rtol: float = 1e-8, max_iter: int = 100000, precond=None, **kw) -> SolveResult:
    """Mean-zero solution of the pure-Neumann system via the Lagrange-multiplier reading.

    The constraint m'q = 0 is kept on every iterate: x0 is projected onto it and each
    preconditioned residual z is projected by z <- z - (m'z / 1'm) 1. In exact arithmetic this
    only shifts the search directions along the null vector 1 (K 1 = 0, 1'r = 0), so alpha,
    beta and the residuals are those of plain PCG; in floating point it stops the null-space
    component of the iterate from drifting, which otherwise stalls the true residual.
    """
    one_m = m.sum()
    lam = b.sum() / one_m
    bc = b - lam * m
    P = precond or jacobi_preconditioner(K)

    def projected(r):
        z = P(r)
        return z - (m @ z) / one_m

    x0p = None if x0 is None else x0 - (m @ x0) / one_m
    res = pcg(K, bc, x0=x0p, rtol=rtol, max_iter=max_iter, precond=projected, **kw)
    res.x = res.x - (m @ res.x) / one_m
    return res


# ---- dense references for tiny meshes (pins) --------------------------------------------------

def dense_cholesky_solve(A: sp.spmatrix, b: np.ndarray) -> np.ndarray:
    import scipy.linalg as sla
    c = sla.cho_factor(A.toarray(), lower=True)
    return sla.cho_solve(c, b)


def dense_augmented_solve(K: sp.spmatrix, m: np.ndarray, b: np.ndarray) -> np.ndarray:
    """Solve [K m; m' 0][q; lambda] = [b; 0] densely (the Lagrange-multiplier system)."""
    n = K.shape[0]
    Aug = np.zeros((n + 1, n + 1))
    Aug[:n, :n] = K.toarray()
    Aug[:n, n] = m
    Aug[n, :n] = m
    rhs = np.concatenate([b, [0.0]])
    sol = np.linalg.solve(Aug, rhs)
    return sol[:n]
