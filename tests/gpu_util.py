"""Helpers shared by the GPU parity tests (test code: may use the oracle)."""
import numpy as np
import scipy.sparse as sp

from paper_1207_0486_gb300.api import SLOT_OFFSETS, NBR_OFFSETS


def slot_columns(nbr: np.ndarray, nz: int):
    """(15, n) neighbour row of every slot (-1 where the slot has no node)."""
    ncols = nbr.shape[0]
    n = ncols * nz
    rows = np.arange(n)
    col = rows // nz
    k = rows % nz
    out = -np.ones((15, n), dtype=np.int64)
    for s, (di, dj, dk) in enumerate(SLOT_OFFSETS):
        q = NBR_OFFSETS.index((di, dj))
        nb = nbr[col, q] if q else col
        kk = k + dk
        ok = (nb >= 0) & (kk >= 0) & (kk < nz)
        out[s, ok] = nb[ok] * nz + kk[ok]
    return out


def ell_to_csr(vals: np.ndarray, nbr: np.ndarray, nz: int, structure=None) -> sp.csr_matrix:
    cols = slot_columns(nbr, nz)
    n = vals.shape[1]
    rows = np.broadcast_to(np.arange(n), (15, n))
    keep = cols >= 0
    if structure is not None:
        bits = ((structure[None, :].astype(np.int64) >> np.arange(15)[:, None]) & 1).astype(bool)
        keep &= bits
    A = sp.csr_matrix((vals[keep], (rows[keep], cols[keep])), shape=(n, n))
    A.sum_duplicates()
    return A


def rel_rowwise(A: sp.spmatrix, B: sp.spmatrix) -> float:
    """max_i max_j |A_ij - B_ij| / max_j |B_ij| over rows."""
    D = (A - B).tocsr()
    Bc = B.tocsr()
    rmax = np.maximum(abs(Bc).max(axis=1).toarray().ravel(), 1e-300)
    dmax = abs(D).max(axis=1).toarray().ravel()
    return float((dmax / rmax).max())


def theta_basin(basin, amp=1e-4):
    """Attach a zonal wind tension theta1 = -amp cos(pi y / Ly) to a basin (in place)."""
    th = np.zeros((2, basin.ny, basin.nx))
    y = np.arange(basin.ny)[:, None] / max(basin.ny - 1, 1)
    th[0] = -amp * np.cos(np.pi * y) * np.ones((1, basin.nx))
    basin.theta = th
    return basin
