"""Oracle mesh: the layered P1 tetrahedral mesh of a thin basin and its boundary sets.

Domain (Section 2): Omega = {(x1, x2) in Gamma_s, -h(x1, x2) < x3 < 0}. A structured
nx x ny x nz node grid with sigma layers z_k = -h (1 - k/(nz-1)) discretises it. Each hex of
the grid (the paper meshes with bricks, Section 5) is split into the six Kuhn tetrahedra that
share its (0,0,0)-(1,1,1) diagonal; the split is the same in every hex, so the mesh conforms.

Boundary sets (Section 2 and Eqs. pred_cl_0 to pred_tr_3):
  Gamma_0 (u = 0): the sea floor (k = 0), coastline columns (next to a land cell), and outer
                   walls that are not declared slip;
  Gamma_1 (u.n = 0, zero tangential stress): outer walls declared slip (artificial limits);
  Gamma_s (surface, k = nz-1): wind tension on u1, u2 and u3 = 0.
Dirichlet sets per velocity component (Dirichlet wins where sets meet):
  c = 1: Gamma_0 and x-normal Gamma_1;  c = 2: Gamma_0 and y-normal Gamma_1;
  c = 3: Gamma_0 and Gamma_s.

Node numbering: active columns in row-major (j, i) order; node id = column * nz + k.

Pins: the exact volume 1'M1 of the sigma mesh (closed form per cell), tet volumes positive,
reference-tet element matrices (tests/test_oracle_fem.py).
"""
from __future__ import annotations

import itertools
from dataclasses import dataclass

import numpy as np

WALL_WEST, WALL_EAST, WALL_SOUTH, WALL_NORTH = 1, 2, 4, 8

# Kuhn split: tetrahedron pi (a permutation of the axes) has vertices v0 = 0, v1 = e_pi0,
# v2 = e_pi0 + e_pi1, v3 = (1, 1, 1) in hex-corner offsets.
PERMS = list(itertools.permutations((0, 1, 2)))


def kuhn_corners():
    """(6, 4, 3) int array: corner offsets (dx, dy, dz) of the 4 vertices of each Kuhn tet."""
    out = np.zeros((6, 4, 3), dtype=np.int64)
    for t, p in enumerate(PERMS):
        v = np.zeros(3, dtype=np.int64)
        out[t, 0] = v
        for a in range(3):
            v = v.copy()
            v[p[a]] += 1
            out[t, a + 1] = v
    return out


@dataclass
class Mesh:
    nx: int
    ny: int
    nz: int
    dx: float
    dy: float
    n: int                 # number of nodes
    ncols: int             # number of active columns
    col_i: np.ndarray      # (ncols,) grid i of each column
    col_j: np.ndarray      # (ncols,) grid j of each column
    colid: np.ndarray      # (ny, nx) column id or -1
    xyz: np.ndarray        # (n, 3) node coordinates
    tets: np.ndarray       # (T, 4) node ids
    dirichlet: np.ndarray  # (3, n) bool, Dirichlet set of velocity component c
    gamma0: np.ndarray     # (n,) bool
    surface: np.ndarray    # (n,) bool, Gamma_s
    colour: np.ndarray     # (n,) int, (i & 1) | (j & 1) << 1 | (k & 1) << 2
    cell_active: np.ndarray  # (ny-1, nx-1) bool
    top_faces: np.ndarray  # (F, 3) node ids of the surface triangles


def build_mesh(basin) -> Mesh:
    nx, ny, nz = basin.nx, basin.ny, basin.nz
    m = basin.mask.astype(bool)
    if nz < 2 or nx < 2 or ny < 2:
        raise ValueError("need at least 2 nodes along each axis")
    cell = m[:-1, :-1] & m[1:, :-1] & m[:-1, 1:] & m[1:, 1:]
    colact = np.zeros_like(m)
    colact[:-1, :-1] |= cell
    colact[1:, :-1] |= cell
    colact[:-1, 1:] |= cell
    colact[1:, 1:] |= cell
    if np.any(basin.depth[colact] <= 0):
        raise ValueError("depth must be positive on ocean columns")

    jj, ii = np.nonzero(colact)           # row-major (j, i) order
    ncols = len(ii)
    colid = -np.ones((ny, nx), dtype=np.int64)
    colid[jj, ii] = np.arange(ncols)
    n = ncols * nz

    ks = np.arange(nz)
    node_col = np.repeat(np.arange(ncols), nz)
    node_k = np.tile(ks, ncols)
    h = basin.depth[jj, ii]
    xyz = np.empty((n, 3))
    xyz[:, 0] = ii[node_col] * basin.dx
    xyz[:, 1] = jj[node_col] * basin.dy
    xyz[:, 2] = -h[node_col] * (1.0 - node_k / (nz - 1))

    # Tetrahedra: every active cell, every layer, six Kuhn tets.
    cj, ci = np.nonzero(cell)
    corners = kuhn_corners()
    tets = []
    for t in range(6):
        verts = []
        for v in range(4):
            a, b, c = corners[t, v]
            col = colid[cj + b, ci + a]            # (ncell,)
            verts.append((col[:, None] * nz + (ks[:-1][None, :] + c)).ravel())
        tets.append(np.stack(verts, axis=1))
    # order: tet type outermost is fine for the oracle (sums are order-independent up to rounding)
    tets = np.concatenate(tets, axis=0)

    # Lateral boundary classification of each column.
    def cell_ok(cj_, ci_):
        inside = (ci_ >= 0) & (ci_ < nx - 1) & (cj_ >= 0) & (cj_ < ny - 1)
        out = np.zeros_like(inside)
        out[inside] = cell[cj_[inside], ci_[inside]]
        return inside, out

    coast = np.zeros(ncols, dtype=bool)
    for (dj, di) in ((-1, -1), (-1, 0), (0, -1), (0, 0)):
        inside, ok = cell_ok(jj + dj, ii + di)
        coast |= inside & ~ok
    west = ii == 0
    east = ii == nx - 1
    south = jj == 0
    north = jj == ny - 1
    sw = basin.slip_walls
    slip = {w: bool(sw & w) for w in (WALL_WEST, WALL_EAST, WALL_SOUTH, WALL_NORTH)}
    noslip_wall = ((west & (not slip[WALL_WEST])) | (east & (not slip[WALL_EAST]))
                   | (south & (not slip[WALL_SOUTH])) | (north & (not slip[WALL_NORTH])))
    g0_col = coast | noslip_wall
    g1x_col = ((west & slip[WALL_WEST]) | (east & slip[WALL_EAST])) & ~g0_col
    g1y_col = ((south & slip[WALL_SOUTH]) | (north & slip[WALL_NORTH])) & ~g0_col

    bottom = node_k == 0
    surface = node_k == nz - 1
    gamma0 = g0_col[node_col] | bottom
    dirichlet = np.zeros((3, n), dtype=bool)
    dirichlet[0] = gamma0 | g1x_col[node_col]
    dirichlet[1] = gamma0 | g1y_col[node_col]
    dirichlet[2] = gamma0 | surface

    colour = (ii[node_col] & 1) | ((jj[node_col] & 1) << 1) | ((node_k & 1) << 2)

    # Surface triangles: the faces of Kuhn tets lying in the top level. In each top cell they
    # split the square along its (0,0)-(1,1) diagonal.
    top = nz - 1
    c00 = colid[cj, ci] * nz + top
    c10 = colid[cj, ci + 1] * nz + top
    c01 = colid[cj + 1, ci] * nz + top
    c11 = colid[cj + 1, ci + 1] * nz + top
    top_faces = np.concatenate([np.stack([c00, c10, c11], 1), np.stack([c00, c01, c11], 1)], 0)

    return Mesh(nx=nx, ny=ny, nz=nz, dx=basin.dx, dy=basin.dy, n=n, ncols=ncols, col_i=ii,
                col_j=jj, colid=colid, xyz=xyz, tets=tets, dirichlet=dirichlet, gamma0=gamma0,
                surface=surface, colour=colour, cell_active=cell, top_faces=top_faces)


def column_field(mesh: Mesh, grid: np.ndarray) -> np.ndarray:
    """Per-node values of a (ny, nx) grid field (constant along each column)."""
    per_col = grid[mesh.col_j, mesh.col_i]
    return np.repeat(per_col, mesh.nz)
