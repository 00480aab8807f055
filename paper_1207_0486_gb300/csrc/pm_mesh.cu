// Host-side mesh construction: ocean columns, neighbour-column table, cell masks and boundary
// flags of the layered basin (Section 2 domain and boundary sets; sigma layers).
#include <cmath>
#include <cstring>
#include <vector>

#include "pm_internal.cuh"

namespace pm {

int build_host_mesh(const pm_mesh_desc* d, const double* coriolis, HostMesh* out) {
  if (!d || !out) return set_error(PM_EINVAL, "null mesh descriptor");
  const int nx = d->nx, ny = d->ny, nz = d->nz;
  if (nx < 2 || ny < 2 || nz < 2) return set_error(PM_EINVAL, "nx, ny, nz must all be >= 2");
  if (!(d->dx > 0.0) || !(d->dy > 0.0)) return set_error(PM_EINVAL, "dx and dy must be > 0");
  if (!d->depth) return set_error(PM_EINVAL, "depth is null");
  if ((int64_t)nx * ny > (int64_t)1 << 28) return set_error(PM_EINVAL, "grid too large");

  auto ocean = [&](int i, int j) -> bool {
    return d->ocean_mask ? d->ocean_mask[(size_t)j * nx + i] != 0 : true;
  };
  const int cx = nx - 1, cy = ny - 1;
  std::vector<uint8_t> cell((size_t)cx * cy, 0);
  size_t ncell = 0;
  for (int j = 0; j < cy; ++j)
    for (int i = 0; i < cx; ++i) {
      const bool a = ocean(i, j) && ocean(i + 1, j) && ocean(i, j + 1) && ocean(i + 1, j + 1);
      cell[(size_t)j * cx + i] = a;
      ncell += a;
    }
  if (ncell == 0) return set_error(PM_EINVAL, "the basin has no ocean cell");

  // Connected components of ocean cells (cells sharing a corner column share nodes).
  {
    std::vector<int32_t> comp((size_t)cx * cy, -1);
    std::vector<int64_t> stack;
    int ncomp = 0;
    for (size_t c0 = 0; c0 < comp.size(); ++c0) {
      if (!cell[c0] || comp[c0] >= 0) continue;
      if (ncomp == 1) {
        return set_error(PM_DISCONNECTED,
                         "the ocean mask has more than one connected component; keep the largest");
      }
      comp[c0] = ncomp;
      stack.push_back((int64_t)c0);
      while (!stack.empty()) {
        const int64_t c = stack.back();
        stack.pop_back();
        const int ci = (int)(c % cx), cj = (int)(c / cx);
        for (int dj = -1; dj <= 1; ++dj)
          for (int di = -1; di <= 1; ++di) {
            const int ii = ci + di, jj = cj + dj;
            if (ii < 0 || jj < 0 || ii >= cx || jj >= cy) continue;
            const size_t cc = (size_t)jj * cx + ii;
            if (cell[cc] && comp[cc] < 0) {
              comp[cc] = ncomp;
              stack.push_back((int64_t)cc);
            }
          }
      }
      ++ncomp;
    }
  }

  auto cell_at = [&](int ci, int cj) -> int {  // -1 outside the grid, else 0/1
    if (ci < 0 || cj < 0 || ci >= cx || cj >= cy) return -1;
    return cell[(size_t)cj * cx + ci];
  };

  std::vector<int32_t> colid((size_t)nx * ny, -1);
  HostMesh& m = *out;
  m.nx = nx;
  m.ny = ny;
  m.nz = nz;
  m.col_i.clear();
  m.col_j.clear();
  for (int j = 0; j < ny; ++j)
    for (int i = 0; i < nx; ++i) {
      const bool act = cell_at(i - 1, j - 1) == 1 || cell_at(i, j - 1) == 1 ||
                       cell_at(i - 1, j) == 1 || cell_at(i, j) == 1;
      if (act) {
        colid[(size_t)j * nx + i] = (int32_t)m.col_i.size();
        m.col_i.push_back(i);
        m.col_j.push_back(j);
      }
    }
  const int ncols = (int)m.col_i.size();
  m.ncols = ncols;
  // Kernels index the 15-slot value arrays with 32-bit integers: 15 * n_pad must stay < 2^31.
  if ((int64_t)ncols * nz > ((int64_t)1 << 27)) return set_error(PM_EINVAL, "too many nodes (limit 2^27 rows)");
  m.nbr.assign((size_t)ncols * NNBR, -1);
  m.depth.resize(ncols);
  m.cellmask.resize(ncols);
  m.colflag.resize(ncols);
  m.coriolis.assign(ncols, 0.0);
  const int sw = d->slip_walls;
  for (int c = 0; c < ncols; ++c) {
    const int i = m.col_i[c], j = m.col_j[c];
    const double h = d->depth[(size_t)j * nx + i];
    if (!(h > 0.0) || !std::isfinite(h)) return set_error(PM_EINVAL, "depth must be > 0 on ocean columns");
    m.depth[c] = h;
    if (coriolis) m.coriolis[c] = coriolis[(size_t)j * nx + i];
    for (int q = 0; q < NNBR; ++q) {
      const int ii = i + q_di(q), jj = j + q_dj(q);
      if (ii < 0 || jj < 0 || ii >= nx || jj >= ny) continue;
      m.nbr[(size_t)c * NNBR + q] = colid[(size_t)jj * nx + ii];
    }
    const int csw = cell_at(i - 1, j - 1), cse = cell_at(i, j - 1);
    const int cnw = cell_at(i - 1, j), cne = cell_at(i, j);
    m.cellmask[c] = (uint8_t)((csw == 1) | ((cse == 1) << 1) | ((cnw == 1) << 2) | ((cne == 1) << 3));
    const bool coast = csw == 0 || cse == 0 || cnw == 0 || cne == 0;
    const bool west = i == 0, east = i == nx - 1, south = j == 0, north = j == ny - 1;
    const bool noslip = (west && !(sw & PM_WALL_WEST)) || (east && !(sw & PM_WALL_EAST)) ||
                        (south && !(sw & PM_WALL_SOUTH)) || (north && !(sw & PM_WALL_NORTH));
    uint8_t f = 0;
    if (coast || noslip) {
      f = CF_GAMMA0;
    } else {
      if ((west && (sw & PM_WALL_WEST)) || (east && (sw & PM_WALL_EAST))) f |= CF_G1X;
      if ((south && (sw & PM_WALL_SOUTH)) || (north && (sw & PM_WALL_NORTH))) f |= CF_G1Y;
    }
    m.colflag[c] = f;
  }
  return PM_OK;
}

}  // namespace pm
