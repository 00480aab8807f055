// Assembly of the P1 operators of Section 5 on the layered Kuhn-tet mesh, Jacobi diagonals and
// the multicolour IC(0) factor (Section 5 remark, item 3).
//
// Assembly is row-owner and deterministic: the thread of row i visits the (at most 24) tets
// that contain node i -- 6 Kuhn tets in each of the 8 hexes around the node, those whose
// vertex set includes the node's corner -- computes each tet's volume and barycentric
// gradients from the sigma-grid coordinates, and adds row i of the element matrix into the 15
// slots. No atomics; every tet is evaluated once per vertex.
//
// Element integrals (exact for P1): M^K_ij = |K| (1 + d_ij)/20, K^K_ij = |K| sum_d nu_d
// d_d phi_i d_d phi_j, G^K_c,ij = |K| d_c phi_j / 4.
#include <cmath>

#include "pm_internal.cuh"

namespace pm {
namespace {

enum Kind { K_AU = 0, K_KI = 1, K_M = 2, K_G0 = 3, K_G1 = 4, K_G2 = 5 };

// Kuhn tet p (axes order pi = p-th permutation of (x, y, z) in lexicographic order) has
// vertex corners v0 = 000, v1 = e_pi0, v2 = e_pi0 + e_pi1, v3 = 111 (bit 0 = x, 1 = y, 2 = z).
__host__ __device__ constexpr int perm_axis(int p, int a) {
  return p == 0 ? (a == 0 ? 0 : a == 1 ? 1 : 2)
       : p == 1 ? (a == 0 ? 0 : a == 1 ? 2 : 1)
       : p == 2 ? (a == 0 ? 1 : a == 1 ? 0 : 2)
       : p == 3 ? (a == 0 ? 1 : a == 1 ? 2 : 0)
       : p == 4 ? (a == 0 ? 2 : a == 1 ? 0 : 1)
       :          (a == 0 ? 2 : a == 1 ? 1 : 0);
}
__host__ __device__ constexpr int vcorner(int p, int w) {
  return w == 0 ? 0 : w == 3 ? 7 : w == 1 ? (1 << perm_axis(p, 0))
                                          : ((1 << perm_axis(p, 0)) | (1 << perm_axis(p, 1)));
}
__host__ __device__ constexpr int local_index(int p, int corner) {
  return vcorner(p, 0) == corner ? 0 : vcorner(p, 1) == corner ? 1
       : vcorner(p, 2) == corner ? 2 : vcorner(p, 3) == corner ? 3 : -1;
}

template <int KIND>
__global__ void __launch_bounds__(128) k_assemble(Geom g, double alpha, double nu0, double nu1,
                                                  double nu2, double* __restrict__ val,
                                                  uint16_t* __restrict__ smask,
                                                  double* __restrict__ rowsum) {
  const int nz = g.nz;
  const double dx = g.dx, dy = g.dy;
  const double nzm1 = (double)(nz - 1);
  for (int64_t row = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; row < g.n;
       row += (int64_t)gridDim.x * blockDim.x) {
    const int col = (int)(row / nz);
    const int k = (int)(row - (int64_t)col * nz);
    double hq[NNBR];
#pragma unroll
    for (int q = 0; q < NNBR; ++q) {
      const int nb = nbr_of(g, col, q);
      hq[q] = nb >= 0 ? g.depth[nb] : 0.0;
    }
    const uint8_t cm = g.cellmask[col];
    double acc[NSLOT];
#pragma unroll
    for (int s = 0; s < NSLOT; ++s) acc[s] = 0.0;
    uint32_t sm = 0;
#pragma unroll
    for (int cn = 0; cn < 8; ++cn) {
      const int a = cn & 1, b = (cn >> 1) & 1, c = (cn >> 2) & 1;
      const int kh = k - c;
      if (kh < 0 || kh > nz - 2) continue;
      const int bit = a ? (b ? 0 : 2) : (b ? 1 : 3);
      if (!((cm >> bit) & 1)) continue;
#pragma unroll
      for (int p = 0; p < 6; ++p) {
        const int v = local_index(p, cn);
        if (v < 0) continue;
        double X[4][3];
        int sl[4];
#pragma unroll
        for (int w = 0; w < 4; ++w) {
          const int vc = vcorner(p, w);
          const int di = (vc & 1) - a, dj = ((vc >> 1) & 1) - b, dk = ((vc >> 2) & 1) - c;
          const int s = slot_of(di, dj, dk);
          sl[w] = s;
          X[w][0] = di * dx;
          X[w][1] = dj * dy;
          X[w][2] = -hq[slot_q(s)] * (1.0 - (double)(k + dk) / nzm1);
        }
        double e[3][3];
#pragma unroll
        for (int r = 0; r < 3; ++r)
#pragma unroll
          for (int d = 0; d < 3; ++d) e[r][d] = X[r + 1][d] - X[0][d];
        // rows of J are e1, e2, e3; grad lambda_a = (e_b x e_c) / det for (a, b, c) cyclic
        double gr[4][3];
        gr[1][0] = e[1][1] * e[2][2] - e[1][2] * e[2][1];
        gr[1][1] = e[1][2] * e[2][0] - e[1][0] * e[2][2];
        gr[1][2] = e[1][0] * e[2][1] - e[1][1] * e[2][0];
        gr[2][0] = e[2][1] * e[0][2] - e[2][2] * e[0][1];
        gr[2][1] = e[2][2] * e[0][0] - e[2][0] * e[0][2];
        gr[2][2] = e[2][0] * e[0][1] - e[2][1] * e[0][0];
        gr[3][0] = e[0][1] * e[1][2] - e[0][2] * e[1][1];
        gr[3][1] = e[0][2] * e[1][0] - e[0][0] * e[1][2];
        gr[3][2] = e[0][0] * e[1][1] - e[0][1] * e[1][0];
        const double det = e[0][0] * gr[1][0] + e[0][1] * gr[1][1] + e[0][2] * gr[1][2];
        const double inv = 1.0 / det;
#pragma unroll
        for (int a2 = 1; a2 < 4; ++a2)
#pragma unroll
          for (int d = 0; d < 3; ++d) gr[a2][d] *= inv;
#pragma unroll
        for (int d = 0; d < 3; ++d) gr[0][d] = -(gr[1][d] + gr[2][d] + gr[3][d]);
        const double vol = fabs(det) / 6.0;
#pragma unroll
        for (int w = 0; w < 4; ++w) {
          double ent;
          if (KIND == K_M) {
            ent = vol * (w == v ? 2.0 : 1.0) / 20.0;
          } else if (KIND == K_KI) {
            ent = vol * (gr[v][0] * gr[w][0] + gr[v][1] * gr[w][1] + gr[v][2] * gr[w][2]);
          } else if (KIND == K_AU) {
            const double kn = vol * (nu0 * gr[v][0] * gr[w][0] + nu1 * gr[v][1] * gr[w][1] +
                                     nu2 * gr[v][2] * gr[w][2]);
            ent = alpha * (vol * (w == v ? 2.0 : 1.0) / 20.0) + kn;
          } else {
            constexpr int cc = KIND - K_G0;
            ent = vol / 4.0 * gr[w][cc];
          }
          acc[sl[w]] += ent;
          sm |= 1u << sl[w];
        }
      }
    }
    double tot = 0.0;
#pragma unroll
    for (int s = 0; s < NSLOT; ++s) {
      val[(int64_t)s * g.npad + row] = acc[s];
      tot += acc[s];
    }
    if (smask) smask[row] = (uint16_t)sm;
    if (rowsum) rowsum[row] = tot;
  }
}

// Jacobi inverse diagonal of a (masked) operator: 1 on Dirichlet rows.
__global__ void k_dinv(Geom g, const double* __restrict__ val, int maskc, double* __restrict__ dinv,
                       float* __restrict__ dinv32) {
  for (int64_t row = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; row < g.n;
       row += (int64_t)gridDim.x * blockDim.x) {
    const int col = (int)(row / g.nz);
    const int k = (int)(row - (int64_t)col * g.nz);
    double d = 1.0;
    if (maskc < 0 || !is_dirichlet(g.colflag[col], k, g.nz, maskc)) d = 1.0 / val[DIAG_SLOT * g.npad + row];
    dinv[row] = d;
    if (dinv32) dinv32[row] = (float)d;
  }
}

// Sum of a vector in a fixed order (one block): used once per basin for 1'm.
__global__ void k_sum_fixed(const double* __restrict__ v, int64_t n, double* out) {
  __shared__ double sh[1024];
  double s = 0.0;
  for (int64_t i = threadIdx.x; i < n; i += blockDim.x) s += v[i];
  sh[threadIdx.x] = s;
  __syncthreads();
  for (int w = blockDim.x / 2; w > 0; w >>= 1) {
    if ((int)threadIdx.x < w) sh[threadIdx.x] += sh[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) *out = sh[0];
}

// ---- multicolour IC(0) ------------------------------------------------------------------------
// Colour of node (i, j, k): (i & 1) | (j & 1) << 1 | (k & 1) << 2; no Kuhn edge joins two nodes
// of one colour, so each colour is one parallel phase. Elimination order: colour 0..7, natural
// order inside a colour (irrelevant: same-colour rows do not couple). Factor storage F[15][n]
// in colour-ordered row positions: for row i, slot s toward neighbour j,
//   F[s][pos(i)] = L_ij when colour(j) < colour(i)   (used by the forward sweep)
//   F[s][pos(i)] = L_ji when colour(j) > colour(i)   (used by the backward sweep)
//   F[1][pos(i)] = L_ii.
// pos(node) = cbase[colour] + clsidx[column] * nlev(kpar) + k / 2, nlev(kpar) = levels of that
// parity.

struct ColourMap {
  int64_t cbase[8];
  int32_t nlev[2];
};

__device__ __forceinline__ int64_t node_pos(const ColourMap& cmap, const int32_t* clsidx, int col,
                                            int colour_cls, int k) {
  const int colour = colour_cls | ((k & 1) << 2);
  return cmap.cbase[colour] + (int64_t)clsidx[col] * cmap.nlev[k & 1] + (k >> 1);
}

template <int colour>
__global__ void __launch_bounds__(128) k_ic0_factor(Geom g, ColourMap cmap,
                                                    const int32_t* __restrict__ cls_cols,
                                                    const int32_t* __restrict__ clsidx,
                                                    const int32_t* __restrict__ coli,
                                                    const int32_t* __restrict__ colj,
                                                    int64_t cls_off, int64_t cls_cnt,
                                                    const double* __restrict__ aval,
                                                    const uint16_t* __restrict__ smask, int maskc,
                                                    double shift, double* __restrict__ F,
                                                    int* __restrict__ breakdown) {
  const int kpar = colour >> 2;
  const int nlev = cmap.nlev[kpar];
  const int64_t total = cls_cnt * nlev;
  const int nz = g.nz;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total;
       t += (int64_t)gridDim.x * blockDim.x) {
    const int col = cls_cols[cls_off + t / nlev];
    const int k = 2 * (int)(t % nlev) + kpar;
    const int64_t row = (int64_t)col * nz + k;
    const int64_t pi = cmap.cbase[colour] + t;
    const uint8_t fi = g.colflag[col];
    const bool di = maskc >= 0 && is_dirichlet(fi, k, nz, maskc);
    const uint32_t smi = smask[row];
    int nbq[NNBR];
#pragma unroll
    for (int q = 0; q < NNBR; ++q) nbq[q] = nbr_of(g, col, q);
    double Lrow[NSLOT];
    double dsum = 0.0;
    // lower slots, visited in increasing neighbour colour
#pragma unroll
    for (int cj = 0; cj < 8; ++cj) {
#pragma unroll
      for (int s = 0; s < NSLOT; ++s) {
        if (s == DIAG_SLOT || (colour ^ slot_flip(s)) != cj || cj >= colour) continue;
        Lrow[s] = 0.0;
        if (!((smi >> s) & 1)) continue;
        const int jcol = nbq[slot_q(s)];
        const int kj = k + slot_dk(s);
        const int64_t rowj = (int64_t)jcol * nz + kj;
        const uint8_t fj = g.colflag[jcol];
        const bool dj = maskc >= 0 && is_dirichlet(fj, kj, nz, maskc);
        double sum = (di || dj) ? 0.0 : aval[(int64_t)s * g.npad + row];
        const uint32_t smj = smask[rowj];
        const int64_t pj = node_pos(cmap, clsidx, jcol, (coli[jcol] & 1) | ((colj[jcol] & 1) << 1), kj);
#pragma unroll
        for (int t2 = 0; t2 < NSLOT; ++t2) {
          if (t2 == DIAG_SLOT || t2 == s) continue;
          const int ck = colour ^ slot_flip(t2);
          if (ck >= cj) continue;       // k must precede j
          if (!((smi >> t2) & 1)) continue;
          const int u = slot_of(slot_di(t2) - slot_di(s), slot_dj(t2) - slot_dj(s),
                                slot_dk(t2) - slot_dk(s));
          if (u < 0 || !((smj >> u) & 1)) continue;
          sum -= Lrow[t2] * F[(int64_t)u * g.n + pj];
        }
        const double l = sum / F[(int64_t)DIAG_SLOT * g.n + pj];
        Lrow[s] = l;
        dsum += l * l;
      }
    }
    const double aii = di ? 1.0 : aval[(int64_t)DIAG_SLOT * g.npad + row];
    const double d = aii * (1.0 + shift) - dsum;
    double lii;
    if (!(d > 0.0)) {
      atomicExch(breakdown, 1);
      lii = 1.0;
    } else {
      lii = sqrt(d);
    }
    F[(int64_t)DIAG_SLOT * g.n + pi] = lii;
#pragma unroll
    for (int s = 0; s < NSLOT; ++s) {
      if (s == DIAG_SLOT) continue;
      const int cj = colour ^ slot_flip(s);
      if (cj >= colour) continue;
      F[(int64_t)s * g.n + pi] = Lrow[s];
      // mirror copy into row j's backward slot
      const int jcol = nbq[slot_q(s)];
      const int kj = k + slot_dk(s);
      if (jcol < 0 || kj < 0 || kj >= nz) continue;
      const int64_t pj = node_pos(cmap, clsidx, jcol, (coli[jcol] & 1) | ((colj[jcol] & 1) << 1), kj);
      F[(int64_t)slot_mirror(s) * g.n + pj] = Lrow[s];
    }
  }
}

// Per velocity component c, per row: bit s set when slot s's neighbour exists and is not in c's
// Dirichlet set (the columns the symmetric elimination keeps), bit 15 set when the row itself is
// a Dirichlet row (an identity row of the eliminated operator).
__global__ void k_keep_masks(Geom g, uint16_t* __restrict__ k0, uint16_t* __restrict__ k1, uint16_t* __restrict__ k2) {
  const int nz = g.nz;
  for (int64_t row = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; row < g.n;
       row += (int64_t)gridDim.x * blockDim.x) {
    const int col = (int)(row / nz);
    const int k = (int)(row - (int64_t)col * nz);
    int nb[NNBR];
    uint8_t fl[NNBR];
#pragma unroll
    for (int q = 0; q < NNBR; ++q) {
      nb[q] = q == 0 ? col : nbr_of(g, col, q);
      fl[q] = nb[q] >= 0 ? g.colflag[nb[q]] : 0;
    }
    uint16_t* outs[3] = {k0, k1, k2};
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      uint32_t m = is_dirichlet(fl[0], k, nz, c) ? 0x8000u : 0u;
#pragma unroll
      for (int s = 0; s < NSLOT; ++s) {
        const int q = slot_q(s);
        const int kk = k + slot_dk(s);
        const bool ok = nb[q] >= 0 && kk >= 0 && kk < nz && !is_dirichlet(fl[q], kk, nz, c);
        m |= (ok ? 1u : 0u) << s;
      }
      outs[c][row] = (uint16_t)m;
    }
  }
}

__global__ void k_recip(double* __restrict__ d, int64_t n) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    d[i] = 1.0 / d[i];
}

int grid_for(int64_t n, int threads, int sms) {
  int64_t gsz = (n + threads - 1) / threads;
  const int64_t cap = (int64_t)sms * 16;
  if (gsz > cap) gsz = cap;
  if (gsz < 1) gsz = 1;
  return (int)gsz;
}

}  // namespace

ColourMap colour_map(const pm_operator* op) {
  ColourMap cm;
  cm.nlev[0] = (op->nz + 1) / 2;
  cm.nlev[1] = op->nz / 2;
  int64_t acc = 0;
  for (int c = 0; c < 8; ++c) {
    cm.cbase[c] = acc;
    acc += (int64_t)op->cls_count[c & 3] * cm.nlev[c >> 2];
  }
  return cm;
}

int launch_assemble(pm_operator* op, cudaStream_t s) {
  Geom g = geom_of(op);
  const int threads = 128;
  const int grid = grid_for(op->n, threads, op->num_sms);
  const double a2 = 1.5 / op->dt, a1 = 1.0 / op->dt;
  const double n0 = op->nu[0], n1 = op->nu[1], n2 = op->nu[2];
  k_assemble<K_AU><<<grid, threads, 0, s>>>(g, a2, n0, n1, n2, op->d_val[VS_AU2], nullptr, nullptr);
  k_assemble<K_AU><<<grid, threads, 0, s>>>(g, a1, n0, n1, n2, op->d_val[VS_AU1], nullptr, nullptr);
  k_assemble<K_KI><<<grid, threads, 0, s>>>(g, 0.0, 1, 1, 1, op->d_val[VS_KI], nullptr, nullptr);
  k_assemble<K_M><<<grid, threads, 0, s>>>(g, 0.0, 0, 0, 0, op->d_val[VS_M], op->d_struct, op->d_m);
  k_assemble<K_G0><<<grid, threads, 0, s>>>(g, 0.0, 0, 0, 0, op->d_val[VS_G0], nullptr, nullptr);
  k_assemble<K_G1><<<grid, threads, 0, s>>>(g, 0.0, 0, 0, 0, op->d_val[VS_G1], nullptr, nullptr);
  k_assemble<K_G2><<<grid, threads, 0, s>>>(g, 0.0, 0, 0, 0, op->d_val[VS_G2], nullptr, nullptr);
  count_launch(7);
  double* d_sum = nullptr;
  int st = cuda_check(cudaMallocAsync((void**)&d_sum, sizeof(double), s), "cudaMallocAsync");
  if (st) return st;
  k_sum_fixed<<<1, 1024, 0, s>>>(op->d_m, op->n, d_sum);
  count_launch();
  st = cuda_check(cudaMemcpyAsync(&op->one_m, d_sum, sizeof(double), cudaMemcpyDeviceToHost, s), "memcpy");
  if (st) return st;
  st = cuda_check(cudaStreamSynchronize(s), "assemble");
  cudaFreeAsync(d_sum, s);
  if (st) return st;
  if ((st = launch_keep_masks(op, s))) return st;
  return cuda_check(cudaGetLastError(), "assemble kernels");
}

int launch_keep_masks(pm_operator* op, cudaStream_t s) {
  for (int c = 0; c < 3; ++c) {
    if (op->d_keep[c]) continue;
    int st = cuda_check(cudaMalloc((void**)&op->d_keep[c], (size_t)op->n * sizeof(uint16_t)), "cudaMalloc keep mask");
    if (st) return st;
    op->device_bytes += op->n * 2;
  }
  Geom g = geom_of(op);
  k_keep_masks<<<grid_for(op->n, 256, op->num_sms), 256, 0, s>>>(g, op->d_keep[0], op->d_keep[1], op->d_keep[2]);
  count_launch();
  return cuda_check(cudaGetLastError(), "k_keep_masks");
}

int launch_dinv(pm_operator* op, int which, cudaStream_t s) {
  if (op->d_dinv[which]) return PM_OK;
  const int vs = which_valset(which);
  double* d = nullptr;
  float* d32 = nullptr;
  int st = cuda_check(cudaMalloc((void**)&d, op->n * sizeof(double)), "cudaMalloc dinv");
  if (st) return st;
  st = cuda_check(cudaMalloc((void**)&d32, op->n * sizeof(float)), "cudaMalloc dinv32");
  if (st) { cudaFree(d); return st; }
  op->device_bytes += op->n * 12;
  Geom g = geom_of(op);
  k_dinv<<<grid_for(op->n, 256, op->num_sms), 256, 0, s>>>(g, op->d_val[vs], which_mask(which), d, d32);
  count_launch();
  op->d_dinv[which] = d;
  op->d_dinv32[which] = d32;
  return cuda_check(cudaGetLastError(), "k_dinv");
}

int launch_ic0_factor(pm_operator* op, int which, double shift, int* breakdown, cudaStream_t s) {
  if (which_valset(which) < 0 || !which_symmetric(which)) return set_error(PM_EINVAL, "IC0 of a non-symmetric operator");
  Ic0Factor& f = op->ic0[which];
  if (!f.F) {
    int st = cuda_check(cudaMalloc((void**)&f.F, (size_t)NSLOT * op->n * sizeof(double)), "cudaMalloc ic0");
    if (st) return st;
    op->device_bytes += (int64_t)NSLOT * op->n * 8;
  }
  cudaMemsetAsync(f.F, 0, (size_t)NSLOT * op->n * sizeof(double), s);
  int* d_bd = nullptr;
  int st = cuda_check(cudaMallocAsync((void**)&d_bd, sizeof(int), s), "cudaMallocAsync");
  if (st) return st;
  cudaMemsetAsync(d_bd, 0, sizeof(int), s);
  Geom g = geom_of(op);
  ColourMap cm = colour_map(op);
  int64_t cls_off[5] = {0, 0, 0, 0, 0};
  for (int c = 0; c < 4; ++c) cls_off[c + 1] = cls_off[c] + op->cls_count[c];
  const int32_t* clsidx = op->d_cls_cols + op->ncols;  // second half: index within class
  const int32_t* coli = clsidx + op->ncols;
  const int32_t* colj = coli + op->ncols;
  for (int colour = 0; colour < 8; ++colour) {
    const int cls = colour & 3;
    const int64_t cnt = op->cls_count[cls];
    const int64_t tot = cnt * cm.nlev[colour >> 2];
    if (tot == 0) continue;
    const int gr = grid_for(tot, 128, op->num_sms);
    const double* av = op->d_val[which_valset(which)];
    const int mc = which_mask(which);
#define PM_IC0F(C)                                                                           \
  case C:                                                                                    \
    k_ic0_factor<C><<<gr, 128, 0, s>>>(g, cm, op->d_cls_cols, clsidx, coli, colj, cls_off[cls], \
                                       cnt, av, op->d_struct, mc, shift, f.F, d_bd);         \
    break;
    switch (colour) {
      PM_IC0F(0) PM_IC0F(1) PM_IC0F(2) PM_IC0F(3) PM_IC0F(4) PM_IC0F(5) PM_IC0F(6) PM_IC0F(7)
    }
#undef PM_IC0F
    count_launch();
  }
  int h_bd = 0;
  st = cuda_check(cudaMemcpyAsync(&h_bd, d_bd, sizeof(int), cudaMemcpyDeviceToHost, s), "memcpy");
  if (!st) st = cuda_check(cudaStreamSynchronize(s), "ic0 factor");
  cudaFreeAsync(d_bd, s);
  if (st) return st;
  *breakdown = h_bd;
  f.shift = shift;
  if (!h_bd) {
    // The sweeps multiply by 1 / L_ii: an FP64 division costs the FP64 pipe about ten times an
    // FMA, and each colour phase has only a few FMAs per row. The factor itself (computed with the
    // divisions above) is unchanged; only its stored diagonal becomes the reciprocal.
    k_recip<<<grid_for(op->n, 256, op->num_sms), 256, 0, s>>>(f.F + (int64_t)DIAG_SLOT * op->n, op->n);
    count_launch();
  }
  f.ok = h_bd == 0;
  return cuda_check(cudaGetLastError(), "k_ic0_factor");
}

}  // namespace pm
