// Batched persistent PCG: many independent systems (basins x right-hand sides) solved by one
// cooperative kernel (Section 5 remark: PCG for every system of the step, here for a whole batch
// of basins at once).
//
// Work is a list of tiles; a tile is up to `tile_cols` whole columns of one system, so the
// vertical-line preconditioner can solve its columns in place. Every iteration is five phases
// separated by a grid barrier:
//   A  tiles: w = A p and the tile partial (p, w)          | REFINE systems: FP64 r = b - A x
//   Ar systems: alpha = rho / (p, w)                      | REFINE: true residual test
//   B  tiles: x += alpha p, r -= alpha w, z = P^{-1} r, partials of (r, r), (r, z), m'z, 1'r
//   Br systems: convergence of the recursive residual, beta (or restart bookkeeping)
//   C  tiles: p = (z - c) + beta p
// Per-system reductions sum the tile partials of that system in tile order (deterministic).
// A system whose recursive residual meets its target moves to REFINE: the FP64 true residual is
// computed; it is DONE when that meets rtol (or the FP64 floor), otherwise it restarts from the
// true residual (x is always FP64; with FP32 values this is iterative refinement).
// The grid barrier spins a bounded number of times; on expiry the kernel records PM_TIMEOUT and
// every block leaves at its next barrier. Vectors that other blocks write during the kernel are
// read with ld.global.cg (L2), never through the non-coherent L1.
#include <cuda_bf16.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstring>
#include <map>
#include <type_traits>
#include <vector>

#include "pm_internal.cuh"

namespace pm {
namespace batch {

enum State : int32_t { ST_ITER = 0, ST_REFINE = 1, ST_RESTART = 2, ST_DONE = 3 };

struct Sys {
  Geom g;
  const void* val;       // T values (FP64 as stored, or FP32 difference form)
  const double* val64;   // FP64 values (true residual)
  const void* dinv;      // T inverse diagonal (Jacobi)
  const void* lineF;     // T line factors (level-major) or null
  const double* m;       // M 1
  const double* b;       // right-hand side (caller's), FP64
  double* bw;            // projected right-hand side (pressure) or == b
  double* x;             // solution, FP64
  void *r, *p, *w, *z;   // Krylov vectors (T)
  double one_m;
  int32_t maskc, proj, prec, tile0, ntiles, pad;
};

struct Scal {
  double rho, alpha, beta, rr, bb, tol2, inner_tol2, proj_c, rel_true, rel_floor, rtol, inner_rtol;
  int32_t iter, outer, state, status, max_iter, first_pass;
};

struct Tile {
  int32_t sys, col0, ncols, pad;
};

struct Ctl {
  uint32_t bar_count, bar_gen;
  int32_t err, active;
};

constexpr int NP = 4;  // partial lanes per tile

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  return v;
}

template <int NV>
__device__ __forceinline__ void block_sum(double (&v)[NV], double* sm) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const int nw = (blockDim.x + 31) >> 5;
  __syncthreads();
#pragma unroll
  for (int i = 0; i < NV; ++i) {
    v[i] = warp_sum(v[i]);
    if (lane == 0) sm[i * 32 + wid] = v[i];
  }
  __syncthreads();
  if (wid == 0) {
#pragma unroll
    for (int i = 0; i < NV; ++i) v[i] = warp_sum(lane < nw ? sm[i * 32 + lane] : 0.0);
  }
  __syncthreads();
}

constexpr long long SPIN_LIMIT = 1ll << 24;  // x ~100 ns sleep: about 2 s

// Bounded grid barrier; returns false (and records PM_TIMEOUT) when the wait expires or another
// block already gave up.
__device__ bool grid_barrier(Ctl* ctl) {
  __shared__ int ok_s;
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) {
    int ok = 1;
    volatile uint32_t* genp = &ctl->bar_gen;
    const uint32_t g0 = *genp;
    __threadfence();
    const uint32_t arrived = atomicAdd(&ctl->bar_count, 1u) + 1u;
    if (arrived == gridDim.x) {
      ctl->bar_count = 0;
      __threadfence();
      atomicAdd(&ctl->bar_gen, 1u);
    } else {
      long long spins = 0;
      while (*genp == g0) {
        if (*((volatile int32_t*)&ctl->err) != 0 || ++spins > SPIN_LIMIT) {
          atomicExch(&ctl->err, PM_TIMEOUT);
          ok = 0;
          break;
        }
        __nanosleep(100);
      }
    }
    __threadfence();
    ok_s = ok && *((volatile int32_t*)&ctl->err) == 0;
  }
  __syncthreads();
  return ok_s != 0;
}

template <typename T>
__device__ __forceinline__ T ldcg(const T* p) { return __ldcg(p); }

template <typename T>
__device__ __forceinline__ T ldv(const T* p, int i) { return __ldg(p + i); }

// Row of A (type T, stored as in the single-system paths: FP64 plain, FP32 difference form).
template <typename T>
__device__ __forceinline__ double row_apply(const Geom& g, const T* __restrict__ val, const T* x, int maskc,
                                            int row, int col, int k) {
  const int nz = g.nz, npad = (int)g.npad;
  int nb[NNBR];
  uint8_t fl[NNBR];
  nb[0] = col;
#pragma unroll
  for (int q = 1; q < NNBR; ++q) nb[q] = __ldg(g.nbr + col * NNBR + q);
#pragma unroll
  for (int q = 0; q < NNBR; ++q) fl[q] = __ldg(g.colflag + (nb[q] >= 0 ? nb[q] : col));
  const T xi = ldcg(x + row);
  if (maskc >= 0 && is_dirichlet(fl[0], k, nz, maskc)) return (double)xi;
  if constexpr (std::is_same<T, double>::value) {
    double sum = 0.0;
#pragma unroll
    for (int s = 0; s < NSLOT; ++s) {
      const int q = slot_q(s), kk = k + slot_dk(s);
      bool ok = nb[q] >= 0;
      if (slot_dk(s) < 0) ok = ok && kk >= 0;
      if (slot_dk(s) > 0) ok = ok && kk < nz;
      if (maskc >= 0) ok = ok && !is_dirichlet(fl[q], kk, nz, maskc);
      const double a = ldv(val, s * npad + row);
      sum = fma(ok ? a : 0.0, ldcg(x + (ok ? nb[q] * nz + kk : row)), sum);
    }
    return sum;
  } else {
    float sum = 0.f, drop = 0.f;
#pragma unroll
    for (int s = 0; s < NSLOT; ++s) {
      if (s == DIAG_SLOT) continue;
      const int q = slot_q(s), kk = k + slot_dk(s);
      bool ok = nb[q] >= 0;
      if (slot_dk(s) < 0) ok = ok && kk >= 0;
      if (slot_dk(s) > 0) ok = ok && kk < nz;
      bool keep = ok;
      const float a = ldv(val, s * npad + row);
      if (maskc >= 0) {
        const bool dj = ok && is_dirichlet(fl[q], kk, nz, maskc);
        keep = ok && !dj;
        drop += dj ? a : 0.f;
      }
      sum = fmaf(keep ? a : 0.f, ldcg(x + (keep ? nb[q] * nz + kk : row)) - xi, sum);
    }
    return (double)fmaf(ldv(val, DIAG_SLOT * npad + row) - drop, xi, sum);
  }
}

// FP64 row with |A||x| (true residual and its floor).
__device__ __forceinline__ double row_apply64_abs(const Geom& g, const double* __restrict__ val, const double* x,
                                                  int maskc, int row, int col, int k, double& asum) {
  const int nz = g.nz, npad = (int)g.npad;
  int nb[NNBR];
  uint8_t fl[NNBR];
  nb[0] = col;
#pragma unroll
  for (int q = 1; q < NNBR; ++q) nb[q] = __ldg(g.nbr + col * NNBR + q);
#pragma unroll
  for (int q = 0; q < NNBR; ++q) fl[q] = __ldg(g.colflag + (nb[q] >= 0 ? nb[q] : col));
  if (maskc >= 0 && is_dirichlet(fl[0], k, nz, maskc)) {
    const double xi = ldcg(x + row);
    asum = fabs(xi);
    return xi;
  }
  double sum = 0.0;
  asum = 0.0;
#pragma unroll
  for (int s = 0; s < NSLOT; ++s) {
    const int q = slot_q(s), kk = k + slot_dk(s);
    bool ok = nb[q] >= 0;
    if (slot_dk(s) < 0) ok = ok && kk >= 0;
    if (slot_dk(s) > 0) ok = ok && kk < nz;
    if (maskc >= 0) ok = ok && !is_dirichlet(fl[q], kk, nz, maskc);
    const double a = ok ? __ldg(val + s * npad + row) : 0.0;
    const double xv = ldcg(x + (ok ? nb[q] * nz + kk : row));
    sum = fma(a, xv, sum);
    asum += fabs(a * xv);
  }
  return sum;
}

// Per-system reduction of tile partials (lane `lane`, tiles [t0, t0 + nt)), one block.
__device__ __forceinline__ double sys_reduce(const double* part, int ntiles_total, int lane, int t0, int nt, double* sm) {
  double v[1] = {0.0};
  for (int t = threadIdx.x; t < nt; t += blockDim.x) v[0] += __ldcg(part + (int64_t)lane * ntiles_total + t0 + t);
  block_sum<1>(v, sm);
  return v[0];  // valid in thread 0
}

// Tiles a block owns (t = blockIdx.x mod gridDim.x) among the systems a phase works on, visited
// system by system so that finished systems cost nothing. mode 0: ITER or REFINE (phase A),
// 1: ITER or RESTART (phase B), 2: ITER (phase C).
__device__ __forceinline__ bool phase_active(int state, int mode) {
  return mode == 0 ? (state == ST_ITER || state == ST_REFINE)
       : mode == 1 ? (state == ST_ITER || state == ST_RESTART) : state == ST_ITER;
}
__device__ __forceinline__ int owned_tile(const Sys* sys, const Scal* scal, int nsys, int s, int mode) {
  const int G = gridDim.x;
  for (; s < nsys; ++s) {
    if (!phase_active(scal[s].state, mode)) continue;
    const int t0 = sys[s].tile0, te = t0 + sys[s].ntiles;
    const int t = t0 + (((int)blockIdx.x - t0) % G + G) % G;
    if (t < te) return t;
  }
  return -1;
}
__device__ __forceinline__ int next_owned(const Sys* sys, const Scal* scal, const Tile* tiles, int nsys, int t,
                                          int mode) {
  const int s = tiles[t].sys;
  const int nt = t + gridDim.x;
  return nt < sys[s].tile0 + sys[s].ntiles ? nt : owned_tile(sys, scal, nsys, s + 1, mode);
}

template <typename T>
__global__ void __launch_bounds__(256, 4) k_batch(const Sys* __restrict__ sys, Scal* scal, int nsys,
                                               const Tile* __restrict__ tiles, int ntiles, double* part, Ctl* ctl,
                                               int quantum, int init) {
  extern __shared__ unsigned char smem_raw[];
  T* smt = reinterpret_cast<T*>(smem_raw);
  __shared__ double red[NP * 32];
  const int tid = threadIdx.x;

  // ---- initialisation: projected right-hand side, r = b' (x = 0), z, p, rho ----------------------
  if (init) {
    // I1: tile partials of 1'b (pressure)
    for (int t = blockIdx.x; t < ntiles; t += gridDim.x) {
      const Tile tl = tiles[t];
      const Sys& S = sys[tl.sys];
      const int nz = S.g.nz, row0 = tl.col0 * nz, rows = tl.ncols * nz;
      double v[1] = {0.0};
      if (S.proj)
        for (int i = tid; i < rows; i += blockDim.x) v[0] += S.b[row0 + i];
      block_sum<1>(v, red);
      if (tid == 0) part[t] = v[0];
    }
    if (!grid_barrier(ctl)) return;
    for (int s = blockIdx.x; s < nsys; s += gridDim.x) {
      const Sys& S = sys[s];
      const double sb = sys_reduce(part, ntiles, 0, S.tile0, S.ntiles, red);
      if (tid == 0) scal[s].proj_c = S.proj ? sb / S.one_m : 0.0;  // lambda, reused below
    }
    if (!grid_barrier(ctl)) return;
    // I2: b' = b - lambda m; x = 0; r = b'; z = P^{-1} r (Jacobi / line) and partials
    for (int t = blockIdx.x; t < ntiles; t += gridDim.x) {
      const Tile tl = tiles[t];
      const Sys& S = sys[tl.sys];
      const int nz = S.g.nz, ld = nz + 1, row0 = tl.col0 * nz, rows = tl.ncols * nz;
      const double lam = scal[tl.sys].proj_c;
      T* r = (T*)S.r;
      T* z = (T*)S.z;
      double v[NP] = {0.0, 0.0, 0.0, 0.0};
      for (int i = tid; i < rows; i += blockDim.x) {
        const int row = row0 + i;
        const double bi = S.proj ? S.b[row] - lam * S.m[row] : S.b[row];
        S.bw[row] = bi;
        S.x[row] = 0.0;
        r[row] = (T)bi;
        v[0] = fma(bi, bi, v[0]);
        if (S.prec == PM_PREC_LINE) smt[(i / nz) * ld + i % nz] = (T)bi;
      }
      __syncthreads();
      if (S.prec == PM_PREC_LINE && tid < tl.ncols) {
        const T* F = (const T*)S.lineF;
        const int col = tl.col0 + tid, nc = S.g.ncols, n = (int)S.g.n;
        T* cs = smt + tid * ld;
        T y = 0;
        for (int k = 0; k < nz; ++k) {
          const int li = k * nc + col;
          y = (cs[k] - F[li] * y) * F[n + li];
          cs[k] = y;
        }
        T zn = y;
        for (int k = nz - 2; k >= 0; --k) {
          const int li = k * nc + col;
          zn = cs[k] - F[2 * n + li] * zn;
          cs[k] = zn;
        }
      }
      __syncthreads();
      for (int i = tid; i < rows; i += blockDim.x) {
        const int row = row0 + i;
        const T ri = r[row];
        const T zi = S.prec == PM_PREC_LINE ? smt[(i / nz) * ld + i % nz] : (T)(((const T*)S.dinv)[row] * ri);
        z[row] = zi;
        v[1] = fma((double)ri, (double)zi, v[1]);
        if (S.proj) {
          v[2] = fma(S.m[row], (double)zi, v[2]);
          v[3] += (double)ri;
        }
      }
      block_sum<NP>(v, red);
      if (tid == 0)
        for (int l = 0; l < NP; ++l) part[(int64_t)l * ntiles + t] = v[l];
      __syncthreads();
    }
    if (!grid_barrier(ctl)) return;
    for (int s = blockIdx.x; s < nsys; s += gridDim.x) {
      const Sys& S = sys[s];
      double tot[NP];
      for (int l = 0; l < NP; ++l) tot[l] = sys_reduce(part, ntiles, l, S.tile0, S.ntiles, red);
      if (tid == 0) {
        Scal& c = scal[s];
        const double cc = S.proj ? tot[2] / S.one_m : 0.0;
        c.bb = tot[0];
        c.rr = tot[0];
        c.tol2 = c.rtol * c.rtol * tot[0];
        c.inner_tol2 = std::is_same<T, double>::value ? c.tol2 : c.inner_rtol * c.inner_rtol * tot[0];
        c.proj_c = cc;
        c.rho = tot[1] - cc * tot[3];
        c.beta = 0.0;
        c.iter = 0;
        c.outer = 0;
        c.status = PM_OK;
        c.state = tot[0] == 0.0 ? ST_DONE : ST_ITER;
        c.rel_true = 0.0;
      }
    }
    if (!grid_barrier(ctl)) return;
    // p = z - c
    for (int t = blockIdx.x; t < ntiles; t += gridDim.x) {
      const Tile tl = tiles[t];
      const Sys& S = sys[tl.sys];
      const int nz = S.g.nz, row0 = tl.col0 * nz, rows = tl.ncols * nz;
      const T c = (T)scal[tl.sys].proj_c;
      for (int i = tid; i < rows; i += blockDim.x) ((T*)S.p)[row0 + i] = ldcg(((const T*)S.z) + row0 + i) - c;
    }
    if (!grid_barrier(ctl)) return;
  }

  for (int it = 0; it < quantum; ++it) {
    if (*((volatile int32_t*)&ctl->active) == 0) return;
    // ---- A: SpMV + (p, w) | REFINE: FP64 residual --------------------------------------------------
    for (int t = owned_tile(sys, scal, nsys, 0, 0); t >= 0; t = next_owned(sys, scal, tiles, nsys, t, 0)) {
      const Tile tl = tiles[t];
      const Sys& S = sys[tl.sys];
      const int state = scal[tl.sys].state;
      const int nz = S.g.nz, row0 = tl.col0 * nz, rows = tl.ncols * nz;
      double v[NP] = {0.0, 0.0, 0.0, 0.0};
      if (state == ST_ITER) {
        const T* p = (const T*)S.p;
        T* w = (T*)S.w;
#pragma unroll 2
        for (int i = tid; i < rows; i += blockDim.x) {
          const int row = row0 + i, col = row / nz, k = row - col * nz;
          const double wi = row_apply<T>(S.g, (const T*)S.val, p, S.maskc, row, col, k);
          w[row] = (T)wi;
          v[0] = fma((double)ldcg(p + row), wi, v[0]);
        }
      } else if (state == ST_REFINE) {
        T* r = (T*)S.r;
        for (int i = tid; i < rows; i += blockDim.x) {
          const int row = row0 + i, col = row / nz, k = row - col * nz;
          double asum;
          const double ax = row_apply64_abs(S.g, S.val64, S.x, S.maskc, row, col, k, asum);
          const double bi = S.bw[row];
          const double ri = bi - ax;
          r[row] = (T)ri;
          v[0] = fma(ri, ri, v[0]);
          const double f = asum + fabs(bi);
          v[1] = fma(f, f, v[1]);
        }
      }
      block_sum<2>(*reinterpret_cast<double(*)[2]>(v), red);
      if (tid == 0) {
        part[t] = v[0];
        part[(int64_t)ntiles + t] = v[1];
      }
    }
    if (!grid_barrier(ctl)) return;
    // ---- Ar ------------------------------------------------------------------------------------------
    for (int s = blockIdx.x; s < nsys; s += gridDim.x) {
      const Sys& S = sys[s];
      Scal& c = scal[s];
      const int state = c.state;
      if (state != ST_ITER && state != ST_REFINE) continue;
      const double a0 = sys_reduce(part, ntiles, 0, S.tile0, S.ntiles, red);
      const double a1 = sys_reduce(part, ntiles, 1, S.tile0, S.ntiles, red);
      if (tid == 0) {
        if (state == ST_ITER) {
          if (!(a0 > 0.0) || !isfinite(a0)) {
            c.status = PM_BREAKDOWN;
            c.state = ST_DONE;
          } else {
            c.alpha = c.rho / a0;
          }
        } else {
          c.outer += 1;
          c.rel_true = sqrt(a0 / c.bb);
          c.rel_floor = ldexp(1.0, -53) * sqrt(a1 / c.bb);
          if (c.rel_true <= fmax(c.rtol, c.rel_floor)) {
            c.state = ST_DONE;
          } else if (c.iter >= c.max_iter || c.outer > 64) {
            c.status = PM_NOT_CONVERGED;
            c.state = ST_DONE;
          } else {
            c.state = ST_RESTART;
            c.inner_tol2 = std::is_same<T, double>::value ? c.tol2 : c.inner_rtol * c.inner_rtol * a0;
            if (c.inner_tol2 < c.tol2) c.inner_tol2 = c.tol2;
          }
        }
      }
    }
    if (!grid_barrier(ctl)) return;
    // ---- B: update + preconditioner + dots | RESTART: preconditioner + dots ---------------------------
    for (int t = owned_tile(sys, scal, nsys, 0, 1); t >= 0; t = next_owned(sys, scal, tiles, nsys, t, 1)) {
      const Tile tl = tiles[t];
      const Sys& S = sys[tl.sys];
      const int state = scal[tl.sys].state;
      double v[NP] = {0.0, 0.0, 0.0, 0.0};
      if (state == ST_ITER || state == ST_RESTART) {
        const int nz = S.g.nz, ld = nz + 1, row0 = tl.col0 * nz, rows = tl.ncols * nz;
        const double alpha = state == ST_ITER ? scal[tl.sys].alpha : 0.0;
        T* r = (T*)S.r;
        T* z = (T*)S.z;
        const T* p = (const T*)S.p;
        const T* w = (const T*)S.w;
        for (int i = tid; i < rows; i += blockDim.x) {
          const int row = row0 + i;
          T ri = ldcg(r + row);
          if (state == ST_ITER) {
            S.x[row] = fma(alpha, (double)ldcg(p + row), S.x[row]);
            ri = ri - (T)alpha * ldcg(w + row);
            r[row] = ri;
          }
          v[0] = fma((double)ri, (double)ri, v[0]);
          if (S.prec == PM_PREC_LINE) smt[(i / nz) * ld + i % nz] = ri;
        }
        __syncthreads();
        if (S.prec == PM_PREC_LINE && tid < tl.ncols) {
          const T* F = (const T*)S.lineF;
          const int col = tl.col0 + tid, nc = S.g.ncols, n = (int)S.g.n;
          T* cs = smt + tid * ld;
          T y = 0;
          for (int k = 0; k < nz; ++k) {
            const int li = k * nc + col;
            y = (cs[k] - F[li] * y) * F[n + li];
            cs[k] = y;
          }
          T zn = y;
          for (int k = nz - 2; k >= 0; --k) {
            const int li = k * nc + col;
            zn = cs[k] - F[2 * n + li] * zn;
            cs[k] = zn;
          }
        }
        __syncthreads();
        for (int i = tid; i < rows; i += blockDim.x) {
          const int row = row0 + i;
          const T ri = ldcg(r + row);
          const T zi = S.prec == PM_PREC_LINE ? smt[(i / nz) * ld + i % nz] : (T)(((const T*)S.dinv)[row] * ri);
          z[row] = zi;
          v[1] = fma((double)ri, (double)zi, v[1]);
          if (S.proj) {
            v[2] = fma(S.m[row], (double)zi, v[2]);
            v[3] += (double)ri;
          }
        }
      }
      block_sum<NP>(v, red);
      if (tid == 0)
        for (int l = 0; l < NP; ++l) part[(int64_t)l * ntiles + t] = v[l];
      __syncthreads();
    }
    if (!grid_barrier(ctl)) return;
    // ---- Br ------------------------------------------------------------------------------------------
    for (int s = blockIdx.x; s < nsys; s += gridDim.x) {
      const Sys& S = sys[s];
      Scal& c = scal[s];
      const int state = c.state;
      if (state != ST_ITER && state != ST_RESTART) continue;
      double tot[NP];
      for (int l = 0; l < NP; ++l) tot[l] = sys_reduce(part, ntiles, l, S.tile0, S.ntiles, red);
      if (tid == 0) {
        const double cc = S.proj ? tot[2] / S.one_m : 0.0;
        const double rho_new = tot[1] - cc * tot[3];
        if (state == ST_RESTART) {
          c.proj_c = cc;
          c.rho = rho_new;
          c.beta = 0.0;
          c.state = ST_ITER;
          if (!(rho_new > 0.0) || !isfinite(rho_new)) {
            c.status = PM_BREAKDOWN;
            c.state = ST_DONE;
          }
        } else {
          c.iter += 1;
          c.rr = tot[0];
          if (tot[0] <= c.inner_tol2) {
            if (c.first_pass == 0) c.first_pass = c.iter;
            c.state = ST_REFINE;
          } else if (c.iter >= c.max_iter) {
            c.state = ST_REFINE;  // final true-residual test, then NOT_CONVERGED
          } else {
            c.proj_c = cc;
            c.beta = rho_new / c.rho;
            c.rho = rho_new;
            if (!(rho_new > 0.0) || !isfinite(rho_new)) {
              c.status = PM_BREAKDOWN;
              c.state = ST_DONE;
            }
          }
        }
      }
    }
    if (!grid_barrier(ctl)) return;
    // ---- C: p = (z - c) + beta p; count active systems ------------------------------------------------
    if (blockIdx.x == 0 && tid == 0) {
      int act = 0;
      for (int s = 0; s < nsys; ++s) act += scal[s].state != ST_DONE;
      ctl->active = act;
    }
    for (int t = owned_tile(sys, scal, nsys, 0, 2); t >= 0; t = next_owned(sys, scal, tiles, nsys, t, 2)) {
      const Tile tl = tiles[t];
      const Sys& S = sys[tl.sys];
      if (scal[tl.sys].state != ST_ITER) continue;
      const int nz = S.g.nz, row0 = tl.col0 * nz, rows = tl.ncols * nz;
      const T beta = (T)scal[tl.sys].beta, c = (T)scal[tl.sys].proj_c;
      T* p = (T*)S.p;
      const T* z = (const T*)S.z;
      for (int i = tid; i < rows; i += blockDim.x) {
        const int row = row0 + i;
        p[row] = (ldcg(z + row) - c) + beta * ldcg(p + row);
      }
    }
    if (!grid_barrier(ctl)) return;
  }
}

// Final pressure shift: x -= m'x / 1'm (per system, tiles reduced like everything else).
__global__ void k_batch_sum_mx(const Sys* sys, const Tile* tiles, int ntiles, double* part) {
  __shared__ double red[32];
  for (int t = blockIdx.x; t < ntiles; t += gridDim.x) {
    const Tile tl = tiles[t];
    const Sys& S = sys[tl.sys];
    const int nz = S.g.nz, row0 = tl.col0 * nz, rows = tl.ncols * nz;
    double v[1] = {0.0};
    if (S.proj)
      for (int i = threadIdx.x; i < rows; i += blockDim.x) v[0] = fma(S.m[row0 + i], S.x[row0 + i], v[0]);
    block_sum<1>(v, red);
    if (threadIdx.x == 0) part[t] = v[0];
  }
}

__global__ void k_batch_shift(const Sys* sys, const Tile* tiles, int ntiles, const double* part) {
  __shared__ double red[32];
  for (int t = blockIdx.x; t < ntiles; t += gridDim.x) {
    const Tile tl = tiles[t];
    const Sys& S = sys[tl.sys];
    if (!S.proj) continue;
    double v[1] = {0.0};
    for (int i = threadIdx.x; i < S.ntiles; i += blockDim.x) v[0] += part[S.tile0 + i];
    block_sum<1>(v, red);
    __shared__ double shift;
    if (threadIdx.x == 0) shift = v[0] / S.one_m;
    __syncthreads();
    const int nz = S.g.nz, row0 = tl.col0 * nz, rows = tl.ncols * nz;
    for (int i = threadIdx.x; i < rows; i += blockDim.x) S.x[row0 + i] -= shift;
    __syncthreads();
  }
}

}  // namespace batch
}  // namespace pm

// ================================= host side ======================================================

struct pm_batch {
  int32_t count = 0;
  int precision = PM_FP64;
  int prec = PM_PREC_JACOBI;
  double rtol = 1e-8, inner_rtol = 1e-2;
  int32_t max_iter = 100000;
  std::vector<pm_operator*> ops;
  std::vector<int32_t> which;
  int tile_cols = 32, block = 256, grid = 0;
  int nz_max = 0;
  int64_t ntiles = 0;
  std::vector<pm::batch::Sys> hsys;
  pm::batch::Sys* d_sys = nullptr;
  pm::batch::Scal* d_scal = nullptr;
  pm::batch::Tile* d_tiles = nullptr;
  pm::batch::Ctl* d_ctl = nullptr;
  double* d_part = nullptr;
  void* work = nullptr;            // r, p, w, z (T) and bw (FP64) for all systems
  size_t work_bytes = 0;
  cudaGraphExec_t graph = nullptr;
  int graph_quantum = 0;
  int device = 0;
  double tuned_ms = 0.0;
};

namespace pm {
int prepare_for_batch(pm_operator* op, int which, int prec, int precision, cudaStream_t s);  // pm_solve.cu

namespace batch {
namespace {

template <typename T>
int max_blocks(int block, size_t smem) {
  int nb = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_batch<T>, block, smem);
  return nb;
}

size_t smem_bytes(const pm_batch* bt) {
  const size_t es = bt->precision == PM_FP64 ? sizeof(double) : sizeof(float);
  return (size_t)bt->tile_cols * (bt->nz_max + 1) * es;
}

void free_layout(pm_batch* bt) {
  if (bt->graph) cudaGraphExecDestroy(bt->graph);
  bt->graph = nullptr;
  cudaFree(bt->d_sys);
  cudaFree(bt->d_scal);
  cudaFree(bt->d_tiles);
  cudaFree(bt->d_ctl);
  cudaFree(bt->d_part);
  cudaFree(bt->work);
  bt->d_sys = nullptr;
  bt->d_scal = nullptr;
  bt->d_tiles = nullptr;
  bt->d_ctl = nullptr;
  bt->d_part = nullptr;
  bt->work = nullptr;
}

// Tiles, descriptors and workspace for the current tile width.
int build_layout(pm_batch* bt) {
  free_layout(bt);
  const bool f32 = bt->precision != PM_FP64;
  const size_t es = f32 ? sizeof(float) : sizeof(double);
  std::vector<Tile> tiles;
  bt->hsys.assign(bt->count, Sys{});
  size_t wb = 0;
  for (int s = 0; s < bt->count; ++s) wb += (size_t)bt->ops[s]->n * (4 * es + sizeof(double)) + 256 * 5;
  int st = cuda_check(cudaMalloc(&bt->work, wb), "batch workspace");
  if (st) return st;
  bt->work_bytes = wb;
  char* cur = (char*)bt->work;
  auto take = [&](size_t bytes) {
    void* p = cur;
    cur += (bytes + 255) / 256 * 256;
    return p;
  };
  bt->nz_max = 0;
  for (int s = 0; s < bt->count; ++s) {
    pm_operator* op = bt->ops[s];
    const int w = bt->which[s];
    const int vs = which_valset(w);
    Sys& S = bt->hsys[s];
    S.g = geom_of(op);
    S.val = f32 ? (const void*)op->d_val32[vs] : (const void*)op->d_val[vs];
    S.val64 = op->d_val[vs];
    S.dinv = f32 ? (const void*)op->d_dinv32[w] : (const void*)op->d_dinv[w];
    S.lineF = bt->prec == PM_PREC_LINE ? (f32 ? (const void*)op->d_line32[w] : (const void*)op->d_line[w]) : nullptr;
    S.m = op->d_m;
    S.one_m = op->one_m;
    S.maskc = which_mask(w);
    S.proj = w == PM_OP_PRESSURE;
    S.prec = bt->prec;
    S.r = take(op->n * es);
    S.p = take(op->n * es);
    S.w = take(op->n * es);
    S.z = take(op->n * es);
    S.bw = (double*)take(op->n * sizeof(double));
    S.tile0 = (int32_t)tiles.size();
    for (int c0 = 0; c0 < op->ncols; c0 += bt->tile_cols) tiles.push_back(Tile{s, c0, std::min(bt->tile_cols, op->ncols - c0), 0});
    S.ntiles = (int32_t)tiles.size() - S.tile0;
    bt->nz_max = std::max(bt->nz_max, op->nz);
  }
  bt->ntiles = (int64_t)tiles.size();
  st = cuda_check(cudaMalloc((void**)&bt->d_sys, bt->count * sizeof(Sys)), "batch sys");
  if (!st) st = cuda_check(cudaMalloc((void**)&bt->d_scal, bt->count * sizeof(Scal)), "batch scal");
  if (!st) st = cuda_check(cudaMalloc((void**)&bt->d_tiles, tiles.size() * sizeof(Tile)), "batch tiles");
  if (!st) st = cuda_check(cudaMalloc((void**)&bt->d_ctl, sizeof(Ctl)), "batch ctl");
  if (!st) st = cuda_check(cudaMalloc((void**)&bt->d_part, (size_t)NP * tiles.size() * sizeof(double)), "batch partials");
  if (st) return st;
  return cuda_check(cudaMemcpy(bt->d_tiles, tiles.data(), tiles.size() * sizeof(Tile), cudaMemcpyHostToDevice), "tiles");
}

template <typename T>
cudaError_t launch(pm_batch* bt, int quantum, int init, cudaStream_t s) {
  const size_t smem = smem_bytes(bt);
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(bt->grid);
  cfg.blockDim = dim3(bt->block);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeCooperative;
  attr[0].val.cooperative = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  count_launch();
  return cudaLaunchKernelEx(&cfg, k_batch<T>, (const Sys*)bt->d_sys, bt->d_scal, (int)bt->count,
                            (const Tile*)bt->d_tiles, (int)bt->ntiles, bt->d_part, bt->d_ctl, quantum, init);
}

int set_grid(pm_batch* bt) {
  const size_t smem = smem_bytes(bt);
  cudaFuncSetAttribute(k_batch<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, 160 * 1024);
  cudaFuncSetAttribute(k_batch<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, 160 * 1024);
  const int per_sm = bt->precision == PM_FP64 ? max_blocks<double>(bt->block, smem) : max_blocks<float>(bt->block, smem);
  int sms = 0;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, bt->device);
  if (per_sm <= 0) return set_error(PM_EINVAL, "batched kernel cannot be resident with this block / tile shape");
  bt->grid = (int)std::max<int64_t>(1, std::min<int64_t>((int64_t)per_sm * sms, std::max<int64_t>(bt->ntiles, bt->count)));
  return PM_OK;
}

// Initialise scalars and control, then the init launch.
int start(pm_batch* bt, cudaStream_t s) {
  std::vector<Scal> hs(bt->count);
  for (int i = 0; i < bt->count; ++i) {
    std::memset(&hs[i], 0, sizeof(Scal));
    hs[i].rtol = bt->rtol;
    hs[i].inner_rtol = bt->inner_rtol;
    hs[i].max_iter = bt->max_iter;
  }
  Ctl c = {0, 0, 0, bt->count};
  int st = cuda_check(cudaMemcpyAsync(bt->d_sys, bt->hsys.data(), bt->count * sizeof(Sys), cudaMemcpyHostToDevice, s), "sys");
  if (!st) st = cuda_check(cudaMemcpyAsync(bt->d_scal, hs.data(), bt->count * sizeof(Scal), cudaMemcpyHostToDevice, s), "scal");
  if (!st) st = cuda_check(cudaMemcpyAsync(bt->d_ctl, &c, sizeof(Ctl), cudaMemcpyHostToDevice, s), "ctl");
  if (st) return st;
  const cudaError_t e = bt->precision == PM_FP64 ? launch<double>(bt, 0, 1, s) : launch<float>(bt, 0, 1, s);
  return cuda_check(e, "batched PCG init launch");
}

int run_to_completion(pm_batch* bt, cudaStream_t s, int quantum) {
  // capture one quantum launch in a CUDA graph once, replay it until no system is active
  if (!bt->graph || bt->graph_quantum != quantum) {
    if (bt->graph) cudaGraphExecDestroy(bt->graph);
    bt->graph = nullptr;
    cudaStream_t cs;
    int st = cuda_check(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking), "capture stream");
    if (st) return st;
    cudaGraph_t g;
    cudaError_t e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
    if (e == cudaSuccess) {
      const cudaError_t le = bt->precision == PM_FP64 ? launch<double>(bt, quantum, 0, cs) : launch<float>(bt, quantum, 0, cs);
      e = cudaStreamEndCapture(cs, &g);
      if (le != cudaSuccess) e = le;
    }
    if (e == cudaSuccess) {
      e = cudaGraphInstantiate(&bt->graph, g, 0);
      cudaGraphDestroy(g);
    }
    cudaStreamDestroy(cs);
    if (e != cudaSuccess) return cuda_check(e, "batched PCG graph capture");
    bt->graph_quantum = quantum;
  }
  Ctl h;
  const int64_t max_quanta = (int64_t)bt->max_iter / quantum + 70;
  for (int64_t q = 0; q < max_quanta; ++q) {
    int st = cuda_check(cudaGraphLaunch(bt->graph, s), "batched PCG graph launch");
    if (st) return st;
    count_launch();
    st = cuda_check(cudaMemcpyAsync(&h, bt->d_ctl, sizeof(Ctl), cudaMemcpyDeviceToHost, s), "ctl");
    if (!st) st = cuda_check(cudaStreamSynchronize(s), "batched PCG");
    if (st) return st;
    if (h.err) return set_error(h.err, "batched PCG: a grid barrier wait expired");
    if (h.active == 0) return PM_OK;
  }
  return set_error(PM_NOT_CONVERGED, "batched PCG: quantum budget exhausted");
}

int finish(pm_batch* bt, pm_solve_stats* stats, cudaStream_t s, double seconds) {
  k_batch_sum_mx<<<bt->grid, 256, 0, s>>>(bt->d_sys, bt->d_tiles, (int)bt->ntiles, bt->d_part);
  k_batch_shift<<<bt->grid, 256, 0, s>>>(bt->d_sys, bt->d_tiles, (int)bt->ntiles, bt->d_part);
  count_launch(2);
  std::vector<Scal> hs(bt->count);
  int st = cuda_check(cudaMemcpyAsync(hs.data(), bt->d_scal, bt->count * sizeof(Scal), cudaMemcpyDeviceToHost, s), "scal");
  if (!st) st = cuda_check(cudaStreamSynchronize(s), "batched PCG finish");
  if (st) return st;
  int worst = PM_OK;
  const double es = bt->precision == PM_FP64 ? 8.0 : 4.0;
  for (int i = 0; i < bt->count; ++i) {
    const Scal& c = hs[i];
    if (c.status != PM_OK && worst == PM_OK) worst = c.status;
    if (stats) {
      pm_solve_stats& o = stats[i];
      o.iters = c.iter;
      o.outer_iters = c.outer;
      o.first_pass_iters = c.first_pass;
      o.status = c.status;
      o.rel_residual_true = c.rel_true;
      o.rel_residual_rec = c.bb > 0 ? std::sqrt(c.rr / c.bb) : 0.0;
      o.rel_residual_floor = c.rel_floor;
      o.seconds = seconds;
      const double n = (double)bt->ops[i]->n;
      o.bytes_moved = c.iter * n * (15 * es + 11 * es + 8 + 8) + c.outer * n * (15 * 8 + 24);
    }
  }
  if (worst != PM_OK) return set_error(worst, "batched PCG: some systems did not converge");
  return PM_OK;
}

struct TuneKey {
  int64_t rows;
  int nsys, precision, prec, nz;
  bool operator<(const TuneKey& o) const {
    return std::tie(rows, nsys, precision, prec, nz) < std::tie(o.rows, o.nsys, o.precision, o.prec, o.nz);
  }
};
std::map<TuneKey, std::pair<int, int>> g_tuned;

// Autotuner: slice width (columns per tile) x block size, timed on 8 iterations of this batch.
int autotune(pm_batch* bt, cudaStream_t s) {
  int64_t rows = 0;
  for (auto* op : bt->ops) rows += op->n;
  int64_t bucket = 1;
  while (bucket < rows) bucket <<= 1;
  TuneKey key{bucket, bt->count, bt->precision, bt->prec, bt->nz_max};
  auto it = g_tuned.find(key);
  if (it != g_tuned.end()) {
    bt->tile_cols = it->second.first;
    bt->block = it->second.second;
    return PM_OK;
  }
  double best = 1e30;
  int bc = 32, bb = 256;
  int64_t nmax = 0;
  for (auto* op : bt->ops) nmax = std::max<int64_t>(nmax, op->n);
  double* xtmp = nullptr;  // scratch solution vector for the timing runs (shared: values unused)
  int st0 = cuda_check(cudaMalloc((void**)&xtmp, nmax * sizeof(double)), "autotune scratch");
  if (st0) return st0;
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  for (int tc : {16, 32, 64}) {
    for (int blk : {128, 256}) {
      if (tc > blk) continue;
      bt->tile_cols = tc;
      bt->block = blk;
      int st = build_layout(bt);
      if (!st) st = set_grid(bt);
      if (st) continue;
      for (int s2 = 0; s2 < bt->count; ++s2) {
        // any right-hand side will do for timing: use the operator's m = M 1
        bt->hsys[s2].b = bt->ops[s2]->d_m;
        bt->hsys[s2].x = xtmp;
      }
      if (start(bt, s)) continue;
      cudaEventRecord(e0, s);
      const cudaError_t le = bt->precision == PM_FP64 ? launch<double>(bt, 8, 0, s) : launch<float>(bt, 8, 0, s);
      cudaEventRecord(e1, s);
      if (le != cudaSuccess || cudaStreamSynchronize(s) != cudaSuccess) continue;
      Ctl h;
      cudaMemcpy(&h, bt->d_ctl, sizeof(Ctl), cudaMemcpyDeviceToHost);
      if (h.err) return set_error(h.err, "batched PCG autotune: grid barrier wait expired");
      float ms = 0.f;
      cudaEventElapsedTime(&ms, e0, e1);
      if (ms < best) {
        best = ms;
        bc = tc;
        bb = blk;
      }
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaFree(xtmp);
  bt->tile_cols = bc;
  bt->block = bb;
  bt->tuned_ms = best;
  g_tuned[key] = {bc, bb};
  return PM_OK;
}

}  // namespace
}  // namespace batch
}  // namespace pm

using namespace pm;

extern "C" int pm_batch_create(pm_operator* const* ops, const pm_which* which, int32_t count,
                               const pm_solve_opts* opts, int32_t autotune, pm_batch** out, pm_stream stream) {
  if (!ops || !which || !opts || !out || count <= 0) return set_error(PM_EINVAL, "bad batch arguments");
  *out = nullptr;
  if (opts->prec != PM_PREC_JACOBI && opts->prec != PM_PREC_LINE && opts->prec != PM_PREC_NONE)
    return set_error(PM_EINVAL, "batched PCG supports PM_PREC_JACOBI, PM_PREC_LINE and PM_PREC_NONE");
  if (opts->precision != PM_FP64 && opts->precision != PM_FP32_REFINE)
    return set_error(PM_EINVAL, "batched PCG supports PM_FP64 and PM_FP32_REFINE");
  if (!(opts->rtol > 0.0)) return set_error(PM_EINVAL, "rtol must be > 0");
  cudaStream_t s = (cudaStream_t)stream;
  pm_batch* bt = new pm_batch();
  bt->count = count;
  bt->precision = opts->precision;
  bt->prec = opts->prec == PM_PREC_NONE ? PM_PREC_JACOBI : opts->prec;
  bt->rtol = opts->rtol;
  bt->inner_rtol = opts->inner_rtol > 0.0 ? opts->inner_rtol : 1e-2;
  bt->max_iter = opts->max_iter > 0 ? opts->max_iter : 100000;
  cudaGetDevice(&bt->device);
  for (int i = 0; i < count; ++i) {
    if (!ops[i] || !which_symmetric((int)which[i])) {
      delete bt;
      return set_error(PM_EINVAL, "batch entry with a null or non-symmetric operator");
    }
    int st = prepare_for_batch(ops[i], (int)which[i], bt->prec, bt->precision, s);
    if (st) {
      delete bt;
      return st;
    }
    bt->ops.push_back(ops[i]);
    bt->which.push_back((int32_t)which[i]);
  }
  int st = cuda_check(cudaStreamSynchronize(s), "batch preparation");
  if (!st && autotune) st = batch::autotune(bt, s);
  if (!st) st = batch::build_layout(bt);
  if (!st) st = batch::set_grid(bt);
  if (st) {
    batch::free_layout(bt);
    delete bt;
    return st;
  }
  *out = bt;
  return PM_OK;
}

extern "C" int pm_batch_solve(pm_batch* bt, const double* const* b, double* const* x, pm_solve_stats* stats,
                              pm_stream stream) {
  if (!bt || !b || !x) return set_error(PM_EINVAL, "null argument");
  auto t0 = std::chrono::steady_clock::now();
  cudaStream_t s = (cudaStream_t)stream;
  for (int i = 0; i < bt->count; ++i) {
    if (!b[i] || !x[i]) return set_error(PM_EINVAL, "null vector in batch");
    bt->hsys[i].b = b[i];
    bt->hsys[i].x = x[i];
  }
  int st = batch::start(bt, s);
  if (!st) st = batch::run_to_completion(bt, s, 64);
  if (st && st != PM_NOT_CONVERGED) return st;
  const double secs = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
  const int fs = batch::finish(bt, stats, s, secs);
  return st ? st : fs;
}

extern "C" int pm_batch_info(const pm_batch* bt, int32_t* tile_cols, int32_t* block, int32_t* grid, int64_t* ntiles) {
  if (!bt) return set_error(PM_EINVAL, "null batch");
  if (tile_cols) *tile_cols = bt->tile_cols;
  if (block) *block = bt->block;
  if (grid) *grid = bt->grid;
  if (ntiles) *ntiles = bt->ntiles;
  return PM_OK;
}

extern "C" void pm_batch_destroy(pm_batch* bt) {
  if (!bt) return;
  batch::free_layout(bt);
  delete bt;
}

extern "C" int pm_pcg_solve_batched(pm_operator* const* ops, const pm_which* which, const double* const* b,
                                    double* const* x, int32_t count, const pm_solve_opts* opts,
                                    pm_solve_stats* stats, pm_stream stream) {
  pm_batch* bt = nullptr;
  int st = pm_batch_create(ops, which, count, opts, 0, &bt, stream);
  if (st) return st;
  st = pm_batch_solve(bt, b, x, stats, stream);
  pm_batch_destroy(bt);
  return st;
}

// Test aid: block 1 leaves without arriving at the barrier, so block 0's bounded wait expires.
__global__ void k_barrier_probe(pm::batch::Ctl* ctl) {
  if (blockIdx.x != 0) return;
  pm::batch::grid_barrier(ctl);
}

extern "C" int pm_debug_barrier_timeout(pm_stream stream) {
  cudaStream_t s = (cudaStream_t)stream;
  pm::batch::Ctl* d = nullptr;
  int st = cuda_check(cudaMalloc((void**)&d, sizeof(pm::batch::Ctl)), "probe ctl");
  if (st) return st;
  cudaMemsetAsync(d, 0, sizeof(pm::batch::Ctl), s);
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(2);
  cfg.blockDim = dim3(32);
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeCooperative;
  attr[0].val.cooperative = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  pm::count_launch();
  st = cuda_check(cudaLaunchKernelEx(&cfg, k_barrier_probe, d), "probe launch");
  pm::batch::Ctl h = {};
  if (!st) st = cuda_check(cudaMemcpyAsync(&h, d, sizeof(h), cudaMemcpyDeviceToHost, s), "probe copy");
  if (!st) st = cuda_check(cudaStreamSynchronize(s), "probe sync");
  cudaFree(d);
  if (st) return st;
  return h.err;
}
