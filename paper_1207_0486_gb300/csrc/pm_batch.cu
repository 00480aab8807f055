// Batched persistent PCG: many independent systems (basins x right-hand sides) solved by one
// cooperative kernel (Section 5 remark: PCG for every system of the step, here for a whole batch
// of basins at once).
//
// Work is a list of tiles; a tile is whole columns of one system (at least `tile_cols`, more for
// shallow columns), so the vertical-line preconditioner can solve its columns in place. Every
// iteration is five phases separated by a grid barrier (IC0 systems: 16 more, one per colour
// sweep, whose rows are dealt to blocks in colour order rather than by tile):
//   A  tiles: w = A p and the tile partial (p, w)          | REFINE systems: FP64 r = b - A x
//   Ar systems: alpha = rho / (p, w)                      | REFINE: true residual test
//   B  tiles: x += alpha p, r -= alpha w, z = P^{-1} r, partials of (r, r), (r, z), m'z, 1'r
//   Br systems: convergence of the recursive residual, beta (or restart bookkeeping)
//   C  tiles: p = (z - c) + beta p
// Per-system reductions sum the tile partials of that system in tile order (deterministic).
// A system whose recursive residual meets its target moves to REFINE: the FP64 true residual is
// computed; it is DONE when that meets rtol (or the FP64 floor), otherwise it restarts from the
// true residual (x is always FP64; with FP32 values this is iterative refinement). A pressure
// system passes through SHIFT (partials of m'x in B) and SHIFT2 (x -= m'x / 1'm in C) on its way
// to DONE. Systems admitted between launches (NEW) are initialised at the start of the next
// launch while the others wait at its barriers.
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

// NEW: admitted, not initialised; PINIT: r, z set, p pending; SHIFT / SHIFT2: converged pressure
// system whose solution is being moved to zero mean (m'x = 0).
enum State : int32_t {
  ST_ITER = 0, ST_REFINE = 1, ST_RESTART = 2, ST_DONE = 3, ST_NEW = 4, ST_PINIT = 5, ST_SHIFT = 6, ST_SHIFT2 = 7
};

struct Sys {
  Geom g;
  const void* val;       // T values (FP64 as stored, or FP32 difference form)
  const double* val64;   // FP64 values (true residual)
  const void* dinv;      // T inverse diagonal (Jacobi)
  const void* lineF;     // T line factors (level-major) or null
  const double* m;       // M 1
  const float2* m2;      // M 1 split into two floats (FP32 systems' m'z), or null
  const double* b;       // right-hand side (caller's), FP64
  double* bw;            // projected right-hand side (pressure) or == b
  double* x;             // solution, FP64
  void *r, *p, *w, *z;   // Krylov vectors (T)
  const void* ic0F;      // T IC0 factor (colour-ordered rows, 1 / L_ii on the diagonal) or null
  const int32_t* cls_cols;  // columns listed parity class by parity class
  int64_t cbase[8];      // first colour-ordered position of each colour
  int32_t cls_off[4];    // first entry of each parity class in cls_cols
  int32_t cls_cnt[4];    // columns of each parity class
  int32_t nlev[2];       // levels of even / odd parity
  double one_m;
  int32_t maskc, proj, prec;
  int32_t tile0, ntiles;  // the system's tiles [tile0, tile0 + ntiles) (partials, block ownership)
  int32_t tw;             // columns per tile (the last tile may have fewer)
  int32_t vbf16;          // FP32 system whose operator values are BF16 (difference form)
};

struct Scal {
  double rho, alpha, beta, rr, bb, tol2, inner_tol2, proj_c, rel_true, rel_floor, rtol, inner_rtol;
  double prev_true;  // true residual of the previous REFINE (-1: none yet)
  int32_t iter, outer, state, status, max_iter, first_pass;
};

struct Tile {
  int32_t sys, col0, ncols;
};

// Tile t of system s: columns [(t - tile0) tw, + tw) of the system, clipped to its columns.
__device__ __forceinline__ Tile tile_of(const Sys& S, int s, int t) {
  const int c0 = (t - S.tile0) * S.tw;
  return Tile{s, c0, min(S.tw, S.g.ncols - c0)};
}

struct Ctl {
  uint32_t bar_count, bar_gen;
  int32_t err, active;   // active: systems not DONE (written by block 0, read at every iteration)
  int32_t pending, pad;  // pending: NEW systems to initialise at the start of the next launch
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

__device__ __forceinline__ double ldval(const double* p) { return __ldg(p); }
__device__ __forceinline__ float ldval(const float* p) { return __ldg(p); }
__device__ __forceinline__ float ldval(const __nv_bfloat16* p) {
  return __bfloat162float(__ushort_as_bfloat16(__ldg(reinterpret_cast<const unsigned short*>(p))));
}

// Row of A for phase A. MASKC: velocity component whose Dirichlet rows are identity rows (0, 1, 2;
// a compile-time constant so the per-slot tests fold), or -1 (pressure: none). The slot values are
// loaded before the neighbour indices are used, and the iterate with plain loads: this file is
// compiled with L2-only default loads, and the iterate is written only in other phases.
template <typename T, int MASKC, typename V = T>
__device__ __forceinline__ T row_spmv(const Geom& g, const V* __restrict__ val, const T* x, int row, int col,
                                           int k) {
  constexpr bool MASK = MASKC >= 0;
  const int nz = g.nz, npad = (int)g.npad;
  int nb[NNBR];
  nb[0] = col;
#pragma unroll
  for (int q = 1; q < NNBR; ++q) nb[q] = nbr_of(g, col, q);
  T a[NSLOT];
#pragma unroll
  for (int s = 0; s < NSLOT; ++s) a[s] = ldval(val + s * npad + row);
  uint8_t fl[NNBR];
  if (MASK) {
#pragma unroll
    for (int q = 0; q < NNBR; ++q) fl[q] = __ldg(g.colflag + (nb[q] >= 0 ? nb[q] : col));
  }
  const T xi = x[row];
  if (MASK && is_dirichlet(fl[0], k, nz, MASKC)) return xi;
  if constexpr (std::is_same<T, double>::value) {
    double sum = 0.0;
#pragma unroll
    for (int s = 0; s < NSLOT; ++s) {
      const int q = slot_q(s), kk = k + slot_dk(s);
      bool ok = nb[q] >= 0;  // geometry only: the load address does not wait for the flags
      if (slot_dk(s) < 0) ok = ok && kk >= 0;
      if (slot_dk(s) > 0) ok = ok && kk < nz;
      const bool keep = MASK ? ok && !is_dirichlet(fl[q], kk, nz, MASKC) : ok;
      sum = fma(keep ? a[s] : 0.0, x[ok ? nb[q] * nz + kk : row], sum);
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
      if (MASK) {
        const bool dj = ok && is_dirichlet(fl[q], kk, nz, MASKC);
        keep = ok && !dj;
        drop += dj ? a[s] : 0.f;
      }
      sum = fmaf(keep ? a[s] : 0.f, x[ok ? nb[q] * nz + kk : row] - xi, sum);
    }
    return fmaf(a[DIAG_SLOT] - drop, xi, sum);
  }
}

// Phase A of one tile: w = A p on its rows, returns the partial (p, w). Two rows per thread are
// computed before either is stored.
template <typename T, int MASKC, typename V = T>
__device__ __forceinline__ double spmv_tile(const Sys& S, int row0, int rows, int nz) {
  const T* p = (const T*)S.p;
  T* w = (T*)S.w;
  const V* val = (const V*)S.val;
  const Geom g = S.g;
  const int bd = blockDim.x;
  AccFor<T> acc;   // FP64 for FP64 systems, compensated FP32 for FP32 ones
  for (int i0 = threadIdx.x; i0 < rows; i0 += 2 * bd) {
    T wv[2];
    T pv[2];
#pragma unroll
    for (int u = 0; u < 2; ++u) {
      const int row = row0 + min(i0 + u * bd, rows - 1), col = row / nz, k = row - col * nz;
      wv[u] = row_spmv<T, MASKC, V>(g, val, p, row, col, k);
      pv[u] = p[row];
    }
#pragma unroll
    for (int u = 0; u < 2; ++u) {
      if (i0 + u * bd < rows) {
        w[row0 + i0 + u * bd] = wv[u];
        acc.add_prod(pv[u], wv[u]);
      }
    }
  }
  return acc.value();
}

// Phase A of a REFINE system's tile: r = b' - A x in FP64, compensated (row_residual_dot2), and
// partials of (r, r) and of the floor (|A||x| + |b|)^2.
template <typename T, int MASKC>
__device__ __forceinline__ void refine_tile(const Sys& S, int row0, int rows, int nz, double& rr, double& ff) {
  T* r = (T*)S.r;
  const Geom g = S.g;
  for (int i = threadIdx.x; i < rows; i += blockDim.x) {
    const int row = row0 + i, col = row / nz, k = row - col * nz;
    double asum;
    const double bi = S.bw[row];
    const double ri = row_residual_dot2<MASKC>(g, S.val64, S.x, bi, row, col, k, asum);
    r[row] = (T)ri;
    rr = fma(ri, ri, rr);
    const double f = asum + fabs(bi);
    ff = fma(f, f, ff);
  }
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
// 1: ITER, RESTART or SHIFT (phase B), 2: ITER or SHIFT2 (phase C), 3: NEW, 4: PINIT.
__device__ __forceinline__ bool phase_active(int state, int mode) {
  switch (mode) {
    case 0: return state == ST_ITER || state == ST_REFINE;
    case 1: return state == ST_ITER || state == ST_RESTART || state == ST_SHIFT;
    case 2: return state == ST_ITER || state == ST_SHIFT2;
    case 3: return state == ST_NEW;
    default: return state == ST_PINIT;
  }
}
// Vertical-line solve of one column in shared memory (cs[0..nz)), level-major factors F: forward
// sweep y_k = (c_k - l_k y_{k-1}) d_k, back substitution z_k = y_k - u_k z_{k+1}. The factors are
// constant during the kernel; they are read CH levels at a time so that CH loads are in flight.
template <typename T>
__device__ __forceinline__ void line_sweep(T* cs, const T* __restrict__ F, int col, int nc, int n, int nz) {
  constexpr int CH = sizeof(T) == 8 ? 4 : 8;
  T y = 0;
  for (int k0 = 0; k0 < nz; k0 += CH) {
    T fl[CH], fd[CH];
#pragma unroll
    for (int u = 0; u < CH; ++u) {
      const int li = min(k0 + u, nz - 1) * nc + col;
      fl[u] = __ldg(F + li);
      fd[u] = __ldg(F + n + li);
    }
#pragma unroll
    for (int u = 0; u < CH; ++u) {
      if (k0 + u < nz) {
        y = (cs[k0 + u] - fl[u] * y) * fd[u];
        cs[k0 + u] = y;
      }
    }
  }
  T zn = y;
  for (int k0 = nz - 2; k0 >= 0; k0 -= CH) {
    T fu[CH];
#pragma unroll
    for (int u = 0; u < CH; ++u) fu[u] = __ldg(F + 2 * n + max(k0 - u, 0) * nc + col);
#pragma unroll
    for (int u = 0; u < CH; ++u) {
      if (k0 - u >= 0) {
        zn = cs[k0 - u] - fu[u] * zn;
        cs[k0 - u] = zn;
      }
    }
  }
}

// One row of an IC0 colour phase (the same update as the single-system sweeps): forward
// y_i = (r_i - sum_{colour(j) < C} L_ij y_j) / L_ii, backward z_i = (y_i - sum_{colour(j) > C} L_ji z_j)
// / L_ii in place on y (natural order; pi: the row's position in colour order, its factor row).
// F's diagonal slot holds 1 / L_ii. Returns the new y_i.
template <typename T, int C, bool FWD>
__device__ __forceinline__ T ic0_value(const Geom& g, int col, int k, int64_t pi, const T* __restrict__ F,
                                       const T* r, const T* y) {
  const int nz = g.nz;
  const int64_t row = (int64_t)col * nz + k;
  T acc = FWD ? r[row] : y[row];
#pragma unroll
  for (int s = 0; s < NSLOT; ++s) {
    if (s == DIAG_SLOT) continue;
    const int cj = C ^ slot_flip(s);
    if (FWD ? (cj > C) : (cj < C)) continue;
    const int kk = k + slot_dk(s);
    if (kk < 0 || kk >= nz) continue;
    const int q = slot_q(s);
    const int nb = q == 0 ? col : nbr_of(g, col, q);
    if (nb < 0) continue;
    acc = fma(-__ldg(F + (int64_t)s * g.n + pi), y[(int64_t)nb * nz + kk], acc);
  }
  return acc * __ldg(F + (int64_t)DIAG_SLOT * g.n + pi);
}

// The rows of colour C of one system in an IC0 colour phase, in the colour-ordered enumeration of
// the single-system sweep (position q of the colour: column cls_cols[cls_off + q / nlev], level
// 2 (q mod nlev) + parity). Chunks of four rows per thread, all computed before any is stored;
// block b takes the chunks ch = (b - tile0) mod G, + G, ... so that the rows of small systems
// spread over the grid, and the block that computes a row never changes its value (no row of a
// colour reads another row of that colour).
template <typename T, int C, bool FWD>
__device__ __forceinline__ void ic0_colour(const Sys& S) {
  constexpr int kpar = C >> 2, cls = C & 3, U = 4;
  const int nlev = S.nlev[kpar];
  const int rows = S.cls_cnt[cls] * nlev;
  if (rows == 0) return;
  const int G = gridDim.x, bd = blockDim.x;
  const int chunk = U * bd;
  const int nch = (rows + chunk - 1) / chunk;
  const T* F = (const T*)S.ic0F;
  const T* r = (const T*)S.r;
  T* y = (T*)S.z;
  const int32_t* cc = S.cls_cols + S.cls_off[cls];
  const int nz = S.g.nz;
  const int64_t cb = S.cbase[C];
  for (int ch = ((int)blockIdx.x - S.tile0 % G + G) % G; ch < nch; ch += G) {
    int col[U], k[U], q[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      q[u] = ch * chunk + u * bd + (int)threadIdx.x;
      const int qq = min(q[u], rows - 1);
      const int t = qq / nlev;
      k[u] = 2 * (qq - t * nlev) + kpar;
      col[u] = __ldg(cc + t);
      q[u] = q[u] < rows ? qq : -1;
    }
    T v[U];
#pragma unroll
    for (int u = 0; u < U; ++u) v[u] = ic0_value<T, C, FWD>(S.g, col[u], k[u], cb + max(q[u], 0), F, r, y);
#pragma unroll
    for (int u = 0; u < U; ++u)
      if (q[u] >= 0) y[(int64_t)col[u] * nz + k[u]] = v[u];
  }
}

// Phase ph of the 16 IC0 colour phases: forward sweeps of colours 0..7, then backward 7..0.
template <typename T>
__device__ __forceinline__ void ic0_phase(const Sys& S, int ph) {
  switch (ph) {
    case 0: ic0_colour<T, 0, true>(S); break;
    case 1: ic0_colour<T, 1, true>(S); break;
    case 2: ic0_colour<T, 2, true>(S); break;
    case 3: ic0_colour<T, 3, true>(S); break;
    case 4: ic0_colour<T, 4, true>(S); break;
    case 5: ic0_colour<T, 5, true>(S); break;
    case 6: ic0_colour<T, 6, true>(S); break;
    case 7: ic0_colour<T, 7, true>(S); break;
    case 8: ic0_colour<T, 7, false>(S); break;
    case 9: ic0_colour<T, 6, false>(S); break;
    case 10: ic0_colour<T, 5, false>(S); break;
    case 11: ic0_colour<T, 4, false>(S); break;
    case 12: ic0_colour<T, 3, false>(S); break;
    case 13: ic0_colour<T, 2, false>(S); break;
    case 14: ic0_colour<T, 1, false>(S); break;
    default: ic0_colour<T, 0, false>(S); break;
  }
}

// Ordered list (shared memory) of the systems s for which want(s) holds, built by every block in
// one parallel pass (one thread per system); returns its length. Blocks build it before each
// phase, so that they visit only the systems they have work in, not every system in turn.
template <typename P>
__device__ int block_list(int nsys, P want, int* list, int* wsum) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  int base = 0;
  for (int s0 = 0; s0 < nsys; s0 += blockDim.x) {
    const int s = s0 + threadIdx.x;
    const bool a = s < nsys && want(s);
    const unsigned m = __ballot_sync(0xffffffffu, a);
    __syncthreads();
    if (lane == 0) wsum[wid] = __popc(m);
    __syncthreads();
    int off = base, tot = base;
    for (int w = 0; w < nw; ++w) {
      off += w < wid ? wsum[w] : 0;
      tot += wsum[w];
    }
    if (a) list[off + __popc(m & ((1u << lane) - 1u))] = s;
    base = tot;
  }
  __syncthreads();
  return base;
}

// Tiles a block owns in a system: t = blockIdx.x mod gridDim.x within the system's range, so
// which block runs a tile never changes the sums.
__device__ __forceinline__ int first_owned(const Sys* sys, int s) {
  const int G = gridDim.x, t0 = sys[s].tile0;
  return t0 + (((int)blockIdx.x - t0) % G + G) % G;
}

// The systems active in phase MODE in which this block owns at least one tile.
__device__ __forceinline__ int phase_list(const Scal* scal, const Sys* sys, int nsys, int mode, int* list, int* wsum) {
  return block_list(
      nsys, [&](int s) { return phase_active(scal[s].state, mode) && first_owned(sys, s) < sys[s].tile0 + sys[s].ntiles; },
      list, wsum);
}

// Whether this block has a chunk of colour c's rows in system S (the first chunk ic0_colour takes).
__device__ __forceinline__ bool owns_ic0_chunk(const Sys& S, int c) {
  const int rows = S.cls_cnt[c & 3] * S.nlev[c >> 2];
  const int chunk = 4 * (int)blockDim.x, G = gridDim.x;
  return (((int)blockIdx.x - S.tile0 % G + G) % G) < (rows + chunk - 1) / chunk;
}

// for (t over the tiles this block owns among the systems active in MODE; tl = tile t)
#define FOR_OWNED_TILES(MODE, t, tl)                                                                \
  for (int a_ = 0, na_ = phase_list(scal, sys, nsys, MODE, slist, wsum); a_ < na_; ++a_)           \
    for (int t = first_owned(sys, slist[a_]), te_ = sys[slist[a_]].tile0 + sys[slist[a_]].ntiles; \
         t < te_; t += gridDim.x)                                                                   \
      if (const Tile tl = tile_of(sys[slist[a_]], slist[a_], t); true)

// The 16 colour phases of an IC0 apply over the IC0 systems active in MODE (SHIFT systems
// skipped), a grid barrier after each: a phase reads rows that the previous phases wrote anywhere
// in the system. Leaves the kernel (return) when a barrier times out.
#define IC0_PHASES(MODE)                                                                            \
  for (int ph_ = 0; ph_ < 16; ++ph_) {                                                              \
    const int c_ = ph_ < 8 ? ph_ : 15 - ph_;                                                        \
    const int na_ = block_list(                                                                     \
        nsys,                                                                                       \
        [&](int s) {                                                                                \
          const int st = scal[s].state;                                                             \
          return phase_active(st, MODE) && st != ST_SHIFT && sys[s].prec == PM_PREC_IC0 &&          \
                 owns_ic0_chunk(sys[s], c_);                                                        \
        },                                                                                          \
        slist, wsum);                                                                               \
    for (int a_ = 0; a_ < na_; ++a_) ic0_phase<T>(sys[slist[a_]], ph_);                             \
    if (!grid_barrier(ctl)) return;                                                                 \
  }

// Resident blocks of 256 threads per SM the register budget is sized for: 3 (80 registers, about
// 1 KB of spills per thread) keeps 24 warps per SM in flight. The kernel is latency-bound, and on
// the batched 64-basin workloads 3 measured faster than 2 (128 registers, no spills): IC0 mass
// systems 0.41 -> 0.36 s, the FP32 line batch 8.84 -> 8.49 s.
#ifndef PM_BATCH_MINB
#define PM_BATCH_MINB 3
#endif

template <typename T>
__global__ void __launch_bounds__(256, PM_BATCH_MINB) k_batch(const Sys* __restrict__ sys, Scal* scal, int nsys,
                                               int ntiles, double* part, Ctl* ctl,
                                               int quantum, int init, int ic0) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  int* slist = reinterpret_cast<int*>(smem_raw);                             // nsys entries
  T* smt = reinterpret_cast<T*>(smem_raw + ((size_t)nsys * 4 + 15) / 16 * 16);  // tile of columns
  __shared__ double red[NP * 32];
  __shared__ int wsum[32];
  const int tid = threadIdx.x;

  // ---- initialisation of NEW systems: projected right-hand side, r = b' (x = 0), z, p, rho --------
  // Runs on the init launch of a batch and, for systems admitted between launches (continuous
  // batching), at the start of the next launch; systems already iterating wait at the barriers.
  if (init || *((volatile int32_t*)&ctl->pending) != 0) {
    // I1: tile partials of 1'b (pressure)
    FOR_OWNED_TILES(3, t, tl) {
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
      if (scal[s].state != ST_NEW) continue;
      const double sb = sys_reduce(part, ntiles, 0, S.tile0, S.ntiles, red);
      if (tid == 0) scal[s].proj_c = S.proj ? sb / S.one_m : 0.0;  // lambda, reused below
    }
    if (!grid_barrier(ctl)) return;
    // I2: b' = b - lambda m; x = 0; r = b'; z = P^{-1} r (Jacobi / line) and partials
    FOR_OWNED_TILES(3, t, tl) {
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
      if (S.prec == PM_PREC_IC0) {   // z comes from the colour phases below; the partials after them
        __syncthreads();
        continue;
      }
      __syncthreads();
      if (S.prec == PM_PREC_LINE && tid < tl.ncols)
        line_sweep<T>(smt + tid * ld, (const T*)S.lineF, tl.col0 + tid, S.g.ncols, (int)S.g.n, nz);
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
    if (ic0) {
      IC0_PHASES(3)
      FOR_OWNED_TILES(3, t, tl) {   // partials of the IC0 systems: (b', b'), (r, z), m'z, 1'r
        const Sys& S = sys[tl.sys];
        if (S.prec != PM_PREC_IC0) continue;
        const int nz = S.g.nz, row0 = tl.col0 * nz, rows = tl.ncols * nz;
        double v[NP] = {0.0, 0.0, 0.0, 0.0};
        for (int i = tid; i < rows; i += blockDim.x) {
          const int row = row0 + i;
          const double bi = S.bw[row];
          const T ri = ((const T*)S.r)[row], zi = ((const T*)S.z)[row];
          v[0] = fma(bi, bi, v[0]);
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
    }
    for (int s = blockIdx.x; s < nsys; s += gridDim.x) {
      const Sys& S = sys[s];
      if (scal[s].state != ST_NEW) continue;
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
        c.state = tot[0] == 0.0 ? ST_DONE : ST_PINIT;
        c.rel_true = 0.0;
        c.prev_true = -1.0;
      }
    }
    if (!grid_barrier(ctl)) return;
    // p = z - c
    FOR_OWNED_TILES(4, t, tl) {
      const Sys& S = sys[tl.sys];
      const int nz = S.g.nz, row0 = tl.col0 * nz, rows = tl.ncols * nz;
      const T c = (T)scal[tl.sys].proj_c;
      for (int i = tid; i < rows; i += blockDim.x) ((T*)S.p)[row0 + i] = ldcg(((const T*)S.z) + row0 + i) - c;
    }
    if (!grid_barrier(ctl)) return;
    for (int s = blockIdx.x; s < nsys; s += gridDim.x)
      if (tid == 0 && scal[s].state == ST_PINIT) scal[s].state = ST_ITER;
    if (blockIdx.x == 0 && tid == 0) ctl->pending = 0;
    if (!grid_barrier(ctl)) return;
  }

  for (int it = 0; it < quantum; ++it) {
    if (*((volatile int32_t*)&ctl->active) == 0) return;
    // ---- A: SpMV + (p, w) | REFINE: FP64 residual --------------------------------------------------
    FOR_OWNED_TILES(0, t, tl) {
      const Sys& S = sys[tl.sys];
      const int state = scal[tl.sys].state;
      const int nz = S.g.nz, row0 = tl.col0 * nz, rows = tl.ncols * nz;
      double v[NP] = {0.0, 0.0, 0.0, 0.0};
      if (state == ST_ITER) {
        if (std::is_same<T, float>::value && S.vbf16) {
          switch (S.maskc) {
            case 0: v[0] = spmv_tile<T, 0, __nv_bfloat16>(S, row0, rows, nz); break;
            case 1: v[0] = spmv_tile<T, 1, __nv_bfloat16>(S, row0, rows, nz); break;
            case 2: v[0] = spmv_tile<T, 2, __nv_bfloat16>(S, row0, rows, nz); break;
            default: v[0] = spmv_tile<T, -1, __nv_bfloat16>(S, row0, rows, nz); break;
          }
        } else {
          switch (S.maskc) {
            case 0: v[0] = spmv_tile<T, 0>(S, row0, rows, nz); break;
            case 1: v[0] = spmv_tile<T, 1>(S, row0, rows, nz); break;
            case 2: v[0] = spmv_tile<T, 2>(S, row0, rows, nz); break;
            default: v[0] = spmv_tile<T, -1>(S, row0, rows, nz); break;
          }
        }
      } else if (state == ST_REFINE) {
        switch (S.maskc) {
          case 0: refine_tile<T, 0>(S, row0, rows, nz, v[0], v[1]); break;
          case 1: refine_tile<T, 1>(S, row0, rows, nz, v[0], v[1]); break;
          case 2: refine_tile<T, 2>(S, row0, rows, nz, v[0], v[1]); break;
          default: refine_tile<T, -1>(S, row0, rows, nz, v[0], v[1]); break;
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
          // done at rtol, or below the FP64 floor once a restart no longer halves the residual
          const bool stalled = c.prev_true >= 0.0 && c.rel_true > 0.5 * c.prev_true;
          const bool last = c.iter >= c.max_iter || c.outer > 64;
          c.prev_true = c.rel_true;
          if (c.rel_true <= c.rtol || (c.rel_true <= c.rel_floor && (stalled || last))) {
            c.state = S.proj ? ST_SHIFT : ST_DONE;
          } else if (last) {
            c.status = PM_NOT_CONVERGED;
            c.state = S.proj ? ST_SHIFT : ST_DONE;
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
    FOR_OWNED_TILES(1, t, tl) {
      const Sys& S = sys[tl.sys];
      const int state = scal[tl.sys].state;
      double v[NP] = {0.0, 0.0, 0.0, 0.0};
      AccFor<T> acc[NP];   // FP64 for FP64 systems, compensated FP32 for FP32 ones
      if (state == ST_SHIFT) {  // partial of m'x for the zero-mean shift
        const int nz = S.g.nz, row0 = tl.col0 * nz, rows = tl.ncols * nz;
        for (int i = tid; i < rows; i += blockDim.x) v[0] = fma(S.m[row0 + i], S.x[row0 + i], v[0]);
      } else if (state == ST_ITER || state == ST_RESTART) {
        const int nz = S.g.nz, ld = nz + 1, row0 = tl.col0 * nz, rows = tl.ncols * nz;
        const double alpha = state == ST_ITER ? scal[tl.sys].alpha : 0.0;
        T* r = (T*)S.r;
        T* z = (T*)S.z;
        const T* p = (const T*)S.p;
        const T* w = (const T*)S.w;
        const int bd = blockDim.x;
        double* xg = S.x;
        constexpr int U = 4;  // rows i0 + u bd: all loads first, then updates and stores
        for (int i0 = tid; i0 < rows; i0 += U * bd) {
          T rv[U], pv[U], wv[U];
          double xv[U];
#pragma unroll
          for (int u = 0; u < U; ++u) {
            const int row = row0 + min(i0 + u * bd, rows - 1);
            rv[u] = ldcg(r + row);
            if (state == ST_ITER) {
              pv[u] = ldcg(p + row);
              wv[u] = ldcg(w + row);
              xv[u] = ldcg(xg + row);
            }
          }
#pragma unroll
          for (int u = 0; u < U; ++u) {
            const int i = i0 + u * bd;
            if (i < rows) {
              const int row = row0 + i;
              T ri = rv[u];
              if (state == ST_ITER) {
                xg[row] = fma(alpha, (double)pv[u], xv[u]);
                ri = ri - (T)alpha * wv[u];
                r[row] = ri;
              }
              acc[0].add_prod(ri, ri);
              if (S.prec == PM_PREC_LINE) smt[(i / nz) * ld + i % nz] = ri;
            }
          }
        }
        __syncthreads();
        if (S.prec == PM_PREC_IC0) {   // z from the colour phases after this one, (r, z), m'z, 1'r after them
          v[0] = acc[0].value();
          goto b_partials;
        }
        if (S.prec == PM_PREC_LINE && tid < tl.ncols)
          line_sweep<T>(smt + tid * ld, (const T*)S.lineF, tl.col0 + tid, S.g.ncols, (int)S.g.n, nz);
        __syncthreads();
        const bool line = S.prec == PM_PREC_LINE;
        const T* dinv = (const T*)S.dinv;
        for (int i0 = tid; i0 < rows; i0 += U * bd) {
          T rv[U], dv[U];
          double mv[U];
          float2 m2v[U];
#pragma unroll
          for (int u = 0; u < U; ++u) {
            const int row = row0 + min(i0 + u * bd, rows - 1);
            rv[u] = ldcg(r + row);
            dv[u] = line ? (T)0 : __ldg(dinv + row);
            if (std::is_same<T, float>::value) m2v[u] = S.proj ? __ldg(S.m2 + row) : make_float2(0.f, 0.f);
            else mv[u] = S.proj ? __ldg(S.m + row) : 0.0;
          }
#pragma unroll
          for (int u = 0; u < U; ++u) {
            const int i = i0 + u * bd;
            if (i < rows) {
              const T ri = rv[u];
              const T zi = line ? smt[(i / nz) * ld + i % nz] : (T)(dv[u] * ri);
              z[row0 + i] = zi;
              acc[1].add_prod(ri, zi);
              if (S.proj) {
                if constexpr (std::is_same<T, float>::value) {
                  acc[2].add_prod(m2v[u].x, zi);
                  acc[2].add_prod(m2v[u].y, zi);
                } else {
                  acc[2].add_prod(mv[u], zi);
                }
                acc[3].add(ri);
              }
            }
          }
        }
        for (int l = 0; l < NP; ++l) v[l] = acc[l].value();
      }
    b_partials:
      block_sum<NP>(v, red);
      if (tid == 0)
        for (int l = 0; l < NP; ++l) part[(int64_t)l * ntiles + t] = v[l];
      __syncthreads();
    }
    if (!grid_barrier(ctl)) return;
    if (ic0) {
      IC0_PHASES(1)
      FOR_OWNED_TILES(1, t, tl) {   // (r, z), m'z, 1'r of IC0 systems' ITER / RESTART tiles into lanes 1..3
        const Sys& S = sys[tl.sys];
        if (scal[tl.sys].state == ST_SHIFT || S.prec != PM_PREC_IC0) continue;
        const int nz = S.g.nz, row0 = tl.col0 * nz, rows = tl.ncols * nz;
        AccFor<T> acc[NP];
        for (int i = tid; i < rows; i += blockDim.x) {
          const int row = row0 + i;
          const T ri = ldcg((const T*)S.r + row), zi = ldcg((const T*)S.z + row);
          acc[1].add_prod(ri, zi);
          if (S.proj) {
            if constexpr (std::is_same<T, float>::value) {
              const float2 m2 = __ldg(S.m2 + row);
              acc[2].add_prod(m2.x, zi);
              acc[2].add_prod(m2.y, zi);
            } else {
              acc[2].add_prod(__ldg(S.m + row), zi);
            }
            acc[3].add(ri);
          }
        }
        double v[NP] = {0.0, acc[1].value(), acc[2].value(), acc[3].value()};
        block_sum<NP>(v, red);
        if (tid == 0)
          for (int l = 1; l < NP; ++l) part[(int64_t)l * ntiles + t] = v[l];
        __syncthreads();
      }
      if (!grid_barrier(ctl)) return;
    }
    // ---- Br ------------------------------------------------------------------------------------------
    for (int s = blockIdx.x; s < nsys; s += gridDim.x) {
      const Sys& S = sys[s];
      Scal& c = scal[s];
      const int state = c.state;
      if (state != ST_ITER && state != ST_RESTART && state != ST_SHIFT) continue;
      double tot[NP];
      for (int l = 0; l < NP; ++l) tot[l] = sys_reduce(part, ntiles, l, S.tile0, S.ntiles, red);
      if (tid == 0) {
        const double cc = S.proj ? tot[2] / S.one_m : 0.0;
        const double rho_new = tot[1] - cc * tot[3];
        if (state == ST_SHIFT) {
          c.proj_c = tot[0] / S.one_m;  // x -= m'x / 1'm in phase C
          c.state = ST_SHIFT2;
        } else if (state == ST_RESTART) {
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
    // ---- C: p = (z - c) + beta p | SHIFT2: x -= shift; count systems still active -----------------------
    if (blockIdx.x == 0) {
      int act = 0;
      for (int s0 = 0; s0 < nsys; s0 += blockDim.x) {
        const int st = s0 + tid < nsys ? scal[s0 + tid].state : (int)ST_DONE;
        act += __syncthreads_count(st != ST_DONE && st != ST_SHIFT2);
      }
      if (tid == 0) ctl->active = act;
    }
    FOR_OWNED_TILES(2, t, tl) {
      const Sys& S = sys[tl.sys];
      const int nz = S.g.nz, row0 = tl.col0 * nz, rows = tl.ncols * nz;
      if (scal[tl.sys].state == ST_SHIFT2) {
        const double sh = scal[tl.sys].proj_c;
        for (int i = tid; i < rows; i += blockDim.x) S.x[row0 + i] -= sh;
        continue;
      }
      const T beta = (T)scal[tl.sys].beta, c = (T)scal[tl.sys].proj_c;
      T* p = (T*)S.p;
      const T* z = (const T*)S.z;
      const int bd = blockDim.x;
      constexpr int U = 4;
      for (int i0 = tid; i0 < rows; i0 += U * bd) {
        T zv[U], pv[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
          const int row = row0 + min(i0 + u * bd, rows - 1);
          zv[u] = ldcg(z + row);
          pv[u] = ldcg(p + row);
        }
#pragma unroll
        for (int u = 0; u < U; ++u)
          if (i0 + u * bd < rows) p[row0 + i0 + u * bd] = (zv[u] - c) + beta * pv[u];
      }
    }
    if (!grid_barrier(ctl)) return;
    // SHIFT2 -> DONE; no phase before the next C reads SHIFT2 or DONE as active, so no barrier
    for (int s = blockIdx.x; s < nsys; s += gridDim.x)
      if (tid == 0 && scal[s].state == ST_SHIFT2) scal[s].state = ST_DONE;
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
  std::vector<int32_t> precs;      // preconditioner of each entry
  bool any_ic0 = false;            // the kernel runs the IC0 colour phases
  int tile_cols = 32, block = 256, grid = 0;
  int nz_max = 0;
  int64_t ntiles = 0;
  std::vector<pm::batch::Sys> hsys;
  pm::batch::Sys* d_sys = nullptr;
  pm::batch::Scal* d_scal = nullptr;
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

// Columns per tile of a system with nz levels: tile_cols, widened for shallow columns toward
// PM_TILE_ROWS_PER_THREAD rows per thread of the block (every tile visit costs a block reduction
// of its partials and a chain of dependent loads, whatever its size; 16 measured faster than 4 on
// the batched mass and line workloads). A line-preconditioned tile keeps at most one column per
// thread for its sweep.
#ifndef PM_TILE_ROWS_PER_THREAD
#define PM_TILE_ROWS_PER_THREAD 16
#endif
int tile_width(int nz, int prec, int tile_cols, int block) {
  int tc = std::max(tile_cols, (PM_TILE_ROWS_PER_THREAD * block + nz - 1) / nz);
  if (prec == PM_PREC_LINE) tc = std::min(tc, block);
  return tc;
}

// Dynamic shared memory: the ordered system list, and a line tile of columns (nz + 1 per column)
// for the widest tile of any nz up to nz_max.
size_t kernel_smem(int nsys, int tile_cols, int block, int nz_max, int precision) {
  const size_t es = precision == PM_FP64 ? sizeof(double) : sizeof(float);
  size_t cols = 0;
  for (int nz = 1; nz <= nz_max; ++nz)
    cols = std::max(cols, (size_t)tile_width(nz, PM_PREC_LINE, tile_cols, block) * (nz + 1));
  return ((size_t)nsys * 4 + 15) / 16 * 16 + cols * es;
}

size_t smem_bytes(const pm_batch* bt) {
  return kernel_smem(bt->count, bt->tile_cols, bt->block, bt->nz_max, bt->precision);
}

// Descriptor of one system: operator values (FP64, or the FP32 difference form), Jacobi
// diagonal, the preconditioner's factors (line: Thomas factors; IC0: factor, column-class index,
// grid parities, colour bases, level counts), mass vector. Vectors and tiles are set by the caller.
void fill_sys(Sys* S, pm_operator* op, int w, int prec, int precision) {
  const int vs = which_valset(w);
  const bool f32 = precision != PM_FP64;
  *S = Sys{};
  S->g = geom_of(op);
  S->val = precision == PM_BF16_REFINE ? (const void*)op->d_val16[vs]
           : f32                       ? (const void*)op->d_val32[vs]
                                       : (const void*)op->d_val[vs];
  S->vbf16 = precision == PM_BF16_REFINE ? 1 : 0;
  S->val64 = op->d_val[vs];
  S->dinv = f32 ? (const void*)op->d_dinv32[w] : (const void*)op->d_dinv[w];
  S->lineF = prec == PM_PREC_LINE ? (f32 ? (const void*)op->d_line32[w] : (const void*)op->d_line[w]) : nullptr;
  S->m = op->d_m;
  S->m2 = op->d_m2f;
  S->one_m = op->one_m;
  S->maskc = which_mask(w);
  S->proj = w == PM_OP_PRESSURE;
  S->prec = prec;
  S->ic0F = nullptr;
  if (prec != PM_PREC_IC0) return;
  S->ic0F = f32 ? (const void*)op->d_ic0_32[w] : (const void*)op->ic0[w].F;
  S->cls_cols = op->d_cls_cols;
  for (int c = 0, off = 0; c < 4; ++c) {
    S->cls_off[c] = off;
    S->cls_cnt[c] = op->cls_count[c];
    off += op->cls_count[c];
  }
  S->nlev[0] = (op->nz + 1) / 2;
  S->nlev[1] = op->nz / 2;
  int64_t acc = 0;
  for (int c = 0; c < 8; ++c) {
    S->cbase[c] = acc;
    acc += (int64_t)op->cls_count[c & 3] * S->nlev[c >> 2];
  }
}

bool known_prec(int p) { return p == PM_PREC_JACOBI || p == PM_PREC_IC0 || p == PM_PREC_NONE || p == PM_PREC_LINE; }

// Preconditioner of one entry: its own choice, or the default for PM_PREC_DEFAULT; NONE runs as
// Jacobi. Both arguments are known preconditioners (or PM_PREC_DEFAULT for `given`).
int entry_prec(int given, int dflt) {
  const int p = given == PM_PREC_DEFAULT ? dflt : given;
  return p == PM_PREC_NONE ? PM_PREC_JACOBI : p;
}

void free_layout(pm_batch* bt) {
  if (bt->graph) cudaGraphExecDestroy(bt->graph);
  bt->graph = nullptr;
  cudaFree(bt->d_sys);
  cudaFree(bt->d_scal);
  cudaFree(bt->d_ctl);
  cudaFree(bt->d_part);
  cudaFree(bt->work);
  bt->d_sys = nullptr;
  bt->d_scal = nullptr;
  bt->d_ctl = nullptr;
  bt->d_part = nullptr;
  bt->work = nullptr;
}

// Tiles, descriptors and workspace for the current tile width.
int build_layout(pm_batch* bt) {
  free_layout(bt);
  const bool f32 = bt->precision != PM_FP64;
  const size_t es = f32 ? sizeof(float) : sizeof(double);
  int64_t ntiles = 0;
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
    Sys& S = bt->hsys[s];
    fill_sys(&S, op, bt->which[s], bt->precs[s], bt->precision);
    S.r = take(op->n * es);
    S.p = take(op->n * es);
    S.w = take(op->n * es);
    S.z = take(op->n * es);
    S.bw = (double*)take(op->n * sizeof(double));
    S.tw = tile_width(op->nz, bt->precs[s], bt->tile_cols, bt->block);
    S.tile0 = (int32_t)ntiles;
    S.ntiles = (op->ncols + S.tw - 1) / S.tw;
    ntiles += S.ntiles;
    bt->nz_max = std::max(bt->nz_max, op->nz);
  }
  bt->ntiles = ntiles;
  st = cuda_check(cudaMalloc((void**)&bt->d_sys, bt->count * sizeof(Sys)), "batch sys");
  if (!st) st = cuda_check(cudaMalloc((void**)&bt->d_scal, bt->count * sizeof(Scal)), "batch scal");
  if (!st) st = cuda_check(cudaMalloc((void**)&bt->d_ctl, sizeof(Ctl)), "batch ctl");
  if (!st) st = cuda_check(cudaMalloc((void**)&bt->d_part, (size_t)NP * ntiles * sizeof(double)), "batch partials");
  return st;
}

template <typename T>
cudaError_t launch_k(int grid, int block, size_t smem, const Sys* d_sys, Scal* d_scal, int nsys, int ntiles, double* d_part, Ctl* d_ctl, int quantum, int init, int ic0, cudaStream_t s) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(grid);
  cfg.blockDim = dim3(block);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeCooperative;
  attr[0].val.cooperative = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  count_launch();
  return cudaLaunchKernelEx(&cfg, k_batch<T>, d_sys, d_scal, nsys, ntiles, d_part, d_ctl, quantum, init, ic0);
}

template <typename T>
cudaError_t launch(pm_batch* bt, int quantum, int init, cudaStream_t s) {
  return launch_k<T>(bt->grid, bt->block, smem_bytes(bt), bt->d_sys, bt->d_scal, (int)bt->count,
                     (int)bt->ntiles, bt->d_part, bt->d_ctl, quantum, init, bt->any_ic0 ? 1 : 0, s);
}

// Capture one launch (made by `fn` on the capture stream) into an executable graph.
template <typename F>
int capture_graph(cudaGraphExec_t* exec, F fn) {
  if (*exec) cudaGraphExecDestroy(*exec);
  *exec = nullptr;
  cudaStream_t cs;
  int st = cuda_check(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking), "capture stream");
  if (st) return st;
  cudaGraph_t g;
  cudaError_t e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
  if (e == cudaSuccess) {
    const cudaError_t le = fn(cs);
    e = cudaStreamEndCapture(cs, &g);
    if (le != cudaSuccess) e = le;
  }
  if (e == cudaSuccess) {
    e = cudaGraphInstantiate(exec, g, 0);
    cudaGraphDestroy(g);
  }
  cudaStreamDestroy(cs);
  return cuda_check(e, "batched PCG graph capture");
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
    hs[i].state = ST_NEW;
  }
  Ctl c = {0, 0, 0, bt->count, 1, 0};
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
    const int st = capture_graph(&bt->graph, [&](cudaStream_t cs) {
      return bt->precision == PM_FP64 ? launch<double>(bt, quantum, 0, cs) : launch<float>(bt, quantum, 0, cs);
    });
    if (st) return st;
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
  std::vector<Scal> hs(bt->count);
  int st = cuda_check(cudaMemcpyAsync(hs.data(), bt->d_scal, bt->count * sizeof(Scal), cudaMemcpyDeviceToHost, s), "scal");
  if (!st) st = cuda_check(cudaStreamSynchronize(s), "batched PCG finish");
  if (st) return st;
  int worst = PM_OK;
  const double es = bt->precision == PM_FP64 ? 8.0 : 4.0;                    // vector bytes
  const double vb = bt->precision == PM_FP64 ? 8.0 : bt->precision == PM_FP32_REFINE ? 4.0 : 2.0;  // values
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
      o.bytes_moved = c.iter * n * (15 * vb + 11 * es + 8 + 8) + c.outer * n * (15 * 8 + 24);
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
  int prec_mask = 0;
  for (int p : bt->precs) prec_mask |= 1 << p;
  TuneKey key{bucket, bt->count, bt->precision, prec_mask, bt->nz_max};
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

extern "C" int pm_batch_create(pm_operator* const* ops, const pm_which* which, const int32_t* prec, int32_t count,
                               const pm_solve_opts* opts, int32_t autotune, pm_batch** out, pm_stream stream) {
  if (!ops || !which || !opts || !out || count <= 0 || count > 4096) return set_error(PM_EINVAL, "bad batch arguments");
  *out = nullptr;
  if (!batch::known_prec(opts->prec)) return set_error(PM_EINVAL, "unknown preconditioner");
  for (int i = 0; prec && i < count; ++i)
    if (prec[i] != PM_PREC_DEFAULT && !batch::known_prec(prec[i]))
      return set_error(PM_EINVAL, "unknown preconditioner in the per-entry list");
  if (opts->precision != PM_FP64 && opts->precision != PM_FP32_REFINE && opts->precision != PM_BF16_REFINE)
    return set_error(PM_EINVAL, "unknown precision");
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
    const int pi = batch::entry_prec(prec ? prec[i] : PM_PREC_DEFAULT, bt->prec);
    int st = prepare_for_batch(ops[i], (int)which[i], pi, bt->precision, s);
    if (st) {
      delete bt;
      return st;
    }
    bt->ops.push_back(ops[i]);
    bt->which.push_back((int32_t)which[i]);
    bt->precs.push_back(pi);
    bt->any_ic0 = bt->any_ic0 || pi == PM_PREC_IC0;
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
  NvtxRange range("pm_batch_solve " + std::to_string(bt->count) + " systems");
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
  std::vector<pm_solve_stats> local(bt->count);
  const int fs = batch::finish(bt, local.data(), s, secs);
  if (stats) std::copy(local.begin(), local.end(), stats);
  if (log_enabled())
    for (int i = 0; i < bt->count; ++i)
      log_solve("batch_solve", bt->ops[i], bt->which[i], bt->precs[i], bt->precision, local[i]);
  const int bs = bounds_status("pm_batch_solve");
  return bs ? bs : st ? st : fs;
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
  int st = pm_batch_create(ops, which, nullptr, count, opts, 0, &bt, stream);
  if (st) return st;
  st = pm_batch_solve(bt, b, x, stats, stream);
  pm_batch_destroy(bt);
  return st;
}

// ================================= continuous batching server ======================================
// A fixed table of slots, each one system (operator x which) with caller-owned vectors and Krylov
// workspace. Systems are admitted and retired between launches of the persistent kernel: a new
// system is initialised at the start of the next launch (state NEW) while the others keep their
// state; a finished one (DONE) frees its slot and its tile range. The kernel takes the whole slot
// table (empty slots are DONE and cost nothing) and the tile capacity (the stride of the partials
// buffer) as arguments, so the captured graph stays valid until that capacity has to grow. Each
// system owns a range of tile indices [tile0, tile0 + ntiles): its partials' slots.

struct pm_server {
  int32_t cap = 0, nz_cap = 0;
  int precision = PM_FP64, prec = PM_PREC_JACOBI;
  double rtol = 1e-8, inner_rtol = 1e-2;
  int32_t max_iter = 100000;
  int tile_cols = 64, block = 128, grid = 0, device = 0;
  std::vector<pm::batch::Sys> hsys;
  std::vector<pm_operator*> ops;
  std::vector<int32_t> which;
  std::vector<int32_t> precs;   // preconditioner of each slot's system
  int32_t n_ic0 = 0;            // used slots with IC0: the kernel runs the colour phases
  int graph_ic0 = 0;
  std::vector<uint8_t> used;
  std::vector<int64_t> tile0, ntiles;
  int64_t tcap = 0;
  pm::batch::Sys* d_sys = nullptr;
  pm::batch::Scal* d_scal = nullptr;
  pm::batch::Ctl* d_ctl = nullptr;
  double* d_part = nullptr;
  pm::batch::Scal* h_scal = nullptr;  // pinned mirror, refreshed after every launch
  pm::batch::Ctl* h_ctl = nullptr;    // pinned: [0] read back, [1] upload staging
  int32_t pending = 0;
  cudaGraphExec_t graph = nullptr;
  int graph_quantum = 0;
  int64_t graph_tcap = 0;
  int64_t launches = 0;
};

namespace pm {
namespace batch {
namespace {

size_t server_smem(const pm_server* sv) {
  return kernel_smem(sv->cap, sv->tile_cols, sv->block, sv->nz_cap, sv->precision);
}

void server_free(pm_server* sv) {
  if (sv->graph) cudaGraphExecDestroy(sv->graph);
  cudaFree(sv->d_sys);
  cudaFree(sv->d_scal);
  cudaFree(sv->d_ctl);
  cudaFree(sv->d_part);
  cudaFreeHost(sv->h_scal);
  cudaFreeHost(sv->h_ctl);
}

// Tile capacity >= want: reallocate the partials (their contents need not survive a launch
// boundary); the graph is re-captured later.
int server_grow_tiles(pm_server* sv, int64_t want) {
  if (want <= sv->tcap) return PM_OK;
  int64_t nc = std::max<int64_t>(sv->tcap * 2, 1024);
  while (nc < want) nc *= 2;
  if (nc > (int64_t)1 << 30) return set_error(PM_ENOMEM, "server tile capacity too large");
  double* np = nullptr;
  const int st = cuda_check(cudaMalloc((void**)&np, (size_t)NP * nc * sizeof(double)), "server partials");
  if (st) return st;
  cudaFree(sv->d_part);
  sv->d_part = np;
  sv->tcap = nc;
  return PM_OK;
}

// First-fit tile range of `need` tiles among the occupied slots' ranges; grows the array if none.
int server_tile_range(pm_server* sv, int64_t need, int64_t* t0) {
  std::vector<std::pair<int64_t, int64_t>> occ;
  for (int i = 0; i < sv->cap; ++i)
    if (sv->used[i]) occ.push_back({sv->tile0[i], sv->tile0[i] + sv->ntiles[i]});
  std::sort(occ.begin(), occ.end());
  int64_t cur = 0;
  for (auto& r : occ) {
    if (r.first - cur >= need) break;
    cur = std::max(cur, r.second);
  }
  if (cur + need > sv->tcap) {
    const int st = server_grow_tiles(sv, cur + need);
    if (st) return st;
  }
  *t0 = cur;
  return PM_OK;
}

}  // namespace
}  // namespace batch
}  // namespace pm

extern "C" size_t pm_server_workspace_bytes(const pm_operator* op, int32_t precision) {
  if (!op) return 0;
  const size_t es = precision == PM_FP64 ? sizeof(double) : sizeof(float);
  auto up = [](size_t b) { return (b + 255) / 256 * 256; };
  return 4 * up((size_t)op->n * es) + up((size_t)op->n * sizeof(double));
}

extern "C" int pm_server_create(int32_t slots, int32_t nz_cap, const pm_solve_opts* opts, int32_t tile_cols,
                                int32_t block, int32_t blocks_per_sm, pm_server** out, pm_stream stream) {
  using namespace pm::batch;
  if (!opts || !out || slots <= 0 || slots > 4096 || nz_cap < 2 || nz_cap > 4096)
    return set_error(PM_EINVAL, "bad server arguments");
  *out = nullptr;
  if (!known_prec(opts->prec)) return set_error(PM_EINVAL, "unknown preconditioner");
  if (opts->precision != PM_FP64 && opts->precision != PM_FP32_REFINE && opts->precision != PM_BF16_REFINE)
    return set_error(PM_EINVAL, "unknown precision");
  if (!(opts->rtol > 0.0)) return set_error(PM_EINVAL, "rtol must be > 0");
  if (tile_cols != 16 && tile_cols != 32 && tile_cols != 64) return set_error(PM_EINVAL, "tile_cols must be 16, 32 or 64");
  if ((block != 128 && block != 256) || tile_cols > block) return set_error(PM_EINVAL, "block must be 128 or 256");
  if (blocks_per_sm < 0) return set_error(PM_EINVAL, "blocks_per_sm must be >= 0");
  pm_server* sv = new pm_server();
  sv->cap = slots;
  sv->nz_cap = nz_cap;
  sv->precision = opts->precision;
  sv->prec = opts->prec == PM_PREC_NONE ? PM_PREC_JACOBI : opts->prec;
  sv->rtol = opts->rtol;
  sv->inner_rtol = opts->inner_rtol > 0.0 ? opts->inner_rtol : 1e-2;
  sv->max_iter = opts->max_iter > 0 ? opts->max_iter : 100000;
  sv->tile_cols = tile_cols;
  sv->block = block;
  cudaGetDevice(&sv->device);
  sv->hsys.assign(slots, Sys{});
  sv->ops.assign(slots, nullptr);
  sv->which.assign(slots, 0);
  sv->precs.assign(slots, 0);
  sv->used.assign(slots, 0);
  sv->tile0.assign(slots, 0);
  sv->ntiles.assign(slots, 0);
  const size_t smem = server_smem(sv);
  int st = smem > 160 * 1024 ? set_error(PM_EINVAL, "tile_cols x (nz_cap + 1) does not fit in shared memory") : PM_OK;
  if (!st) {
    cudaFuncSetAttribute(k_batch<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, 160 * 1024);
    cudaFuncSetAttribute(k_batch<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, 160 * 1024);
    const int per_sm = sv->precision == PM_FP64 ? max_blocks<double>(block, smem) : max_blocks<float>(block, smem);
    int sms = 0;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, sv->device);
    if (per_sm <= 0) st = set_error(PM_EINVAL, "server kernel cannot be resident with this block / tile shape");
    sv->grid = sms * (blocks_per_sm > 0 ? std::min(per_sm, (int)blocks_per_sm) : per_sm);
  }
  if (!st) st = cuda_check(cudaMalloc((void**)&sv->d_sys, slots * sizeof(Sys)), "server sys");
  if (!st) st = cuda_check(cudaMalloc((void**)&sv->d_scal, slots * sizeof(Scal)), "server scal");
  if (!st) st = cuda_check(cudaMalloc((void**)&sv->d_ctl, sizeof(Ctl)), "server ctl");
  if (!st) st = cuda_check(cudaMallocHost((void**)&sv->h_scal, slots * sizeof(Scal)), "server scal mirror");
  if (!st) st = cuda_check(cudaMallocHost((void**)&sv->h_ctl, 2 * sizeof(Ctl)), "server ctl mirror");
  if (!st) st = server_grow_tiles(sv, 1024);
  if (!st) {
    for (int i = 0; i < slots; ++i) {
      std::memset(&sv->h_scal[i], 0, sizeof(Scal));
      sv->h_scal[i].state = ST_DONE;
    }
    std::memset(sv->h_ctl, 0, 2 * sizeof(Ctl));
    cudaStream_t s = (cudaStream_t)stream;
    st = cuda_check(cudaMemcpyAsync(sv->d_scal, sv->h_scal, slots * sizeof(Scal), cudaMemcpyHostToDevice, s), "scal");
    if (!st) st = cuda_check(cudaMemcpyAsync(sv->d_sys, sv->hsys.data(), slots * sizeof(Sys), cudaMemcpyHostToDevice, s), "sys");
    if (!st) st = cuda_check(cudaMemcpyAsync(sv->d_ctl, sv->h_ctl, sizeof(Ctl), cudaMemcpyHostToDevice, s), "ctl");
    if (!st) st = cuda_check(cudaStreamSynchronize(s), "server create");
  }
  if (st) {
    server_free(sv);
    delete sv;
    return st;
  }
  *out = sv;
  return PM_OK;
}

extern "C" int pm_server_admit(pm_server* sv, pm_operator* op, pm_which which, int32_t prec, const double* b,
                               double* x, void* work, size_t work_bytes, int32_t* slot, pm_stream stream) {
  using namespace pm::batch;
  if (!sv || !op || !b || !x || !work || !slot) return set_error(PM_EINVAL, "null server argument");
  *slot = -1;
  if (prec != PM_PREC_DEFAULT && !known_prec(prec)) return set_error(PM_EINVAL, "unknown preconditioner");
  const int pi = entry_prec(prec, sv->prec);
  if (!which_symmetric((int)which)) return set_error(PM_EINVAL, "server entry with a non-symmetric operator");
  if (op->nz > sv->nz_cap) return set_error(PM_EINVAL, "operator has more levels than the server's nz_cap");
  if (work_bytes < pm_server_workspace_bytes(op, sv->precision)) return set_error(PM_EINVAL, "workspace too small");
  if (((uintptr_t)work & 255) != 0) return set_error(PM_EINVAL, "workspace must be 256-byte aligned");
  int s_i = -1;
  for (int i = 0; i < sv->cap; ++i)
    if (!sv->used[i]) {
      s_i = i;
      break;
    }
  if (s_i < 0) return set_error(PM_EBUSY, "no free server slot");
  cudaStream_t s = (cudaStream_t)stream;
  int st = prepare_for_batch(op, (int)which, pi, sv->precision, s);
  if (st) return st;
  const int tw = tile_width(op->nz, pi, sv->tile_cols, sv->block);
  const int64_t need = (op->ncols + tw - 1) / tw;
  int64_t t0 = 0;
  if ((st = server_tile_range(sv, need, &t0))) return st;
  const bool f32 = sv->precision != PM_FP64;
  const size_t es = f32 ? sizeof(float) : sizeof(double);
  char* cur = (char*)work;
  auto take = [&](size_t bytes) {
    void* p = cur;
    cur += (bytes + 255) / 256 * 256;
    return p;
  };
  Sys& S = sv->hsys[s_i];
  fill_sys(&S, op, (int)which, pi, sv->precision);
  S.r = take(op->n * es);
  S.p = take(op->n * es);
  S.w = take(op->n * es);
  S.z = take(op->n * es);
  S.bw = (double*)take(op->n * sizeof(double));
  S.b = b;
  S.x = x;
  S.tile0 = (int32_t)t0;
  S.ntiles = (int32_t)need;
  S.tw = tw;
  Scal c;
  std::memset(&c, 0, sizeof(c));
  c.rtol = sv->rtol;
  c.inner_rtol = sv->inner_rtol;
  c.max_iter = sv->max_iter;
  c.state = ST_NEW;
  st = cuda_check(cudaMemcpyAsync(sv->d_sys + s_i, &S, sizeof(Sys), cudaMemcpyHostToDevice, s), "sys");
  if (!st) st = cuda_check(cudaMemcpyAsync(sv->d_scal + s_i, &c, sizeof(Scal), cudaMemcpyHostToDevice, s), "scal");
  if (st) return st;
  sv->h_scal[s_i] = c;
  sv->used[s_i] = 1;
  sv->ops[s_i] = op;
  sv->which[s_i] = (int32_t)which;
  sv->precs[s_i] = pi;
  sv->n_ic0 += pi == PM_PREC_IC0;
  sv->tile0[s_i] = t0;
  sv->ntiles[s_i] = need;
  sv->pending += 1;
  *slot = s_i;
  return PM_OK;
}

extern "C" int pm_server_run(pm_server* sv, int32_t quantum, int32_t* active, pm_stream stream) {
  using namespace pm::batch;
  if (!sv || quantum <= 0 || quantum > 4096) return set_error(PM_EINVAL, "bad server run arguments");
  cudaStream_t s = (cudaStream_t)stream;
  int busy = 0;
  for (int i = 0; i < sv->cap; ++i) busy += sv->used[i] && sv->h_scal[i].state != ST_DONE;
  if (busy == 0) {
    if (active) *active = 0;
    return PM_OK;
  }
  int st = PM_OK;
  if (sv->pending) {  // active / pending fields only; the barrier words and err stay as they are
    sv->h_ctl[1].active = busy;
    sv->h_ctl[1].pending = 1;
    st = cuda_check(cudaMemcpyAsync(&sv->d_ctl->active, &sv->h_ctl[1].active, 2 * sizeof(int32_t),
                                    cudaMemcpyHostToDevice, s), "ctl");
    if (st) return st;
  }
  const int ic0 = sv->n_ic0 > 0 ? 1 : 0;
  if (!sv->graph || sv->graph_quantum != quantum || sv->graph_tcap != sv->tcap || sv->graph_ic0 != ic0) {
    const size_t smem = server_smem(sv);
    st = capture_graph(&sv->graph, [&](cudaStream_t cs) {
      return sv->precision == PM_FP64
                 ? launch_k<double>(sv->grid, sv->block, smem, sv->d_sys, sv->d_scal, sv->cap,
                                    (int)sv->tcap, sv->d_part, sv->d_ctl, quantum, 0, ic0, cs)
                 : launch_k<float>(sv->grid, sv->block, smem, sv->d_sys, sv->d_scal, sv->cap,
                                   (int)sv->tcap, sv->d_part, sv->d_ctl, quantum, 0, ic0, cs);
    });
    if (st) return st;
    sv->graph_quantum = quantum;
    sv->graph_tcap = sv->tcap;
    sv->graph_ic0 = ic0;
  }
  NvtxRange range("pm_server_run");
  st = cuda_check(cudaGraphLaunch(sv->graph, s), "server graph launch");
  if (st) return st;
  count_launch();
  sv->launches += 1;
  sv->pending = 0;
  st = cuda_check(cudaMemcpyAsync(sv->h_scal, sv->d_scal, sv->cap * sizeof(Scal), cudaMemcpyDeviceToHost, s), "scal");
  if (!st) st = cuda_check(cudaMemcpyAsync(sv->h_ctl, sv->d_ctl, sizeof(Ctl), cudaMemcpyDeviceToHost, s), "ctl");
  if (!st) st = cuda_check(cudaStreamSynchronize(s), "server quantum");
  if (st) return st;
  if (sv->h_ctl[0].err) return set_error(sv->h_ctl[0].err, "server: a grid barrier wait expired");
  if ((st = bounds_status("pm_server_run"))) return st;
  busy = 0;
  for (int i = 0; i < sv->cap; ++i) busy += sv->used[i] && sv->h_scal[i].state != ST_DONE;
  if (active) *active = busy;
  return PM_OK;
}

extern "C" int pm_server_poll(pm_server* sv, int32_t* slots, pm_solve_stats* stats, int32_t max_out, int32_t* n_out) {
  using namespace pm::batch;
  if (!sv || !slots || !n_out || max_out < 0) return set_error(PM_EINVAL, "bad server poll arguments");
  int n = 0;
  const double es = sv->precision == PM_FP64 ? 8.0 : 4.0;                    // vector bytes
  const double vb = sv->precision == PM_FP64 ? 8.0 : sv->precision == PM_FP32_REFINE ? 4.0 : 2.0;  // values
  for (int i = 0; i < sv->cap && n < max_out; ++i) {
    if (!sv->used[i] || sv->h_scal[i].state != ST_DONE) continue;
    const Scal& c = sv->h_scal[i];
    slots[n] = i;
    if (stats) {
      pm_solve_stats& o = stats[n];
      std::memset(&o, 0, sizeof(o));
      o.iters = c.iter;
      o.outer_iters = c.outer;
      o.first_pass_iters = c.first_pass;
      o.status = c.status;
      o.rel_residual_true = c.rel_true;
      o.rel_residual_rec = c.bb > 0 ? std::sqrt(c.rr / c.bb) : 0.0;
      o.rel_residual_floor = c.rel_floor;
      const double nr = (double)sv->ops[i]->n;
      o.bytes_moved = c.iter * nr * (15 * vb + 11 * es + 8 + 8) + c.outer * nr * (15 * 8 + 24);
      if (log_enabled()) log_solve("server_solve", sv->ops[i], sv->which[i], sv->precs[i], sv->precision, o);
    }
    sv->used[i] = 0;
    sv->n_ic0 -= sv->precs[i] == PM_PREC_IC0;
    sv->ops[i] = nullptr;
    sv->ntiles[i] = 0;
    ++n;
  }
  *n_out = n;
  return PM_OK;
}

extern "C" int pm_server_info(const pm_server* sv, int32_t* tile_cols, int32_t* block, int32_t* grid, int64_t* tile_capacity,
                              int64_t* launches) {
  if (!sv) return set_error(PM_EINVAL, "null server");
  if (tile_cols) *tile_cols = sv->tile_cols;
  if (block) *block = sv->block;
  if (grid) *grid = sv->grid;
  if (tile_capacity) *tile_capacity = sv->tcap;
  if (launches) *launches = sv->launches;
  return PM_OK;
}

extern "C" void pm_server_destroy(pm_server* sv) {
  if (!sv) return;
  pm::batch::server_free(sv);
  delete sv;
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
