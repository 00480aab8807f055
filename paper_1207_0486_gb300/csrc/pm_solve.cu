// SpMV, preconditioner apply and preconditioned conjugate gradient on the column-sliced ELL
// layout (Section 5 remark: the linear systems are solved by PCG; IC0 for the velocity and mass
// systems, DIAG (Jacobi) for the pressure system with a zero-mean Lagrange multiplier).
//
// PCG follows Saad's preconditioned CG step for step (same order of updates, same stopping test
// ||r|| <= rtol ||b|| on the recursive residual, then a true-residual check with restarts):
//   K1 k_cg_spmv   : w = A p and the grid reduction (p, w); the last block forms alpha
//   K2 k_cg_update : x += alpha p, r -= alpha w, z = D^{-1} r (Jacobi, never stored), the grid
//                    reductions (r, r), (r, z) [and m'z, 1'r for the pressure]; the last block
//                    tests convergence and forms beta
//   K3 k_cg_pupd   : p = z + beta p
// IC0 replaces the inline z by 8 forward and 8 backward colour sweeps plus a (r, z) reduction.
// Grid reductions are deterministic: each block reduces its rows in a fixed tree, writes one
// partial, and the last block to arrive (atomic ticket) sums the partials in block order.
// All scalars (alpha, beta, rho, status) stay on the device; the host reads one small struct
// every few dozen iterations to see whether the solve has finished. Kernels of iterations
// issued after convergence return at once (the device "done" flag), so the result is the same
// as testing after every iteration.
#include <cuda_bf16.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <chrono>
#include <type_traits>

#include "pm_internal.cuh"

namespace pm {

struct SolveCtx {
  int64_t n = 0;
  int line_slots = 0, line_slots_nz = -1;  // resident blocks of the fused line kernel (per nz)
  double *r = nullptr, *p = nullptr, *w = nullptr, *z = nullptr, *bw = nullptr;
  double* partials = nullptr;
  PcgScalars* sc = nullptr;
  PcgScalars* sc_host = nullptr;
  // mixed precision (allocated on first use)
  float *r32 = nullptr, *p32 = nullptr, *w32 = nullptr, *z32 = nullptr, *d32 = nullptr;
  PcgScalars* sc_in = nullptr;
  PcgScalars* sc_in_host = nullptr;
  void* small_out = nullptr;        // SmallOut of the resident solve (device)
  void* small_out_host = nullptr;   // pinned host copy
};

struct ColourMap;  // pm_assemble.cu
}  // namespace pm

namespace pm {

// ---- live kernel timing (CUDA events on the launching stream) ------------------------------------
// When enabled, the host PCG loop brackets each launch of the timed kernel classes with a pair of
// events on the solve's stream; elapsed times are collected where that loop synchronises anyway.
// Process-global, not thread-safe: enable it from one host thread only.
struct KernelTimer {
  bool on = false;
  std::vector<cudaEvent_t> pool;
  struct Pending { cudaEvent_t a, b; int kind; int launches; };
  std::vector<Pending> pending;
  double total_ms[PM_KT_COUNT] = {};
  int64_t launches[PM_KT_COUNT] = {};
};
static KernelTimer g_kt;

static cudaEvent_t kt_event() {
  if (!g_kt.pool.empty()) {
    cudaEvent_t e = g_kt.pool.back();
    g_kt.pool.pop_back();
    return e;
  }
  cudaEvent_t e;
  cudaEventCreate(&e);
  return e;
}

struct KtScope {
  cudaEvent_t a = nullptr;
  cudaStream_t s;
  int kind, launches;
  KtScope(int kind_, int launches_, cudaStream_t s_) : s(s_), kind(kind_), launches(launches_) {
    if (g_kt.on) {
      a = kt_event();
      cudaEventRecord(a, s);
    }
  }
  ~KtScope() {
    if (a) {
      cudaEvent_t b = kt_event();
      cudaEventRecord(b, s);
      g_kt.pending.push_back({a, b, kind, launches});
    }
  }
};

static void kt_collect() {
  for (auto& p : g_kt.pending) {
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, p.a, p.b) == cudaSuccess) {
      g_kt.total_ms[p.kind] += ms;
      g_kt.launches[p.kind] += p.launches;
    }
    g_kt.pool.push_back(p.a);
    g_kt.pool.push_back(p.b);
  }
  g_kt.pending.clear();
}

namespace {

constexpr int TPB = 256;

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  return v;
}

// Reduce NV per-thread values over the block; thread 0 receives the sums. sm: NV * 32 doubles.
template <int NV>
__device__ __forceinline__ void block_sum(double (&v)[NV], double* sm) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const int nw = (blockDim.x + 31) >> 5;
#pragma unroll
  for (int i = 0; i < NV; ++i) {
    v[i] = warp_sum(v[i]);
    if (lane == 0) sm[i * 32 + wid] = v[i];
  }
  __syncthreads();
  if (wid == 0) {
#pragma unroll
    for (int i = 0; i < NV; ++i) {
      double t = lane < nw ? sm[i * 32 + lane] : 0.0;
      v[i] = warp_sum(t);
    }
  }
  __syncthreads();
}

// Grid reduction with a last-block finish. Returns true in the last block; there, thread 0 holds
// the grid totals in v. partials: NV * gridDim.x doubles; ticket: a zero-initialised counter
// that the last block resets.
template <int NV>
__device__ __forceinline__ bool grid_sum(double (&v)[NV], double* partials, uint32_t* ticket) {
  __shared__ double sm[NV * 32];
  __shared__ bool last;
  block_sum<NV>(v, sm);
  if (threadIdx.x == 0) {
#pragma unroll
    for (int i = 0; i < NV; ++i) partials[i * gridDim.x + blockIdx.x] = v[i];
    __threadfence();
    last = atomicAdd(ticket, 1u) == gridDim.x - 1;
  }
  __syncthreads();
  if (!last) return false;
  __threadfence();
  double acc[NV];
#pragma unroll
  for (int i = 0; i < NV; ++i) {
    double a = 0.0;
    for (int b = threadIdx.x; b < (int)gridDim.x; b += blockDim.x) a += __ldcg(partials + i * gridDim.x + b);
    acc[i] = a;
  }
  block_sum<NV>(acc, sm);
  if (threadIdx.x == 0) {
#pragma unroll
    for (int i = 0; i < NV; ++i) v[i] = acc[i];
    *ticket = 0;
  }
  return true;
}

__device__ __forceinline__ bool sc_done(const PcgScalars* sc) {
  return *((volatile const int32_t*)&sc->done) != 0;
}

// Row r of the (optionally masked) operator times x. MASKC >= 0: symmetric elimination of
// component MASKC's Dirichlet set (identity row, zero column).
// Branch-free: all 15 value loads are unconditional (absent slots hold 0), an absent or
// eliminated neighbour reads x[row] and multiplies a selected 0, so every load of a row can be
// in flight at once. 32-bit indices: the library caps n so that 15 * n_pad < 2^31.
template <int MASKC, typename TV, typename TX>
__device__ __forceinline__ double row_dot(const Geom& g, const TV* __restrict__ val, const TX* __restrict__ x,
                                          int row, int col, int k, bool& is_dir) {
  const int nz = g.nz;
  const int npad = (int)g.npad;
  int nb[NNBR];
  uint8_t fl[NNBR];
  nb[0] = col;
#pragma unroll
  for (int q = 1; q < NNBR; ++q) nb[q] = nbr_of(g, col, q);
  if (MASKC >= 0) {
#pragma unroll
    for (int q = 0; q < NNBR; ++q) fl[q] = __ldg(g.colflag + (nb[q] >= 0 ? nb[q] : col));
  }
  TV a[NSLOT];
#pragma unroll
  for (int s = 0; s < NSLOT; ++s) a[s] = __ldg(val + s * npad + row);
  double sum = 0.0;
#pragma unroll
  for (int s = 0; s < NSLOT; ++s) {
    const int q = slot_q(s);
    const int kk = k + slot_dk(s);
    bool ok = nb[q] >= 0;
    if (slot_dk(s) < 0) ok = ok && kk >= 0;
    if (slot_dk(s) > 0) ok = ok && kk < nz;
    if (MASKC >= 0) ok = ok && !is_dirichlet(fl[q], kk, nz, MASKC);
    const double xv = (double)x[ok ? nb[q] * nz + kk : row];
    const double av = ok ? (double)a[s] : 0.0;
    sum = fma(av, xv, sum);
  }
  if (MASKC >= 0) {
    is_dir = is_dirichlet(fl[0], k, nz, MASKC);
    if (is_dir) sum = (double)x[row];
  }
  return sum;
}

// Row r of component c's eliminated velocity operator times x, with the kept slots of the row
// read from its precomputed mask (bit s: slot s's neighbour present and not Dirichlet; bit 15:
// identity row). Same result as row_dot<c>, without the dependent column-flag loads.
template <typename TV, typename TX>
__device__ __forceinline__ double row_dot_keep(const Geom& g, const TV* __restrict__ val, const TX* __restrict__ x,
                                               const uint16_t* __restrict__ keep, int row, int col, int k) {
  const int nz = g.nz;
  const int npad = (int)g.npad;
  const uint32_t km = __ldg(keep + row);
  if (km & 0x8000u) return (double)x[row];
  int nb[NNBR];
  nb[0] = col;
#pragma unroll
  for (int q = 1; q < NNBR; ++q) nb[q] = nbr_of(g, col, q);
  TV a[NSLOT];
#pragma unroll
  for (int s = 0; s < NSLOT; ++s) a[s] = __ldg(val + s * npad + row);
  double sum = 0.0;
#pragma unroll
  for (int s = 0; s < NSLOT; ++s) {
    const bool ok = (km >> s) & 1u;
    const double xv = (double)x[ok ? nb[slot_q(s)] * nz + k + slot_dk(s) : row];
    sum = fma(ok ? (double)a[s] : 0.0, xv, sum);
  }
  return sum;
}

template <int MASKC>
__global__ void __launch_bounds__(TPB) k_spmv(Geom g, const double* __restrict__ val,
                                              const double* __restrict__ x, double* __restrict__ y) {
  const int n = (int)g.n;
  for (int row = blockIdx.x * blockDim.x + threadIdx.x; row < n; row += gridDim.x * blockDim.x) {
    const int col = row / g.nz;
    const int k = row - col * g.nz;
    bool d = false;
    y[row] = row_dot<MASKC>(g, val, x, row, col, k, d);
  }
}

// ---- PCG setup ---------------------------------------------------------------------------------

// Pressure only: lam = 1'b / 1'm, xshift = m'x / 1'm.
__global__ void __launch_bounds__(TPB) k_cg_press_sums(int64_t n, const double* __restrict__ b,
                                                       const double* __restrict__ x, const double* __restrict__ m,
                                                       int use_x, double* partials, PcgScalars* sc) {
  double v[2] = {0.0, 0.0};
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    v[0] += b[i];
    if (use_x) v[1] = fma(m[i], x[i], v[1]);
  }
  if (grid_sum<2>(v, partials, &sc->count[0]) && threadIdx.x == 0) {
    sc->lam = v[0] / sc->one_m;
    sc->xshift = use_x ? v[1] / sc->one_m : 0.0;
  }
}

// bw = b - lam m (pressure) and x = x - xshift (pressure) or x = 0 (no guess).
__global__ void k_cg_prepare(int64_t n, const double* __restrict__ b, const double* __restrict__ m,
                             double* __restrict__ bw, double* __restrict__ x, int press, int use_x,
                             const PcgScalars* sc) {
  const double lam = press ? sc->lam : 0.0, xs = press ? sc->xshift : 0.0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    if (press) bw[i] = b[i] - lam * m[i];
    x[i] = use_x ? x[i] - xs : 0.0;
  }
}

// r = bw - A x, row by row in compensated arithmetic (row_residual_dot2); grid sums (bw, bw),
// (r, r) and the floor's (|A||x| + |bw|)^2. MODE 0: first setup (also sets tol2, zero_rhs and
// the initial convergence test); MODE 1: true residual at exit (stores (r, r) in aux[0]).
template <int MASKC, int MODE>
__global__ void __launch_bounds__(TPB) k_cg_residual(Geom g, const double* __restrict__ val,
                                                     const double* __restrict__ bw, const double* __restrict__ x,
                                                     double* __restrict__ r, double rtol, double* partials,
                                                     PcgScalars* sc) {
  double v[3] = {0.0, 0.0, 0.0};
  const int n = (int)g.n;
  for (int row = blockIdx.x * blockDim.x + threadIdx.x; row < n; row += gridDim.x * blockDim.x) {
    const int col = row / g.nz;
    const int k = row - col * g.nz;
    double asum = 0.0;
    const double bi = bw[row];
    const double ri = row_residual_dot2<MASKC>(g, val, x, bi, row, col, k, asum);
    r[row] = ri;
    v[0] = fma(bi, bi, v[0]);
    v[1] = fma(ri, ri, v[1]);
    if (MODE == 1) {
      const double f = asum + fabs(bi);
      v[2] = fma(f, f, v[2]);
    }
  }
  if (grid_sum<3>(v, partials, &sc->count[1]) && threadIdx.x == 0) {
    if (MODE == 0) {
      sc->bb = v[0];
      sc->rr = v[1];
      sc->tol2 = rtol * rtol * v[0];
      sc->zero_rhs = v[0] == 0.0;
      sc->iter = 0;
      sc->status = PM_OK;
      sc->done = (v[0] == 0.0 || v[1] <= sc->tol2) ? 1 : 0;
      if (!sc->done && sc->max_iter == 0) {  // no iteration allowed: report the initial residual
        sc->status = PM_NOT_CONVERGED;
        sc->done = 1;
      }
    } else {
      sc->aux[0] = v[1];
      sc->aux[1] = v[2];
    }
  }
}

// First preconditioned residual (Jacobi or stored z): rho = (r, z') with z' = z - c 1,
// c = m'z / 1'm for the pressure (PROJ), p = z'. STORED: z read from zbuf.
template <int PROJ, int STORED>
__global__ void __launch_bounds__(TPB) k_cg_rho(int64_t n, const double* __restrict__ r, const double* __restrict__ dinv,
                                                const double* __restrict__ zbuf, const double* __restrict__ m,
                                                double* partials, PcgScalars* sc, int is_first) {
  if (!is_first && sc_done(sc)) return;
  double v[3] = {0.0, 0.0, 0.0};
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const double ri = r[i];
    const double zi = STORED ? zbuf[i] : dinv[i] * ri;
    v[0] = fma(ri, zi, v[0]);
    if (PROJ) {
      v[1] = fma(m[i], zi, v[1]);
      v[2] += ri;
    }
  }
  if (grid_sum<3>(v, partials, &sc->count[2]) && threadIdx.x == 0) {
    const double c = PROJ ? v[1] / sc->one_m : 0.0;
    const double rho_new = v[0] - c * v[2];
    sc->proj_c = c;
    if (is_first) {
      sc->rho = rho_new;
      sc->beta = 0.0;
    } else {
      sc->beta = rho_new / sc->rho;
      sc->rho = rho_new;
    }
    if (!(rho_new > 0.0) || !isfinite(rho_new)) {
      if (!sc->done) {
        sc->status = PM_BREAKDOWN;
        sc->done = 1;
      }
    }
  }
}

// p = (z - c) + beta p; beta = 0 on the first step. STORED: z from zbuf, else dinv r.
template <int STORED>
__global__ void __launch_bounds__(TPB) k_cg_pupd(int64_t n, const double* __restrict__ r, const double* __restrict__ dinv,
                                                 const double* __restrict__ zbuf, double* __restrict__ p,
                                                 const PcgScalars* sc, int is_first) {
  if (!is_first && sc_done(sc)) return;
  const double beta = sc->beta, c = sc->proj_c;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const double zi = (STORED ? zbuf[i] : dinv[i] * r[i]) - c;
    p[i] = is_first ? zi : fma(beta, p[i], zi);
  }
}

// ---- PCG iteration -----------------------------------------------------------------------------

// 256 threads, at most 64 registers: 4 blocks (32 warps) per SM to hide the gather latency.
template <int MASKC>
__global__ void __launch_bounds__(TPB, 4) k_cg_spmv(Geom g, const double* __restrict__ val, const double* __restrict__ p,
                                                    double* __restrict__ w, const uint16_t* __restrict__ keep,
                                                    double* partials, PcgScalars* sc) {
  if (sc_done(sc)) return;
  double v[1] = {0.0};
  const int n = (int)g.n;
  for (int row = blockIdx.x * blockDim.x + threadIdx.x; row < n; row += gridDim.x * blockDim.x) {
    const int col = row / g.nz;
    const int k = row - col * g.nz;
    bool d = false;
    const double wi = MASKC >= 0 ? row_dot_keep(g, val, p, keep, row, col, k) : row_dot<MASKC>(g, val, p, row, col, k, d);
    w[row] = wi;
    v[0] = fma(p[row], wi, v[0]);
  }
  if (grid_sum<1>(v, partials, &sc->count[3]) && threadIdx.x == 0) {
    const double pap = v[0];
    sc->pAp = pap;
    if (!(pap > 0.0) || !isfinite(pap)) {
      sc->status = PM_BREAKDOWN;
      sc->done = 1;
    } else {
      sc->alpha = sc->rho / pap;
    }
  }
}

// x += alpha p; r -= alpha w; (Jacobi, INLINE_Z) z = dinv r and its dots, else only (r, r).
template <int PROJ, int INLINE_Z>
__global__ void __launch_bounds__(TPB) k_cg_update(int64_t n, double* __restrict__ x, double* __restrict__ r,
                                                   const double* __restrict__ p, const double* __restrict__ w,
                                                   const double* __restrict__ dinv, const double* __restrict__ m,
                                                   double* partials, PcgScalars* sc) {
  if (sc_done(sc)) return;
  const double alpha = sc->alpha;
  double v[4] = {0.0, 0.0, 0.0, 0.0};
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    x[i] = fma(alpha, p[i], x[i]);
    const double ri = fma(-alpha, w[i], r[i]);
    r[i] = ri;
    v[0] = fma(ri, ri, v[0]);
    if (INLINE_Z) {
      const double zi = dinv[i] * ri;
      v[1] = fma(ri, zi, v[1]);
      if (PROJ) {
        v[2] = fma(m[i], zi, v[2]);
        v[3] += ri;
      }
    }
  }
  if (grid_sum<4>(v, partials, &sc->count[4]) && threadIdx.x == 0) {
    sc->iter += 1;
    sc->rr = v[0];
    if (v[0] <= sc->tol2) {
      sc->done = 1;
    } else if (sc->iter >= sc->max_iter) {
      sc->status = PM_NOT_CONVERGED;
      sc->done = 1;
    } else if (v[0] <= sc->aux[2]) {
      sc->done = 2;  // residual replacement requested (mixed precision): the host finishes the step
    } else if (INLINE_Z) {
      const double c = PROJ ? v[2] / sc->one_m : 0.0;
      const double rho_new = v[1] - c * v[3];
      sc->proj_c = c;
      sc->beta = rho_new / sc->rho;
      sc->rho = rho_new;
      if (!(rho_new > 0.0) || !isfinite(rho_new)) {
        sc->status = PM_BREAKDOWN;
        sc->done = 1;
      }
    }
  }
}

// ---- IC0 colour sweeps -------------------------------------------------------------------------
struct CMap {
  int64_t cbase[8];
  int32_t nlev[2];
};

// Forward (FWD = 1): y_i = (r_i - sum_{colour(j) < c} L_ij y_j) / L_ii over rows of colour c.
// Backward (FWD = 0): z_i = (y_i - sum_{colour(j) > c} L_ji z_j) / L_ii, in place on y.
// The factor's diagonal slot holds 1 / L_ii (a multiply instead of an FP64 division).
// Position t of colour COLOUR: column cls_cols[cls_off + t / nlev], level 2 (t % nlev) + parity.
// ic0_value returns the row's new value and its index; ic0_row stores it.
template <int COLOUR, int FWD, typename T>
__device__ __forceinline__ T ic0_value(const Geom& g, const CMap& cm, const int32_t* __restrict__ cls_cols,
                                       int64_t cls_off, int64_t t, const T* __restrict__ F,
                                       const T* __restrict__ r, const T* y, int64_t* row_out) {
  constexpr int kpar = COLOUR >> 2;
  const int nlev = cm.nlev[kpar];
  const int nz = g.nz;
  const int col = __ldg(cls_cols + cls_off + t / nlev);
  const int k = 2 * (int)(t % nlev) + kpar;
  const int64_t row = (int64_t)col * nz + k;
  const int64_t pi = cm.cbase[COLOUR] + t;
  T acc = FWD ? r[row] : y[row];
#pragma unroll
  for (int s = 0; s < NSLOT; ++s) {
    if (s == DIAG_SLOT) continue;
    const int cj = COLOUR ^ slot_flip(s);
    if (FWD ? (cj > COLOUR) : (cj < COLOUR)) continue;
    const int q = slot_q(s);
    const int kk = k + slot_dk(s);
    if (kk < 0 || kk >= nz) continue;
    const int nb = q == 0 ? col : nbr_of(g, col, q);
    if (nb < 0) continue;
    acc = fma(-F[(int64_t)s * g.n + pi], y[(int64_t)nb * nz + kk], acc);
  }
  *row_out = row;
  return acc * F[(int64_t)DIAG_SLOT * g.n + pi];
}

template <int COLOUR, int FWD>
__device__ __forceinline__ void ic0_row(const Geom& g, const CMap& cm, const int32_t* __restrict__ cls_cols,
                                        int64_t cls_off, int64_t t, const double* __restrict__ F,
                                        const double* __restrict__ r, double* __restrict__ y) {
  int64_t row;
  const double v = ic0_value<COLOUR, FWD>(g, cm, cls_cols, cls_off, t, F, r, y, &row);
  y[row] = v;
}

// One colour phase: two rows per thread (t and t + stride), both computed before either is
// stored (no row of a colour reads another row of that colour), so that each thread has both
// rows' neighbour gathers in flight. Launched over half the rows.
template <int COLOUR, int FWD, typename T>
__global__ void __launch_bounds__(TPB) k_ic0_sweep(Geom g, CMap cm, const int32_t* __restrict__ cls_cols,
                                                   int64_t cls_off, int64_t cls_cnt, const T* __restrict__ F,
                                                   const T* __restrict__ r, T* __restrict__ y,
                                                   const PcgScalars* sc, int check_done) {
  if (check_done && sc_done(sc)) return;
  const int64_t total = cls_cnt * cm.nlev[COLOUR >> 2];
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total; t += 2 * stride) {
    const bool two = t + stride < total;
    int64_t r0, r1 = 0;
    const T v0 = ic0_value<COLOUR, FWD>(g, cm, cls_cols, cls_off, t, F, r, y, &r0);
    T v1 = 0;
    if (two) v1 = ic0_value<COLOUR, FWD>(g, cm, cls_cols, cls_off, t + stride, F, r, y, &r1);
    y[r0] = v0;
    if (two) y[r1] = v1;
  }
}

// Grid of the reduction kernels: at most MAX_GRID blocks (the size of the partials buffer).
// ---- vertical-line block Jacobi ----------------------------------------------------------------
// P = block diagonal of A made of each column's tridiagonal block (rows k, couplings k-1 / k+1
// inside the column, the same Dirichlet elimination as A). Thomas factors per row, stored
// level-major (index k * ncols + column) so that one thread per column reads them coalesced:
//   lo_k = A[k, k-1],  w_k = 1 / (A[k, k] - lo_k cp_{k-1}),  cp_k = A[k, k+1] w_k.
__global__ void k_line_factor(Geom g, const double* __restrict__ val, int maskc, double* __restrict__ F,
                              int* __restrict__ breakdown) {
  const int nz = g.nz;
  const int64_t n = g.n;
  for (int64_t col = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; col < g.ncols;
       col += (int64_t)gridDim.x * blockDim.x) {
    const uint8_t fl = g.colflag[col];
    double cprev = 0.0;
    for (int k = 0; k < nz; ++k) {
      const int64_t row = col * nz + k;
      const bool di = maskc >= 0 && is_dirichlet(fl, k, nz, maskc);
      const double d = di ? 1.0 : val[(int64_t)DIAG_SLOT * g.npad + row];
      double lo = 0.0, up = 0.0;
      if (k > 0 && !di && !(maskc >= 0 && is_dirichlet(fl, k - 1, nz, maskc))) lo = val[row];
      if (k < nz - 1 && !di && !(maskc >= 0 && is_dirichlet(fl, k + 1, nz, maskc)))
        up = val[2 * g.npad + row];
      double piv = d - lo * cprev;
      if (!(piv > 0.0)) {
        atomicExch(breakdown, 1);
        piv = 1.0;
      }
      const double w = 1.0 / piv;
      const double cp = up * w;
      const int64_t li = (int64_t)k * g.ncols + col;
      F[li] = lo;
      F[n + li] = w;
      F[2 * n + li] = cp;
      cprev = cp;
    }
  }
}

constexpr int LINE_COLS = 64;
constexpr int LINE_TPB = 128;

// z = P^{-1} r for whole columns staged in shared memory, fused with the (r, z) [m'z, 1'r]
// reductions and the beta update (as k_cg_rho).
template <int PROJ>
__global__ void __launch_bounds__(LINE_TPB) k_line_rho(Geom g, const double* __restrict__ F,
                                                       const double* __restrict__ r, double* __restrict__ z,
                                                       const double* __restrict__ m, double* partials,
                                                       PcgScalars* sc, int is_first) {
  extern __shared__ double smem[];
  if (!is_first && sc_done(sc)) return;
  const int nz = g.nz, ld = nz + 1;
  double* sr = smem;
  double* sz = smem + LINE_COLS * ld;
  const int64_t n = g.n;
  const int64_t ntiles = (g.ncols + LINE_COLS - 1) / LINE_COLS;
  double v[3] = {0.0, 0.0, 0.0};
  for (int64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    const int64_t c0 = tile * LINE_COLS;
    const int cc = (int)min((int64_t)LINE_COLS, (int64_t)g.ncols - c0);
    const int64_t row0 = c0 * nz;
    const int rows = cc * nz;
    for (int i = threadIdx.x; i < rows; i += blockDim.x) sr[(i / nz) * ld + i % nz] = r[row0 + i];
    __syncthreads();
    if ((int)threadIdx.x < cc) {
      const int64_t col = c0 + threadIdx.x;
      const int base = threadIdx.x * ld;
      double y = 0.0;
      for (int k = 0; k < nz; ++k) {
        const int64_t li = (int64_t)k * g.ncols + col;
        y = (sr[base + k] - F[li] * y) * F[n + li];
        sz[base + k] = y;
      }
      double zn = sz[base + nz - 1];
      for (int k = nz - 2; k >= 0; --k) {
        const int64_t li = (int64_t)k * g.ncols + col;
        zn = fma(-F[2 * n + li], zn, sz[base + k]);
        sz[base + k] = zn;
      }
    }
    __syncthreads();
    for (int i = threadIdx.x; i < rows; i += blockDim.x) {
      const int si = (i / nz) * ld + i % nz;
      const double zi = sz[si], ri = sr[si];
      z[row0 + i] = zi;
      v[0] = fma(ri, zi, v[0]);
      if (PROJ) {
        v[1] = fma(m[row0 + i], zi, v[1]);
        v[2] += ri;
      }
    }
    __syncthreads();
  }
  if (grid_sum<3>(v, partials, &sc->count[2]) && threadIdx.x == 0) {
    const double c = PROJ ? v[1] / sc->one_m : 0.0;
    const double rho_new = v[0] - c * v[2];
    sc->proj_c = c;
    if (is_first) {
      sc->rho = rho_new;
      sc->beta = 0.0;
    } else {
      sc->beta = rho_new / sc->rho;
      sc->rho = rho_new;
    }
    if (!(rho_new > 0.0) || !isfinite(rho_new)) {
      if (!sc->done) {
        sc->status = PM_BREAKDOWN;
        sc->done = 1;
      }
    }
  }
}

// One PCG iteration's update with the vertical-line preconditioner fused in:
//   x += alpha p, r -= alpha w (rows of LINE_UCOLS whole columns, staged in shared memory),
//   z = P^{-1} r column by column (one thread per column, in place), then the reductions
//   (r, r), (r, z) [m'z, 1'r]. The last block tests convergence on (r, r) and forms beta, as
//   k_cg_update + k_line_rho would; the z of the converged iteration is simply not used.
constexpr int LINE_UCOLS = 128;   // FP32 fused kernel: columns (= threads) per block
#ifndef PM_LINE_FCOLS
#define PM_LINE_FCOLS 64
#endif
#ifndef PM_LINE_UNROLL
#define PM_LINE_UNROLL 8
#endif
constexpr int LINE_FCOLS = PM_LINE_FCOLS;  // FP64 fused kernel: columns per block (128 threads stage them)
constexpr int LINE_FTPB = 128;
constexpr int LINE_UNROLL = PM_LINE_UNROLL;  // levels of Thomas factors in flight per sweep thread

// NZ > 0: compile-time column height (shifts instead of divisions); NZ == 0: g.nz at run time.
template <int PROJ, int NZ>
__global__ void __launch_bounds__(LINE_FTPB) k_update_line(Geom g, const double* __restrict__ F,
                                                         double* __restrict__ x, double* __restrict__ r,
                                                         const double* __restrict__ p, const double* __restrict__ w,
                                                         double* __restrict__ z, const double* __restrict__ m,
                                                         double* partials, PcgScalars* sc, int nfull_max) {
  extern __shared__ double smem[];
  if (sc_done(sc)) return;
  const double alpha = sc->alpha;
  const int nz = NZ > 0 ? NZ : g.nz, ld = nz + 1;
  const int ncols = g.ncols;
  const int n = (int)g.n;
  const int ntiles = (ncols + LINE_FCOLS - 1) / LINE_FCOLS;
  double v[4] = {0.0, 0.0, 0.0, 0.0};
  // Tiles 0 .. nfull-1 are LINE_FCOLS columns wide (one per resident block: the first wave); the
  // columns left after them go in half-width tiles, so the second wave is short.
  const int nfull = min(ntiles, nfull_max);
  const int rest0 = nfull * LINE_FCOLS;
  const int nhalf = rest0 < ncols ? (ncols - rest0 + LINE_FCOLS / 2 - 1) / (LINE_FCOLS / 2) : 0;
  for (int tile = blockIdx.x; tile < nfull + nhalf; tile += gridDim.x) {
    const int c0 = tile < nfull ? tile * LINE_FCOLS : rest0 + (tile - nfull) * (LINE_FCOLS / 2);
    const int cc = min(tile < nfull ? LINE_FCOLS : LINE_FCOLS / 2, ncols - c0);
    const int row0 = c0 * nz;
    const int rows = cc * nz;
    for (int i = threadIdx.x; i < rows; i += blockDim.x) {
      const int row = row0 + i;
      x[row] = fma(alpha, p[row], x[row]);
      const double ri = fma(-alpha, w[row], r[row]);
      r[row] = ri;
      smem[(i / nz) * ld + i % nz] = ri;
      v[0] = fma(ri, ri, v[0]);
    }
    __syncthreads();
    if ((int)threadIdx.x < cc) {
      const int col = c0 + threadIdx.x;
      double* col_s = smem + threadIdx.x * ld;
      double y = 0.0;
#pragma unroll (LINE_UNROLL)
      for (int k = 0; k < nz; ++k) {
        const int li = k * ncols + col;
        y = (col_s[k] - F[li] * y) * F[n + li];
        col_s[k] = y;
      }
      double zn = y;
#pragma unroll (LINE_UNROLL)
      for (int k = nz - 2; k >= 0; --k) {
        const int li = k * ncols + col;
        zn = fma(-F[2 * n + li], zn, col_s[k]);
        col_s[k] = zn;
      }
    }
    __syncthreads();
    for (int i = threadIdx.x; i < rows; i += blockDim.x) {
      const int row = row0 + i;
      const double zi = smem[(i / nz) * ld + i % nz];
      const double ri = r[row];
      z[row] = zi;
      v[1] = fma(ri, zi, v[1]);
      if (PROJ) {
        v[2] = fma(m[row], zi, v[2]);
        v[3] += ri;
      }
    }
    __syncthreads();
  }
  if (grid_sum<4>(v, partials, &sc->count[4]) && threadIdx.x == 0) {
    sc->iter += 1;
    sc->rr = v[0];
    if (v[0] <= sc->tol2) {
      sc->done = 1;
    } else if (sc->iter >= sc->max_iter) {
      sc->status = PM_NOT_CONVERGED;
      sc->done = 1;
    } else {
      const double c = PROJ ? v[2] / sc->one_m : 0.0;
      const double rho_new = v[1] - c * v[3];
      sc->proj_c = c;
      sc->beta = rho_new / sc->rho;
      sc->rho = rho_new;
      if (!(rho_new > 0.0) || !isfinite(rho_new)) {
        sc->status = PM_BREAKDOWN;
        sc->done = 1;
      }
    }
  }
}

// The same fused iteration for 32-level columns, organised by warp instead of by block. A task is
// TCOLS = 32 whole columns (TCOLS * 32 consecutive rows, since node id = column * 32 + k); every
// warp owns an even, contiguous share of the tasks and the grid is exactly the resident blocks,
// so each SM gets the same work. Per task:
//   A (all lanes, coalesced): x += alpha p, r -= alpha w for level k = lane of each column, r
//     staged into the warp's own shared-memory tile [column][level];
//   B (lane = column): the Thomas sweep down and up the column in that tile;
//   C (all lanes, coalesced): z written, m'z.
// Warps never wait for one another (only __syncwarp), so one warp's sequential sweep overlaps
// other warps' streaming. (r, z) comes out of the sweep without reading r again: with the factors
// T = L U of the column block (L lower bidiagonal, diagonal 1/w_k, sub-diagonal lo_k; U unit
// upper bidiagonal, cp_k), a symmetric T has U = diag(w) L^T, so with t_k = r_k - lo_k y_{k-1},
// y_k = t_k w_k and z = U^{-1} y,  (r, z) = y' diag(1/w) y = sum_k t_k y_k.
constexpr int LINE_WNZ = 32;
constexpr int LINE_WTPB = 256;   // 8 warps per block
template <int PROJ, int TCOLS>
__global__ void __launch_bounds__(LINE_WTPB, TCOLS == 32 ? 3 : 4) k_update_line_w(
    Geom g, const double* __restrict__ F, double* __restrict__ x, double* __restrict__ r,
    const double* __restrict__ p, const double* __restrict__ w, double* __restrict__ z,
    const double* __restrict__ m, double* partials, PcgScalars* sc) {
  constexpr int NZ = LINE_WNZ, LD = NZ + 1;
  extern __shared__ double smem[];
  if (sc_done(sc)) return;
  const double alpha = sc->alpha;
  const int lane = threadIdx.x & 31;
  const int wib = threadIdx.x >> 5;
  double* ws = smem + wib * (TCOLS * LD);
  const int ncols = g.ncols;
  const int n = (int)g.n;
  const int nwarps = gridDim.x * (LINE_WTPB / 32);
  const int wg = blockIdx.x * (LINE_WTPB / 32) + wib;
  // this warp's tasks (TCOLS columns each, the last one ragged): an even split of all tasks over
  // all warps, so every block, hence every SM, gets the same work and every lane sweeps a column
  const int ntask = (ncols + TCOLS - 1) / TCOLS;
  const int tbeg = (int)((int64_t)ntask * wg / nwarps);
  const int tend = (int)((int64_t)ntask * (wg + 1) / nwarps);
  double v[4] = {0.0, 0.0, 0.0, 0.0};   // (r, r), (r, z), m'z, 1'r
  for (int t = tbeg; t < tend; ++t) {
    const int c0 = t * TCOLS;
    const int cc = min(TCOLS, ncols - c0);
    const int row0 = c0 * NZ + lane;
#pragma unroll 8
    for (int j = 0; j < cc; ++j) {
      const int row = row0 + j * NZ;
      x[row] = fma(alpha, p[row], x[row]);
      const double ri = fma(-alpha, w[row], r[row]);
      r[row] = ri;
      ws[j * LD + lane] = ri;
      v[0] = fma(ri, ri, v[0]);
      if (PROJ) v[3] += ri;
    }
    __syncwarp();
    if (lane < cc) {
      const int col = c0 + lane;
      double* cs = ws + lane * LD;
      double y = 0.0, rz = 0.0;
#pragma unroll 8
      for (int k = 0; k < NZ; ++k) {
        const int li = k * ncols + col;
        const double tk = fma(-F[li], y, cs[k]);
        y = tk * F[n + li];
        rz = fma(tk, y, rz);
        cs[k] = y;
      }
      double zn = y;
#pragma unroll 8
      for (int k = NZ - 2; k >= 0; --k) {
        const int li = k * ncols + col;
        zn = fma(-F[2 * n + li], zn, cs[k]);
        cs[k] = zn;
      }
      v[1] += rz;
    }
    __syncwarp();
#pragma unroll 8
    for (int j = 0; j < cc; ++j) {
      const int row = row0 + j * NZ;
      const double zi = ws[j * LD + lane];
      z[row] = zi;
      if (PROJ) v[2] = fma(m[row], zi, v[2]);
    }
    __syncwarp();
  }
  if (grid_sum<4>(v, partials, &sc->count[4]) && threadIdx.x == 0) {
    sc->iter += 1;
    sc->rr = v[0];
    if (v[0] <= sc->tol2) {
      sc->done = 1;
    } else if (sc->iter >= sc->max_iter) {
      sc->status = PM_NOT_CONVERGED;
      sc->done = 1;
    } else {
      const double c = PROJ ? v[2] / sc->one_m : 0.0;
      const double rho_new = v[1] - c * v[3];
      sc->proj_c = c;
      sc->beta = rho_new / sc->rho;
      sc->rho = rho_new;
      if (!(rho_new > 0.0) || !isfinite(rho_new)) {
        sc->status = PM_BREAKDOWN;
        sc->done = 1;
      }
    }
  }
}

// Columns per task: 32, so that every lane of a warp sweeps a column (an FP64 instruction costs the
// FP64 pipe the same with idle lanes, and the sweep is a third of the kernel's FP64 work), unless
// that leaves fewer tasks than resident warps (basins under about 600 x 600 columns of 32 levels):
// then 16, twice the warps and half the lanes sweeping. line_w_slots gives the resident tasks of
// one choice.
template <int TC>
int line_w_slots(const void* kernel, int num_sms) {
  const size_t smem = (size_t)(LINE_WTPB / 32) * TC * (LINE_WNZ + 1) * sizeof(double);
  cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  int per_sm = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, LINE_WTPB, smem);
  return std::max(1, per_sm) * num_sms;
}

template <int TC>
void launch_line_w(pm_operator* op, int which, bool proj, double* x, int slots, cudaStream_t s) {
  SolveCtx* c = op->ctx;
  Geom g = geom_of(op);
  const size_t smem = (size_t)(LINE_WTPB / 32) * TC * (LINE_WNZ + 1) * sizeof(double);
  int64_t blocks = std::min<int64_t>(slots, (int64_t)NPART * MAX_GRID / 4);
  const int64_t ntask = (op->ncols + TC - 1) / TC;
  blocks = std::min<int64_t>(blocks, (ntask + LINE_WTPB / 32 - 1) / (LINE_WTPB / 32));
  const int grid = (int)std::max<int64_t>(1, blocks);
  const double* F = op->d_line[which];
  if (proj)
    k_update_line_w<1, TC><<<grid, LINE_WTPB, smem, s>>>(g, F, x, c->r, c->p, c->w, c->z, op->d_m, c->partials, c->sc);
  else
    k_update_line_w<0, TC><<<grid, LINE_WTPB, smem, s>>>(g, F, x, c->r, c->p, c->w, c->z, op->d_m, c->partials, c->sc);
}

// Launch of k_update_line_w: exactly the resident blocks (capped by the partials buffer, 4 lanes
// per block, and by one task per warp).
void update_line_w(pm_operator* op, int which, bool proj, double* x, cudaStream_t s) {
  static int slots32 = 0, slots16 = 0;
  if (!slots32) {
    slots32 = line_w_slots<32>((const void*)k_update_line_w<1, 32>, op->num_sms);
    line_w_slots<32>((const void*)k_update_line_w<0, 32>, op->num_sms);
    slots16 = line_w_slots<16>((const void*)k_update_line_w<1, 16>, op->num_sms);
    line_w_slots<16>((const void*)k_update_line_w<0, 16>, op->num_sms);
  }
  const int64_t tasks32 = (op->ncols + 31) / 32;
  if (tasks32 >= (int64_t)slots32 * (LINE_WTPB / 32)) launch_line_w<32>(op, which, proj, x, slots32, s);
  else launch_line_w<16>(op, which, proj, x, slots16, s);
  count_launch();
}

void update_line(pm_operator* op, int which, bool proj, double* x, cudaStream_t s) {
  if (op->nz == LINE_WNZ) {
    update_line_w(op, which, proj, x, s);
    return;
  }
  SolveCtx* c = op->ctx;
  Geom g = geom_of(op);
  const size_t smem = (size_t)LINE_FCOLS * (op->nz + 1) * sizeof(double);
  static bool attr_set = false;
  if (!attr_set) {
    cudaFuncSetAttribute(k_update_line<0, 0>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
    cudaFuncSetAttribute(k_update_line<1, 0>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
    attr_set = true;
  }
  // resident blocks of this shape: the full-width tiles fill exactly one wave of them
  if (c->line_slots_nz != op->nz) {
    int per_sm = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_update_line<1, 0>, LINE_FTPB, smem);
    c->line_slots = std::max(1, per_sm) * op->num_sms;
    c->line_slots_nz = op->nz;
  }
  // four partial lanes per block must fit the partials buffer (NPART x MAX_GRID doubles)
  const int nfull_max = (int)std::min<int64_t>(c->line_slots, (int64_t)NPART * MAX_GRID / 4);
  const int64_t nt_full = (op->ncols + LINE_FCOLS - 1) / LINE_FCOLS;
  const int64_t nfull = std::min<int64_t>(nt_full, nfull_max);
  const int64_t rest = std::max<int64_t>(0, op->ncols - nfull * LINE_FCOLS);
  const int64_t ntiles = nfull + (rest + LINE_FCOLS / 2 - 1) / (LINE_FCOLS / 2);
  int grid = (int)std::min<int64_t>(ntiles, nfull_max);
  if (grid < 1) grid = 1;
  const double* F = op->d_line[which];
#define PM_UL(P, NZ)                                                                                     \
  k_update_line<P, NZ><<<grid, LINE_FTPB, smem, s>>>(g, F, x, c->r, c->p, c->w, c->z, op->d_m, c->partials, c->sc, \
                                                     nfull_max)
  if (op->nz == 32) {
    if (proj) PM_UL(1, 32);
    else PM_UL(0, 32);
  } else {
    if (proj) PM_UL(1, 0);
    else PM_UL(0, 0);
  }
#undef PM_UL
  count_launch();
}

void line_apply_rho(pm_operator* op, int which, bool proj, int is_first, cudaStream_t s) {
  SolveCtx* c = op->ctx;
  Geom g = geom_of(op);
  const int64_t ntiles = (op->ncols + LINE_COLS - 1) / LINE_COLS;
  int grid = (int)std::min<int64_t>(ntiles, std::min<int64_t>((int64_t)op->num_sms * 8, MAX_GRID));
  if (grid < 1) grid = 1;
  const size_t smem = 2 * (size_t)LINE_COLS * (op->nz + 1) * sizeof(double);
  static bool attr_set = false;
  if (!attr_set) {
    cudaFuncSetAttribute(k_line_rho<0>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
    cudaFuncSetAttribute(k_line_rho<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
    attr_set = true;
  }
  if (proj)
    k_line_rho<1><<<grid, LINE_TPB, smem, s>>>(g, op->d_line[which], c->r, c->z, op->d_m, c->partials, c->sc, is_first);
  else
    k_line_rho<0><<<grid, LINE_TPB, smem, s>>>(g, op->d_line[which], c->r, c->z, op->d_m, c->partials, c->sc, is_first);
  count_launch();
}

int line_factor(pm_operator* op, int which, cudaStream_t s) {
  if (op->line_ok[which]) return PM_OK;
  int st;
  if (!op->d_line[which]) {
    if ((st = cuda_check(cudaMalloc((void**)&op->d_line[which], 3 * (size_t)op->n * sizeof(double)), "cudaMalloc line")))
      return st;
    op->device_bytes += 3 * op->n * 8;
  }
  int* d_bd = nullptr;
  if ((st = cuda_check(cudaMallocAsync((void**)&d_bd, sizeof(int), s), "cudaMallocAsync"))) return st;
  cudaMemsetAsync(d_bd, 0, sizeof(int), s);
  Geom g = geom_of(op);
  int grid = (int)std::min<int64_t>((op->ncols + 127) / 128, (int64_t)op->num_sms * 16);
  if (grid < 1) grid = 1;
  k_line_factor<<<grid, 128, 0, s>>>(g, op->d_val[which_valset(which)], which_mask(which), op->d_line[which], d_bd);
  count_launch();
  int h = 0;
  st = cuda_check(cudaMemcpyAsync(&h, d_bd, sizeof(int), cudaMemcpyDeviceToHost, s), "memcpy");
  if (!st) st = cuda_check(cudaStreamSynchronize(s), "line factor");
  cudaFreeAsync(d_bd, s);
  if (st) return st;
  if (h) return set_error(PM_BREAKDOWN, "vertical-line preconditioner: non-positive pivot");
  op->line_ok[which] = true;
  return cuda_check(cudaGetLastError(), "k_line_factor");
}

int grid_for(int64_t n, int threads, int sms) {
  int64_t gsz = (n + threads - 1) / threads;
  int64_t cap = (int64_t)sms * 8;
  if (cap > MAX_GRID) cap = MAX_GRID;
  if (gsz > cap) gsz = cap;
  if (gsz < 1) gsz = 1;
  return (int)gsz;
}

CMap cmap_of(const pm_operator* op) {
  CMap cm;
  cm.nlev[0] = (op->nz + 1) / 2;
  cm.nlev[1] = op->nz / 2;
  int64_t acc = 0;
  for (int c = 0; c < 8; ++c) {
    cm.cbase[c] = acc;
    acc += (int64_t)op->cls_count[c & 3] * cm.nlev[c >> 2];
  }
  return cm;
}

void ic0_apply(pm_operator* op, int which, const double* r, double* z, const PcgScalars* sc,
               int check_done, cudaStream_t s) {
  Geom g = geom_of(op);
  CMap cm = cmap_of(op);
  const double* F = op->ic0[which].F;
  int64_t off[5] = {0, 0, 0, 0, 0};
  for (int c = 0; c < 4; ++c) off[c + 1] = off[c] + op->cls_count[c];
#define PM_SWEEP(C, FW)                                                                        \
  {                                                                                            \
    const int64_t cnt = op->cls_count[(C) & 3];                                                \
    const int64_t tot = cnt * cm.nlev[(C) >> 2];                                               \
    if (tot > 0) {                                                                             \
      k_ic0_sweep<C, FW, double><<<grid_for((tot + 1) / 2, TPB, op->num_sms), TPB, 0, s>>>(     \
          g, cm, op->d_cls_cols, off[(C) & 3], cnt, F, r, z, sc, check_done);                  \
      count_launch();                                                                          \
    }                                                                                          \
  }
  PM_SWEEP(0, 1) PM_SWEEP(1, 1) PM_SWEEP(2, 1) PM_SWEEP(3, 1)
  PM_SWEEP(4, 1) PM_SWEEP(5, 1) PM_SWEEP(6, 1) PM_SWEEP(7, 1)
  PM_SWEEP(7, 0) PM_SWEEP(6, 0) PM_SWEEP(5, 0) PM_SWEEP(4, 0)
  PM_SWEEP(3, 0) PM_SWEEP(2, 0) PM_SWEEP(1, 0) PM_SWEEP(0, 0)
#undef PM_SWEEP
}

int ensure_ctx(pm_operator* op) {
  if (op->ctx) return PM_OK;
  SolveCtx* c = new SolveCtx();
  c->n = op->n;
  const size_t vb = (size_t)op->n * sizeof(double);
  cudaError_t e = cudaSuccess;
  e = e ? e : cudaMalloc((void**)&c->r, vb);
  e = e ? e : cudaMalloc((void**)&c->p, vb);
  e = e ? e : cudaMalloc((void**)&c->w, vb);
  e = e ? e : cudaMalloc((void**)&c->z, vb);
  e = e ? e : cudaMalloc((void**)&c->bw, vb);
  e = e ? e : cudaMalloc((void**)&c->partials, (size_t)NPART * MAX_GRID * sizeof(double));
  e = e ? e : cudaMalloc((void**)&c->sc, sizeof(PcgScalars));
  e = e ? e : cudaMallocHost((void**)&c->sc_host, sizeof(PcgScalars));
  e = e ? e : cudaMalloc(&c->small_out, 64);
  e = e ? e : cudaMallocHost(&c->small_out_host, 64);
  if (e == cudaSuccess) e = cudaMemset(c->sc, 0, sizeof(PcgScalars));
  op->ctx = c;
  if (e != cudaSuccess) return cuda_check(e, "solve workspace");
  op->device_bytes += 5 * (int64_t)vb + (int64_t)NPART * MAX_GRID * 8 + (int64_t)sizeof(PcgScalars);
  return PM_OK;
}

template <int MASKC>
void launch_iter(pm_operator* op, int which, const double* val, double* x, bool proj, int prec,
                 const double* dinv, cudaStream_t s) {
  SolveCtx* c = op->ctx;
  Geom g = geom_of(op);
  const int G = grid_for(op->n, TPB, op->num_sms);
  const bool ic0 = prec == PM_PREC_IC0;
  {
    KtScope t(PM_KT_SPMV, 1, s);
    k_cg_spmv<MASKC><<<G, TPB, 0, s>>>(g, val, c->p, c->w, MASKC >= 0 ? op->d_keep[MASKC < 0 ? 0 : MASKC] : nullptr,
                                       c->partials, c->sc);
  }
  if (prec == PM_PREC_LINE) {
    {
      KtScope t(PM_KT_LINE, 1, s);
      update_line(op, which, proj, x, s);
    }
    {
      KtScope t(PM_KT_PUPDATE, 1, s);
      k_cg_pupd<1><<<G, TPB, 0, s>>>(op->n, c->r, dinv, c->z, c->p, c->sc, 0);
    }
    count_launch(1);
  } else if (!ic0) {
    {
      KtScope t(PM_KT_UPDATE, 1, s);
      if (proj) {
        k_cg_update<1, 1><<<G, TPB, 0, s>>>(op->n, x, c->r, c->p, c->w, dinv, op->d_m, c->partials, c->sc);
      } else {
        k_cg_update<0, 1><<<G, TPB, 0, s>>>(op->n, x, c->r, c->p, c->w, dinv, op->d_m, c->partials, c->sc);
      }
    }
    {
      KtScope t(PM_KT_PUPDATE, 1, s);
      k_cg_pupd<0><<<G, TPB, 0, s>>>(op->n, c->r, dinv, nullptr, c->p, c->sc, 0);
    }
    count_launch(3);
  } else {
    {
      KtScope t(PM_KT_UPDATE, 1, s);
      k_cg_update<0, 0><<<G, TPB, 0, s>>>(op->n, x, c->r, c->p, c->w, dinv, op->d_m, c->partials, c->sc);
    }
    count_launch(1);
    {
      KtScope t(PM_KT_IC0, 16, s);
      ic0_apply(op, which, c->r, c->z, c->sc, 1, s);
    }
    {
      KtScope t(PM_KT_PUPDATE, 2, s);
      if (proj) {
        k_cg_rho<1, 1><<<G, TPB, 0, s>>>(op->n, c->r, dinv, c->z, op->d_m, c->partials, c->sc, 0);
      } else {
        k_cg_rho<0, 1><<<G, TPB, 0, s>>>(op->n, c->r, dinv, c->z, op->d_m, c->partials, c->sc, 0);
      }
      k_cg_pupd<1><<<G, TPB, 0, s>>>(op->n, c->r, dinv, c->z, c->p, c->sc, 0);
    }
    count_launch(2);
  }
}

template <int MASKC>
void launch_residual(pm_operator* op, const double* val, const double* bw, const double* x, double rtol,
                     int mode, cudaStream_t s) {
  SolveCtx* c = op->ctx;
  Geom g = geom_of(op);
  const int G = grid_for(op->n, TPB, op->num_sms);
  if (mode == 0)
    k_cg_residual<MASKC, 0><<<G, TPB, 0, s>>>(g, val, bw, x, c->r, rtol, c->partials, c->sc);
  else
    k_cg_residual<MASKC, 1><<<G, TPB, 0, s>>>(g, val, bw, x, c->r, rtol, c->partials, c->sc);
  count_launch();
}

// z, p, rho from the current r (first step or restart). The kernels run even when "done" is
// set by the setup so that a zero initial residual still leaves consistent scalars.
void launch_first(pm_operator* op, int which, bool proj, int prec, const double* dinv, cudaStream_t s) {
  SolveCtx* c = op->ctx;
  const int G = grid_for(op->n, TPB, op->num_sms);
  if (prec == PM_PREC_LINE) {
    line_apply_rho(op, which, proj, 1, s);
    k_cg_pupd<1><<<G, TPB, 0, s>>>(op->n, c->r, dinv, c->z, c->p, c->sc, 1);
    count_launch(1);
    return;
  }
  if (prec == PM_PREC_IC0) {
    ic0_apply(op, which, c->r, c->z, c->sc, 0, s);
    if (proj) k_cg_rho<1, 1><<<G, TPB, 0, s>>>(op->n, c->r, dinv, c->z, op->d_m, c->partials, c->sc, 1);
    else k_cg_rho<0, 1><<<G, TPB, 0, s>>>(op->n, c->r, dinv, c->z, op->d_m, c->partials, c->sc, 1);
    k_cg_pupd<1><<<G, TPB, 0, s>>>(op->n, c->r, dinv, c->z, c->p, c->sc, 1);
  } else {
    if (proj) k_cg_rho<1, 0><<<G, TPB, 0, s>>>(op->n, c->r, dinv, nullptr, op->d_m, c->partials, c->sc, 1);
    else k_cg_rho<0, 0><<<G, TPB, 0, s>>>(op->n, c->r, dinv, nullptr, op->d_m, c->partials, c->sc, 1);
    k_cg_pupd<0><<<G, TPB, 0, s>>>(op->n, c->r, dinv, nullptr, c->p, c->sc, 1);
  }
  count_launch(2);
}

__global__ void k_fill(double* x, int64_t n, double v) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) x[i] = v;
}
__global__ void k_shift_by(double* x, int64_t n, const PcgScalars* sc) {
  const double v = sc->xshift;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) x[i] -= v;
}

int read_scalars(SolveCtx* c, cudaStream_t s) {
  int st = cuda_check(cudaMemcpyAsync(c->sc_host, c->sc, sizeof(PcgScalars), cudaMemcpyDeviceToHost, s), "scalars");
  if (st) return st;
  st = cuda_check(cudaStreamSynchronize(s), "pcg sync");
  if (!st && !g_kt.pending.empty()) kt_collect();
  return st;
}

// Algorithmic bytes of one PCG iteration per row (FP64), each array once per pass:
//   SpMV: 15 values + p read + w write = 136;
//   Jacobi: update x, r read/write + p, w, dinv read (z = dinv r inline) = 56, p-update r, dinv,
//           p read + p write = 32;
//   IC0: update x, r read/write + p, w read = 48, the factor (8 of its 15 slots per row in each
//        sweep direction) 128 and r, y, z traffic 32, the (r, z) pass 16, p-update z, p, p = 24;
//   LINE: update 48, the three line factors and the z write 32 (fused with the update), p-update 24.
// The pressure adds m (8) where m'z is taken.
double bytes_per_iter(const pm_operator* op, int prec, bool proj) {
  const double n = (double)op->n;
  double b = n * (15 * 8 + 8 + 8);
  if (prec == PM_PREC_IC0) b += n * (48 + 2 * 8 * 8 + 4 * 8 + 16 + 24);
  else if (prec == PM_PREC_LINE) b += n * (48 + 3 * 8 + 8 + 24);
  else b += n * (56 + 32);
  if (proj) b += n * 8;
  return b;
}

template <int MASKC>
int pcg_run(pm_operator* op, int which, const double* b, double* x, const pm_solve_opts* o,
            pm_solve_stats* stats, cudaStream_t s) {
  auto t0 = std::chrono::steady_clock::now();
  SolveCtx* c = op->ctx;
  const bool proj = which == PM_OP_PRESSURE;
  const bool ic0 = o->prec == PM_PREC_IC0;
  const int prec = o->prec;
  const double* val = op->d_val[which_valset(which)];
  int st;
  // Preconditioner set-up.
  const double* dinv = nullptr;
  if ((st = launch_dinv(op, which, s))) return st;
  dinv = op->d_dinv[which];
  double* ones_buf = nullptr;
  if (o->prec == PM_PREC_NONE) {
    ones_buf = c->z;  // plain CG: z = r, held as dinv = 1 in a scratch vector
    k_fill<<<grid_for(op->n, TPB, op->num_sms), TPB, 0, s>>>(ones_buf, op->n, 1.0);
    count_launch();
    dinv = ones_buf;
  }
  if (ic0) {
    Ic0Factor& f = op->ic0[which];
    if (!f.ok) {
      int bd = 0;
      double shift = 0.0;
      for (int m = -1; m <= 10; ++m) {
        shift = m < 0 ? 0.0 : 1e-3 * std::pow(2.0, m);
        if ((st = launch_ic0_factor(op, which, shift, &bd, s))) return st;
        if (!bd) break;
      }
      if (bd) return set_error(PM_BREAKDOWN, "IC0 pivot failure after the shift limit");
    }
  }
  if (prec == PM_PREC_LINE && (st = line_factor(op, which, s))) return st;
  // Right-hand side and initial guess.
  const int G = grid_for(op->n, TPB, op->num_sms);
  PcgScalars init;
  std::memset(&init, 0, sizeof(init));
  init.one_m = op->one_m;
  init.max_iter = o->max_iter;
  if ((st = cuda_check(cudaMemcpyAsync(c->sc, &init, sizeof(init), cudaMemcpyHostToDevice, s), "scalars init"))) return st;
  const double* bw = b;
  if (proj) {
    k_cg_press_sums<<<G, TPB, 0, s>>>(op->n, b, x, op->d_m, o->x0_is_guess ? 1 : 0, c->partials, c->sc);
    k_cg_prepare<<<G, TPB, 0, s>>>(op->n, b, op->d_m, c->bw, x, 1, o->x0_is_guess ? 1 : 0, c->sc);
    count_launch(2);
    bw = c->bw;
  } else if (!o->x0_is_guess) {
    k_cg_prepare<<<G, TPB, 0, s>>>(op->n, b, op->d_m, nullptr, x, 0, 0, c->sc);
    count_launch();
  }
  launch_residual<MASKC>(op, val, bw, x, o->rtol, 0, s);
  launch_first(op, which, proj, prec, dinv, s);
  if ((st = read_scalars(c, s))) return st;
  int restarts = 0;
  int first_pass = 0;
  int status = PM_OK;
  double rel_true = 0.0, rel_floor = 0.0, prev_true = -1.0;
  bool accepted = false;
  if (c->sc_host->zero_rhs) {
    k_fill<<<G, TPB, 0, s>>>(x, op->n, 0.0);
    count_launch();
    if ((st = read_scalars(c, s))) return st;
  } else {
    int64_t issued = 0;
    for (;;) {
      int chunk = 4;
      while (!c->sc_host->done) {
        // the device stops itself at max_iter; this bound only guards the host loop
        if (issued > (int64_t)o->max_iter + 4096)
          return set_error(PM_ECUDA, "PCG driver: device never reported completion");
        for (int it = 0; it < chunk; ++it) launch_iter<MASKC>(op, which, val, x, proj, prec, dinv, s);
        issued += chunk;
        if ((st = read_scalars(c, s))) return st;
        if (chunk < 64) chunk *= 2;
      }
      status = c->sc_host->status;
      if (restarts == 0) first_pass = c->sc_host->iter;
      // true residual
      launch_residual<MASKC>(op, val, bw, x, o->rtol, 1, s);
      if ((st = read_scalars(c, s))) return st;
      rel_true = std::sqrt(c->sc_host->aux[0] / c->sc_host->bb);
      rel_floor = std::ldexp(1.0, -53) * std::sqrt(c->sc_host->aux[1] / c->sc_host->bb);
      // Accepted when the (compensated, hence exact to one rounding) true residual meets rtol,
      // or when it lies below the floor that rounding x to FP64 alone can cause (backward error
      // at the unit roundoff) and restarts no longer lower it: the last restart did not halve
      // it, or no restart is left.
      const bool stalled = prev_true >= 0.0 && rel_true > 0.5 * prev_true;
      const bool last = restarts >= o->max_restarts || c->sc_host->iter >= o->max_iter;
      accepted = rel_true <= o->rtol || (rel_true <= rel_floor && (stalled || last));
      if (status != PM_OK || accepted || last) break;
      prev_true = rel_true;
      ++restarts;
      // restart from the true residual held in r
      PcgScalars* hs = c->sc_host;
      hs->done = 0;
      hs->rr = hs->aux[0];
      if ((st = cuda_check(cudaMemcpyAsync(c->sc, hs, sizeof(PcgScalars), cudaMemcpyHostToDevice, s), "scalars"))) return st;
      launch_first(op, which, proj, prec, dinv, s);
      if ((st = read_scalars(c, s))) return st;
    }
    if (status == PM_OK && !accepted) status = PM_NOT_CONVERGED;
  }
  if (proj) {
    // keep m'x = 0 exactly as returned result
    k_cg_press_sums<<<G, TPB, 0, s>>>(op->n, b, x, op->d_m, 1, c->partials, c->sc);
    k_shift_by<<<G, TPB, 0, s>>>(x, op->n, c->sc);
    count_launch(2);
    if ((st = read_scalars(c, s))) return st;
  }
  const PcgScalars* h = c->sc_host;
  if (stats) {
    stats->iters = h->iter;
    stats->outer_iters = restarts;
    stats->first_pass_iters = first_pass;
    stats->rel_residual_floor = rel_floor;
    stats->status = status;
    stats->rel_residual_true = h->zero_rhs ? 0.0 : rel_true;
    stats->rel_residual_rec = h->zero_rhs ? 0.0 : std::sqrt(h->rr / h->bb);
    stats->bytes_moved = h->iter * bytes_per_iter(op, prec, proj);
    stats->seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
  }
  if ((st = cuda_check(cudaGetLastError(), "pcg kernels"))) return st;
  if (status != PM_OK) {
    return set_error(status, status == PM_NOT_CONVERGED ? "PCG did not reach rtol within max_iter"
                                                        : "PCG breakdown: (p, Ap) <= 0 or non-finite");
  }
  return PM_OK;
}

// ---- resident solve of a small system: one block runs the whole PCG ----------------------------
// The multi-kernel solve costs about twenty launches per IC0 iteration; on a few thousand rows each
// of them is a few microseconds of launch latency around far less work. Here one block of
// SMALL_TPB threads runs every step of the same PCG (the same preconditioners, projection,
// stopping rule and true-residual restarts) with __syncthreads between phases, and writes its
// statistics to device memory once. The FP64 work of one SM bounds it; it is used where that
// is cheaper than the launches (n <= SMALL_AUTO_ROWS by default).
constexpr int SMALL_TPB = 256;
constexpr int64_t SMALL_AUTO_ROWS = 16384;   // automatic choice of the resident solve
constexpr int64_t SMALL_MAX_ROWS = 1 << 20;  // accepted when requested explicitly

struct SmallArgs {
  double rtol, one_m;
  int32_t max_iter, max_restarts, x0_is_guess, proj;
  const double* dinv;     // Jacobi inverse diagonal (ones for PM_PREC_NONE)
  const uint16_t* keep;   // keep mask of the velocity component (MASKC >= 0)
  const double* m;        // M 1
  const double* Fic;      // IC0 factor (colour-ordered rows)
  const double* Fl;       // line factors (level-major)
  const int32_t* cls_cols;
  CMap cm;
  int64_t cls_off[4], cls_cnt[4];
};

struct SmallOut {
  int32_t iters, restarts, first_pass, status, zero_rhs, pad;
  double rel_true, rel_rec, floor;
};

// Sum of NV values over the block; every thread receives the totals. red: NV * 32 + NV doubles.
// FP64 adds are what the reduction costs on this GPU (its FP64 pipe runs at 1/64 of FP32): the
// warps' partials are added by one thread per value, in warp order (deterministic), and the
// totals are read back from shared memory, rather than every thread adding them again.
template <int NV>
__device__ __forceinline__ void small_sum(double (&v)[NV], double* red) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const int nw = blockDim.x >> 5;
#pragma unroll
  for (int i = 0; i < NV; ++i) {
    double t = warp_sum(v[i]);
    if (lane == 0) red[i * 32 + wid] = t;
  }
  __syncthreads();
  if (threadIdx.x < NV) {
    double t = 0.0;
    for (int wv = 0; wv < nw; ++wv) t += red[threadIdx.x * 32 + wv];
    red[NV * 32 + threadIdx.x] = t;
  }
  __syncthreads();
#pragma unroll
  for (int i = 0; i < NV; ++i) v[i] = red[NV * 32 + i];
  __syncthreads();
}

template <int MASKC>
__device__ __forceinline__ double small_row(const Geom& g, const double* __restrict__ val, const double* x,
                                            const uint16_t* __restrict__ keep, int row) {
  const int col = row / g.nz, k = row - col * g.nz;
  bool d = false;
  return MASKC >= 0 ? row_dot_keep(g, val, x, keep, row, col, k) : row_dot<MASKC>(g, val, x, row, col, k, d);
}

// z = P^{-1} r for the whole system; leaves (r, z), m'z and 1'r in v (block totals).
template <int PREC>
__device__ __forceinline__ void small_precond(const Geom& g, const SmallArgs& a, const double* r, double* z,
                                              double (&v)[3], double* red) {
  const int n = (int)g.n, T = blockDim.x, tid = threadIdx.x;
  if (PREC == PM_PREC_IC0) {
#define PM_SMALL_PHASE(C, FW)                                                                            \
  {                                                                                                      \
    const int64_t tot = a.cls_cnt[(C) & 3] * a.cm.nlev[(C) >> 2];                                        \
    for (int64_t t = tid; t < tot; t += T) ic0_row<C, FW>(g, a.cm, a.cls_cols, a.cls_off[(C) & 3], t, a.Fic, r, z); \
    __syncthreads();                                                                                     \
  }
    PM_SMALL_PHASE(0, 1) PM_SMALL_PHASE(1, 1) PM_SMALL_PHASE(2, 1) PM_SMALL_PHASE(3, 1)
    PM_SMALL_PHASE(4, 1) PM_SMALL_PHASE(5, 1) PM_SMALL_PHASE(6, 1) PM_SMALL_PHASE(7, 1)
    PM_SMALL_PHASE(7, 0) PM_SMALL_PHASE(6, 0) PM_SMALL_PHASE(5, 0) PM_SMALL_PHASE(4, 0)
    PM_SMALL_PHASE(3, 0) PM_SMALL_PHASE(2, 0) PM_SMALL_PHASE(1, 0) PM_SMALL_PHASE(0, 0)
#undef PM_SMALL_PHASE
  } else if (PREC == PM_PREC_LINE) {
    const int nz = g.nz, ncols = g.ncols;
    for (int col = tid; col < ncols; col += T) {
      double y = 0.0;
      for (int k = 0; k < nz; ++k) {
        const int li = k * ncols + col;
        y = (r[col * nz + k] - a.Fl[li] * y) * a.Fl[n + li];
        z[col * nz + k] = y;
      }
      double zn = y;
      for (int k = nz - 2; k >= 0; --k) {
        const int li = k * ncols + col;
        zn = fma(-a.Fl[2 * n + li], zn, z[col * nz + k]);
        z[col * nz + k] = zn;
      }
    }
    __syncthreads();
  } else {
    for (int i = tid; i < n; i += T) z[i] = PREC == PM_PREC_NONE ? r[i] : a.dinv[i] * r[i];
    __syncthreads();
  }
  v[0] = v[1] = v[2] = 0.0;
  for (int i = tid; i < n; i += T) {
    const double zi = z[i], ri = r[i];
    v[0] = fma(ri, zi, v[0]);
    if (a.proj) {
      v[1] = fma(a.m[i], zi, v[1]);
      v[2] += ri;
    }
  }
  small_sum<3>(v, red);
}

template <int MASKC, int PREC>
__global__ void __launch_bounds__(SMALL_TPB, 1) k_small_pcg(Geom g, const double* __restrict__ val,
                                                           const double* __restrict__ b, double* x, double* r,
                                                           double* p, double* w, double* z, double* bw,
                                                           SmallArgs a, SmallOut* out) {
  __shared__ double red[3 * 32 + 3];
  const int n = (int)g.n, T = blockDim.x, tid = threadIdx.x;
  // right-hand side and initial guess (pressure: b - (1'b / 1'm) m, x shifted to m'x = 0)
  double v[3] = {0.0, 0.0, 0.0};
  if (a.proj) {
    for (int i = tid; i < n; i += T) {
      v[0] += b[i];
      if (a.x0_is_guess) v[1] = fma(a.m[i], x[i], v[1]);
    }
    small_sum<3>(v, red);
  }
  const double lam = a.proj ? v[0] / a.one_m : 0.0, xs = a.proj && a.x0_is_guess ? v[1] / a.one_m : 0.0;
  const double* bb_ = b;
  for (int i = tid; i < n; i += T) {
    if (a.proj) bw[i] = b[i] - lam * a.m[i];
    x[i] = a.x0_is_guess ? x[i] - xs : 0.0;
  }
  if (a.proj) bb_ = bw;
  __syncthreads();
  // r = b - A x (compensated), ||b||^2, ||r||^2
  v[0] = v[1] = v[2] = 0.0;
  for (int i = tid; i < n; i += T) {
    const int col = i / g.nz, k = i - col * g.nz;
    double asum;
    const double bi = bb_[i];
    const double ri = row_residual_dot2<MASKC>(g, val, x, bi, i, col, k, asum);
    r[i] = ri;
    v[0] = fma(bi, bi, v[0]);
    v[1] = fma(ri, ri, v[1]);
  }
  small_sum<3>(v, red);
  const double bb = v[0], tol2 = a.rtol * a.rtol * bb;
  double rr = v[1];
  int iter = 0, restarts = 0, first_pass = -1, status = PM_OK;
  double rel_true = 0.0, floor = 0.0, prev_true = -1.0;
  bool accepted = false;
  // as pcg_run: x0 may already meet rtol (no iteration), max_iter = 0 allows none
  bool skip = rr <= tol2;
  if (!skip && a.max_iter == 0) status = PM_NOT_CONVERGED;
  if (bb == 0.0) {
    for (int i = tid; i < n; i += T) x[i] = 0.0;
  }
  while (bb != 0.0) {
    if (status == PM_OK && !skip) {
      // z = P^{-1} r, rho = (r, z'), p = z' (z' = z - c 1, c = m'z / 1'm for the pressure)
      small_precond<PREC>(g, a, r, z, v, red);
      double c = a.proj ? v[1] / a.one_m : 0.0;
      double rho = v[0] - c * v[2];
      if (!(rho > 0.0) || !isfinite(rho)) status = PM_BREAKDOWN;
      for (int i = tid; i < n; i += T) p[i] = z[i] - c;
      __syncthreads();
      bool converged = false;
      while (status == PM_OK && iter < a.max_iter) {
        // w = A p, (p, w)
        double pw[1] = {0.0};
        for (int i = tid; i < n; i += T) {
          const double wi = small_row<MASKC>(g, val, p, a.keep, i);
          w[i] = wi;
          pw[0] = fma(p[i], wi, pw[0]);
        }
        small_sum<1>(pw, red);
        if (!(pw[0] > 0.0) || !isfinite(pw[0])) {
          status = PM_BREAKDOWN;
          break;
        }
        const double alpha = rho / pw[0];
        double rv[1] = {0.0};
        for (int i = tid; i < n; i += T) {
          x[i] = fma(alpha, p[i], x[i]);
          const double ri = fma(-alpha, w[i], r[i]);
          r[i] = ri;
          rv[0] = fma(ri, ri, rv[0]);
        }
        small_sum<1>(rv, red);
        rr = rv[0];
        ++iter;
        if (rr <= tol2) {
          converged = true;
          break;
        }
        if (iter >= a.max_iter) break;
        small_precond<PREC>(g, a, r, z, v, red);
        c = a.proj ? v[1] / a.one_m : 0.0;
        const double rho_new = v[0] - c * v[2];
        if (!(rho_new > 0.0) || !isfinite(rho_new)) {
          status = PM_BREAKDOWN;
          break;
        }
        const double beta = rho_new / rho;
        rho = rho_new;
        for (int i = tid; i < n; i += T) p[i] = fma(beta, p[i], z[i] - c);
        __syncthreads();
      }
      if (status == PM_OK && !converged) status = PM_NOT_CONVERGED;   // iteration cap
    }
    skip = false;
    if (first_pass < 0) first_pass = iter;
    // true residual, compensated (into r, the restart's starting residual), and the acceptance
    // rule of pcg_run
    v[0] = v[1] = v[2] = 0.0;
    for (int i = tid; i < n; i += T) {
      const int col = i / g.nz, k = i - col * g.nz;
      double asum;
      const double bi = bb_[i];
      const double ri = row_residual_dot2<MASKC>(g, val, x, bi, i, col, k, asum);
      r[i] = ri;
      v[0] = fma(ri, ri, v[0]);
      const double f = asum + fabs(bi);
      v[1] = fma(f, f, v[1]);
    }
    small_sum<3>(v, red);
    rel_true = sqrt(v[0] / bb);
    floor = ldexp(1.0, -53) * sqrt(v[1] / bb);
    const bool stalled = prev_true >= 0.0 && rel_true > 0.5 * prev_true;
    const bool last = restarts >= a.max_restarts || iter >= a.max_iter;
    accepted = rel_true <= a.rtol || (rel_true <= floor && (stalled || last));
    if (status != PM_OK || accepted || last) break;
    prev_true = rel_true;
    ++restarts;
  }
  if (bb != 0.0 && status == PM_OK && !accepted) status = PM_NOT_CONVERGED;
  if (a.proj) {   // the returned pressure has m'x = 0
    __syncthreads();
    v[0] = v[1] = v[2] = 0.0;
    for (int i = tid; i < n; i += T) v[0] = fma(a.m[i], x[i], v[0]);
    small_sum<3>(v, red);
    const double sh = v[0] / a.one_m;
    for (int i = tid; i < n; i += T) x[i] -= sh;
  }
  if (tid == 0) {
    out->iters = iter;
    out->restarts = restarts;
    out->first_pass = first_pass < 0 ? iter : first_pass;
    out->status = status;
    out->zero_rhs = bb == 0.0;
    out->rel_true = bb == 0.0 ? 0.0 : rel_true;
    out->rel_rec = bb == 0.0 ? 0.0 : sqrt(rr / bb);
    out->floor = floor;
  }
}

static_assert(sizeof(SmallOut) <= 64, "SmallOut buffer");

template <int MASKC>
int small_run(pm_operator* op, int which, const double* b, double* x, const pm_solve_opts* o,
              pm_solve_stats* stats, cudaStream_t s) {
  auto t0 = std::chrono::steady_clock::now();
  SolveCtx* c = op->ctx;
  const bool proj = which == PM_OP_PRESSURE;
  const int prec = o->prec;
  int st;
  if ((st = launch_dinv(op, which, s))) return st;
  if (prec == PM_PREC_IC0 && !op->ic0[which].ok) {
    int bd = 0;
    for (int m = -1; m <= 10; ++m) {
      if ((st = launch_ic0_factor(op, which, m < 0 ? 0.0 : 1e-3 * std::pow(2.0, m), &bd, s))) return st;
      if (!bd) break;
    }
    if (bd) return set_error(PM_BREAKDOWN, "IC0 pivot failure after the shift limit");
  }
  if (prec == PM_PREC_LINE && (st = line_factor(op, which, s))) return st;
  SmallArgs a;
  std::memset(&a, 0, sizeof(a));
  a.rtol = o->rtol;
  a.one_m = op->one_m;
  a.max_iter = o->max_iter;
  a.max_restarts = o->max_restarts;
  a.x0_is_guess = o->x0_is_guess ? 1 : 0;
  a.proj = proj ? 1 : 0;
  a.dinv = op->d_dinv[which];
  a.keep = MASKC >= 0 ? op->d_keep[MASKC < 0 ? 0 : MASKC] : nullptr;
  a.m = op->d_m;
  a.Fic = op->ic0[which].F;
  a.Fl = op->d_line[which];
  a.cls_cols = op->d_cls_cols;
  a.cm = cmap_of(op);
  int64_t off = 0;
  for (int q = 0; q < 4; ++q) {
    a.cls_off[q] = off;
    a.cls_cnt[q] = op->cls_count[q];
    off += op->cls_count[q];
  }
  Geom g = geom_of(op);
  const double* val = op->d_val[which_valset(which)];
  SmallOut* dout = static_cast<SmallOut*>(c->small_out);
#define PM_SMALL(P) k_small_pcg<MASKC, P><<<1, SMALL_TPB, 0, s>>>(g, val, b, x, c->r, c->p, c->w, c->z, c->bw, a, dout)
  switch (prec) {
    case PM_PREC_IC0: PM_SMALL(PM_PREC_IC0); break;
    case PM_PREC_LINE: PM_SMALL(PM_PREC_LINE); break;
    case PM_PREC_NONE: PM_SMALL(PM_PREC_NONE); break;
    default: PM_SMALL(PM_PREC_JACOBI); break;
  }
#undef PM_SMALL
  count_launch();
  if ((st = cuda_check(cudaGetLastError(), "k_small_pcg"))) return st;
  if ((st = cuda_check(cudaMemcpyAsync(c->small_out_host, c->small_out, sizeof(SmallOut), cudaMemcpyDeviceToHost, s),
                       "small stats")))
    return st;
  if ((st = cuda_check(cudaStreamSynchronize(s), "small pcg"))) return st;
  const SmallOut& h = *static_cast<const SmallOut*>(c->small_out_host);
  if (stats) {
    stats->iters = h.iters;
    stats->outer_iters = h.restarts;
    stats->first_pass_iters = h.first_pass;
    stats->status = h.status;
    stats->rel_residual_true = h.rel_true;
    stats->rel_residual_rec = h.rel_rec;
    stats->rel_residual_floor = h.floor;
    stats->bytes_moved = h.iters * bytes_per_iter(op, prec, proj);
    stats->seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
  }
  if (h.status != PM_OK)
    return set_error(h.status, h.status == PM_NOT_CONVERGED ? "PCG did not reach rtol within max_iter"
                                                            : "PCG breakdown: (p, Ap) <= 0 or non-finite");
  return PM_OK;
}

// ---- mixed precision: FP32 / BF16 operator values, FP32 inner PCG, FP64 outer refinement -------
// Outer (FP64): r = b - A x with the FP64 operator; stop when ||r|| <= rtol ||b|| or below the
// FP64 floor. Inner: PCG on A d = r with the operator values in FP32 (or BF16), FP32 vectors and
// FP32 SpMV / preconditioner arithmetic, FP64 dot products and alpha / beta, to a relative
// reduction inner_rtol; then x += d in FP64.

// m'z with m held exactly as two floats (hi + lo = m in FP64 to 48 bits) for the FP32 kernels.
__device__ __forceinline__ void add_mz(DF& acc, float2 m2, float z) {
  acc.add_prod(m2.x, z);
  acc.add_prod(m2.y, z);
}

__device__ __forceinline__ float ldv(const float* p, int i) { return __ldg(p + i); }
__device__ __forceinline__ float ldv(const __nv_bfloat16* p, int i) { return __bfloat162float(p[i]); }

// Low-precision operator in difference form. The low-precision copy keeps the 14 off-diagonal
// values and stores, in the diagonal slot, the FP64 row sum rs_i = sum_j a_ij (0 for the pure-
// Neumann pressure operator). Then
//   (A x)_i = (rs_i - sum_{j eliminated} a_ij) x_i + sum_{j kept, j != i} a_ij (x_j - x_i),
// which is A x exactly, but rounds each a_ij (x_j - x_i) instead of cancelling large a_ij x_j
// terms: for vectors that are smooth along the strong (vertical) couplings this keeps the
// relative accuracy that FP32 / BF16 would otherwise lose on the thin-domain operators, and the
// constant null space of the pressure operator is exact in any precision.
template <int MASKC, typename TV>
__device__ __forceinline__ float row_dot32(const Geom& g, const TV* __restrict__ val, const float* __restrict__ x,
                                           int row, int col, int k) {
  const int nz = g.nz;
  const int npad = (int)g.npad;
  int nb[NNBR];
  uint8_t fl[NNBR];
  nb[0] = col;
#pragma unroll
  for (int q = 1; q < NNBR; ++q) nb[q] = nbr_of(g, col, q);
  if (MASKC >= 0) {
#pragma unroll
    for (int q = 0; q < NNBR; ++q) fl[q] = __ldg(g.colflag + (nb[q] >= 0 ? nb[q] : col));
    if (is_dirichlet(fl[0], k, nz, MASKC)) return x[row];
  }
  float a[NSLOT];
#pragma unroll
  for (int s = 0; s < NSLOT; ++s) a[s] = ldv(val, s * npad + row);
  const float xi = x[row];
  float sum = 0.f, drop = 0.f;
#pragma unroll
  for (int s = 0; s < NSLOT; ++s) {
    if (s == DIAG_SLOT) continue;
    const int q = slot_q(s);
    const int kk = k + slot_dk(s);
    bool ok = nb[q] >= 0;
    if (slot_dk(s) < 0) ok = ok && kk >= 0;
    if (slot_dk(s) > 0) ok = ok && kk < nz;
    bool keep = ok;
    if (MASKC >= 0) {
      const bool dj = ok && is_dirichlet(fl[q], kk, nz, MASKC);
      keep = ok && !dj;
      drop += dj ? a[s] : 0.f;
    }
    const float xv = x[keep ? nb[q] * nz + kk : row];
    sum = fmaf(keep ? a[s] : 0.f, xv - xi, sum);
  }
  return fmaf(a[DIAG_SLOT] - drop, xi, sum);
}

// row_dot32 for a velocity component through its keep mask (see row_dot_keep): a slot whose
// neighbour is present but eliminated adds its value to the drop term.
template <typename TV>
__device__ __forceinline__ float row_dot32_keep(const Geom& g, const TV* __restrict__ val, const float* __restrict__ x,
                                                const uint16_t* __restrict__ keep, int row, int col, int k) {
  const int nz = g.nz;
  const int npad = (int)g.npad;
  const uint32_t km = __ldg(keep + row);
  if (km & 0x8000u) return x[row];
  int nb[NNBR];
  nb[0] = col;
#pragma unroll
  for (int q = 1; q < NNBR; ++q) nb[q] = nbr_of(g, col, q);
  float a[NSLOT];
#pragma unroll
  for (int s = 0; s < NSLOT; ++s) a[s] = ldv(val, s * npad + row);
  const float xi = x[row];
  float sum = 0.f, drop = 0.f;
#pragma unroll
  for (int s = 0; s < NSLOT; ++s) {
    if (s == DIAG_SLOT) continue;
    const int q = slot_q(s);
    const int kk = k + slot_dk(s);
    bool exists = nb[q] >= 0;
    if (slot_dk(s) < 0) exists = exists && kk >= 0;
    if (slot_dk(s) > 0) exists = exists && kk < nz;
    const bool keep_s = (km >> s) & 1u;
    drop += (exists && !keep_s) ? a[s] : 0.f;
    const float xv = x[keep_s ? nb[q] * nz + kk : row];
    sum = fmaf(keep_s ? a[s] : 0.f, xv - xi, sum);
  }
  return fmaf(a[DIAG_SLOT] - drop, xi, sum);
}

// Low-precision copy in difference form: off-diagonals rounded, diagonal slot = FP64 row sum
// (zero_rowsum: exactly 0, the pure-Neumann operator).
template <typename T>
__global__ void k_cvt_diff(int64_t n, int64_t npad, const double* __restrict__ val, T* __restrict__ out,
                           int zero_rowsum) {
  for (int64_t row = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; row < npad; row += (int64_t)gridDim.x * blockDim.x) {
    double rs = 0.0;
#pragma unroll
    for (int s = 0; s < NSLOT; ++s) {
      const double v = val[s * npad + row];
      rs += v;
      if (s != DIAG_SLOT) {
        if constexpr (std::is_same<T, float>::value) out[s * npad + row] = (float)v;
        else out[s * npad + row] = __double2bfloat16(v);
      }
    }
    if (zero_rowsum || row >= n) rs = 0.0;
    if constexpr (std::is_same<T, float>::value) out[DIAG_SLOT * npad + row] = (float)rs;
    else out[DIAG_SLOT * npad + row] = __double2bfloat16(rs);
  }
}

template <int MASKC, typename TV>
__global__ void __launch_bounds__(TPB, 4) k32_spmv(Geom g, const TV* __restrict__ val, const float* __restrict__ p,
                                                   float* __restrict__ w, const uint16_t* __restrict__ keep,
                                                   double* partials, PcgScalars* sc) {
  if (sc_done(sc)) return;
  double v[1] = {0.0};
  DF a0;
  const int n = (int)g.n;
  for (int row = blockIdx.x * blockDim.x + threadIdx.x; row < n; row += gridDim.x * blockDim.x) {
    const int col = row / g.nz;
    const int k = row - col * g.nz;
    const float wi = MASKC >= 0 ? row_dot32_keep<TV>(g, val, p, keep, row, col, k) : row_dot32<MASKC, TV>(g, val, p, row, col, k);
    w[row] = wi;
    a0.add_prod(p[row], wi);
  }
  v[0] = a0.value();
  if (grid_sum<1>(v, partials, &sc->count[3]) && threadIdx.x == 0) {
    const double pap = v[0];
    sc->pAp = pap;
    if (!(pap > 0.0) || !isfinite(pap)) {
      sc->status = PM_BREAKDOWN;
      sc->done = 1;
    } else {
      sc->alpha = sc->rho / pap;
    }
  }
}

// d += alpha p, r -= alpha w (FP32; d is the correction since the last residual replacement,
// folded into the FP64 x there); INLINE_Z: z = dinv r (Jacobi) and its reductions.
template <int PROJ, int INLINE_Z>
__global__ void __launch_bounds__(TPB) k32_update(int64_t n, float* __restrict__ d, float* __restrict__ r,
                                                  const float* __restrict__ p, const float* __restrict__ w,
                                                  const float* __restrict__ dinv, const float2* __restrict__ m2,
                                                  double* partials, PcgScalars* sc) {
  if (sc_done(sc)) return;
  const double alpha_d = sc->alpha;
  const float alpha = (float)alpha_d;
  DF a[4];
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    d[i] = fmaf(alpha, p[i], d[i]);
    const float ri = fmaf(-alpha, w[i], r[i]);
    r[i] = ri;
    a[0].add_prod(ri, ri);
    if (INLINE_Z) {
      const float zi = dinv[i] * ri;
      a[1].add_prod(ri, zi);
      if (PROJ) {
        add_mz(a[2], m2[i], zi);
        a[3].add(ri);
      }
    }
  }
  double v[4] = {a[0].value(), a[1].value(), a[2].value(), a[3].value()};
  if (grid_sum<4>(v, partials, &sc->count[4]) && threadIdx.x == 0) {
    sc->iter += 1;
    sc->rr = v[0];
    if (v[0] <= sc->tol2) {
      sc->done = 1;
    } else if (sc->iter >= sc->max_iter) {
      sc->status = PM_NOT_CONVERGED;
      sc->done = 1;
    } else if (v[0] <= sc->aux[2]) {
      sc->done = 2;  // residual replacement requested (mixed precision): the host finishes the step
    } else if (INLINE_Z) {
      const double c = PROJ ? v[2] / sc->one_m : 0.0;
      const double rho_new = v[1] - c * v[3];
      sc->proj_c = c;
      sc->beta = rho_new / sc->rho;
      sc->rho = rho_new;
      if (!(rho_new > 0.0) || !isfinite(rho_new)) {
        sc->status = PM_BREAKDOWN;
        sc->done = 1;
      }
    }
  }
}

// rho = (r, z') with z' = z - c (pressure) from stored or inline z; first: beta = 0.
template <int PROJ, int STORED>
__global__ void __launch_bounds__(TPB) k32_rho(int64_t n, const float* __restrict__ r, const float* __restrict__ dinv,
                                               const float* __restrict__ zbuf, const float2* __restrict__ m2,
                                               double* partials, PcgScalars* sc, int is_first) {
  if (!is_first && sc_done(sc)) return;
  DF a[3];
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const float ri = r[i];
    const float zi = STORED ? zbuf[i] : dinv[i] * ri;
    a[0].add_prod(ri, zi);
    if (PROJ) {
      add_mz(a[1], m2[i], zi);
      a[2].add(ri);
    }
  }
  double v[3] = {a[0].value(), a[1].value(), a[2].value()};
  if (grid_sum<3>(v, partials, &sc->count[2]) && threadIdx.x == 0) {
    const double c = PROJ ? v[1] / sc->one_m : 0.0;
    const double rho_new = v[0] - c * v[2];
    sc->proj_c = c;
    if (is_first) {
      sc->rho = rho_new;
      sc->beta = 0.0;
    } else {
      sc->beta = rho_new / sc->rho;
      sc->rho = rho_new;
    }
    if ((!(rho_new > 0.0) || !isfinite(rho_new)) && !sc->done) {
      sc->status = PM_BREAKDOWN;
      sc->done = 1;
    }
  }
}

template <int STORED>
__global__ void __launch_bounds__(TPB) k32_pupd(int64_t n, const float* __restrict__ r, const float* __restrict__ dinv,
                                                const float* __restrict__ zbuf, float* __restrict__ p,
                                                const PcgScalars* sc, int is_first) {
  if (!is_first && sc_done(sc)) return;
  const float beta = (float)sc->beta, c = (float)sc->proj_c;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const float zi = (STORED ? zbuf[i] : dinv[i] * r[i]) - c;
    p[i] = is_first ? zi : fmaf(beta, p[i], zi);
  }
}

// m = hi + lo as two floats (hi = fl32(m), lo = fl32(m - hi)) for the FP32 kernels' m'z.
__global__ void k_split_m(int64_t n, const double* __restrict__ m, float2* __restrict__ m2) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const float hi = (float)m[i];
    m2[i] = make_float2(hi, (float)(m[i] - (double)hi));
  }
}

// x += d (FP64), d = 0: the inner solve's FP32 correction folded into the FP64 iterate.
__global__ void k32_fold(int64_t n, double* __restrict__ x, float* __restrict__ d) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    x[i] += (double)d[i];
    d[i] = 0.f;
  }
}

__global__ void k32_from64(int64_t n, const double* __restrict__ r64, float* __restrict__ r32) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    r32[i] = (float)r64[i];
}

__global__ void k_fill32(float* x, int64_t n, float v) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) x[i] = v;
}

template <typename T>
__global__ void k_cvt(int64_t n, const double* __restrict__ in, T* __restrict__ out) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    if constexpr (std::is_same<T, float>::value) out[i] = (float)in[i];
    else out[i] = __double2bfloat16(in[i]);
  }
}

// FP32 vertical-line solve fused with the inner update (as k_update_line).
template <int PROJ>
__global__ void __launch_bounds__(LINE_UCOLS) k32_update_line(Geom g, const float* __restrict__ F,
                                                            float* __restrict__ d, float* __restrict__ r,
                                                            const float* __restrict__ p, const float* __restrict__ w,
                                                            float* __restrict__ z, const float2* __restrict__ m2,
                                                            double* partials, PcgScalars* sc, int mode) {
  // mode 0: first step (z, rho, beta = 0); 1: a full iteration (d, r update, z, rho, beta)
  extern __shared__ float smf[];
  const int update = mode == 1;
  if (mode != 0 && sc_done(sc)) return;
  const double alpha_d = update ? sc->alpha : 0.0;
  const float alpha = (float)alpha_d;
  const int nz = g.nz, ld = nz + 1;
  const int ncols = g.ncols;
  const int n = (int)g.n;
  const int ntiles = (ncols + LINE_UCOLS - 1) / LINE_UCOLS;
  DF a[4];
  for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    const int c0 = tile * LINE_UCOLS;
    const int cc = min(LINE_UCOLS, ncols - c0);
    const int row0 = c0 * nz;
    const int rows = cc * nz;
    for (int i = threadIdx.x; i < rows; i += blockDim.x) {
      const int row = row0 + i;
      float ri = r[row];
      if (update) {
        d[row] = fmaf(alpha, p[row], d[row]);
        ri = fmaf(-alpha, w[row], ri);
        r[row] = ri;
      }
      smf[(i / nz) * ld + i % nz] = ri;
      a[0].add_prod(ri, ri);
    }
    __syncthreads();
    if ((int)threadIdx.x < cc) {
      const int col = c0 + threadIdx.x;
      float* col_s = smf + threadIdx.x * ld;
      float y = 0.f;
#pragma unroll 4
      for (int k = 0; k < nz; ++k) {
        const int li = k * ncols + col;
        y = (col_s[k] - F[li] * y) * F[n + li];
        col_s[k] = y;
      }
      float zn = y;
#pragma unroll 4
      for (int k = nz - 2; k >= 0; --k) {
        const int li = k * ncols + col;
        zn = fmaf(-F[2 * n + li], zn, col_s[k]);
        col_s[k] = zn;
      }
    }
    __syncthreads();
    for (int i = threadIdx.x; i < rows; i += blockDim.x) {
      const int row = row0 + i;
      const float zi = smf[(i / nz) * ld + i % nz];
      const float ri = r[row];
      z[row] = zi;
      a[1].add_prod(ri, zi);
      if (PROJ) {
        add_mz(a[2], m2[row], zi);
        a[3].add(ri);
      }
    }
    __syncthreads();
  }
  double v[4] = {a[0].value(), a[1].value(), a[2].value(), a[3].value()};
  if (grid_sum<4>(v, partials, &sc->count[4]) && threadIdx.x == 0) {
    const double c = PROJ ? v[2] / sc->one_m : 0.0;
    const double rho_new = v[1] - c * v[3];
    if (mode == 0) {
      sc->proj_c = c;
      sc->rho = rho_new;
      sc->beta = 0.0;
      if ((!(rho_new > 0.0) || !isfinite(rho_new)) && !sc->done) {
        sc->status = PM_BREAKDOWN;
        sc->done = 1;
      }
    } else {
      sc->iter += 1;
      sc->rr = v[0];
      if (v[0] <= sc->tol2) {
        sc->done = 1;
      } else if (sc->iter >= sc->max_iter) {
        sc->status = PM_NOT_CONVERGED;
        sc->done = 1;
      } else if (v[0] <= sc->aux[2]) {
        sc->done = 2;
      } else {
        sc->proj_c = c;
        sc->beta = rho_new / sc->rho;
        sc->rho = rho_new;
        if (!(rho_new > 0.0) || !isfinite(rho_new)) {
          sc->status = PM_BREAKDOWN;
          sc->done = 1;
        }
      }
    }
  }
}

// FP32 version of k_update_line_w (32-level columns, warp tasks of TC columns, no block
// barriers); the FP32 correction d takes alpha p (folded into the FP64 x at each refinement) and
// the dots are accumulated in compensated FP32. mode as k32_update_line: 0 first step, 1 a full
// iteration. (r, z) = sum_k t_k y_k from the sweep (symmetric column blocks, see k_update_line_w).
template <int PROJ, int TC>
__global__ void __launch_bounds__(LINE_WTPB, 4) k32_update_line_w(Geom g, const float* __restrict__ F,
                                                              float* __restrict__ d, float* __restrict__ r,
                                                              const float* __restrict__ p, const float* __restrict__ w,
                                                              float* __restrict__ z, const float2* __restrict__ m2,
                                                              double* partials, PcgScalars* sc, int mode) {
  constexpr int NZ = LINE_WNZ, LD = NZ + 1;
  extern __shared__ float smf[];
  const int update = mode == 1;
  if (mode != 0 && sc_done(sc)) return;
  const double alpha_d = update ? sc->alpha : 0.0;
  const float alpha = (float)alpha_d;
  const int lane = threadIdx.x & 31;
  const int wib = threadIdx.x >> 5;
  float* ws = smf + wib * (TC * LD);
  const int ncols = g.ncols;
  const int n = (int)g.n;
  const int nwarps = gridDim.x * (LINE_WTPB / 32);
  const int wg = blockIdx.x * (LINE_WTPB / 32) + wib;
  const int ntask = (ncols + TC - 1) / TC;
  const int tbeg = (int)((int64_t)ntask * wg / nwarps);
  const int tend = (int)((int64_t)ntask * (wg + 1) / nwarps);
  DF a[4];   // (r, r), (r, z), m'z, 1'r
  for (int t = tbeg; t < tend; ++t) {
    const int c0 = t * TC;
    const int cc = min(TC, ncols - c0);
    const int row0 = c0 * NZ + lane;
#pragma unroll 8
    for (int j = 0; j < cc; ++j) {
      const int row = row0 + j * NZ;
      float ri = r[row];
      if (update) {
        d[row] = fmaf(alpha, p[row], d[row]);
        ri = fmaf(-alpha, w[row], ri);
        r[row] = ri;
      }
      ws[j * LD + lane] = ri;
      a[0].add_prod(ri, ri);
      if (PROJ) a[3].add(ri);
    }
    __syncwarp();
    if (lane < cc) {
      const int col = c0 + lane;
      float* cs = ws + lane * LD;
      float y = 0.f;
#pragma unroll 8
      for (int k = 0; k < NZ; ++k) {
        const int li = k * ncols + col;
        const float tk = fmaf(-F[li], y, cs[k]);
        y = tk * F[n + li];
        a[1].add_prod(tk, y);
        cs[k] = y;
      }
      float zn = y;
#pragma unroll 8
      for (int k = NZ - 2; k >= 0; --k) {
        const int li = k * ncols + col;
        zn = fmaf(-F[2 * n + li], zn, cs[k]);
        cs[k] = zn;
      }
    }
    __syncwarp();
#pragma unroll 8
    for (int j = 0; j < cc; ++j) {
      const int row = row0 + j * NZ;
      const float zi = ws[j * LD + lane];
      z[row] = zi;
      if (PROJ) add_mz(a[2], m2[row], zi);
    }
    __syncwarp();
  }
  double v[4] = {a[0].value(), a[1].value(), a[2].value(), a[3].value()};
  if (grid_sum<4>(v, partials, &sc->count[4]) && threadIdx.x == 0) {
    const double c = PROJ ? v[2] / sc->one_m : 0.0;
    const double rho_new = v[1] - c * v[3];
    if (mode == 0) {
      sc->proj_c = c;
      sc->rho = rho_new;
      sc->beta = 0.0;
      if ((!(rho_new > 0.0) || !isfinite(rho_new)) && !sc->done) {
        sc->status = PM_BREAKDOWN;
        sc->done = 1;
      }
    } else {
      sc->iter += 1;
      sc->rr = v[0];
      if (v[0] <= sc->tol2) {
        sc->done = 1;
      } else if (sc->iter >= sc->max_iter) {
        sc->status = PM_NOT_CONVERGED;
        sc->done = 1;
      } else if (v[0] <= sc->aux[2]) {
        sc->done = 2;
      } else {
        sc->proj_c = c;
        sc->beta = rho_new / sc->rho;
        sc->rho = rho_new;
        if (!(rho_new > 0.0) || !isfinite(rho_new)) {
          sc->status = PM_BREAKDOWN;
          sc->done = 1;
        }
      }
    }
  }
}

// The FP32 fused update + line solve (mode as k32_update_line): warp tasks for 32-level columns,
// the block kernel otherwise. One launch; the caller counts it.
void update_line32(pm_operator* op, int which, bool proj, int mode, cudaStream_t s) {
  SolveCtx* c = op->ctx;
  Geom g = geom_of(op);
  if (op->nz == LINE_WNZ) {
    static int slots32 = 0, slots16 = 0;
    auto slots_of = [&](const void* kern, int tc) {
      const size_t sm = (size_t)(LINE_WTPB / 32) * tc * (LINE_WNZ + 1) * sizeof(float);
      cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
      int per_sm = 0;
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, LINE_WTPB, sm);
      return std::max(1, per_sm) * op->num_sms;
    };
    if (!slots32) {
      slots32 = slots_of((const void*)k32_update_line_w<1, 32>, 32);
      slots_of((const void*)k32_update_line_w<0, 32>, 32);
      slots16 = slots_of((const void*)k32_update_line_w<1, 16>, 16);
      slots_of((const void*)k32_update_line_w<0, 16>, 16);
    }
    // 32-column tasks while they fill the resident warps, else 16 (as update_line_w)
    const bool wide = (op->ncols + 31) / 32 >= (int64_t)slots32 * (LINE_WTPB / 32);
    const int tc = wide ? 32 : 16;
    const size_t smem = (size_t)(LINE_WTPB / 32) * tc * (LINE_WNZ + 1) * sizeof(float);
    int64_t blocks = std::min<int64_t>(wide ? slots32 : slots16, (int64_t)NPART * MAX_GRID / 4);
    const int64_t ntask = (op->ncols + tc - 1) / tc;
    blocks = std::min<int64_t>(blocks, (ntask + LINE_WTPB / 32 - 1) / (LINE_WTPB / 32));
    const int grid = (int)std::max<int64_t>(1, blocks);
#define PM_UL32(P, TCV)                                                                                   \
  k32_update_line_w<P, TCV><<<grid, LINE_WTPB, smem, s>>>(g, op->d_line32[which], c->d32, c->r32, c->p32, c->w32, \
                                                           c->z32, op->d_m2f, c->partials, c->sc_in, mode)
    if (wide) {
      if (proj) PM_UL32(1, 32);
      else PM_UL32(0, 32);
    } else {
      if (proj) PM_UL32(1, 16);
      else PM_UL32(0, 16);
    }
#undef PM_UL32
    return;
  }
  const int64_t ntiles = (op->ncols + LINE_UCOLS - 1) / LINE_UCOLS;
  int grid = (int)std::min<int64_t>(ntiles, std::min<int64_t>((int64_t)op->num_sms * 8, MAX_GRID));
  const size_t smem = (size_t)LINE_UCOLS * (op->nz + 1) * sizeof(float);
  if (proj)
    k32_update_line<1><<<grid, LINE_UCOLS, smem, s>>>(g, op->d_line32[which], c->d32, c->r32, c->p32, c->w32, c->z32,
                                                      op->d_m2f, c->partials, c->sc_in, mode);
  else
    k32_update_line<0><<<grid, LINE_UCOLS, smem, s>>>(g, op->d_line32[which], c->d32, c->r32, c->p32, c->w32, c->z32,
                                                      op->d_m2f, c->partials, c->sc_in, mode);
}

// FP32 IC0 apply: the same colour sweeps (k_ic0_sweep<.., float>) on the FP32 copy of the factor.
void ic0_apply32(pm_operator* op, int which, const float* r, float* z, const PcgScalars* sc, int check_done,
                 cudaStream_t s) {
  Geom g = geom_of(op);
  CMap cm = cmap_of(op);
  const float* F = op->d_ic0_32[which];
  int64_t off[5] = {0, 0, 0, 0, 0};
  for (int c = 0; c < 4; ++c) off[c + 1] = off[c] + op->cls_count[c];
#define PM_SWEEP32(C, FW)                                                                      \
  {                                                                                            \
    const int64_t cnt = op->cls_count[(C) & 3];                                                \
    const int64_t tot = cnt * cm.nlev[(C) >> 2];                                               \
    if (tot > 0) {                                                                             \
      k_ic0_sweep<C, FW, float><<<grid_for((tot + 1) / 2, TPB, op->num_sms), TPB, 0, s>>>(     \
          g, cm, op->d_cls_cols, off[(C) & 3], cnt, F, r, z, sc, check_done);                  \
      count_launch();                                                                          \
    }                                                                                          \
  }
  PM_SWEEP32(0, 1) PM_SWEEP32(1, 1) PM_SWEEP32(2, 1) PM_SWEEP32(3, 1)
  PM_SWEEP32(4, 1) PM_SWEEP32(5, 1) PM_SWEEP32(6, 1) PM_SWEEP32(7, 1)
  PM_SWEEP32(7, 0) PM_SWEEP32(6, 0) PM_SWEEP32(5, 0) PM_SWEEP32(4, 0)
  PM_SWEEP32(3, 0) PM_SWEEP32(2, 0) PM_SWEEP32(1, 0) PM_SWEEP32(0, 0)
#undef PM_SWEEP32
}

int ensure_mixed(pm_operator* op, int which, int precision, int prec, cudaStream_t s) {
  SolveCtx* c = op->ctx;
  const size_t fb = (size_t)op->n * sizeof(float);
  if (!c->r32) {
    cudaError_t e = cudaSuccess;
    e = e ? e : cudaMalloc((void**)&c->r32, fb);
    e = e ? e : cudaMalloc((void**)&c->p32, fb);
    e = e ? e : cudaMalloc((void**)&c->w32, fb);
    e = e ? e : cudaMalloc((void**)&c->z32, fb);
    e = e ? e : cudaMalloc((void**)&c->d32, fb);
    e = e ? e : cudaMalloc((void**)&c->sc_in, sizeof(PcgScalars));
    e = e ? e : cudaMallocHost((void**)&c->sc_in_host, sizeof(PcgScalars));
    if (e != cudaSuccess) return cuda_check(e, "mixed-precision workspace");
    op->device_bytes += 5 * (int64_t)fb;
  }
  if (!op->d_m2f) {
    int st = cuda_check(cudaMalloc((void**)&op->d_m2f, (size_t)op->n * sizeof(float2)), "cudaMalloc m split");
    if (st) return st;
    op->device_bytes += op->n * 8;
    k_split_m<<<grid_for(op->n, TPB, op->num_sms), TPB, 0, s>>>(op->n, op->d_m, op->d_m2f);
    count_launch();
  }
  const int vs = which_valset(which);
  const int64_t nv = (int64_t)NSLOT * op->npad;
  const int G = grid_for(nv, TPB, op->num_sms);
  const int zero_rs = vs == VS_KI ? 1 : 0;
  const int Gr = grid_for(op->npad, TPB, op->num_sms);
  (void)G;
  if (precision == PM_FP32_REFINE && !op->d_val32[vs]) {
    int st = cuda_check(cudaMalloc((void**)&op->d_val32[vs], nv * sizeof(float)), "cudaMalloc fp32 values");
    if (st) return st;
    op->device_bytes += nv * 4;
    k_cvt_diff<float><<<Gr, TPB, 0, s>>>(op->n, op->npad, op->d_val[vs], op->d_val32[vs], zero_rs);
    count_launch();
  }
  if (precision == PM_BF16_REFINE && !op->d_val16[vs]) {
    int st = cuda_check(cudaMalloc((void**)&op->d_val16[vs], nv * sizeof(uint16_t)), "cudaMalloc bf16 values");
    if (st) return st;
    op->device_bytes += nv * 2;
    k_cvt_diff<__nv_bfloat16><<<Gr, TPB, 0, s>>>(op->n, op->npad, op->d_val[vs],
                                                reinterpret_cast<__nv_bfloat16*>(op->d_val16[vs]), zero_rs);
    count_launch();
  }
  if (prec == PM_PREC_LINE && !op->d_line32[which]) {
    int st = cuda_check(cudaMalloc((void**)&op->d_line32[which], 3 * fb), "cudaMalloc fp32 line");
    if (st) return st;
    op->device_bytes += 3 * (int64_t)fb;
    k_cvt<float><<<grid_for(3 * op->n, TPB, op->num_sms), TPB, 0, s>>>(3 * op->n, op->d_line[which], op->d_line32[which]);
    count_launch();
  }
  if (prec == PM_PREC_IC0 && !op->d_ic0_32[which]) {
    int st = cuda_check(cudaMalloc((void**)&op->d_ic0_32[which], (size_t)NSLOT * fb), "cudaMalloc fp32 ic0");
    if (st) return st;
    op->device_bytes += (int64_t)NSLOT * fb;
    k_cvt<float><<<grid_for(NSLOT * op->n, TPB, op->num_sms), TPB, 0, s>>>(NSLOT * op->n, op->ic0[which].F,
                                                                          op->d_ic0_32[which]);
    count_launch();
  }
  return cuda_check(cudaGetLastError(), "mixed set-up");
}

int read_inner(SolveCtx* c, cudaStream_t s) {
  int st = cuda_check(cudaMemcpyAsync(c->sc_in_host, c->sc_in, sizeof(PcgScalars), cudaMemcpyDeviceToHost, s), "scalars");
  if (st) return st;
  st = cuda_check(cudaStreamSynchronize(s), "mixed pcg sync");
  if (!st && !g_kt.pending.empty()) kt_collect();
  return st;
}

// Algorithmic bytes per inner iteration per row (values at vbytes each; vectors FP32, the
// correction d read and written in FP32).
double bytes_per_inner(const pm_operator* op, int prec, int vbytes, bool proj) {
  const double n = (double)op->n;
  double b = n * (15 * vbytes + 4 + 4);                       // SpMV: values, p, w
  if (prec == PM_PREC_LINE) b += n * (8 + 8 + 4 + 4 + 12 + 4 + 12);  // d, r r/w; p, w; factors; z; p-update
  else if (prec == PM_PREC_IC0) b += n * (8 + 8 + 4 + 4 + 2 * 8 * 4 + 4 * 4 + 8 + 12);
  else b += n * (8 + 8 + 4 + 4 + 4 + 4 * 4);                   // Jacobi update (z inline), p-update
  if (proj) b += n * 8;                                         // m'z
  return b;
}

template <int MASKC, typename TV>
void inner_iter(pm_operator* op, int which, const TV* val32, bool proj, int prec, const float* dinv32,
                cudaStream_t s) {
  SolveCtx* c = op->ctx;
  Geom g = geom_of(op);
  const int G = grid_for(op->n, TPB, op->num_sms);
  {
    KtScope t(PM_KT_SPMV, 1, s);
    k32_spmv<MASKC, TV><<<G, TPB, 0, s>>>(g, val32, c->p32, c->w32, MASKC >= 0 ? op->d_keep[MASKC < 0 ? 0 : MASKC] : nullptr,
                                          c->partials, c->sc_in);
  }
  if (prec == PM_PREC_LINE) {
    {
      KtScope t(PM_KT_LINE, 1, s);
      update_line32(op, which, proj, 1, s);
    }
    {
      KtScope t(PM_KT_PUPDATE, 1, s);
      k32_pupd<1><<<G, TPB, 0, s>>>(op->n, c->r32, dinv32, c->z32, c->p32, c->sc_in, 0);
    }
    count_launch(3);
  } else if (prec == PM_PREC_IC0) {
    {
      KtScope t(PM_KT_UPDATE, 1, s);
      k32_update<0, 0><<<G, TPB, 0, s>>>(op->n, c->d32, c->r32, c->p32, c->w32, dinv32, op->d_m2f, c->partials, c->sc_in);
    }
    {
      KtScope t(PM_KT_IC0, 16, s);
      ic0_apply32(op, which, c->r32, c->z32, c->sc_in, 1, s);
    }
    {
      KtScope t(PM_KT_PUPDATE, 2, s);
      if (proj) k32_rho<1, 1><<<G, TPB, 0, s>>>(op->n, c->r32, dinv32, c->z32, op->d_m2f, c->partials, c->sc_in, 0);
      else k32_rho<0, 1><<<G, TPB, 0, s>>>(op->n, c->r32, dinv32, c->z32, op->d_m2f, c->partials, c->sc_in, 0);
      k32_pupd<1><<<G, TPB, 0, s>>>(op->n, c->r32, dinv32, c->z32, c->p32, c->sc_in, 0);
    }
    count_launch(4);
  } else {
    {
      KtScope t(PM_KT_UPDATE, 1, s);
      if (proj) k32_update<1, 1><<<G, TPB, 0, s>>>(op->n, c->d32, c->r32, c->p32, c->w32, dinv32, op->d_m2f, c->partials, c->sc_in);
      else k32_update<0, 1><<<G, TPB, 0, s>>>(op->n, c->d32, c->r32, c->p32, c->w32, dinv32, op->d_m2f, c->partials, c->sc_in);
    }
    {
      KtScope t(PM_KT_PUPDATE, 1, s);
      k32_pupd<0><<<G, TPB, 0, s>>>(op->n, c->r32, dinv32, nullptr, c->p32, c->sc_in, 0);
    }
    count_launch(3);
  }
}

// z = P^{-1} r32, rho = (r, z'), beta = 0, p = z': the first step of an inner solve.
void inner_first(pm_operator* op, int which, bool proj, int prec, const float* dinv32, cudaStream_t s) {
  SolveCtx* c = op->ctx;
  const int G = grid_for(op->n, TPB, op->num_sms);
  if (prec == PM_PREC_LINE) {
    update_line32(op, which, proj, 0, s);
    k32_pupd<1><<<G, TPB, 0, s>>>(op->n, c->r32, dinv32, c->z32, c->p32, c->sc_in, 1);
  } else if (prec == PM_PREC_IC0) {
    ic0_apply32(op, which, c->r32, c->z32, c->sc_in, 0, s);
    if (proj) k32_rho<1, 1><<<G, TPB, 0, s>>>(op->n, c->r32, dinv32, c->z32, op->d_m2f, c->partials, c->sc_in, 1);
    else k32_rho<0, 1><<<G, TPB, 0, s>>>(op->n, c->r32, dinv32, c->z32, op->d_m2f, c->partials, c->sc_in, 1);
    k32_pupd<1><<<G, TPB, 0, s>>>(op->n, c->r32, dinv32, c->z32, c->p32, c->sc_in, 1);
  } else {
    if (proj) k32_rho<1, 0><<<G, TPB, 0, s>>>(op->n, c->r32, dinv32, nullptr, op->d_m2f, c->partials, c->sc_in, 1);
    else k32_rho<0, 0><<<G, TPB, 0, s>>>(op->n, c->r32, dinv32, nullptr, op->d_m2f, c->partials, c->sc_in, 1);
    k32_pupd<0><<<G, TPB, 0, s>>>(op->n, c->r32, dinv32, nullptr, c->p32, c->sc_in, 1);
  }
  count_launch(2);
}

template <int MASKC, typename TV>
int mixed_run(pm_operator* op, int which, const double* b, double* x, const pm_solve_opts* o, pm_solve_stats* stats,
              cudaStream_t s) {
  auto t0 = std::chrono::steady_clock::now();
  SolveCtx* c = op->ctx;
  const bool proj = which == PM_OP_PRESSURE;
  const int prec = o->prec;
  const double* val64 = op->d_val[which_valset(which)];
  int st;
  if ((st = launch_dinv(op, which, s))) return st;
  if (prec == PM_PREC_IC0 && !op->ic0[which].ok) {
    int bd = 0;
    for (int m = -1; m <= 10; ++m) {
      if ((st = launch_ic0_factor(op, which, m < 0 ? 0.0 : 1e-3 * std::pow(2.0, m), &bd, s))) return st;
      if (!bd) break;
    }
    if (bd) return set_error(PM_BREAKDOWN, "IC0 pivot failure after the shift limit");
  }
  if (prec == PM_PREC_LINE && (st = line_factor(op, which, s))) return st;
  if ((st = ensure_mixed(op, which, o->precision, prec, s))) return st;
  const int vs = which_valset(which);
  const TV* val32 = std::is_same<TV, float>::value ? reinterpret_cast<const TV*>(op->d_val32[vs])
                                                   : reinterpret_cast<const TV*>(op->d_val16[vs]);
  const float* dinv32 = op->d_dinv32[which];
  if (prec == PM_PREC_NONE) {  // plain CG: z = r, held as an all-ones diagonal in z32
    k_fill32<<<grid_for(op->n, TPB, op->num_sms), TPB, 0, s>>>(c->z32, op->n, 1.f);
    count_launch();
    dinv32 = c->z32;
  }
  // residual replacement each time the recursive residual has dropped by this factor
  const double inner_rtol = o->inner_rtol > 0.0 ? o->inner_rtol : 1e-2;
  const int G = grid_for(op->n, TPB, op->num_sms);
  PcgScalars init;
  std::memset(&init, 0, sizeof(init));
  init.one_m = op->one_m;
  init.max_iter = o->max_iter;
  if ((st = cuda_check(cudaMemcpyAsync(c->sc, &init, sizeof(init), cudaMemcpyHostToDevice, s), "scalars init"))) return st;
  const double* bw = b;
  if (proj) {
    k_cg_press_sums<<<G, TPB, 0, s>>>(op->n, b, x, op->d_m, o->x0_is_guess ? 1 : 0, c->partials, c->sc);
    k_cg_prepare<<<G, TPB, 0, s>>>(op->n, b, op->d_m, c->bw, x, 1, o->x0_is_guess ? 1 : 0, c->sc);
    count_launch(2);
    bw = c->bw;
  } else if (!o->x0_is_guess) {
    k_cg_prepare<<<G, TPB, 0, s>>>(op->n, b, op->d_m, nullptr, x, 0, 0, c->sc);
    count_launch();
  }
  launch_residual<MASKC>(op, val64, bw, x, o->rtol, 0, s);
  if ((st = read_scalars(c, s))) return st;
  const double bb = c->sc_host->bb;
  int outer = 0, inner_total = 0, status = PM_OK;
  double rel_true = 0.0, rel_floor = 0.0, bytes = 0.0;
  const int vbytes = std::is_same<TV, float>::value ? 4 : 2;
  if (c->sc_host->zero_rhs) {
    k_fill<<<G, TPB, 0, s>>>(x, op->n, 0.0);
    count_launch();
  } else if (c->sc_host->done) {
    // x0 already meets rtol (PM_OK), or max_iter = 0 (PM_NOT_CONVERGED): no inner solve runs
    status = c->sc_host->status;
    rel_true = std::sqrt(c->sc_host->rr / bb);
  } else {
    // Restarted refinement: inner PCG solves with r, p, w, z and the correction d in FP32 (dots
    // in compensated FP32 reduced in FP64, alpha and beta in FP64). Each time the recursive
    // residual has dropped by inner_rtol, or claims convergence, d is folded into the FP64 x, the
    // FP64 true residual b - A x (compensated) is formed, and a new inner solve starts from it.
    const double rr_drop = inner_rtol * inner_rtol;
    PcgScalars in;
    std::memset(&in, 0, sizeof(in));
    in.one_m = op->one_m;
    in.max_iter = o->max_iter;
    in.tol2 = c->sc_host->tol2;
    in.bb = bb;
    in.aux[2] = rr_drop * c->sc_host->rr;   // replacement threshold on the recursive (r, r)
    if ((st = cuda_check(cudaMemcpyAsync(c->sc_in, &in, sizeof(in), cudaMemcpyHostToDevice, s), "scalars"))) return st;
    k32_from64<<<G, TPB, 0, s>>>(op->n, c->r, c->r32);
    count_launch();
    if ((st = cuda_check(cudaMemsetAsync(c->d32, 0, (size_t)op->n * sizeof(float), s), "d32"))) return st;
    inner_first(op, which, proj, prec, dinv32, s);
    if ((st = read_inner(c, s))) return st;
    int64_t issued = 0;
    const int32_t zero = 0;
    int stalled = 0;
    double prev_true = 1e300;
    for (;;) {
      int chunk = 4;
      while (!c->sc_in_host->done) {
        if (issued > (int64_t)o->max_iter + 4096) return set_error(PM_ECUDA, "mixed PCG: device never reported completion");
        for (int it = 0; it < chunk; ++it) inner_iter<MASKC, TV>(op, which, val32, proj, prec, dinv32, s);
        issued += chunk;
        if ((st = read_inner(c, s))) return st;
        if (chunk < 64) chunk *= 2;
      }
      // fold the FP32 correction into x, then the FP64 true residual into c->r
      k32_fold<<<G, TPB, 0, s>>>(op->n, x, c->d32);
      count_launch();
      launch_residual<MASKC>(op, val64, bw, x, o->rtol, 1, s);
      if ((st = read_scalars(c, s))) return st;
      ++outer;
      bytes += (double)op->n * (15 * 8 + 3 * 8 + 16 + 8);   // FP64 residual; the fold of d into x
      rel_true = std::sqrt(c->sc_host->aux[0] / bb);
      rel_floor = std::ldexp(1.0, -53) * std::sqrt(c->sc_host->aux[1] / bb);
      // the refinement step did not halve the (compensated) true residual
      const bool stalled_now = rel_true > 0.5 * prev_true;
      if (rel_true <= o->rtol || (rel_true <= rel_floor && stalled_now)) break;
      // stagnation above the floor: three replacements in a row that did not halve it
      stalled = stalled_now ? stalled + 1 : 0;
      prev_true = rel_true;
      if (stalled >= 3) {
        status = PM_NOT_CONVERGED;
        break;
      }
      if (c->sc_in_host->status == PM_BREAKDOWN) {
        status = PM_BREAKDOWN;
        break;
      }
      if (c->sc_in_host->iter >= o->max_iter) {  // no iteration left: accepted only below the floor
        status = rel_true <= rel_floor ? PM_OK : PM_NOT_CONVERGED;
        break;
      }
      // the next inner solve starts from r32 = (float)(b - A x)
      const double thr = rr_drop * c->sc_host->aux[0];
      if ((st = cuda_check(cudaMemcpyAsync(&c->sc_in->done, &zero, sizeof(zero), cudaMemcpyHostToDevice, s), "scalars")))
        return st;
      if ((st = cuda_check(cudaMemcpyAsync(&c->sc_in->aux[2], &thr, sizeof(thr), cudaMemcpyHostToDevice, s), "scalars")))
        return st;
      k32_from64<<<G, TPB, 0, s>>>(op->n, c->r, c->r32);
      count_launch();
      inner_first(op, which, proj, prec, dinv32, s);
      if ((st = read_inner(c, s))) return st;
    }
    inner_total = c->sc_in_host->iter;
    bytes += inner_total * bytes_per_inner(op, prec, vbytes, proj);
  }
  if (proj) {
    k_cg_press_sums<<<G, TPB, 0, s>>>(op->n, b, x, op->d_m, 1, c->partials, c->sc);
    k_shift_by<<<G, TPB, 0, s>>>(x, op->n, c->sc);
    count_launch(2);
    if ((st = read_scalars(c, s))) return st;
  }
  if (stats) {
    stats->iters = inner_total;
    stats->outer_iters = outer;
    stats->first_pass_iters = inner_total;
    stats->status = status;
    stats->rel_residual_true = c->sc_host->zero_rhs ? 0.0 : rel_true;
    stats->rel_residual_rec = stats->rel_residual_true;
    stats->rel_residual_floor = rel_floor;
    stats->bytes_moved = bytes;
    stats->seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
  }
  if ((st = cuda_check(cudaGetLastError(), "mixed pcg kernels"))) return st;
  if (status != PM_OK)
    return set_error(status, status == PM_NOT_CONVERGED ? "mixed-precision PCG did not reach rtol"
                                                        : "mixed-precision PCG breakdown");
  return PM_OK;
}

}  // namespace

int spmv(pm_operator* op, int which, const double* x, double* y, cudaStream_t s) {
  const int vs = which_valset(which);
  if (vs < 0) return set_error(PM_EINVAL, "unknown operator");
  Geom g = geom_of(op);
  const int G = grid_for(op->n, TPB, op->num_sms);
  switch (which_mask(which)) {
    case 0: k_spmv<0><<<G, TPB, 0, s>>>(g, op->d_val[vs], x, y); break;
    case 1: k_spmv<1><<<G, TPB, 0, s>>>(g, op->d_val[vs], x, y); break;
    case 2: k_spmv<2><<<G, TPB, 0, s>>>(g, op->d_val[vs], x, y); break;
    default: k_spmv<-1><<<G, TPB, 0, s>>>(g, op->d_val[vs], x, y); break;
  }
  count_launch();
  return cuda_check(cudaGetLastError(), "k_spmv");
}

namespace {
// r = b - A x by row_residual_dot2, with the grid sums (r, r), (|A||x| + |b|)^2 and (b, b) left
// in aux[2..4] of the operator's scalar block (ticket 5).
template <int MASKC>
__global__ void __launch_bounds__(TPB) k_residual_any(Geom g, const double* __restrict__ val,
                                                      const double* __restrict__ b, const double* __restrict__ x,
                                                      double* __restrict__ r, double* partials, PcgScalars* sc) {
  double v[3] = {0.0, 0.0, 0.0};
  const int n = (int)g.n;
  for (int row = blockIdx.x * blockDim.x + threadIdx.x; row < n; row += gridDim.x * blockDim.x) {
    const int col = row / g.nz;
    const int k = row - col * g.nz;
    double asum = 0.0;
    const double bi = b[row];
    const double ri = row_residual_dot2<MASKC>(g, val, x, bi, row, col, k, asum);
    r[row] = ri;
    v[0] = fma(ri, ri, v[0]);
    const double f = asum + fabs(bi);
    v[1] = fma(f, f, v[1]);
    v[2] = fma(bi, bi, v[2]);
  }
  if (grid_sum<3>(v, partials, &sc->count[5]) && threadIdx.x == 0) {
    sc->aux[2] = v[0];
    sc->aux[3] = v[1];
    sc->aux[4] = v[2];
  }
}
}  // namespace

int residual(pm_operator* op, int which, const double* b, const double* x, double* r, double* norms,
             cudaStream_t s) {
  const int vs = which_valset(which);
  if (vs < 0) return set_error(PM_EINVAL, "unknown operator");
  int st = ensure_ctx(op);
  if (st) return st;
  SolveCtx* c = op->ctx;
  Geom g = geom_of(op);
  const int G = grid_for(op->n, TPB, op->num_sms);
  switch (which_mask(which)) {
    case 0: k_residual_any<0><<<G, TPB, 0, s>>>(g, op->d_val[vs], b, x, r, c->partials, c->sc); break;
    case 1: k_residual_any<1><<<G, TPB, 0, s>>>(g, op->d_val[vs], b, x, r, c->partials, c->sc); break;
    case 2: k_residual_any<2><<<G, TPB, 0, s>>>(g, op->d_val[vs], b, x, r, c->partials, c->sc); break;
    default: k_residual_any<-1><<<G, TPB, 0, s>>>(g, op->d_val[vs], b, x, r, c->partials, c->sc); break;
  }
  count_launch();
  if ((st = cuda_check(cudaGetLastError(), "k_residual_any"))) return st;
  if (!norms) return PM_OK;
  if ((st = read_scalars(c, s))) return st;
  norms[0] = c->sc_host->aux[2];
  norms[1] = c->sc_host->aux[3];
  norms[2] = c->sc_host->aux[4];
  return PM_OK;
}

int pcg_solve(pm_operator* op, int which, const double* b, double* x, const pm_solve_opts* o,
              pm_solve_stats* st, cudaStream_t s) {
  if (!which_symmetric(which)) return set_error(PM_EINVAL, "pcg needs a symmetric operator");
  if (o->prec < 0 || o->prec > PM_PREC_LINE) return set_error(PM_EINVAL, "unknown preconditioner");
  if (!(o->rtol > 0.0) || o->max_iter < 0) return set_error(PM_EINVAL, "rtol must be > 0, max_iter >= 0");
  if (o->precision < PM_FP64 || o->precision > PM_BF16_REFINE) return set_error(PM_EINVAL, "unknown precision");
  if (o->kernel < PM_KERNEL_AUTO || o->kernel > PM_KERNEL_RESIDENT) return set_error(PM_EINVAL, "unknown kernel choice");
  NvtxRange range(std::string("pcg ") + which_name(which) + " " + prec_name(o->prec) + " " + precision_name(o->precision));
  int r = ensure_ctx(op);
  if (r) return r;
  if (o->precision == PM_FP32_REFINE) {
    switch (which_mask(which)) {
      case 0: return mixed_run<0, float>(op, which, b, x, o, st, s);
      case 1: return mixed_run<1, float>(op, which, b, x, o, st, s);
      case 2: return mixed_run<2, float>(op, which, b, x, o, st, s);
      default: return mixed_run<-1, float>(op, which, b, x, o, st, s);
    }
  }
  if (o->precision == PM_BF16_REFINE) {
    switch (which_mask(which)) {
      case 0: return mixed_run<0, __nv_bfloat16>(op, which, b, x, o, st, s);
      case 1: return mixed_run<1, __nv_bfloat16>(op, which, b, x, o, st, s);
      case 2: return mixed_run<2, __nv_bfloat16>(op, which, b, x, o, st, s);
      default: return mixed_run<-1, __nv_bfloat16>(op, which, b, x, o, st, s);
    }
  }
  const bool resident = o->kernel == PM_KERNEL_RESIDENT || (o->kernel == PM_KERNEL_AUTO && op->n <= SMALL_AUTO_ROWS);
  if (resident) {
    if (op->n > SMALL_MAX_ROWS)
      return set_error(PM_EINVAL, "PM_KERNEL_RESIDENT: at most " + std::to_string(SMALL_MAX_ROWS) + " rows");
    switch (which_mask(which)) {
      case 0: return small_run<0>(op, which, b, x, o, st, s);
      case 1: return small_run<1>(op, which, b, x, o, st, s);
      case 2: return small_run<2>(op, which, b, x, o, st, s);
      default: return small_run<-1>(op, which, b, x, o, st, s);
    }
  }
  switch (which_mask(which)) {
    case 0: return pcg_run<0>(op, which, b, x, o, st, s);
    case 1: return pcg_run<1>(op, which, b, x, o, st, s);
    case 2: return pcg_run<2>(op, which, b, x, o, st, s);
    default: return pcg_run<-1>(op, which, b, x, o, st, s);
  }
}

// Everything a batched solve reads from one operator: Jacobi diagonals, line or IC0 factors, and
// for FP32 the difference-form values and FP32 factors.
int prepare_for_batch(pm_operator* op, int which, int prec, int precision, cudaStream_t s) {
  int st = ensure_ctx(op);
  if (st) return st;
  if ((st = launch_dinv(op, which, s))) return st;
  if (prec == PM_PREC_LINE && (st = line_factor(op, which, s))) return st;
  if (prec == PM_PREC_IC0 && !op->ic0[which].ok) {
    int bd = 0;
    for (int m = -1; m <= 10; ++m) {
      if ((st = launch_ic0_factor(op, which, m < 0 ? 0.0 : 1e-3 * std::pow(2.0, m), &bd, s))) return st;
      if (!bd) break;
    }
    if (bd) return set_error(PM_BREAKDOWN, "IC0 pivot failure after the shift limit");
  }
  if (precision != PM_FP64 && (st = ensure_mixed(op, which, precision, prec, s))) return st;
  return PM_OK;
}

}  // namespace pm

extern "C" int pm_kernel_timing(int32_t enable) {
  using namespace pm;
  if (!g_kt.pending.empty()) {
    cudaDeviceSynchronize();
    kt_collect();
  }
  g_kt.on = enable != 0;
  for (int k = 0; k < PM_KT_COUNT; ++k) {
    g_kt.total_ms[k] = 0.0;
    g_kt.launches[k] = 0;
  }
  return PM_OK;
}

extern "C" int pm_kernel_timing_get(int32_t kind, double* total_ms, int64_t* launches) {
  using namespace pm;
  if (kind < 0 || kind >= PM_KT_COUNT) return set_error(PM_EINVAL, "unknown kernel class");
  if (!g_kt.pending.empty()) {
    cudaDeviceSynchronize();
    kt_collect();
  }
  if (total_ms) *total_ms = g_kt.total_ms[kind];
  if (launches) *launches = g_kt.launches[kind];
  return PM_OK;
}

namespace pm {

void destroy_ctx(pm_operator* op) {
  SolveCtx* c = op->ctx;
  if (!c) return;
  cudaFree(c->r);
  cudaFree(c->p);
  cudaFree(c->w);
  cudaFree(c->z);
  cudaFree(c->bw);
  cudaFree(c->partials);
  cudaFree(c->sc);
  cudaFreeHost(c->sc_host);
  cudaFree(c->r32);
  cudaFree(c->p32);
  cudaFree(c->w32);
  cudaFree(c->z32);
  cudaFree(c->d32);
  cudaFree(c->sc_in);
  if (c->sc_in_host) cudaFreeHost(c->sc_in_host);
  cudaFree(c->small_out);
  if (c->small_out_host) cudaFreeHost(c->small_out_host);
  delete c;
  op->ctx = nullptr;
}

}  // namespace pm
