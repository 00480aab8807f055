// pm_pcg_solve_noalloc: the Jacobi / plain PCG solve with every scratch buffer taken from one
// file-scope device array instead of allocated memory.
//
// Some callers cannot allocate device memory while they solve: hosts whose device memory is
// owned by a custom pool or a framework allocator (a cudaMalloc behind its back would escape its
// accounting or fail against its reservation), and embedded callers that must not grow the
// device footprint after start-up. This entry point serves them. It calls no cudaMalloc,
// cudaFree, cudaMallocHost or any other allocating routine (torch's included): the Krylov
// vectors r, p, w, the projected right-hand side, the Jacobi inverse diagonal, the reduction
// partials and the device scalars all live in g_pm_noalloc_scratch below, which every GPU that
// loads the library holds until the process exits (about 21 MB). Host-side scalars are read into
// stack memory.
//
// Limits and sharing rules:
//   - n (rows) <= PM_NOALLOC_MAX_ROWS; larger systems are rejected with PM_EINVAL.
//   - Jacobi or no preconditioner, FP64 (the IC0 and line factors would need storage).
//   - The operator's device must be the current device (PM_EINVAL otherwise).
//   - The call reads convergence scalars back to the host and synchronises the stream every few
//     iterations, so it is rejected with PM_EINVAL when the stream is being captured.
//   - All calls on a device share the one array, which keeps the last call's contents; every
//     call re-initialises what must start at zero (reduction tickets, scalars). Calls that
//     overlap on the GPU (different streams, or different host threads) race on the array.
//   - The first call on a device (with that device current) looks the array's device address up
//     with cudaGetSymbolAddress.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstring>
#include <mutex>

#include "pm_internal.cuh"

namespace pm {
namespace na {

constexpr int64_t MAXR = PM_NOALLOC_MAX_ROWS;
constexpr int TPB = 256;
constexpr int64_t OFF_R = 0;
constexpr int64_t OFF_P = 1 * MAXR;
constexpr int64_t OFF_W = 2 * MAXR;
constexpr int64_t OFF_BW = 3 * MAXR;
constexpr int64_t OFF_DINV = 4 * MAXR;
constexpr int64_t OFF_PART = 5 * MAXR;
constexpr int64_t OFF_SC = OFF_PART + ((int64_t)NPART * MAX_GRID + 31) / 32 * 32;
constexpr int64_t TOTAL = OFF_SC + ((int64_t)sizeof(PcgScalars) + 255) / 256 * 32;

}  // namespace na
}  // namespace pm

// The scratch array. In host code its name is only a stand-in: the device address comes from
// cudaGetSymbolAddress (see scratch_for_current_device).
static __device__ __align__(256) double g_pm_noalloc_scratch[pm::na::TOTAL];

namespace pm {
namespace na {
namespace {

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  return v;
}

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
    for (int i = 0; i < NV; ++i) v[i] = warp_sum(lane < nw ? sm[i * 32 + lane] : 0.0);
  }
  __syncthreads();
}

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

__device__ __forceinline__ bool done_(const PcgScalars* sc) { return *((volatile const int32_t*)&sc->done) != 0; }

template <int MASKC>
__device__ __forceinline__ double row_dot(const Geom& g, const double* __restrict__ val, const double* __restrict__ x,
                                          int64_t row, int col, int k) {
  const int nz = g.nz;
  if (MASKC >= 0 && is_dirichlet(g.colflag[col], k, nz, MASKC)) return x[row];
  int nb[NNBR];
  uint8_t fl[NNBR];
#pragma unroll
  for (int q = 0; q < NNBR; ++q) {
    nb[q] = q == 0 ? col : nbr_of(g, col, q);
    if (MASKC >= 0) fl[q] = nb[q] >= 0 ? g.colflag[nb[q]] : 0;
  }
  double sum = 0.0;
#pragma unroll
  for (int s = 0; s < NSLOT; ++s) {
    const int q = slot_q(s);
    const int kk = k + slot_dk(s);
    if (nb[q] < 0 || kk < 0 || kk >= nz) continue;
    if (MASKC >= 0 && is_dirichlet(fl[q], kk, nz, MASKC)) continue;
    sum = fma(val[(int64_t)s * g.npad + row], x[(int64_t)nb[q] * nz + kk], sum);
  }
  return sum;
}

// Jacobi inverse diagonal (1 on Dirichlet rows); prec NONE: all ones.
__global__ void k_dinv(Geom g, const double* __restrict__ val, int maskc, int none, double* __restrict__ dinv) {
  for (int64_t row = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; row < g.n; row += (int64_t)gridDim.x * blockDim.x) {
    const int col = (int)(row / g.nz), k = (int)(row - (int64_t)col * g.nz);
    double d = 1.0;
    if (!none && (maskc < 0 || !is_dirichlet(g.colflag[col], k, g.nz, maskc))) d = 1.0 / val[DIAG_SLOT * g.npad + row];
    dinv[row] = d;
  }
}

__global__ void k_press_sums(int64_t n, const double* __restrict__ b, const double* __restrict__ x,
                             const double* __restrict__ m, int use_x, double* partials, PcgScalars* sc) {
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

__global__ void k_prepare(int64_t n, const double* __restrict__ b, const double* __restrict__ m, double* __restrict__ bw,
                          double* __restrict__ x, int press, int use_x, const PcgScalars* sc) {
  const double lam = press ? sc->lam : 0.0, xs = press ? sc->xshift : 0.0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    if (press) bw[i] = b[i] - lam * m[i];
    x[i] = use_x ? x[i] - xs : 0.0;
  }
}

template <int MASKC, int MODE>
__global__ void k_residual(Geom g, const double* __restrict__ val, const double* __restrict__ bw,
                           const double* __restrict__ x, double* __restrict__ r, double rtol, double* partials,
                           PcgScalars* sc) {
  double v[3] = {0.0, 0.0, 0.0};
  for (int64_t row = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; row < g.n; row += (int64_t)gridDim.x * blockDim.x) {
    const int col = (int)(row / g.nz), k = (int)(row - (int64_t)col * g.nz);
    double asum = 0.0;
    const double bi = bw[row];
    const double ri = row_residual_dot2<MASKC>(g, val, x, bi, (int)row, col, k, asum);   // compensated
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

template <int PROJ>
__global__ void k_first(int64_t n, const double* __restrict__ r, const double* __restrict__ dinv, const double* __restrict__ m,
                        double* __restrict__ p, double* partials, PcgScalars* sc) {
  double v[3] = {0.0, 0.0, 0.0};
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const double ri = r[i], zi = dinv[i] * ri;
    v[0] = fma(ri, zi, v[0]);
    if (PROJ) {
      v[1] = fma(m[i], zi, v[1]);
      v[2] += ri;
    }
  }
  if (grid_sum<3>(v, partials, &sc->count[2]) && threadIdx.x == 0) {
    const double c = PROJ ? v[1] / sc->one_m : 0.0;
    const double rho = v[0] - c * v[2];
    sc->proj_c = c;
    sc->rho = rho;
    sc->beta = 0.0;
    if ((!(rho > 0.0) || !isfinite(rho)) && !sc->done) {
      sc->status = PM_BREAKDOWN;
      sc->done = 1;
    }
  }
}

__global__ void k_pupd(int64_t n, const double* __restrict__ r, const double* __restrict__ dinv, double* __restrict__ p,
                       const PcgScalars* sc, int first) {
  if (!first && done_(sc)) return;
  const double beta = sc->beta, c = sc->proj_c;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const double zi = dinv[i] * r[i] - c;
    p[i] = first ? zi : fma(beta, p[i], zi);
  }
}

template <int MASKC>
__global__ void k_spmv_dot(Geom g, const double* __restrict__ val, const double* __restrict__ p, double* __restrict__ w,
                           double* partials, PcgScalars* sc) {
  if (done_(sc)) return;
  double v[1] = {0.0};
  for (int64_t row = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; row < g.n; row += (int64_t)gridDim.x * blockDim.x) {
    const int col = (int)(row / g.nz), k = (int)(row - (int64_t)col * g.nz);
    const double wi = row_dot<MASKC>(g, val, p, row, col, k);
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

template <int PROJ>
__global__ void k_update(int64_t n, double* __restrict__ x, double* __restrict__ r, const double* __restrict__ p,
                         const double* __restrict__ w, const double* __restrict__ dinv, const double* __restrict__ m,
                         double* partials, PcgScalars* sc) {
  if (done_(sc)) return;
  const double alpha = sc->alpha;
  double v[4] = {0.0, 0.0, 0.0, 0.0};
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    x[i] = fma(alpha, p[i], x[i]);
    const double ri = fma(-alpha, w[i], r[i]);
    r[i] = ri;
    v[0] = fma(ri, ri, v[0]);
    const double zi = dinv[i] * ri;
    v[1] = fma(ri, zi, v[1]);
    if (PROJ) {
      v[2] = fma(m[i], zi, v[2]);
      v[3] += ri;
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

__global__ void k_fill(double* x, int64_t n, double v) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) x[i] = v;
}
__global__ void k_shift(double* x, int64_t n, const PcgScalars* sc) {
  const double v = sc->xshift;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) x[i] -= v;
}

int grid_of(int64_t n, int sms) {
  int64_t g = (n + TPB - 1) / TPB;
  int64_t cap = std::min<int64_t>((int64_t)sms * 8, MAX_GRID);
  return (int)std::max<int64_t>(1, std::min(g, cap));
}

// Device address of the scratch array for the current device, looked up once per device.
double* scratch_for_current_device() {
  static std::mutex mu;
  static double* addr[256] = {};
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 256) return nullptr;
  std::lock_guard<std::mutex> lk(mu);
  if (!addr[dev]) {
    double* p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress((void**)&p, g_pm_noalloc_scratch);
    if (e != cudaSuccess) {
      cuda_check(e, "cudaGetSymbolAddress(g_pm_noalloc_scratch)");
      return nullptr;
    }
    addr[dev] = p;
  }
  return addr[dev];
}

struct View {
  double *r, *p, *w, *bw, *dinv, *part;
  PcgScalars* sc;
};

template <int MASKC>
int run(pm_operator* op, int which, const double* b, double* x, const pm_solve_opts* o, pm_solve_stats* stats,
        cudaStream_t s, const View& v) {
  auto t0 = std::chrono::steady_clock::now();
  Geom g = geom_of(op);
  const int64_t n = op->n;
  const int G = grid_of(n, op->num_sms);
  const bool proj = which == PM_OP_PRESSURE;
  const double* val = op->d_val[which_valset(which)];
  PcgScalars h;
  std::memset(&h, 0, sizeof(h));
  h.one_m = op->one_m;
  h.max_iter = o->max_iter;
  int st = cuda_check(cudaMemcpyAsync(v.sc, &h, sizeof(h), cudaMemcpyHostToDevice, s), "scalars init");
  if (st) return st;
  k_dinv<<<G, TPB, 0, s>>>(g, val, which_mask(which), o->prec == PM_PREC_NONE ? 1 : 0, v.dinv);
  const double* bw = b;
  if (proj) {
    k_press_sums<<<G, TPB, 0, s>>>(n, b, x, op->d_m, o->x0_is_guess ? 1 : 0, v.part, v.sc);
    k_prepare<<<G, TPB, 0, s>>>(n, b, op->d_m, v.bw, x, 1, o->x0_is_guess ? 1 : 0, v.sc);
    bw = v.bw;
  } else if (!o->x0_is_guess) {
    k_prepare<<<G, TPB, 0, s>>>(n, b, op->d_m, nullptr, x, 0, 0, v.sc);
  }
  k_residual<MASKC, 0><<<G, TPB, 0, s>>>(g, val, bw, x, v.r, o->rtol, v.part, v.sc);
  auto first = [&]() {
    if (proj) k_first<1><<<G, TPB, 0, s>>>(n, v.r, v.dinv, op->d_m, v.p, v.part, v.sc);
    else k_first<0><<<G, TPB, 0, s>>>(n, v.r, v.dinv, op->d_m, v.p, v.part, v.sc);
    k_pupd<<<G, TPB, 0, s>>>(n, v.r, v.dinv, v.p, v.sc, 1);
  };
  auto read = [&]() -> int {
    int e = cuda_check(cudaMemcpyAsync(&h, v.sc, sizeof(h), cudaMemcpyDeviceToHost, s), "scalars");
    return e ? e : cuda_check(cudaStreamSynchronize(s), "noalloc pcg sync");
  };
  first();
  count_launch(6);
  if ((st = read())) return st;
  int restarts = 0, first_pass = 0, status = PM_OK;
  double rel_true = 0.0, rel_floor = 0.0, prev_true = -1.0;
  bool accepted = false;
  if (h.zero_rhs) {
    k_fill<<<G, TPB, 0, s>>>(x, n, 0.0);
    count_launch();
    if ((st = read())) return st;
  } else {
    int64_t issued = 0;
    for (;;) {
      int chunk = 4;
      while (!h.done) {
        if (issued > (int64_t)o->max_iter + 4096) return set_error(PM_ECUDA, "PCG driver: device never reported completion");
        for (int it = 0; it < chunk; ++it) {
          k_spmv_dot<MASKC><<<G, TPB, 0, s>>>(g, val, v.p, v.w, v.part, v.sc);
          if (proj) k_update<1><<<G, TPB, 0, s>>>(n, x, v.r, v.p, v.w, v.dinv, op->d_m, v.part, v.sc);
          else k_update<0><<<G, TPB, 0, s>>>(n, x, v.r, v.p, v.w, v.dinv, op->d_m, v.part, v.sc);
          k_pupd<<<G, TPB, 0, s>>>(n, v.r, v.dinv, v.p, v.sc, 0);
          count_launch(3);
        }
        issued += chunk;
        if ((st = read())) return st;
        if (chunk < 64) chunk *= 2;
      }
      status = h.status;
      if (restarts == 0) first_pass = h.iter;
      k_residual<MASKC, 1><<<G, TPB, 0, s>>>(g, val, bw, x, v.r, o->rtol, v.part, v.sc);
      count_launch();
      if ((st = read())) return st;
      rel_true = std::sqrt(h.aux[0] / h.bb);
      rel_floor = std::ldexp(1.0, -53) * std::sqrt(h.aux[1] / h.bb);
      // as pm_pcg_solve: rtol met, or below the FP64 floor once restarts stop halving it
      const bool stalled = prev_true >= 0.0 && rel_true > 0.5 * prev_true;
      const bool last = restarts >= o->max_restarts || h.iter >= o->max_iter;
      accepted = rel_true <= o->rtol || (rel_true <= rel_floor && (stalled || last));
      if (status != PM_OK || accepted || last) break;
      prev_true = rel_true;
      ++restarts;
      h.done = 0;
      h.rr = h.aux[0];
      if ((st = cuda_check(cudaMemcpyAsync(v.sc, &h, sizeof(h), cudaMemcpyHostToDevice, s), "scalars"))) return st;
      first();
      count_launch(2);
      if ((st = read())) return st;
    }
    if (status == PM_OK && !accepted) status = PM_NOT_CONVERGED;
  }
  if (proj) {
    k_press_sums<<<G, TPB, 0, s>>>(n, b, x, op->d_m, 1, v.part, v.sc);
    k_shift<<<G, TPB, 0, s>>>(x, n, v.sc);
    count_launch(2);
    if ((st = read())) return st;
  }
  if (stats) {
    stats->iters = h.iter;
    stats->outer_iters = restarts;
    stats->first_pass_iters = first_pass;
    stats->status = status;
    stats->rel_residual_true = h.zero_rhs ? 0.0 : rel_true;
    stats->rel_residual_rec = h.zero_rhs ? 0.0 : std::sqrt(h.rr / h.bb);
    stats->rel_residual_floor = rel_floor;
    stats->bytes_moved = (double)h.iter * (double)n * (15 * 8 + 8 + 8 + 5 * 8 + 2 * 8 + 3 * 8 + 8);
    stats->seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
  }
  if ((st = cuda_check(cudaGetLastError(), "noalloc pcg kernels"))) return st;
  if (status != PM_OK)
    return set_error(status, status == PM_NOT_CONVERGED ? "PCG did not reach rtol within max_iter"
                                                        : "PCG breakdown: (p, Ap) <= 0 or non-finite");
  return PM_OK;
}

}  // namespace
}  // namespace na
}  // namespace pm

extern "C" int pm_pcg_solve_noalloc(pm_operator* op, pm_which which, const double* b, double* x,
                                    const pm_solve_opts* opts, pm_solve_stats* stats, pm_stream stream) {
  using namespace pm;
  if (!op || !b || !x || !opts) return set_error(PM_EINVAL, "null argument");
  if (!which_symmetric((int)which)) return set_error(PM_EINVAL, "pcg needs a symmetric operator");
  if (opts->prec != PM_PREC_JACOBI && opts->prec != PM_PREC_NONE)
    return set_error(PM_EINVAL, "pm_pcg_solve_noalloc supports PM_PREC_JACOBI and PM_PREC_NONE only");
  if (opts->precision != PM_FP64) return set_error(PM_EINVAL, "pm_pcg_solve_noalloc solves in FP64 only");
  if (!(opts->rtol > 0.0) || opts->max_iter < 0) return set_error(PM_EINVAL, "rtol must be > 0, max_iter >= 0");
  if (op->n > na::MAXR)
    return set_error(PM_EINVAL, "pm_pcg_solve_noalloc: the system has " + std::to_string(op->n) +
                                    " rows, more than PM_NOALLOC_MAX_ROWS = " + std::to_string(na::MAXR));
  cudaStream_t s = (cudaStream_t)stream;
  cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
  int st = cuda_check(cudaStreamIsCapturing(s, &cap), "cudaStreamIsCapturing");
  if (st) return st;
  if (cap != cudaStreamCaptureStatusNone)
    return set_error(PM_EINVAL, "pm_pcg_solve_noalloc synchronises its stream; it cannot be called on a stream "
                                "that is being captured");
  int dev = -1;
  if ((st = cuda_check(cudaGetDevice(&dev), "cudaGetDevice"))) return st;
  if (dev != op->device)
    return set_error(PM_EINVAL, "pm_pcg_solve_noalloc: the operator lives on device " + std::to_string(op->device) +
                                    ", the current device is " + std::to_string(dev));
  double* base = na::scratch_for_current_device();
  if (!base) return PM_ECUDA;
  na::View v;
  v.r = base + na::OFF_R;
  v.p = base + na::OFF_P;
  v.w = base + na::OFF_W;
  v.bw = base + na::OFF_BW;
  v.dinv = base + na::OFF_DINV;
  v.part = base + na::OFF_PART;
  v.sc = reinterpret_cast<PcgScalars*>(base + na::OFF_SC);
  NvtxRange range(std::string("pcg_noalloc ") + which_name((int)which) + " " + prec_name(opts->prec));
  pm_solve_stats local = {};
  switch (which_mask((int)which)) {
    case 0: st = na::run<0>(op, (int)which, b, x, opts, &local, s, v); break;
    case 1: st = na::run<1>(op, (int)which, b, x, opts, &local, s, v); break;
    case 2: st = na::run<2>(op, (int)which, b, x, opts, &local, s, v); break;
    default: st = na::run<-1>(op, (int)which, b, x, opts, &local, s, v); break;
  }
  const int bs = bounds_status("pm_pcg_solve_noalloc");
  if (bs) st = bs;
  if (stats) *stats = local;
  if (log_enabled()) log_solve("pcg_solve_noalloc", op, (int)which, opts->prec, PM_FP64, local);
  return st;
}
