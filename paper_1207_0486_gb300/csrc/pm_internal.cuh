// Internal declarations of the GB300 projection-method library: data layout, device helpers
// and the host-side launchers each translation unit provides.
//
// Layout in HBM ("column-sliced ELL"): node id = column * nz + k over the ocean columns.
// Every row has exactly 15 slots at fixed stencil offsets; a slot's column index is never
// stored: it is nbr[column][q] * nz + k + dk. Values are slot-major, values[s * n_pad + row],
// so a warp over consecutive rows reads each slot as one contiguous 256-byte line.
//
// The 15 slots are the node itself and its 14 Kuhn neighbours (edges of the six tetrahedra of
// each hex split along its (0,0,0)-(1,1,1) diagonal): offsets (di, dj, dk) =
//   s : 0        1       2       3       4       5          6        7       8       9
//       (0,0,-1) (0,0,0) (0,0,1) (1,0,0) (1,0,1) (-1,0,-1) (-1,0,0) (0,1,0) (0,1,1) (0,-1,-1)
//   s : 10        11      12      13          14
//       (0,-1,0) (1,1,0) (1,1,1) (-1,-1,-1) (-1,-1,0)
// They lie in 7 columns q: 0 (0,0), 1 (+1,0), 2 (-1,0), 3 (0,+1), 4 (0,-1), 5 (+1,+1), 6 (-1,-1).
#pragma once

#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "../../include/pm.h"

namespace pm {

// Host-side NVTX range for the lifetime of a scope: profilers show the library's assemblies,
// solves, steps and their stages on the timeline. Without a profiler attached the calls return
// at once.
struct NvtxRange {
  explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
  explicit NvtxRange(const std::string& name) { nvtxRangePushA(name.c_str()); }
  ~NvtxRange() { nvtxRangePop(); }
  NvtxRange(const NvtxRange&) = delete;
  NvtxRange& operator=(const NvtxRange&) = delete;
};

// ---- checked build (PM_CHECKED): device-side index checks --------------------------------------
// Every neighbour-column index a kernel reads is checked against the column count; the first bad
// one is recorded (site, value, limit) and read as "no neighbour", so the kernel skips the access
// instead of faulting, and the entry point that launched it returns PM_EBOUNDS. Each translation
// unit has its own record (no relocatable device code) and registers a reader for it at load time.
enum BoundsSite { SITE_NONE = 0, SITE_NBR = 1 };
struct BoundsRecord {
  int32_t flag, site;
  int64_t value, limit;
};
using BoundsReader = int (*)(BoundsRecord*);
void register_bounds_reader(BoundsReader r);   // pm_trace.cu
// PM_EBOUNDS with a message when a checked kernel recorded a bad index since the last call
// (clears the records); PM_OK otherwise, and always in an unchecked build.
int bounds_status(const char* where);
#ifdef PM_CHECKED
namespace {
__device__ BoundsRecord g_bounds_tu;
__device__ __noinline__ void record_bad_index(int site, int64_t value, int64_t limit) {
  if (atomicCAS(&g_bounds_tu.flag, 0, 1) == 0) {
    g_bounds_tu.site = site;
    g_bounds_tu.value = value;
    g_bounds_tu.limit = limit;
  }
}
int read_bounds_tu(BoundsRecord* out) {
  if (cudaMemcpyFromSymbol(out, g_bounds_tu, sizeof(BoundsRecord)) != cudaSuccess) return 0;
  if (out->flag) {
    const BoundsRecord zero = {0, 0, 0, 0};
    cudaMemcpyToSymbol(g_bounds_tu, &zero, sizeof(BoundsRecord));
  }
  return out->flag;
}
struct BoundsRegistration {
  BoundsRegistration() { register_bounds_reader(&read_bounds_tu); }
} g_bounds_registration_tu;
}  // namespace
#endif

// ---- per-solve JSON log (pm_set_log) -------------------------------------------------------------
const char* which_name(int which);
const char* prec_name(int prec);
const char* precision_name(int precision);
bool log_enabled();
// One JSON line for one solved system: event name, basin size, system, options and its stats.
void log_solve(const char* event, const pm_operator* op, int which, int prec, int precision,
               const pm_solve_stats& st);

constexpr int NSLOT = 15;
constexpr int NNBR = 7;
constexpr int DIAG_SLOT = 1;

// Column flags (per ocean column).
constexpr uint8_t CF_GAMMA0 = 1;  // coastline or no-slip outer wall: Gamma_0 on every level
constexpr uint8_t CF_G1X = 2;     // x-normal slip wall (Gamma_1)
constexpr uint8_t CF_G1Y = 4;     // y-normal slip wall (Gamma_1)

__host__ __device__ constexpr int slot_q(int s) {
  return s < 3 ? 0 : s < 5 ? 1 : s < 7 ? 2 : s < 9 ? 3 : s < 11 ? 4 : s < 13 ? 5 : 6;
}
__host__ __device__ constexpr int slot_dk(int s) {
  return s == 0 ? -1 : s == 1 ? 0 : s == 2 ? 1 : s == 3 ? 0 : s == 4 ? 1 : s == 5 ? -1 :
         s == 6 ? 0 : s == 7 ? 0 : s == 8 ? 1 : s == 9 ? -1 : s == 10 ? 0 : s == 11 ? 0 :
         s == 12 ? 1 : s == 13 ? -1 : 0;
}
__host__ __device__ constexpr int q_di(int q) {
  return q == 1 || q == 5 ? 1 : q == 2 || q == 6 ? -1 : 0;
}
__host__ __device__ constexpr int q_dj(int q) {
  return q == 3 || q == 5 ? 1 : q == 4 || q == 6 ? -1 : 0;
}
__host__ __device__ constexpr int slot_di(int s) { return q_di(slot_q(s)); }
__host__ __device__ constexpr int slot_dj(int s) { return q_dj(slot_q(s)); }
// Slot whose offset is the negative of s's.
__host__ __device__ constexpr int slot_mirror(int s) {
  return s == 0 ? 2 : s == 2 ? 0 : s == 1 ? 1 : s == 3 ? 6 : s == 6 ? 3 : s == 4 ? 5 :
         s == 5 ? 4 : s == 7 ? 10 : s == 10 ? 7 : s == 8 ? 9 : s == 9 ? 8 : s == 11 ? 14 :
         s == 14 ? 11 : s == 12 ? 13 : 12;
}
// Slot of offset (di, dj, dk), or -1 when the offset is not a Kuhn edge.
__host__ __device__ constexpr int slot_of(int di, int dj, int dk) {
  return (di == 0 && dj == 0) ? (dk == -1 ? 0 : dk == 0 ? 1 : 2)
       : (di == 1 && dj == 0) ? (dk == 0 ? 3 : dk == 1 ? 4 : -1)
       : (di == -1 && dj == 0) ? (dk == -1 ? 5 : dk == 0 ? 6 : -1)
       : (di == 0 && dj == 1) ? (dk == 0 ? 7 : dk == 1 ? 8 : -1)
       : (di == 0 && dj == -1) ? (dk == -1 ? 9 : dk == 0 ? 10 : -1)
       : (di == 1 && dj == 1) ? (dk == 0 ? 11 : dk == 1 ? 12 : -1)
       : (di == -1 && dj == -1) ? (dk == -1 ? 13 : dk == 0 ? 14 : -1)
       : -1;
}
// Multicolour parity flip of a slot: colour(neighbour) = colour(row) ^ slot_flip(s).
__host__ __device__ constexpr int slot_flip(int s) {
  return (slot_di(s) & 1) | ((slot_dj(s) & 1) << 1) | ((slot_dk(s) & 1) << 2);
}

// Homogeneous Dirichlet set of velocity component c (0, 1, 2) at level k of a column.
__host__ __device__ inline bool is_dirichlet(uint8_t flag, int k, int nz, int c) {
  if (k == 0 || (flag & CF_GAMMA0)) return true;
  if (c == 0) return (flag & CF_G1X) != 0;
  if (c == 1) return (flag & CF_G1Y) != 0;
  return k == nz - 1;
}

// ---- compensated residual (Ogita, Rump & Oishi, "Accurate sum and dot product", 2005) --------
// Error-free transformations in FP64. The _rn intrinsics are never contracted into an FMA, which
// would change what the transformations compute.
__device__ __forceinline__ double two_sum(double a, double b, double& err) {
  const double s = __dadd_rn(a, b);
  const double bv = __dsub_rn(s, a);
  err = __dadd_rn(__dsub_rn(a, __dsub_rn(s, bv)), __dsub_rn(b, bv));
  return s;
}
// a * b = p + err exactly (one FMA gives the rounding error of the product).
__device__ __forceinline__ double two_product(double a, double b, double& err) {
  const double p = __dmul_rn(a, b);
  err = fma(a, b, -p);
  return p;
}

// Compensated FP32 ("double-float") accumulation of the mixed-precision dot products. GB300's
// FP64 pipe runs at 1/64 of its FP32 rate, and an FP64 dot of FP32 vectors costs two conversions
// and an FP64 FMA per term on that pipe, which made the FP32 kernels FP64-bound. Here each product
// a b is split exactly into p + e by one FP32 FMA (TwoProduct), p is added to the running sum by
// TwoSum, and both rounding errors go into a second FP32 word: a thread's partial sum keeps about
// 48 significant bits (relative error of order n u32^2 for its n terms, u32 = 2^-24) and becomes
// an FP64 number once, where the FP64 block and grid reductions take over.
struct DF {
  float hi = 0.f, lo = 0.f;
  __device__ __forceinline__ void add(float a) {
    const float s = __fadd_rn(hi, a);
    const float bv = __fsub_rn(s, hi);
    const float e = __fadd_rn(__fsub_rn(hi, __fsub_rn(s, bv)), __fsub_rn(a, bv));
    hi = s;
    lo = __fadd_rn(lo, e);
  }
  __device__ __forceinline__ void add_prod(float a, float b) {
    const float pr = __fmul_rn(a, b);
    const float pe = fmaf(a, b, -pr);
    add(pr);
    lo = __fadd_rn(lo, pe);
  }
  __device__ __forceinline__ double value() const { return (double)hi + (double)lo; }
};

// The same interface accumulating in FP64 (the FP64 kernels' dots), so that a kernel templated on
// its vector type can pick its accumulator: AccFor<float> = DF, AccFor<double> = Acc64.
struct Acc64 {
  double v = 0.0;
  __device__ __forceinline__ void add(double a) { v += a; }
  __device__ __forceinline__ void add_prod(double a, double b) { v = fma(a, b, v); }
  __device__ __forceinline__ double value() const { return v; }
};
template <typename T> struct AccSel { using type = Acc64; };
template <> struct AccSel<float> { using type = DF; };
template <typename T> using AccFor = typename AccSel<T>::type;

// Device view of a basin's mesh.
struct Geom {
  int32_t ncols, nz;
  int64_t n, npad;
  double dx, dy;
  const int32_t* nbr;       // [ncols * 7], -1 absent (entry q = 0 is the column itself)
  const double* depth;      // [ncols]
  const uint8_t* cellmask;  // [ncols] bit0 cell(i-1,j-1), bit1 cell(i,j-1), bit2 cell(i-1,j), bit3 cell(i,j)
  const uint8_t* colflag;   // [ncols] CF_*
  const double* coriolis;   // [ncols] or null
};

// Neighbour column q of column col (-1: none; q = 0 is col itself). Checked builds validate it.
__device__ __forceinline__ int nbr_of(const Geom& g, int64_t col, int q) {
  const int nb = __ldg(g.nbr + col * NNBR + q);
#ifdef PM_CHECKED
  if (nb < -1 || nb >= g.ncols) {
    record_bad_index(SITE_NBR, nb, g.ncols);
    return -1;
  }
#endif
  return nb;
}

// r_i = b_i - (A x)_i for one row of the column-sliced operator, by Dot2 (Ogita, Rump & Oishi):
// every product a_ij x_j is split exactly into p + e (two_product), the -p are summed into b_i by
// two_sum, and both rounding errors are accumulated and added once at the end. The result is as
// accurate as b_i - (A x)_i formed in twice the working precision and rounded once; the plain
// FP64 residual of a nearly converged x is wrong by up to u (|A||x|)_i, which for the thin
// basins' pressure operator is of the order of the residuals a solve aims for.
// abs_sum receives (|A||x|)_i (the FP64 floor). MASKC >= 0: component MASKC's symmetric
// Dirichlet elimination (identity row, zero column), as the solvers apply it.
template <int MASKC>
__device__ __forceinline__ double row_residual_dot2(const Geom& g, const double* __restrict__ val,
                                                    const double* x, double bi, int row, int col, int k,
                                                    double& abs_sum) {
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
    if (is_dirichlet(fl[0], k, nz, MASKC)) {
      const double xi = x[row];
      abs_sum = fabs(xi);
      return __dsub_rn(bi, xi);
    }
  }
  double s = bi, c = 0.0, asum = 0.0;
#pragma unroll
  for (int sl = 0; sl < NSLOT; ++sl) {
    const int q = slot_q(sl);
    const int kk = k + slot_dk(sl);
    bool ok = nb[q] >= 0;
    if (slot_dk(sl) < 0) ok = ok && kk >= 0;
    if (slot_dk(sl) > 0) ok = ok && kk < nz;
    if (MASKC >= 0) ok = ok && !is_dirichlet(fl[q], kk, nz, MASKC);
    const double av = ok ? __ldg(val + sl * npad + row) : 0.0;
    const double xv = x[ok ? nb[q] * nz + kk : row];
    double pe, se;
    const double p = two_product(av, xv, pe);
    s = two_sum(s, -p, se);
    c = __dadd_rn(c, __dsub_rn(se, pe));
    asum += fabs(p);
  }
  abs_sum = asum;
  return __dadd_rn(s, c);
}

// Operator value sets held per basin.
enum ValSet { VS_AU2 = 0, VS_AU1 = 1, VS_KI = 2, VS_M = 3, VS_G0 = 4, VS_G1 = 5, VS_G2 = 6, VS_COUNT = 7 };

// Scalars of one PCG solve, device-resident.
struct PcgScalars {
  double rho;        // (r, z) of the current iterate
  double pAp;
  double alpha, beta;
  double rr;         // ||r||^2 (recursive)
  double bb;         // ||b||^2 of the (projected) right-hand side
  double tol2;       // (rtol ||b||)^2
  double proj_c;     // pressure: m'z / 1'm of the current preconditioned residual
  double one_m;      // 1'm
  double lam;        // pressure: 1'b / 1'm
  double xshift;     // pressure: m'x0 / 1'm
  double aux[5];
  int32_t iter, max_iter, done, status;
  int32_t zero_rhs, pad0;
  uint32_t count[8]; // last-block counters of the grid reductions
};

constexpr int MAX_GRID = 152 * 8;
constexpr int NPART = 6;  // partial-sum lanes per reduction kernel

// ---- host-side bookkeeping -------------------------------------------------------------------
struct DevBuf {
  void* p = nullptr;
  size_t bytes = 0;
};

struct Ic0Factor {
  double* F = nullptr;     // [15][n] colour-ordered rows (row position = colour base + index)
  double shift = 0.0;
  bool ok = false;
};

struct SolveCtx;  // per-operator PCG workspace

}  // namespace pm

struct pm_operator {
  int32_t nx, ny, nz, ncols;
  int32_t slip_walls;
  int64_t n, npad;
  double dx, dy, nu[3], dt;
  std::vector<int32_t> col_i, col_j;
  std::vector<int32_t> cls_count;   // columns per parity class (i&1 | (j&1)<<1)
  int device;
  // device arrays
  int32_t* d_nbr = nullptr;
  double* d_depth = nullptr;
  uint8_t* d_cellmask = nullptr;
  uint8_t* d_colflag = nullptr;
  double* d_coriolis = nullptr;
  int32_t* d_cls_cols = nullptr;    // columns grouped by parity class, [ncols]
  uint16_t* d_struct = nullptr;     // structural slot bits per row
  uint16_t* d_keep[3] = {};         // per velocity component: bit s = slot s kept (neighbour present and
                                    // not in the component's Dirichlet set), bit 15 = Dirichlet row
  double* d_val[pm::VS_COUNT] = {};
  float* d_val32[pm::VS_COUNT] = {};
  uint16_t* d_val16[pm::VS_COUNT] = {};  // bf16 bit patterns
  double* d_m = nullptr;            // M 1
  float2* d_m2f = nullptr;          // M 1 split into two floats (mixed-precision kernels)
  double* d_dinv[8] = {};           // Jacobi inverse diagonals per (op, mask)
  float* d_dinv32[8] = {};
  pm::Ic0Factor ic0[8];
  double* d_line[8] = {};           // vertical-line factors per (op, mask): 3 x n, level-major
  bool line_ok[8] = {};
  float* d_line32[8] = {};          // FP32 copies for mixed-precision inner solves
  float* d_ic0_32[8] = {};
  pm::SolveCtx* ctx = nullptr;
  double one_m = 0.0;
  int64_t device_bytes = 0;
  int num_sms = 0;
};

struct pm_state {
  pm_operator* op;
  double* u[3];
  double* u_prev[3];
  double* p;
  double* q;
  double* ut[3];    // u~ (prediction)
  double* b[3];     // velocity right-hand sides
  double* bp;       // pressure right-hand side
  double* diag;     // diagnostics partials: PM_DIAG_COUNT lanes x MAX_GRID blocks, then the totals
  int32_t step;
};

namespace pm {

// error reporting (pm_api.cu)
int set_error(int status, const std::string& msg);
int cuda_check(cudaError_t e, const char* what);
void count_launch(int n = 1);

// geometry view
Geom geom_of(const pm_operator* op);

// pm_mesh.cu: host mesh build
struct HostMesh {
  int32_t nx, ny, nz, ncols;
  std::vector<int32_t> col_i, col_j;
  std::vector<int32_t> nbr;        // ncols * 7
  std::vector<double> depth;       // ncols
  std::vector<uint8_t> cellmask;   // ncols
  std::vector<uint8_t> colflag;    // ncols
  std::vector<double> coriolis;    // ncols
};
int build_host_mesh(const pm_mesh_desc* d, const double* coriolis, HostMesh* out);

// pm_assemble.cu
int launch_assemble(pm_operator* op, cudaStream_t s);
int launch_ic0_factor(pm_operator* op, int which, double shift, int* breakdown, cudaStream_t s);
int launch_dinv(pm_operator* op, int which, cudaStream_t s);
int launch_keep_masks(pm_operator* op, cudaStream_t s);

// pm_solve.cu
int spmv(pm_operator* op, int which, const double* x, double* y, cudaStream_t s);
int residual(pm_operator* op, int which, const double* b, const double* x, double* r, double* norms,
             cudaStream_t s);
int pcg_solve(pm_operator* op, int which, const double* b, double* x, const pm_solve_opts* o,
              pm_solve_stats* st, cudaStream_t s);
void destroy_ctx(pm_operator* op);

// pm_step.cu
int step_diagnostics(pm_operator* op, const pm_state* st, double* out, cudaStream_t s);
int project_step(pm_operator* op, pm_state* st, const double* th1, const double* th2,
                 const pm_solve_opts* vel, const pm_solve_opts* pres, int correction,
                 pm_solve_stats* stats, cudaStream_t s);

// which -> value set / mask component / solvable
inline int which_valset(int w) {
  switch (w) {
    case PM_OP_VEL_U1: case PM_OP_VEL_U2: case PM_OP_VEL_U3: return VS_AU2;
    case PM_OP_VEL1_U1: case PM_OP_VEL1_U2: case PM_OP_VEL1_U3: return VS_AU1;
    case PM_OP_PRESSURE: return VS_KI;
    case PM_OP_MASS: return VS_M;
    case PM_OP_GRAD_X: return VS_G0;
    case PM_OP_GRAD_Y: return VS_G1;
    case PM_OP_GRAD_Z: return VS_G2;
  }
  return -1;
}
inline int which_mask(int w) {
  switch (w) {
    case PM_OP_VEL_U1: case PM_OP_VEL1_U1: return 0;
    case PM_OP_VEL_U2: case PM_OP_VEL1_U2: return 1;
    case PM_OP_VEL_U3: case PM_OP_VEL1_U3: return 2;
  }
  return -1;
}
inline bool which_symmetric(int w) { return w >= 0 && w <= PM_OP_VEL1_U3; }

}  // namespace pm
