// C ABI entry points of libpm_gb300 (declared in include/pm.h): argument checks, operator and
// state lifetime, host<->device transfers; the numerical work is in pm_assemble.cu,
// pm_solve.cu and pm_step.cu.
#include <atomic>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "pm_internal.cuh"

namespace pm {

static thread_local std::string g_last_error;
static std::atomic<int64_t> g_launches{0};

int set_error(int status, const std::string& msg) {
  g_last_error = msg;
  return status;
}

int cuda_check(cudaError_t e, const char* what) {
  if (e == cudaSuccess) return PM_OK;
  g_last_error = std::string(what) + ": " + cudaGetErrorString(e);
  if (e == cudaErrorMemoryAllocation) return PM_ENOMEM;
  return PM_ECUDA;
}

void count_launch(int n) { g_launches.fetch_add(n, std::memory_order_relaxed); }

Geom geom_of(const pm_operator* op) {
  Geom g;
  g.ncols = op->ncols;
  g.nz = op->nz;
  g.n = op->n;
  g.npad = op->npad;
  g.dx = op->dx;
  g.dy = op->dy;
  g.nbr = op->d_nbr;
  g.depth = op->d_depth;
  g.cellmask = op->d_cellmask;
  g.colflag = op->d_colflag;
  g.coriolis = op->d_coriolis;
  return g;
}

static int64_t padded(int64_t n) { return (n + 31) / 32 * 32; }

template <typename T>
static int dalloc(pm_operator* op, T** p, size_t count) {
  const size_t bytes = count * sizeof(T);
  cudaError_t e = cudaMalloc((void**)p, bytes > 0 ? bytes : 1);
  if (e != cudaSuccess) return cuda_check(e, "cudaMalloc");
  op->device_bytes += (int64_t)bytes;
  return PM_OK;
}

static void free_operator(pm_operator* op) {
  if (!op) return;
  destroy_ctx(op);
  cudaFree(op->d_nbr);
  cudaFree(op->d_depth);
  cudaFree(op->d_cellmask);
  cudaFree(op->d_colflag);
  cudaFree(op->d_coriolis);
  cudaFree(op->d_cls_cols);
  cudaFree(op->d_struct);
  cudaFree(op->d_m2f);
  for (int c = 0; c < 3; ++c) cudaFree(op->d_keep[c]);
  cudaFree(op->d_m);
  for (int v = 0; v < VS_COUNT; ++v) {
    cudaFree(op->d_val[v]);
    cudaFree(op->d_val32[v]);
    cudaFree(op->d_val16[v]);
  }
  for (int w = 0; w < 8; ++w) {
    cudaFree(op->d_dinv[w]);
    cudaFree(op->d_dinv32[w]);
    cudaFree(op->ic0[w].F);
    cudaFree(op->d_line[w]);
    cudaFree(op->d_line32[w]);
    cudaFree(op->d_ic0_32[w]);
  }
  delete op;
}

}  // namespace pm

using namespace pm;

extern "C" {

const char* pm_status_string(int s) {
  switch (s) {
    case PM_OK: return "ok";
    case PM_EINVAL: return "invalid argument";
    case PM_ENOMEM: return "out of memory";
    case PM_ECUDA: return "CUDA error";
    case PM_NOT_CONVERGED: return "not converged";
    case PM_BREAKDOWN: return "breakdown";
    case PM_TIMEOUT: return "device wait timed out";
    case PM_DISCONNECTED: return "ocean is not connected";
    case PM_EBUSY: return "no free server slot";
    case PM_EBOUNDS: return "bad index caught by a checked build";
  }
  return "unknown status";
}

int pm_last_error(char* buf, int32_t len) {
  const int n = (int)g_last_error.size();
  if (buf && len > 0) {
    const int m = n < len - 1 ? n : len - 1;
    std::memcpy(buf, g_last_error.data(), (size_t)m);
    buf[m] = 0;
  }
  return n;
}

int64_t pm_kernel_launch_count(void) { return g_launches.load(); }

int64_t pm_operator_bytes(const pm_mesh_desc* d) {
  if (!d || d->nx < 2 || d->ny < 2 || d->nz < 2) return -1;
  // ocean columns: corners of ocean cells
  int64_t ncols = 0;
  const int nx = d->nx, ny = d->ny;
  auto ocean = [&](int i, int j) { return d->ocean_mask ? d->ocean_mask[(size_t)j * nx + i] != 0 : true; };
  auto cell = [&](int ci, int cj) {
    if (ci < 0 || cj < 0 || ci >= nx - 1 || cj >= ny - 1) return false;
    return ocean(ci, cj) && ocean(ci + 1, cj) && ocean(ci, cj + 1) && ocean(ci + 1, cj + 1);
  };
  for (int j = 0; j < ny; ++j)
    for (int i = 0; i < nx; ++i)
      if (cell(i - 1, j - 1) || cell(i, j - 1) || cell(i - 1, j) || cell(i, j)) ++ncols;
  const int64_t n = ncols * d->nz, np = padded(n);
  int64_t b = 0;
  b += (int64_t)VS_COUNT * NSLOT * np * 8;     // FP64 operators
  b += 3 * (int64_t)NSLOT * np * 4;            // FP32 copies of the solved operators (mixed precision)
  b += 3 * (int64_t)NSLOT * n * 8;             // IC0 factors of the three BDF2 velocity systems
  b += 4 * n * 12;                             // Jacobi diagonals
  b += n * (8 + 2 + 3 * 2) + ncols * (7 * 4 + 8 + 8 + 2 + 16);   // m, structure, keep masks; columns
  b += 5 * n * 8 + (int64_t)NPART * MAX_GRID * 8;   // PCG workspace
  return b;
}

int pm_assemble_operator(const pm_mesh_desc* mesh, const pm_physics* phys, pm_operator** out,
                         pm_stream stream) {
  if (!mesh || !phys || !out) return set_error(PM_EINVAL, "null argument");
  NvtxRange range("pm_assemble_operator");
  *out = nullptr;
  if (!(phys->dt > 0.0)) return set_error(PM_EINVAL, "dt must be > 0");
  for (int d = 0; d < 3; ++d)
    if (!(phys->nu[d] >= 0.0)) return set_error(PM_EINVAL, "nu must be >= 0");
  HostMesh hm;
  int st = build_host_mesh(mesh, phys->coriolis, &hm);
  if (st) return st;
  cudaStream_t s = (cudaStream_t)stream;
  pm_operator* op = new pm_operator();
  op->nx = mesh->nx;
  op->ny = mesh->ny;
  op->nz = mesh->nz;
  op->ncols = hm.ncols;
  op->slip_walls = mesh->slip_walls;
  op->n = (int64_t)hm.ncols * mesh->nz;
  op->npad = padded(op->n);
  op->dx = mesh->dx;
  op->dy = mesh->dy;
  for (int d = 0; d < 3; ++d) op->nu[d] = phys->nu[d];
  op->dt = phys->dt;
  op->col_i = hm.col_i;
  op->col_j = hm.col_j;
  cudaGetDevice(&op->device);
  cudaDeviceGetAttribute(&op->num_sms, cudaDevAttrMultiProcessorCount, op->device);
  if (op->num_sms <= 0) op->num_sms = 1;
  // parity classes of columns: cls = (i & 1) | (j & 1) << 1, columns listed class by class
  op->cls_count.assign(4, 0);
  std::vector<int32_t> cls_cols, clsidx(hm.ncols);
  for (int cls = 0; cls < 4; ++cls)
    for (int c = 0; c < hm.ncols; ++c)
      if (((hm.col_i[c] & 1) | ((hm.col_j[c] & 1) << 1)) == cls) {
        clsidx[c] = op->cls_count[cls]++;
        cls_cols.push_back(c);
      }
  const int nc = hm.ncols;
  std::vector<int32_t> packed;
  packed.reserve((size_t)4 * nc);
  packed.insert(packed.end(), cls_cols.begin(), cls_cols.end());
  packed.insert(packed.end(), clsidx.begin(), clsidx.end());
  packed.insert(packed.end(), hm.col_i.begin(), hm.col_i.end());
  packed.insert(packed.end(), hm.col_j.begin(), hm.col_j.end());
#define PM_TRY(x)           \
  do {                      \
    int _e = (x);           \
    if (_e) {               \
      free_operator(op);    \
      return _e;            \
    }                       \
  } while (0)
  PM_TRY(dalloc(op, &op->d_nbr, (size_t)nc * NNBR));
  PM_TRY(dalloc(op, &op->d_depth, (size_t)nc));
  PM_TRY(dalloc(op, &op->d_cellmask, (size_t)nc));
  PM_TRY(dalloc(op, &op->d_colflag, (size_t)nc));
  PM_TRY(dalloc(op, &op->d_coriolis, (size_t)nc));
  PM_TRY(dalloc(op, &op->d_cls_cols, (size_t)4 * nc));
  PM_TRY(dalloc(op, &op->d_struct, (size_t)op->n));
  PM_TRY(dalloc(op, &op->d_m, (size_t)op->n));
  for (int v = 0; v < VS_COUNT; ++v) PM_TRY(dalloc(op, &op->d_val[v], (size_t)NSLOT * op->npad));
  PM_TRY(cuda_check(cudaMemcpyAsync(op->d_nbr, hm.nbr.data(), hm.nbr.size() * 4, cudaMemcpyHostToDevice, s), "upload"));
  PM_TRY(cuda_check(cudaMemcpyAsync(op->d_depth, hm.depth.data(), nc * 8, cudaMemcpyHostToDevice, s), "upload"));
  PM_TRY(cuda_check(cudaMemcpyAsync(op->d_cellmask, hm.cellmask.data(), nc, cudaMemcpyHostToDevice, s), "upload"));
  PM_TRY(cuda_check(cudaMemcpyAsync(op->d_colflag, hm.colflag.data(), nc, cudaMemcpyHostToDevice, s), "upload"));
  PM_TRY(cuda_check(cudaMemcpyAsync(op->d_coriolis, hm.coriolis.data(), nc * 8, cudaMemcpyHostToDevice, s), "upload"));
  PM_TRY(cuda_check(cudaMemcpyAsync(op->d_cls_cols, packed.data(), packed.size() * 4, cudaMemcpyHostToDevice, s), "upload"));
  // padding rows of the value arrays stay zero
  for (int v = 0; v < VS_COUNT; ++v)
    PM_TRY(cuda_check(cudaMemsetAsync(op->d_val[v], 0, (size_t)NSLOT * op->npad * 8, s), "memset"));
  PM_TRY(launch_assemble(op, s));
  PM_TRY(bounds_status("pm_assemble_operator"));
#undef PM_TRY
  *out = op;
  return PM_OK;
}

int pm_operator_info_get(const pm_operator* op, pm_operator_info* info) {
  if (!op || !info) return set_error(PM_EINVAL, "null argument");
  info->n = op->n;
  info->n_pad = op->npad;
  info->ncols = op->ncols;
  info->nz = op->nz;
  info->nx = op->nx;
  info->ny = op->ny;
  info->device_bytes = op->device_bytes;
  return PM_OK;
}

int pm_operator_columns(const pm_operator* op, int32_t* col_i, int32_t* col_j) {
  if (!op) return set_error(PM_EINVAL, "null operator");
  if (col_i) std::memcpy(col_i, op->col_i.data(), op->col_i.size() * 4);
  if (col_j) std::memcpy(col_j, op->col_j.data(), op->col_j.size() * 4);
  return PM_OK;
}

int pm_operator_export(const pm_operator* op, pm_which which, double* values, int32_t* nbr,
                       uint16_t* structure) {
  if (!op) return set_error(PM_EINVAL, "null operator");
  const int vs = which_valset(which);
  if (vs < 0) return set_error(PM_EINVAL, "unknown operator");
  int st = cuda_check(cudaDeviceSynchronize(), "export sync");
  if (st) return st;
  std::vector<int32_t> hn((size_t)op->ncols * NNBR);
  st = cuda_check(cudaMemcpy(hn.data(), op->d_nbr, hn.size() * 4, cudaMemcpyDeviceToHost), "export");
  if (st) return st;
  if (nbr) std::memcpy(nbr, hn.data(), hn.size() * 4);
  if (structure) {
    st = cuda_check(cudaMemcpy(structure, op->d_struct, op->n * 2, cudaMemcpyDeviceToHost), "export");
    if (st) return st;
  }
  if (values) {
    std::vector<double> hv((size_t)NSLOT * op->npad);
    st = cuda_check(cudaMemcpy(hv.data(), op->d_val[vs], hv.size() * 8, cudaMemcpyDeviceToHost), "export");
    if (st) return st;
    std::vector<uint8_t> fl(op->ncols);
    st = cuda_check(cudaMemcpy(fl.data(), op->d_colflag, op->ncols, cudaMemcpyDeviceToHost), "export");
    if (st) return st;
    const int mc = which_mask(which);
    const int nz = op->nz;
    for (int64_t row = 0; row < op->n; ++row) {
      const int col = (int)(row / nz), k = (int)(row % nz);
      const bool dr = mc >= 0 && is_dirichlet(fl[col], k, nz, mc);
      for (int s = 0; s < NSLOT; ++s) {
        double v = hv[(size_t)s * op->npad + row];
        if (mc >= 0) {
          const int q = slot_q(s), kk = k + slot_dk(s);
          const int nb = hn[(size_t)col * NNBR + q];
          bool dc = false;
          if (nb >= 0 && kk >= 0 && kk < nz) dc = is_dirichlet(fl[nb], kk, nz, mc);
          if (dr || dc) v = (s == DIAG_SLOT && dr) ? 1.0 : 0.0;
        }
        values[(size_t)s * op->n + row] = v;
      }
    }
  }
  return PM_OK;
}

int pm_spmv(pm_operator* op, pm_which which, const double* x, double* y, pm_stream stream) {
  if (!op || !x || !y) return set_error(PM_EINVAL, "null argument");
  return spmv(op, (int)which, x, y, (cudaStream_t)stream);
}

int pm_residual(pm_operator* op, pm_which which, const double* b, const double* x, double* r, double* norms,
                pm_stream stream) {
  if (!op || !b || !x || !r) return set_error(PM_EINVAL, "null argument");
  const int st = residual(op, (int)which, b, x, r, norms, (cudaStream_t)stream);
  const int bs = bounds_status("pm_residual");
  return bs ? bs : st;
}

int pm_pcg_solve(pm_operator* op, pm_which which, const double* b, double* x,
                 const pm_solve_opts* opts, pm_solve_stats* stats, pm_stream stream) {
  if (!op || !b || !x || !opts) return set_error(PM_EINVAL, "null argument");
  pm_solve_stats local = {};
  int r = pcg_solve(op, (int)which, b, x, opts, &local, (cudaStream_t)stream);
  const int bs = bounds_status("pm_pcg_solve");
  if (bs) r = bs;
  if (stats) *stats = local;
  if (log_enabled() && r != PM_EINVAL) log_solve("pcg_solve", op, (int)which, opts->prec, opts->precision, local);
  return r;
}

int pm_state_create(pm_operator* op, pm_state** out) {
  if (!op || !out) return set_error(PM_EINVAL, "null argument");
  *out = nullptr;
  pm_state* st = new pm_state();
  std::memset(st, 0, sizeof(pm_state));
  st->op = op;
  double** fields[] = {&st->u[0], &st->u[1], &st->u[2], &st->u_prev[0], &st->u_prev[1], &st->u_prev[2],
                       &st->p, &st->q, &st->ut[0], &st->ut[1], &st->ut[2], &st->b[0], &st->b[1],
                       &st->b[2], &st->bp};
  for (double** f : fields) {
    cudaError_t e = cudaMalloc((void**)f, op->n * sizeof(double));
    if (e == cudaSuccess) e = cudaMemset(*f, 0, op->n * sizeof(double));
    if (e != cudaSuccess) {
      pm_state_destroy(st);
      return cuda_check(e, "state allocation");
    }
  }
  cudaError_t e = cudaMalloc((void**)&st->diag, ((size_t)PM_DIAG_COUNT * MAX_GRID + PM_DIAG_COUNT) * sizeof(double));
  if (e != cudaSuccess) {
    pm_state_destroy(st);
    return cuda_check(e, "state allocation");
  }
  *out = st;
  return PM_OK;
}

int pm_state_get(const pm_state* st, double* u1, double* u2, double* u3, double* p, pm_stream stream) {
  if (!st) return set_error(PM_EINVAL, "null state");
  cudaStream_t s = (cudaStream_t)stream;
  const size_t b = st->op->n * sizeof(double);
  double* outs[4] = {u1, u2, u3, p};
  const double* ins[4] = {st->u[0], st->u[1], st->u[2], st->p};
  for (int i = 0; i < 4; ++i)
    if (outs[i]) {
      int r = cuda_check(cudaMemcpyAsync(outs[i], ins[i], b, cudaMemcpyDeviceToDevice, s), "state get");
      if (r) return r;
    }
  return PM_OK;
}

int pm_state_field(const pm_state* st, int32_t field, double* dst, pm_stream stream) {
  if (!st || !dst) return set_error(PM_EINVAL, "null argument");
  const double* src = nullptr;
  switch (field) {
    case PM_FIELD_U1: case PM_FIELD_U2: case PM_FIELD_U3: src = st->u[field - PM_FIELD_U1]; break;
    case PM_FIELD_U1_PREV: case PM_FIELD_U2_PREV: case PM_FIELD_U3_PREV: src = st->u_prev[field - PM_FIELD_U1_PREV]; break;
    case PM_FIELD_P: src = st->p; break;
    case PM_FIELD_Q: src = st->q; break;
    case PM_FIELD_UT1: case PM_FIELD_UT2: case PM_FIELD_UT3: src = st->ut[field - PM_FIELD_UT1]; break;
    case PM_FIELD_BP: src = st->bp; break;
    default: return set_error(PM_EINVAL, "unknown state field");
  }
  return cuda_check(cudaMemcpyAsync(dst, src, st->op->n * sizeof(double), cudaMemcpyDeviceToDevice,
                                    (cudaStream_t)stream), "state field");
}

int pm_state_set_field(pm_state* st, int32_t field, const double* src, pm_stream stream) {
  if (!st || !src) return set_error(PM_EINVAL, "null argument");
  double* dst = nullptr;
  switch (field) {
    case PM_FIELD_U1: case PM_FIELD_U2: case PM_FIELD_U3: dst = st->u[field - PM_FIELD_U1]; break;
    case PM_FIELD_U1_PREV: case PM_FIELD_U2_PREV: case PM_FIELD_U3_PREV: dst = st->u_prev[field - PM_FIELD_U1_PREV]; break;
    case PM_FIELD_P: dst = st->p; break;
    case PM_FIELD_Q: dst = st->q; break;
    default: return set_error(PM_EINVAL, "only u^k, u^{k-1}, p and q can be set");
  }
  return cuda_check(cudaMemcpyAsync(dst, src, st->op->n * sizeof(double), cudaMemcpyDeviceToDevice,
                                    (cudaStream_t)stream), "state set field");
}

int pm_state_set_step_index(pm_state* st, int32_t step_index) {
  if (!st || step_index < 0) return set_error(PM_EINVAL, "bad argument");
  st->step = step_index;
  return PM_OK;
}

int pm_state_diagnostics(pm_operator* op, const pm_state* st, double* out, pm_stream stream) {
  if (!op || !st || !out || st->op != op) return set_error(PM_EINVAL, "bad argument");
  return step_diagnostics(op, st, out, (cudaStream_t)stream);
}

int pm_state_set(pm_state* st, const double* u1, const double* u2, const double* u3, const double* p,
                 int32_t step_index, pm_stream stream) {
  if (!st || step_index < 0) return set_error(PM_EINVAL, "bad argument");
  cudaStream_t s = (cudaStream_t)stream;
  const size_t b = st->op->n * sizeof(double);
  const double* ins[4] = {u1, u2, u3, p};
  double* outs[4] = {st->u[0], st->u[1], st->u[2], st->p};
  for (int i = 0; i < 4; ++i) {
    int r = ins[i] ? cuda_check(cudaMemcpyAsync(outs[i], ins[i], b, cudaMemcpyDeviceToDevice, s), "state set")
                   : cuda_check(cudaMemsetAsync(outs[i], 0, b, s), "state set");
    if (r) return r;
    if (i < 3) {
      r = cuda_check(cudaMemcpyAsync(st->u_prev[i], outs[i], b, cudaMemcpyDeviceToDevice, s), "state set");
      if (r) return r;
    }
  }
  int r = cuda_check(cudaMemsetAsync(st->q, 0, b, s), "state set");
  if (r) return r;
  st->step = step_index;
  return PM_OK;
}

int32_t pm_state_step_index(const pm_state* st) { return st ? st->step : -1; }

int pm_project_step(pm_operator* op, pm_state* st, const double* theta1, const double* theta2,
                    const pm_solve_opts* vel, const pm_solve_opts* pres, int32_t correction,
                    pm_solve_stats* stats, pm_stream stream) {
  if (!op || !st || !vel || !pres || st->op != op) return set_error(PM_EINVAL, "bad argument");
  if (correction != PM_STEP_LUMPED && correction != PM_STEP_CONSISTENT)
    return set_error(PM_EINVAL, "unknown correction");
  NvtxRange range("pm_project_step");
  const int first = st->step == 0 ? PM_OP_VEL1_U1 : PM_OP_VEL_U1;
  pm_solve_stats local[7] = {};
  int r = project_step(op, st, theta1, theta2, vel, pres, correction, local, (cudaStream_t)stream);
  const int bs = bounds_status("pm_project_step");
  if (bs) r = bs;
  if (stats)
    for (int i = 0; i < 7; ++i) stats[i] = local[i];
  if (log_enabled() && r != PM_EINVAL)
    for (int i = 0; i < (correction == PM_STEP_CONSISTENT ? 7 : 4); ++i) {
      const pm_solve_opts& o = i == 3 ? *pres : *vel;
      const int w = i < 3 ? first + i : i == 3 ? PM_OP_PRESSURE : PM_OP_MASS;
      log_solve("project_step", op, w, o.prec, o.precision, local[i]);
    }
  return r;
}

void pm_operator_destroy(pm_operator* op) { free_operator(op); }

void pm_state_destroy(pm_state* st) {
  if (!st) return;
  double* fields[] = {st->u[0], st->u[1], st->u[2], st->u_prev[0], st->u_prev[1], st->u_prev[2],
                      st->p, st->q, st->ut[0], st->ut[1], st->ut[2], st->b[0], st->b[1], st->b[2], st->bp};
  for (double* f : fields) cudaFree(f);
  cudaFree(st->diag);
  delete st;
}

}  // extern "C"
