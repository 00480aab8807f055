// Tracing and checking around the solver: the per-solve JSON log (pm_set_log), the registry of
// the checked build's device index records (PM_CHECKED) and the build flags query.
#include <cmath>
#include <cstdio>
#include <mutex>
#include <string>
#include <vector>

#include "pm_internal.cuh"

namespace pm {
namespace {

std::mutex g_log_mu;
FILE* g_log = nullptr;
double g_log_peak = 0.0;

std::vector<BoundsReader>& readers() {
  static std::vector<BoundsReader> r;
  return r;
}

// JSON has no inf / nan: such values are written as null.
std::string num(double v) {
  if (!std::isfinite(v)) return "null";
  char b[32];
  std::snprintf(b, sizeof b, "%.6g", v);
  return b;
}

}  // namespace

const char* which_name(int w) {
  switch (w) {
    case PM_OP_VEL_U1: return "velocity_u1";
    case PM_OP_VEL_U2: return "velocity_u2";
    case PM_OP_VEL_U3: return "velocity_u3";
    case PM_OP_PRESSURE: return "pressure";
    case PM_OP_MASS: return "mass";
    case PM_OP_VEL1_U1: return "velocity_bdf1_u1";
    case PM_OP_VEL1_U2: return "velocity_bdf1_u2";
    case PM_OP_VEL1_U3: return "velocity_bdf1_u3";
  }
  return "other";
}

const char* prec_name(int p) {
  switch (p) {
    case PM_PREC_JACOBI: return "jacobi";
    case PM_PREC_IC0: return "ic0";
    case PM_PREC_NONE: return "none";
    case PM_PREC_LINE: return "line";
  }
  return "other";
}

const char* precision_name(int p) {
  switch (p) {
    case PM_FP64: return "fp64";
    case PM_FP32_REFINE: return "fp32_refine";
    case PM_BF16_REFINE: return "bf16_refine";
  }
  return "other";
}

void register_bounds_reader(BoundsReader r) { readers().push_back(r); }

int bounds_status(const char* where) {
  if (readers().empty()) return PM_OK;
  cudaDeviceSynchronize();
  for (BoundsReader r : readers()) {
    BoundsRecord rec = {0, 0, 0, 0};
    if (r(&rec))
      return set_error(PM_EBOUNDS, std::string(where) + ": a checked kernel read a bad neighbour index " +
                                       std::to_string(rec.value) + " (limit " + std::to_string(rec.limit) + ")");
  }
  return PM_OK;
}

bool log_enabled() { return g_log != nullptr; }

void log_solve(const char* event, const pm_operator* op, int which, int prec, int precision,
               const pm_solve_stats& st) {
  std::lock_guard<std::mutex> lock(g_log_mu);
  if (!g_log) return;
  const double gbs = st.seconds > 0.0 ? st.bytes_moved / st.seconds * 1e-9 : 0.0;
  std::string js = std::string("{\"event\":\"") + event + "\",\"rows\":" + std::to_string(op ? op->n : 0) +
                   ",\"system\":\"" + which_name(which) + "\",\"preconditioner\":\"" + prec_name(prec) +
                   "\",\"precision\":\"" + precision_name(precision) + "\",\"status\":\"" +
                   pm_status_string(st.status) + "\",\"iters\":" + std::to_string(st.iters) +
                   ",\"outer_iters\":" + std::to_string(st.outer_iters) +
                   ",\"first_pass_iters\":" + std::to_string(st.first_pass_iters) +
                   ",\"rel_residual_true\":" + num(st.rel_residual_true) +
                   ",\"rel_residual_floor\":" + num(st.rel_residual_floor) + ",\"seconds\":" + num(st.seconds) +
                   ",\"bytes_moved\":" + num(st.bytes_moved) + ",\"gbs\":" + num(gbs);
  if (g_log_peak > 0.0) js += ",\"pct_of_peak\":" + num(100.0 * gbs / g_log_peak);
  js += "}\n";
  std::fputs(js.c_str(), g_log);
  std::fflush(g_log);
}

}  // namespace pm

extern "C" int pm_set_log(const char* path, double hbm_peak_gbs) {
  using namespace pm;
  std::lock_guard<std::mutex> lock(g_log_mu);
  if (g_log) std::fclose(g_log);
  g_log = nullptr;
  g_log_peak = 0.0;
  if (!path) return PM_OK;
  g_log = std::fopen(path, "a");
  if (!g_log) return set_error(PM_EINVAL, std::string("cannot open log file '") + path + "'");
  g_log_peak = hbm_peak_gbs > 0.0 ? hbm_peak_gbs : 0.0;
  return PM_OK;
}

extern "C" int32_t pm_build_flags(void) {
#ifdef PM_CHECKED
  return PM_BUILD_CHECKED;
#else
  return 0;
#endif
}
