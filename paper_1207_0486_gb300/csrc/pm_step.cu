// The BDF2 velocity-correction projection step (Section 3) on the GPU:
//   k_rhs_vel     right-hand side of the velocity prediction (Eq. fofa_velo_pred_h), per row from
//                 the incident tets: history (1/dt) M (2 u^k - u^{k-1}/2) (BDF1: (1/dt) M u^k),
//                 advection - sum_d (d_d u_c)|_K (M^K u_d)_i, Coriolis +-f_i (M u)_i,
//                 pressure (G_c^T p^k)_i = sum_K |K|/4 d_c phi_i sum_{j in K} p_j, and the wind
//                 tension on Gamma_s with the surface P1 mass |F| (1 + d_ij)/12; Dirichlet rows 0
//   k_div_rhs     b_p = -alpha sum_c G_c u~_c (Eq. fofa_q_cor_h), the three G_c on one stencil
//   k_correct     u_c = u~_c - (G_c q)_i / (alpha m_i), lumped mass m = M 1
//                 (Eq. fofa_velo_cor_h), then the Dirichlet sets. The minus sign is the one
//                 Eq. correc_velo_u fixes, (3/(2 dt)) (u - u~) + grad q = 0, and the one from
//                 which Eq. press_cor follows; the "+" printed in Eq. fofa_velo_cor_h and at the
//                 end of Section 3 would add the gradient the correction exists to remove.
//   k_axpy        p^{k+1} = p^k + q (Eq. fofa_pres_cor_h: the L2 projection onto P_h is the
//                 identity for q, p^k in P_h)
#include <algorithm>
#include <chrono>
#include <cmath>

#include "pm_internal.cuh"

namespace pm {
namespace {

constexpr int TPB = 128;

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

struct StepIn {
  const double* u[3];
  const double* up[3];
  const double* p;
  const double* th[2];   // per column, may be null
  double* b[3];
  double inv_dt;
  int bdf1;
};

__global__ void __launch_bounds__(TPB) k_rhs_vel(Geom g, StepIn in) {
  const int nz = g.nz;
  const double dx = g.dx, dy = g.dy;
  const double nzm1 = (double)(nz - 1);
  for (int64_t row = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; row < g.n;
       row += (int64_t)gridDim.x * blockDim.x) {
    const int col = (int)(row / nz);
    const int k = (int)(row - (int64_t)col * nz);
    int nb[NNBR];
    double hq[NNBR];
#pragma unroll
    for (int q = 0; q < NNBR; ++q) {
      nb[q] = nbr_of(g, col, q);
      hq[q] = nb[q] >= 0 ? g.depth[nb[q]] : 0.0;
    }
    const uint8_t cm = g.cellmask[col];
    double hist[3] = {0, 0, 0}, adv[3] = {0, 0, 0}, mu[2] = {0, 0}, pr[3] = {0, 0, 0};
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
        double U[3][4], H[3][4], P[4];
#pragma unroll
        for (int w = 0; w < 4; ++w) {
          const int vc = vcorner(p, w);
          const int di = (vc & 1) - a, dj = ((vc >> 1) & 1) - b, dk = ((vc >> 2) & 1) - c;
          const int s = slot_of(di, dj, dk);
          const int64_t nrow = (int64_t)nb[slot_q(s)] * nz + k + dk;
          X[w][0] = di * dx;
          X[w][1] = dj * dy;
          X[w][2] = -hq[slot_q(s)] * (1.0 - (double)(k + dk) / nzm1);
#pragma unroll
          for (int cc = 0; cc < 3; ++cc) {
            const double uk = in.u[cc][nrow];
            U[cc][w] = uk;
            H[cc][w] = in.bdf1 ? uk : 2.0 * uk - 0.5 * in.up[cc][nrow];
          }
          P[w] = in.p[nrow];
        }
        double e[3][3];
#pragma unroll
        for (int r = 0; r < 3; ++r)
#pragma unroll
          for (int d = 0; d < 3; ++d) e[r][d] = X[r + 1][d] - X[0][d];
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
        // (M^K y)_v = vol/20 (y_v + sum_w y_w)
        double MU[3], MH[3], psum = 0.0;
#pragma unroll
        for (int cc = 0; cc < 3; ++cc) {
          double su = 0.0, sh = 0.0;
#pragma unroll
          for (int w = 0; w < 4; ++w) {
            su += U[cc][w];
            sh += H[cc][w];
          }
          MU[cc] = vol / 20.0 * (su + U[cc][v]);
          MH[cc] = vol / 20.0 * (sh + H[cc][v]);
        }
#pragma unroll
        for (int w = 0; w < 4; ++w) psum += P[w];
#pragma unroll
        for (int cc = 0; cc < 3; ++cc) {
          double gu[3];
#pragma unroll
          for (int d = 0; d < 3; ++d) {
            double t = 0.0;
#pragma unroll
            for (int w = 0; w < 4; ++w) t = fma(U[cc][w], gr[w][d], t);
            gu[d] = t;
          }
          hist[cc] += MH[cc];
          adv[cc] += gu[0] * MU[0] + gu[1] * MU[1] + gu[2] * MU[2];
          pr[cc] += vol / 4.0 * gr[v][cc] * psum;
        }
        mu[0] += MU[0];
        mu[1] += MU[1];
      }
    }
    const double f = g.coriolis ? g.coriolis[col] : 0.0;
    double bc[3];
#pragma unroll
    for (int cc = 0; cc < 3; ++cc) bc[cc] = in.inv_dt * hist[cc] - adv[cc] + pr[cc];
    bc[0] += f * mu[1];
    bc[1] -= f * mu[0];
    if (k == nz - 1) {
      // surface tension on the top triangles (each cell split along its (0,0)-(1,1) diagonal)
      const double area = 0.5 * dx * dy;
#pragma unroll
      for (int cc = 0; cc < 2; ++cc) {
        const double* th = in.th[cc];
        if (!th) continue;
        auto T = [&](int q) -> double { return th[nb[q]]; };
        const double t0 = th[col];
        double s = 0.0;
        // SW cell (i-1, j-1): node is corner 11; triangles (00,10,11) and (00,01,11)
        if (cm & 1) {
          const double t00 = T(6);
          // corner 10 of that cell is (i, j-1) -> q 4; corner 01 is (i-1, j) -> q 2
          s += 2 * t0 + t00 + T(4);
          s += 2 * t0 + t00 + T(2);
        }
        // SE cell (i, j-1): node is corner 01; triangle (00,01,11): 00 = (i, j-1) q4, 11 = (i+1, j) q1
        if (cm & 2) s += 2 * t0 + T(4) + T(1);
        // NW cell (i-1, j): node is corner 10; triangle (00,10,11): 00 = (i-1, j) q2, 11 = (i, j+1) q3
        if (cm & 4) s += 2 * t0 + T(2) + T(3);
        // NE cell (i, j): node is corner 00; triangles (00,10,11), (00,01,11): 11 = (i+1, j+1) q5
        if (cm & 8) {
          s += 2 * t0 + T(1) + T(5);
          s += 2 * t0 + T(3) + T(5);
        }
        bc[cc] += area / 12.0 * s;
      }
    }
    const uint8_t fl = g.colflag[col];
#pragma unroll
    for (int cc = 0; cc < 3; ++cc) in.b[cc][row] = is_dirichlet(fl, k, nz, cc) ? 0.0 : bc[cc];
  }
}

struct GradIn {
  const double* gv[3];  // G_c values, slot-major
  const double* u[3];
  double* out[3];
};

// b_p = -alpha sum_c G_c u~_c.
__global__ void __launch_bounds__(TPB) k_div_rhs(Geom g, GradIn in, double alpha, double* __restrict__ bp) {
  const int nz = g.nz;
  for (int64_t row = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; row < g.n;
       row += (int64_t)gridDim.x * blockDim.x) {
    const int col = (int)(row / nz);
    const int k = (int)(row - (int64_t)col * nz);
    int nb[NNBR];
#pragma unroll
    for (int q = 0; q < NNBR; ++q) nb[q] = q == 0 ? col : nbr_of(g, col, q);
    double s = 0.0;
#pragma unroll
    for (int sl = 0; sl < NSLOT; ++sl) {
      const int q = slot_q(sl);
      const int kk = k + slot_dk(sl);
      if (nb[q] < 0 || kk < 0 || kk >= nz) continue;
      const int64_t j = (int64_t)nb[q] * nz + kk;
#pragma unroll
      for (int c = 0; c < 3; ++c) s = fma(in.gv[c][(int64_t)sl * g.npad + row], in.u[c][j], s);
    }
    bp[row] = -alpha * s;
  }
}

// u_c = u~_c - (G_c q)_i / (alpha m_i) on non-Dirichlet rows, 0 on Dirichlet rows.
__global__ void __launch_bounds__(TPB) k_correct(Geom g, GradIn in, const double* __restrict__ q,
                                                 const double* __restrict__ m, double inv_alpha) {
  const int nz = g.nz;
  for (int64_t row = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; row < g.n;
       row += (int64_t)gridDim.x * blockDim.x) {
    const int col = (int)(row / nz);
    const int k = (int)(row - (int64_t)col * nz);
    int nb[NNBR];
#pragma unroll
    for (int qq = 0; qq < NNBR; ++qq) nb[qq] = qq == 0 ? col : nbr_of(g, col, qq);
    double s[3] = {0, 0, 0};
#pragma unroll
    for (int sl = 0; sl < NSLOT; ++sl) {
      const int qq = slot_q(sl);
      const int kk = k + slot_dk(sl);
      if (nb[qq] < 0 || kk < 0 || kk >= nz) continue;
      const double qj = q[(int64_t)nb[qq] * nz + kk];
#pragma unroll
      for (int c = 0; c < 3; ++c) s[c] = fma(in.gv[c][(int64_t)sl * g.npad + row], qj, s[c]);
    }
    const uint8_t fl = g.colflag[col];
    const double sc = inv_alpha / m[row];
#pragma unroll
    for (int c = 0; c < 3; ++c)
      in.out[c][row] = is_dirichlet(fl, k, nz, c) ? 0.0 : fma(-s[c], sc, in.u[c][row]);
  }
}

// Right-hand side of the consistent-mass correction: M u~_c - (G_c q) / alpha.
__global__ void __launch_bounds__(TPB) k_correct_rhs(Geom g, GradIn in, const double* __restrict__ mval,
                                                     const double* __restrict__ q, double inv_alpha) {
  const int nz = g.nz;
  for (int64_t row = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; row < g.n;
       row += (int64_t)gridDim.x * blockDim.x) {
    const int col = (int)(row / nz);
    const int k = (int)(row - (int64_t)col * nz);
    int nb[NNBR];
#pragma unroll
    for (int qq = 0; qq < NNBR; ++qq) nb[qq] = qq == 0 ? col : nbr_of(g, col, qq);
    double s[3] = {0, 0, 0}, mu[3] = {0, 0, 0};
#pragma unroll
    for (int sl = 0; sl < NSLOT; ++sl) {
      const int qq = slot_q(sl);
      const int kk = k + slot_dk(sl);
      if (nb[qq] < 0 || kk < 0 || kk >= nz) continue;
      const int64_t j = (int64_t)nb[qq] * nz + kk;
      const double qj = q[j];
      const double mv = mval[(int64_t)sl * g.npad + row];
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        s[c] = fma(in.gv[c][(int64_t)sl * g.npad + row], qj, s[c]);
        mu[c] = fma(mv, in.u[c][j], mu[c]);
      }
    }
#pragma unroll
    for (int c = 0; c < 3; ++c) in.out[c][row] = fma(-s[c], inv_alpha, mu[c]);
  }
}

__global__ void k_mask(Geom g, double* __restrict__ u, int c) {
  for (int64_t row = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; row < g.n;
       row += (int64_t)gridDim.x * blockDim.x) {
    const int col = (int)(row / g.nz);
    const int k = (int)(row - (int64_t)col * g.nz);
    if (is_dirichlet(g.colflag[col], k, g.nz, c)) u[row] = 0.0;
  }
}

__global__ void k_axpy(int64_t n, double a, const double* __restrict__ x, double* __restrict__ y) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    y[i] = fma(a, x[i], y[i]);
}

int grid_for(int64_t n, int threads, int sms) {
  int64_t gsz = (n + threads - 1) / threads;
  const int64_t cap = (int64_t)sms * 16;
  if (gsz > cap) gsz = cap;
  if (gsz < 1) gsz = 1;
  return (int)gsz;
}

// Diagnostics of a state, per row i: u_c,i (M u_c)_i for the kinetic energy, the discrete
// divergences (sum_c G_c u_c)_i of u^k and (sum_c G_c u~_c)_i of the last prediction, and m_i p_i.
// Each block writes its partial sums (lane-major, PM_DIAG_COUNT lanes); k_diag_total adds them in
// block order (deterministic).
__global__ void __launch_bounds__(TPB) k_diagnostics(Geom g, const double* __restrict__ mval,
                                                     const double* __restrict__ gv0, const double* __restrict__ gv1,
                                                     const double* __restrict__ gv2, StepIn u, StepIn ut,
                                                     const double* __restrict__ m, const double* __restrict__ p,
                                                     double* __restrict__ part) {
  const int nz = g.nz;
  double acc[PM_DIAG_COUNT] = {0.0, 0.0, 0.0, 0.0};
  const double* gv[3] = {gv0, gv1, gv2};
  for (int64_t row = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; row < g.n;
       row += (int64_t)gridDim.x * blockDim.x) {
    const int col = (int)(row / nz);
    const int k = (int)(row - (int64_t)col * nz);
    int nb[NNBR];
#pragma unroll
    for (int q = 0; q < NNBR; ++q) nb[q] = q == 0 ? col : nbr_of(g, col, q);
    double mu[3] = {0, 0, 0}, du = 0.0, dut = 0.0;
#pragma unroll
    for (int sl = 0; sl < NSLOT; ++sl) {
      const int q = slot_q(sl);
      const int kk = k + slot_dk(sl);
      if (nb[q] < 0 || kk < 0 || kk >= nz) continue;
      const int64_t j = (int64_t)nb[q] * nz + kk;
      const double mv = mval[(int64_t)sl * g.npad + row];
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        const double gcv = gv[c][(int64_t)sl * g.npad + row];
        mu[c] = fma(mv, u.u[c][j], mu[c]);
        du = fma(gcv, u.u[c][j], du);
        dut = fma(gcv, ut.u[c][j], dut);
      }
    }
    double e = 0.0;
#pragma unroll
    for (int c = 0; c < 3; ++c) e = fma(u.u[c][row], mu[c], e);
    acc[PM_DIAG_KINETIC_ENERGY] += 0.5 * e;
    acc[PM_DIAG_DIV_U] = fma(du, du, acc[PM_DIAG_DIV_U]);
    acc[PM_DIAG_DIV_UT] = fma(dut, dut, acc[PM_DIAG_DIV_UT]);
    acc[PM_DIAG_P_MEAN] = fma(m[row], p[row], acc[PM_DIAG_P_MEAN]);
  }
  __shared__ double sm[PM_DIAG_COUNT][TPB / 32];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
  for (int l = 0; l < PM_DIAG_COUNT; ++l) {
    double v = acc[l];
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    if (lane == 0) sm[l][wid] = v;
  }
  __syncthreads();
  if (threadIdx.x < PM_DIAG_COUNT) {
    double v = 0.0;
    for (int w = 0; w < TPB / 32; ++w) v += sm[threadIdx.x][w];
    part[(int64_t)threadIdx.x * MAX_GRID + blockIdx.x] = v;
  }
}

// One block: totals of the block partials, in block order; the two divergences as 2-norms and the
// mean pressure m'p / 1'm.
__global__ void k_diag_total(const double* __restrict__ part, int nblocks, double one_m, double* __restrict__ out) {
  if (threadIdx.x >= PM_DIAG_COUNT) return;
  double v = 0.0;
  for (int b = 0; b < nblocks; ++b) v += part[(int64_t)threadIdx.x * MAX_GRID + b];
  if (threadIdx.x == PM_DIAG_DIV_U || threadIdx.x == PM_DIAG_DIV_UT) v = sqrt(v);
  if (threadIdx.x == PM_DIAG_P_MEAN) v /= one_m;
  out[threadIdx.x] = v;
}

}  // namespace

int step_diagnostics(pm_operator* op, const pm_state* st, double* out, cudaStream_t s) {
  Geom g = geom_of(op);
  const int G = std::min(grid_for(op->n, TPB, op->num_sms), MAX_GRID);
  StepIn u, ut;
  for (int c = 0; c < 3; ++c) {
    u.u[c] = st->u[c];
    ut.u[c] = st->ut[c];
  }
  k_diagnostics<<<G, TPB, 0, s>>>(g, op->d_val[VS_M], op->d_val[VS_G0], op->d_val[VS_G1], op->d_val[VS_G2], u, ut,
                                  op->d_m, st->p, st->diag);
  double* tot = st->diag + (int64_t)PM_DIAG_COUNT * MAX_GRID;
  k_diag_total<<<1, 32, 0, s>>>(st->diag, G, op->one_m, tot);
  count_launch(2);
  int r = cuda_check(cudaMemcpyAsync(out, tot, PM_DIAG_COUNT * sizeof(double), cudaMemcpyDeviceToHost, s), "diagnostics");
  if (!r) r = cuda_check(cudaStreamSynchronize(s), "diagnostics");
  return r;
}

int project_step(pm_operator* op, pm_state* st, const double* th1, const double* th2,
                 const pm_solve_opts* vel, const pm_solve_opts* pres, int correction,
                 pm_solve_stats* stats, cudaStream_t s) {
  Geom g = geom_of(op);
  const int G = grid_for(op->n, TPB, op->num_sms);
  const bool bdf1 = st->step == 0;
  const double alpha = bdf1 ? 1.0 / op->dt : 1.5 / op->dt;
  StepIn in;
  for (int c = 0; c < 3; ++c) {
    in.u[c] = st->u[c];
    in.up[c] = st->u_prev[c];
    in.b[c] = st->b[c];
  }
  in.p = st->p;
  in.th[0] = th1;
  in.th[1] = th2;
  in.inv_dt = 1.0 / op->dt;
  in.bdf1 = bdf1 ? 1 : 0;
  {
    NvtxRange range("velocity right-hand sides");
    k_rhs_vel<<<G, TPB, 0, s>>>(g, in);
    count_launch();
  }
  int st_all = PM_OK;
  pm_solve_stats local[7];
  for (int i = 0; i < 7; ++i) local[i] = pm_solve_stats{};
  for (int c = 0; c < 3; ++c) {
    cudaMemcpyAsync(st->ut[c], st->u[c], op->n * sizeof(double), cudaMemcpyDeviceToDevice, s);
    pm_solve_opts o = *vel;
    o.x0_is_guess = 1;
    const int which = (bdf1 ? PM_OP_VEL1_U1 : PM_OP_VEL_U1) + c;
    const int r = pcg_solve(op, which, st->b[c], st->ut[c], &o, &local[c], s);
    if (r != PM_OK && st_all == PM_OK) st_all = r;
    if (r != PM_OK && r != PM_NOT_CONVERGED) return r;
  }
  GradIn gi;
  for (int c = 0; c < 3; ++c) {
    gi.gv[c] = op->d_val[VS_G0 + c];
    gi.u[c] = st->ut[c];
    gi.out[c] = st->u_prev[c];  // u^{k-1} is no longer needed: it receives u^{k+1}
  }
  {
    NvtxRange range("divergence right-hand side");
    k_div_rhs<<<G, TPB, 0, s>>>(g, gi, alpha, st->bp);
    count_launch();
  }
  {
    pm_solve_opts o = *pres;
    o.x0_is_guess = 1;
    const int r = pcg_solve(op, PM_OP_PRESSURE, st->bp, st->q, &o, &local[3], s);
    if (r != PM_OK && st_all == PM_OK) st_all = r;
    if (r != PM_OK && r != PM_NOT_CONVERGED) return r;
  }
  k_axpy<<<G, TPB, 0, s>>>(op->n, 1.0, st->q, st->p);
  count_launch();
  NvtxRange correction_range(correction == PM_STEP_CONSISTENT ? "consistent-mass correction" : "lumped correction");
  if (correction == PM_STEP_CONSISTENT) {
    // b[c] <- M u~_c - G_c q / alpha, then M u_c = b[c] by PCG with x0 = u~_c
    GradIn gr = gi;
    for (int c = 0; c < 3; ++c) gr.out[c] = st->b[c];
    k_correct_rhs<<<G, TPB, 0, s>>>(g, gr, op->d_val[VS_M], st->q, 1.0 / alpha);
    count_launch();
    for (int c = 0; c < 3; ++c) {
      cudaMemcpyAsync(st->u_prev[c], st->ut[c], op->n * sizeof(double), cudaMemcpyDeviceToDevice, s);
      pm_solve_opts o = *vel;
      o.x0_is_guess = 1;
      const int r = pcg_solve(op, PM_OP_MASS, st->b[c], st->u_prev[c], &o, &local[4 + c], s);
      if (r != PM_OK && st_all == PM_OK) st_all = r;
      if (r != PM_OK && r != PM_NOT_CONVERGED) return r;
      k_mask<<<G, TPB, 0, s>>>(g, st->u_prev[c], c);
      count_launch();
    }
  } else {
    k_correct<<<G, TPB, 0, s>>>(g, gi, st->q, op->d_m, 1.0 / alpha);
    count_launch();
  }
  for (int c = 0; c < 3; ++c) {
    double* t = st->u[c];
    st->u[c] = st->u_prev[c];
    st->u_prev[c] = t;
  }
  st->step += 1;
  if (stats)
    for (int i = 0; i < 7; ++i) stats[i] = local[i];
  int r = cuda_check(cudaStreamSynchronize(s), "project_step");
  if (r) return r;
  return st_all;
}

}  // namespace pm
