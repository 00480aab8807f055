/* pm.h -- C ABI of the GB300 projection-method FEM solver library (libpm_gb300.so).
 *
 * The library implements the per-time-step linear algebra of a BDF2 velocity-correction
 * projection method for the anisotropic Navier-Stokes equations in a thin layered basin
 * (Besson & Straubhaar, "Wind driven 3D Navier-Stokes circulation in the Atlantic"):
 *   - P1 finite element operators on a layered (sigma) grid whose hexes are split into six
 *     Kuhn tetrahedra (Section 5, Eqs. fofa_velo_pred_h .. fofa_velo_cor_h);
 *   - preconditioned conjugate gradient solves of the velocity prediction and pressure
 *     increment systems (Section 5 remark, items 1-3);
 *   - the projection step itself (Section 3, Eqs. pred_velo .. press_cor_cl).
 *
 * Conventions shared by every entry point:
 *   - Status: every int-returning call returns a PM_* status code; nothing throws or exits.
 *     pm_last_error() gives a one-line message for the calling thread's last failure.
 *   - Node order: ocean columns in row-major (j, i) order of the grid, and node id =
 *     column * nz + k, k = 0 at the sea floor and k = nz-1 at the surface. pm_operator_columns()
 *     returns the (i, j) of each column.
 *   - Device vectors: caller-owned device pointers to contiguous FP64 arrays of length n (or
 *     ncols for per-column surface fields) in that node order. The library never frees them.
 *   - Streams: all GPU work of a call is enqueued on the given stream (a cudaStream_t; NULL =
 *     legacy default stream). Calls that report convergence (pm_pcg_solve, pm_project_step,
 *     pm_pcg_solve_batched, pm_batch_solve, pm_server_run) synchronise that stream before
 *     returning; pm_spmv and the kernels-only calls are asynchronous.
 *   - Handles (pm_operator, pm_state, pm_batch, pm_server) are owned by the library and released
 *     by their destroy call. One handle must not be used from two host threads at once; different
 *     handles may be.
 */
#ifndef PM_GB300_H
#define PM_GB300_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct CUstream_st* pm_stream; /* identical to cudaStream_t */
typedef struct pm_operator pm_operator;
typedef struct pm_state pm_state;
typedef struct pm_batch pm_batch;
typedef struct pm_server pm_server;

/* ---- status codes ------------------------------------------------------------------------ */
enum {
  PM_OK = 0,
  PM_EINVAL = 1,        /* bad size, null pointer, depth <= 0, empty basin, unknown enum     */
  PM_ENOMEM = 2,        /* device or host allocation failed                                   */
  PM_ECUDA = 3,         /* a CUDA runtime call failed (message in pm_last_error)              */
  PM_NOT_CONVERGED = 4, /* iteration cap reached; x holds the last iterate, stats are filled   */
  PM_BREAKDOWN = 5,     /* (p, Ap) <= 0 or non-finite, or IC0 pivot failure after 11 shifts    */
  PM_TIMEOUT = 6,       /* a bounded device-side wait ran out (persistent kernels)            */
  PM_DISCONNECTED = 7,  /* the ocean has more than one connected component                    */
  PM_EBUSY = 8,         /* no free server slot; retry after a pm_server_poll frees one         */
  PM_EBOUNDS = 9        /* checked build only: a kernel read a bad neighbour index (skipped)   */
};

/* Lateral outer walls that are artificial slip boundaries Gamma_1 (Section 2, Eq. prim_bot_1:
 * u.n = 0 and zero tangential stress). Outer walls not listed, and coastlines, belong to
 * Gamma_0 (u = 0, Eq. prim_bot_0), as does the sea floor. */
enum { PM_WALL_WEST = 1, PM_WALL_EAST = 2, PM_WALL_SOUTH = 4, PM_WALL_NORTH = 8 };

/* Basin geometry (Section 2: Omega = {(x1,x2) in Gamma_s, -h(x1,x2) < x3 < 0}).
 * Grid nodes sit at x = i dx, y = j dy, z_k = -depth[j,i] (1 - k/(nz-1)). A hex cell is ocean
 * when its four corner columns are ocean; columns that touch no ocean cell are dropped.
 * ocean_mask, depth: host arrays [ny][nx] (row-major, index j*nx + i); read during the call only.
 * ocean_mask may be NULL (all ocean); depth must be > 0 on every kept column. */
typedef struct pm_mesh_desc {
  int32_t nx, ny, nz;        /* nodes per axis, each >= 2                                   */
  int32_t slip_walls;        /* PM_WALL_* bits                                              */
  double dx, dy;             /* horizontal node spacing (> 0)                               */
  const uint8_t* ocean_mask; /* host [ny][nx], 1 = ocean column, or NULL                    */
  const double* depth;       /* host [ny][nx], h > 0                                        */
} pm_mesh_desc;

/* Physics of Sections 2-3: Delta_nu = sum_j nu_j d^2/dx_j^2, time step dt, Coriolis parameter
 * f = 2 omega_3 per grid column (host [ny][nx], NULL = 0). */
typedef struct pm_physics {
  double nu[3];
  double dt;
  const double* coriolis;
} pm_physics;

/* Operators stored for a basin.
 * VEL_Uc  : 3/(2 dt) M + K_nu with component c's homogeneous Dirichlet set eliminated
 *           symmetrically (BDF2 prediction, Eq. fofa_velo_pred_h). Dirichlet sets: c = 1:
 *           Gamma_0 + x-normal Gamma_1; c = 2: Gamma_0 + y-normal Gamma_1; c = 3: Gamma_0 +
 *           Gamma_s (Eqs. pred_cl_0, pred_cl_1_u, pred_tr_3).
 * VEL1_Uc : 1/dt M + K_nu, same sets (BDF1 start step).
 * PRESSURE: K_I, the pure-Neumann Laplacian (Eq. fofa_q_cor_h). Solves impose zero mean.
 * MASS    : consistent P1 mass M (Eq. fofa_velo_cor_h).
 * GRAD_c  : G_c,ij = integral of (d phi_j / dx_c) phi_i (not symmetric; pm_spmv only).      */
typedef enum pm_which {
  PM_OP_VEL_U1 = 0, PM_OP_VEL_U2 = 1, PM_OP_VEL_U3 = 2,
  PM_OP_PRESSURE = 3, PM_OP_MASS = 4,
  PM_OP_VEL1_U1 = 5, PM_OP_VEL1_U2 = 6, PM_OP_VEL1_U3 = 7,
  PM_OP_GRAD_X = 8, PM_OP_GRAD_Y = 9, PM_OP_GRAD_Z = 10
} pm_which;

/* Preconditioners (Section 5 remark): IC0 is the paper's choice for the velocity and mass
 * systems (zero fill, multicolour order: colour = (i&1) | (j&1)<<1 | (k&1)<<2); JACOBI is the
 * diagonal ("DIAG") and the labelled fallback; NONE is plain CG. LINE is vertical-line block
 * Jacobi -- each column's tridiagonal block of A solved exactly -- a labelled reading for the
 * pressure system of a thin layered domain (the paper's "DIAG + LS CGS OPT" is not defined in
 * it), not the paper's method. */
enum { PM_PREC_JACOBI = 0, PM_PREC_IC0 = 1, PM_PREC_NONE = 2, PM_PREC_LINE = 3 };
/* In per-entry preconditioner arguments (batches, server admission): use the options' choice. */
#define PM_PREC_DEFAULT (-1)
/* Arithmetic of the inner iteration. FP64 throughout, or FP32 (BF16) operator values with FP32
 * vectors inside PCG, dot products accumulated per thread in compensated FP32 (two floats, about
 * 48 significant bits) and reduced in FP64, FP64 alpha / beta, and FP64 outer iterative
 * refinement on the true residual until rtol is met. */
enum { PM_FP64 = 0, PM_FP32_REFINE = 1, PM_BF16_REFINE = 2 };

typedef struct pm_solve_opts {
  double rtol;           /* stop when ||b - A x||_2 <= rtol ||b||_2 (recursive residual,
                            then confirmed on the true residual)                           */
  int32_t max_iter;      /* cap on PCG iterations (all restarts / outer steps together)     */
  int32_t prec;          /* PM_PREC_*                                                       */
  int32_t precision;     /* PM_FP64, PM_FP32_REFINE, PM_BF16_REFINE                         */
  int32_t x0_is_guess;   /* 1: x holds the initial guess; 0: start from x = 0               */
  int32_t max_restarts;  /* true-residual restarts after the recursive test passes (FP64)   */
  double inner_rtol;     /* mixed precision: relative reduction asked of each inner solve  */
  int32_t kernel;        /* FP64 solves: PM_KERNEL_AUTO (resident for n <= 16384 rows),
                            PM_KERNEL_STREAM (one launch per PCG phase, every SM), or
                            PM_KERNEL_RESIDENT (one block runs the whole solve, n <= 2^20)   */
  int32_t pad;
} pm_solve_opts;

/* How an FP64 solve runs on the GPU (no paper counterpart; the iterates are those of the Section 5
 * PCG either way). STREAM issues one kernel per phase of every PCG iteration over the whole GPU;
 * RESIDENT runs the whole solve in one block of one SM, with block barriers between phases and one
 * read-back at the end: for small systems, whose stream iterations are bound by launch latency. */
enum { PM_KERNEL_AUTO = 0, PM_KERNEL_STREAM = 1, PM_KERNEL_RESIDENT = 2 };

typedef struct pm_solve_stats {
  int32_t iters;              /* PCG iterations (summed over restarts / inner solves)       */
  int32_t outer_iters;        /* refinement steps (mixed precision), restarts (FP64)        */
  int32_t status;             /* PM_* of this solve                                         */
  int32_t first_pass_iters;   /* iterations until the recursive residual first met rtol    */
  double rel_residual_true;   /* ||b - A x|| / ||b|| in FP64 at exit                         */
  double rel_residual_rec;    /* recursive residual estimate at exit                        */
  double seconds;             /* host wall time of the call                                 */
  double bytes_moved;         /* algorithmic bytes (values, vectors) the iterations moved   */
  double rel_residual_floor;  /* u || |A||x| + |b| ||_2 / ||b||_2, u = 2^-53: the relative
                                 residual that rounding x to FP64 alone can cause           */
} pm_solve_stats;

typedef struct pm_operator_info {
  int64_t n;          /* nodes (rows)                                     */
  int64_t n_pad;      /* row stride of the slot-major value arrays         */
  int32_t ncols, nz;  /* ocean columns, nodes per column                   */
  int32_t nx, ny;
  int64_t device_bytes; /* device memory held by the operator now         */
} pm_operator_info;

/* ---- operator ------------------------------------------------------------------------------ */

/* Build the layered mesh, boundary sets and all operators of a basin on the GPU: element
 * integrals of Section 5 assembled row by row into a 15-slot column-sliced ELL layout.
 * *out receives a new handle. Errors: PM_EINVAL, PM_DISCONNECTED, PM_ENOMEM, PM_ECUDA. */
int pm_assemble_operator(const pm_mesh_desc* mesh, const pm_physics* phys, pm_operator** out,
                         pm_stream stream);

/* Device bytes pm_assemble_operator would hold for this mesh (operators, factors, workspace),
 * for admission control by free HBM; -1 on invalid input. Host-only. */
int64_t pm_operator_bytes(const pm_mesh_desc* mesh);

int pm_operator_info_get(const pm_operator* op, pm_operator_info* info);

/* Grid indices of each ocean column (host arrays of length ncols). */
int pm_operator_columns(const pm_operator* op, int32_t* col_i, int32_t* col_j);

/* Copy one operator to host for inspection: values[s * n + row] (15 slots at the offsets listed
 * in api.SLOT_OFFSETS and csrc/pm_internal.cuh), nbr[col * 7 + q] neighbour columns (-1 = none), structural slot bits per row
 * (bit s set when row and slot neighbour share a tetrahedron). Any output may be NULL.
 * Dirichlet elimination is applied to the VEL values as the solver sees them. Synchronous. */
int pm_operator_export(const pm_operator* op, pm_which which, double* values, int32_t* nbr,
                       uint16_t* structure);

/* y = A x for one operator (VEL_* with its Dirichlet elimination), device vectors. Async. */
int pm_spmv(pm_operator* op, pm_which which, const double* x, double* y, pm_stream stream);

/* r = b - A x for one operator (VEL_* with its Dirichlet elimination), every row formed in
 * compensated arithmetic: the Dot2 scheme of Ogita, Rump and Oishi ("Accurate sum and dot
 * product", SIAM J. Sci. Comput. 26, 2005) splits each product a_ij x_j exactly into p + e with
 * one FMA, sums the p by TwoSum and carries both rounding errors, so r is as accurate as if formed
 * in twice the working precision and rounded once. This is how the solvers measure the true
 * residual. b, x, r: device vectors of length n (r must not alias x). norms: NULL (the call is
 * asynchronous) or a host array of 3 that receives ||r||^2, || |A||x| + |b| ||^2 (the square of
 * the FP64 floor's numerator) and ||b||^2; the call then synchronises the stream. The paper
 * states no stopping rule; this measures the one the solvers use (Section 5 remark). */
int pm_residual(pm_operator* op, pm_which which, const double* b, const double* x, double* r,
                double* norms, pm_stream stream);

/* Solve A x = b by PCG (Section 5 remark). For PM_OP_PRESSURE the zero-mean Lagrange multiplier
 * reading applies: b is replaced by b - (1'b / 1'm) m (m = M 1), the iterate is kept on
 * m'x = 0, and the returned x has m'x = 0. b and x are device vectors of length n; b is not
 * modified. stats may be NULL. Synchronises the stream. */
int pm_pcg_solve(pm_operator* op, pm_which which, const double* b, double* x,
                 const pm_solve_opts* opts, pm_solve_stats* stats, pm_stream stream);

/* Same solve as pm_pcg_solve, restricted to PM_PREC_JACOBI / PM_PREC_NONE in FP64, that
 * allocates nothing. (The paper has no counterpart: this is a deployment aid.) It is meant for
 * callers that cannot allocate device memory at solve time: processes whose device memory is
 * owned by a framework allocator or a fixed pool (an allocation behind the pool's back escapes its
 * accounting, or fails against its reservation), and embedded users that must not grow the device
 * footprint after start-up.
 * All scratch (Krylov vectors, Jacobi diagonal, reduction partials, device scalars) lives in one
 * static device array of PM_NOALLOC_MAX_ROWS rows (about 21 MB), held by every GPU that loads the
 * library until the process exits; no cudaMalloc, cudaFree or other allocating routine is called.
 * Errors: PM_EINVAL for systems with more than PM_NOALLOC_MAX_ROWS rows, another preconditioner
 * or precision, an operator that lives on a device other than the current one, or a stream that
 * is being captured (the call reads scalars back and synchronises the stream every few
 * iterations). The first call on a device looks up the array's address (cudaGetSymbolAddress)
 * with that device current. Every call shares the one array and re-initialises what must start
 * at zero; calls that overlap on the GPU (other streams or threads) race. max_iter = 0 runs no
 * iteration (PM_NOT_CONVERGED unless x already meets rtol). The operator itself must already be
 * assembled. Synchronises the stream. */
#define PM_NOALLOC_MAX_ROWS 524288
int pm_pcg_solve_noalloc(pm_operator* op, pm_which which, const double* b, double* x,
                         const pm_solve_opts* opts, pm_solve_stats* stats, pm_stream stream);

/* ---- batched solves (many basins x right-hand sides in one persistent launch) ---------------- */

/* A batch of independent systems (operator ops[i] with which[i]), solved together by one
 * persistent cooperative kernel per quantum of iterations, captured once in a CUDA graph and
 * replayed: PCG of the Section 5 remark for every system, all systems advancing together, each
 * with its own alpha / beta / convergence. Preconditioners: PM_PREC_JACOBI, PM_PREC_LINE,
 * PM_PREC_IC0 (PM_PREC_NONE maps to Jacobi), opts->prec for every entry, or prec[i] per entry
 * (prec may be NULL; an entry of PM_PREC_DEFAULT takes opts->prec), so that one batch can hold a
 * step's IC0 velocity and mass systems next to line-preconditioned pressure systems. IC0 applies
 * the same multicolour factor as the single-system solve: its 16 colour sweeps run as 16 phases of
 * the persistent kernel with a grid barrier after each, so a batch holding an IC0 system waits at
 * 22 grid barriers per iteration instead of 5. Precision: PM_FP64, PM_FP32_REFINE (FP32
 * difference-form values and vectors, FP64 x, dots and true-residual restarts), or
 * PM_BF16_REFINE (the same with BF16 difference-form values: FP32 vectors and factors). Starts from x = 0;
 * the pressure zero-mean reading applies to PM_OP_PRESSURE entries. autotune != 0 times the tile
 * width (columns per tile: 16, 32, 64) x block size (128, 256) on this batch once and caches the
 * choice per size bucket. Grid waits are bounded: an expired wait returns PM_TIMEOUT. The batch
 * keeps its own workspace; the operators must outlive it. count: 1..4096 systems. Errors:
 * PM_EINVAL (null or non-symmetric entry, unknown preconditioner or precision, rtol <= 0),
 * PM_BREAKDOWN (an IC0 factor that fails after the shift limit), PM_ENOMEM, PM_ECUDA. */
int pm_batch_create(pm_operator* const* ops, const pm_which* which, const int32_t* prec, int32_t count,
                    const pm_solve_opts* opts, int32_t autotune, pm_batch** out, pm_stream stream);
/* Solve all systems: b[i], x[i] device vectors of ops[i]'s length. stats: NULL or count entries.
 * Synchronises the stream. */
int pm_batch_solve(pm_batch* batch, const double* const* b, double* const* x, pm_solve_stats* stats,
                   pm_stream stream);
int pm_batch_info(const pm_batch* batch, int32_t* tile_cols, int32_t* block, int32_t* grid,
                  int64_t* ntiles);
void pm_batch_destroy(pm_batch* batch);
/* Test aid for failure detection: launches a two-block cooperative kernel in which one block
 * leaves without reaching the grid barrier, so the other block's bounded wait expires (about 2 s).
 * Returns the status that wait recorded: PM_TIMEOUT. Nothing faults, traps or hangs, and the
 * context stays usable. */
int pm_debug_barrier_timeout(pm_stream stream);
/* One-shot: create (no autotuning), solve, destroy. */
int pm_pcg_solve_batched(pm_operator* const* ops, const pm_which* which, const double* const* b,
                         double* const* x, int32_t count, const pm_solve_opts* opts,
                         pm_solve_stats* stats, pm_stream stream);

/* ---- continuous batching server ------------------------------------------------------------ */

/* A resident solve server: a table of `slots` systems advanced together by the persistent kernel
 * of the batched solves. Systems are admitted and retired between launches, so requests that
 * arrive while others are on the GPU join at the next quantum instead of waiting for the batch to
 * drain; each system's iterates depend on nothing but its own tiles (bit-identical whatever else
 * is resident, for a fixed tile_cols and block). No paper counterpart: the paper solves one basin;
 * this serves many basins' PCG solves (Section 5) at once.
 * opts: as pm_batch_create (PM_PREC_JACOBI / PM_PREC_LINE / PM_PREC_IC0 / PM_PREC_NONE; PM_FP64,
 * PM_FP32_REFINE or PM_BF16_REFINE); every system uses them unless its admission names its own
 * preconditioner. nz_cap: the largest nz admitted (sizes shared memory).
 * tile_cols: 16, 32 or 64 columns per tile; block: 128 or 256 threads; blocks_per_sm: resident
 * blocks per SM of the kernel (0 = as many as fit). Errors: PM_EINVAL, PM_ENOMEM, PM_ECUDA. */
int pm_server_create(int32_t slots, int32_t nz_cap, const pm_solve_opts* opts, int32_t tile_cols,
                     int32_t block, int32_t blocks_per_sm, pm_server** out, pm_stream stream);
/* Device bytes of Krylov workspace one system of `op` needs at `precision` (0 for NULL). */
size_t pm_server_workspace_bytes(const pm_operator* op, int32_t precision);
/* Admit one system: solve A x = b for op / which from x = 0, preconditioned by prec
 * (PM_PREC_DEFAULT: the server's opts->prec). b, x: device vectors of op's length;
 * work: device workspace of at least pm_server_workspace_bytes bytes, 256-byte aligned. All three
 * are the caller's and must stay valid until the slot is returned by pm_server_poll; nothing is
 * allocated per system except when the tile array has to grow. *slot receives the slot index.
 * Errors: PM_EINVAL (non-symmetric which, nz > nz_cap, small or misaligned workspace),
 * PM_EBUSY (all slots taken), PM_ENOMEM, PM_ECUDA. Async on `stream`. */
int pm_server_admit(pm_server* srv, pm_operator* op, pm_which which, int32_t prec, const double* b,
                    double* x, void* work, size_t work_bytes, int32_t* slot, pm_stream stream);
/* One launch of `quantum` iterations for every resident system (systems admitted since the last
 * launch are initialised first). *active receives the number of systems still iterating.
 * Synchronises the stream. An expired grid wait returns PM_TIMEOUT (the server is then unusable:
 * destroy it). */
int pm_server_run(pm_server* srv, int32_t quantum, int32_t* active, pm_stream stream);
/* Retire finished systems: up to max_out of them are written to slots[] / stats[] (stats may be
 * NULL) and their slots freed; *n_out receives the count. Host only. */
int pm_server_poll(pm_server* srv, int32_t* slots, pm_solve_stats* stats, int32_t max_out,
                   int32_t* n_out);
int pm_server_info(const pm_server* srv, int32_t* tile_cols, int32_t* block, int32_t* grid,
                   int64_t* tile_capacity, int64_t* launches);
void pm_server_destroy(pm_server* srv);

/* ---- projection step ---------------------------------------------------------------------- */

/* Time-step state u^k, u^{k-1}, p^k (device, owned by the handle). Created at rest:
 * u^0 = 0 (Eq. prim_ci), p^0 = 0, step index 0. */
int pm_state_create(pm_operator* op, pm_state** out);
/* Copy state fields to / from caller device vectors (any pointer may be NULL). Async.
 * pm_state_set sets u^k and p^k from the given vectors (NULL = 0), sets u^{k-1} = u^k, clears
 * the pressure-increment warm start, and sets the step index (0 = the next step is BDF1). */
int pm_state_get(const pm_state* st, double* u1, double* u2, double* u3, double* p,
                 pm_stream stream);
int pm_state_set(pm_state* st, const double* u1, const double* u2, const double* u3,
                 const double* p, int32_t step_index, pm_stream stream);
int32_t pm_state_step_index(const pm_state* st);

/* One field of the state, copied to a caller device vector of length n. Async. Besides u^k,
 * u^{k-1} and p^k, the last step's intermediate fields stay available until the next step: the
 * prediction u~ (Eq. fofa_velo_pred_h), the pressure increment q and its right-hand side
 * b_p = -alpha sum_c G_c u~_c (Eq. fofa_q_cor_h). Before the first step they are 0. */
enum { PM_FIELD_U1 = 0, PM_FIELD_U2 = 1, PM_FIELD_U3 = 2,
       PM_FIELD_U1_PREV = 3, PM_FIELD_U2_PREV = 4, PM_FIELD_U3_PREV = 5,
       PM_FIELD_P = 6, PM_FIELD_Q = 7, PM_FIELD_UT1 = 8, PM_FIELD_UT2 = 9, PM_FIELD_UT3 = 10,
       PM_FIELD_BP = 11 };
int pm_state_field(const pm_state* st, int32_t field, double* dst, pm_stream stream);
/* Set one field (PM_FIELD_U1 .. PM_FIELD_Q) from a caller device vector of length n, and the step
 * index (0: the next step is the BDF1 start step). With these, a state can be restored exactly
 * (u^k, u^{k-1}, p^k, the pressure-increment warm start q). Async. */
int pm_state_set_field(pm_state* st, int32_t field, const double* src, pm_stream stream);
int pm_state_set_step_index(pm_state* st, int32_t step_index);

/* Checkpoint and resume of a time loop (Section 3's BDF2 recurrence needs u^k and u^{k-1}).
 * pm_state_save writes u^k (3), u^{k-1} (3), p^k, q and the step index of `st` to `path`: a
 * 4096-byte ASCII header (one JSON object, space padded, ending in a newline) followed by the
 * eight fields as little-endian IEEE-754 float64 arrays of n values, in that order. The header
 * records the format version, n, the grid (nx, ny, nz, ncols, dx, dy), dt, nu, an FNV-1a 64-bit
 * hash of the ocean column list and of the payload. The file is written under a temporary name
 * and renamed, so an interrupted save leaves any previous checkpoint intact.
 * pm_state_load reads such a file into `st`, whose operator must be the same basin (grid, column
 * list, dt, nu): otherwise, or for a wrong version, size or payload hash, PM_EINVAL and `st` is
 * unchanged. A state saved and loaded continues bit for bit as the uninterrupted run would.
 * Both synchronise the stream. Errors: PM_EINVAL, PM_ENOMEM, PM_ECUDA (I/O errors: PM_EINVAL with
 * the system's message in pm_last_error). */
int pm_state_save(const pm_state* st, const char* path, pm_stream stream);
int pm_state_load(pm_state* st, const char* path, pm_stream stream);

/* Diagnostics of the state after a step (no paper counterpart; they monitor the time loop of
 * Section 3): out[PM_DIAG_KINETIC_ENERGY] = (1/2) sum_c u_c' M u_c, out[PM_DIAG_DIV_U] =
 * || sum_c G_c u_c ||_2 (the integral of div u^k against every basis function; the correction of
 * Eq. correc_velo_u exists to make it small), out[PM_DIAG_DIV_UT] = the same for the last
 * prediction u~, out[PM_DIAG_P_MEAN] = m'p / 1'm. Synchronises the stream. */
enum { PM_DIAG_KINETIC_ENERGY = 0, PM_DIAG_DIV_U = 1, PM_DIAG_DIV_UT = 2, PM_DIAG_P_MEAN = 3,
       PM_DIAG_COUNT = 4 };
int pm_state_diagnostics(pm_operator* op, const pm_state* st, double* out, pm_stream stream);

enum { PM_STEP_LUMPED = 0, PM_STEP_CONSISTENT = 1 };

/* One BDF2 velocity-correction step (Section 3; BDF1 on the first step):
 *   b_c = velocity right-hand side (history, advection, Coriolis, G_c^T p^k, wind tension)
 *   (alpha M + K_nu) u~_c = b_c, c = 1..3               (velocity PCG, x0 = u^k_c)
 *   K_I q = -alpha sum_c G_c u~_c, zero mean            (pressure PCG, x0 = previous q)
 *   p^{k+1} = p^k + q;  u_c = u~_c - M^{-1} G_c q / alpha, then the Dirichlet sets
 *   (the correction takes the sign of Eq. correc_velo_u, from which Eq. press_cor follows;
 *   Eq. fofa_velo_cor_h prints "+", which would add the gradient instead of removing it)
 * theta1, theta2: device arrays [ncols], kinematic wind tension at the surface node of each
 * column (NULL = 0). correction: PM_STEP_LUMPED (diag(M 1)) or PM_STEP_CONSISTENT (PCG on M
 * with vel's options). stats: NULL or 7 entries (u1, u2, u3, q, mass1, mass2, mass3).
 * Synchronises the stream. */
int pm_project_step(pm_operator* op, pm_state* st, const double* theta1, const double* theta2,
                    const pm_solve_opts* vel, const pm_solve_opts* pres, int32_t correction,
                    pm_solve_stats* stats, pm_stream stream);

void pm_operator_destroy(pm_operator* op);
void pm_state_destroy(pm_state* st);

/* ---- misc --------------------------------------------------------------------------------- */
const char* pm_status_string(int status);
/* Copies the calling thread's last error message (NUL-terminated) into buf; returns its length. */
int pm_last_error(char* buf, int32_t len);
/* Number of kernels this process has launched through the library (all threads). */
int64_t pm_kernel_launch_count(void);

/* Live kernel timing. When enabled, the PCG driver brackets every launch of the kernel classes
 * below with CUDA events on the solve's stream and accumulates their elapsed times at its own
 * synchronisation points. pm_kernel_timing(enable) switches it and resets the totals;
 * pm_kernel_timing_get returns the total milliseconds and launch count of one class. Process-
 * global and not thread-safe; a measurement aid, off by default. */
enum { PM_KT_SPMV = 0,    /* SpMV + (p, Ap) reduction, one launch per PCG iteration      */
       PM_KT_UPDATE = 1,  /* x, r update + residual reductions                           */
       PM_KT_PUPDATE = 2, /* search-direction update (with the (r, z) reduction for IC0) */
       PM_KT_IC0 = 3,     /* the 16 IC0 colour sweeps of one preconditioner apply        */
       PM_KT_LINE = 4,    /* the vertical-line solve fused with the (r, z) reduction     */
       PM_KT_COUNT = 5 };
int pm_kernel_timing(int32_t enable);
int pm_kernel_timing_get(int32_t kind, double* total_ms, int64_t* launches);

/* Per-solve JSON log. With a path, every solved system appends one line to that file (opened in
 * append mode): the entry point ("pcg_solve", "pcg_solve_noalloc", "project_step",
 * "batch_solve", "server_solve"), rows, system, preconditioner, precision, status, iterations
 * (total, outer, first pass), true and floor relative residuals, seconds, algorithmic bytes, GB/s,
 * and, when hbm_peak_gbs > 0, GB/s as a percentage of it. NULL closes the log. Process-global,
 * lines written under a lock. Errors: PM_EINVAL (the file cannot be opened; logging is then off).
 * The library also marks its assemblies, solves, steps and their stages as NVTX ranges, which
 * profilers show on their timelines. */
int pm_set_log(const char* path, double hbm_peak_gbs);

/* Build flags: PM_BUILD_CHECKED when the library was compiled with device index checks
 * (PM_CHECKED). In that build every neighbour-column index a kernel reads is checked against the
 * column count; a bad one is recorded and skipped (read as "no neighbour"), nothing faults, and
 * the entry point that launched the kernel returns PM_EBOUNDS with the value in pm_last_error. */
enum { PM_BUILD_CHECKED = 1 };
int32_t pm_build_flags(void);

#ifdef __cplusplus
}
#endif
#endif /* PM_GB300_H */
