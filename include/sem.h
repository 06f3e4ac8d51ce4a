/*
 * sem.h -- C ABI of libsem, a GB300 (sm_103a) matrix-free spectral-element
 * solver for the monodomain equation of cardiac electrophysiology.
 *
 * What it computes (arXiv 2205.05136):
 *   - Section 2, Eq. (monodomain) and Eq. (diffusiontensor): the monodomain
 *     equation with homogeneous Neumann data and the anisotropic conductivity
 *     D = sigma_t I + (sigma_l - sigma_t) f f^T (sigma_n = sigma_t), fibre
 *     f = (cos theta, sin theta, 0) per element.
 *   - Section 3: Q_p spectral elements on hexahedra with the LGL nodal basis;
 *     SEM integrates with the (p+1)-point Legendre-Gauss rule, SEM-NI with the
 *     (p+1)-point Legendre-Gauss-Lobatto rule (diagonal mass).
 *   - Section 3, Eqs. (ionic_discr), (monodomain_discr), (algebraic_ionic),
 *     (linsys), (matrix_rhs): the partitioned semi-implicit BDF2 step with the
 *     extrapolated potential u* = 2u^n - u^{n-1}.
 *   - Section 4 and Algorithm 1: the matrix-free application of
 *     A = alpha M + K by a cell loop with sum factorization, inside CG.
 *
 * Conventions
 *   - Every function returns an int status: SEM_OK (0) or a negative
 *     SEM_ERR_* code.  sem_last_error() returns a message for the last failure
 *     on a context.  No function exits the process or traps on the device.
 *   - "device" pointers point to memory of the context's CUDA device (for
 *     example torch tensors); they are checked with cudaPointerGetAttributes and
 *     rejected with SEM_ERR_ARG when they are host memory.  The library never
 *     frees caller memory.
 *   - Vectors over the global nodes have length ndofs (sem_num_dofs), node
 *     (I, J, K) of the (p nx + 1) x (p ny + 1) x (p nz + 1) lattice at index
 *     I + (p nx + 1) (J + (p ny + 1) K).  Per-element arrays have length
 *     nx ny nz, element (ex, ey, ez) at ex + nx (ey + ny ez).
 *   - `stream` is a cudaStream_t passed as void* (NULL = legacy default
 *     stream).  Work is enqueued on it; functions that return host scalars
 *     (iteration counts, residuals) synchronise that stream only.
 *   - Memory for mesh data, metric terms and solver work vectors is owned by
 *     the context (cudaMalloc at creation or on first use) and released by
 *     sem_destroy.
 */
#ifndef SEM_H
#define SEM_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define SEM_OK 0
#define SEM_ERR_ARG (-1)           /* bad argument: null, size, range, host pointer */
#define SEM_ERR_CUDA (-2)          /* a CUDA runtime call failed */
#define SEM_ERR_BAD_MESH (-3)      /* det J <= 0 at some quadrature point */
#define SEM_ERR_NOT_CONVERGED (-4) /* CG reached maxit; x holds the last iterate */
#define SEM_ERR_NONFINITE (-5)     /* NaN or Inf met in a CG inner product */
#define SEM_ERR_UNSUPPORTED (-6)   /* valid request that this library does not provide */
#define SEM_ERR_NOMEM (-7)         /* device allocation failed */
#define SEM_ERR_TIMEOUT (-8)       /* a kernel's bounded wait for its own copy gave up (reported by the
                                      next multigrid solve; the context stays usable) */

#define SEM_QUAD_LG 0  /* SEM: (p+1)-point Legendre-Gauss quadrature */
#define SEM_QUAD_LGL 1 /* SEM-NI: (p+1)-point Legendre-Gauss-Lobatto quadrature */

#define SEM_PREC_FP64 0      /* double vectors, double metric, double arithmetic */
#define SEM_PREC_FP32 1      /* float vectors, float metric, float arithmetic */
#define SEM_PREC_FP32_BF16 2 /* float vectors, bfloat16 metric, float arithmetic */
#define SEM_PREC_DF64 3      /* double vectors, metric split into float pairs, double-float
                                arithmetic on the FP32 pipe (FP64 results to ~1e-14) */
#define SEM_PREC_BF16_TC 4   /* float vectors, bfloat16 metric, the sum-factorization
                                contractions on the tensor cores (bf16 operands, FP32
                                accumulation): SEM-NI (SEM_QUAD_LGL) at p = 2..4 */

#define SEM_PC_NONE 0
#define SEM_PC_JACOBI 1
#define SEM_PC_GMG 2

#define SEM_REGION_BOX 0    /* params: x0 y0 z0 x1 y1 z1 (closed box) */
#define SEM_REGION_SPHERE 1 /* params: cx cy cz r (closed ball) */

typedef struct sem_ctx sem_ctx;
typedef struct sem_state sem_state;

/* Parameters of the two-variable stand-in ionic model (the paper's TTP06
 * equations are not printed in it):
 *   v = (u - u_rest) / u_amp
 *   I_ion = -u_amp (h v^2 (1 - v) / tau_in - v / tau_out)
 *   s(v) = 1 / (1 + exp(-(v - v_gate) / kappa))
 *   dh/dt = (1 - s)(1 - h) / tau_open - s h / tau_close
 * Units: mV and ms, chi = C_m = 1 as in Section 2. */
typedef struct {
  double u_rest, u_amp, tau_in, tau_out, tau_open, tau_close, v_gate, kappa;
} sem_ionic_params;

/* Counters filled by sem_step and sem_cg_solve. */
typedef struct {
  int64_t steps;          /* time steps taken by this call */
  int64_t cg_iters;       /* CG iterations summed over the call */
  double last_residual;   /* ||r||_2 at the end of the last solve */
  double apply_ms;        /* device time of operator-apply kernels (when timing on) */
  int64_t n_apply;        /* operator-apply launches timed (one per sampled solve, see sem_set_timing) */
  int64_t kernel_launches; /* libsem kernels launched by the call */
  double smoother_apply_ms;   /* device time of timed fine-level multigrid smoother applies */
  int64_t n_smoother_apply;   /* fine-level smoother applies timed (one per sampled solve) */
  int64_t carried_solves;     /* time-step solves whose initial residual came from the
                                 previous step's solve (no operator apply) */
} sem_stats;

/* Library version string (static storage). */
const char* sem_version(void);

/* Create a context for a structured hexahedral slab of nx x ny x nz elements.
 * vertices: HOST array of (nx+1)(ny+1)(nz+1) points x y z, x fastest; element
 *   (ex, ey, ez) is the trilinear image of [-1,1]^3 through its 8 lattice
 *   vertices (Section 3).  The vertices are copied.
 * p: polynomial degree 1..6.  quad: SEM_QUAD_LG or SEM_QUAD_LGL.
 * device: CUDA device ordinal; the context uses it for every call.
 * Tissue defaults to sigma_l = 0.12, sigma_t = 0.03 mm^2/ms, theta = 0.
 * Errors: SEM_ERR_ARG, SEM_ERR_BAD_MESH (det J <= 0), SEM_ERR_CUDA, SEM_ERR_NOMEM.
 * On failure *out is NULL. */
int sem_create(sem_ctx** out, int nx, int ny, int nz, const double* vertices, int p, int quad,
               int device);

/* Release every resource of the context (waits for its work to finish). */
int sem_destroy(sem_ctx* ctx);

/* Message of the last failing call on ctx (or of the last failed creation when
 * ctx is NULL).  Static/ctx-owned storage, valid until the next call. */
const char* sem_last_error(const sem_ctx* ctx);

int sem_num_dofs(const sem_ctx* ctx, int64_t* ndofs);
int sem_num_elements(const sem_ctx* ctx, int64_t* nelem);

/* Physical coordinates of the global nodes: device double xyz[3 * ndofs] laid
 * out as x[ndofs], y[ndofs], z[ndofs]. */
int sem_dof_coords(sem_ctx* ctx, double* xyz, void* stream);

/* Per-element conductivities and fibre angle (device double arrays of length
 * nelem; theta in radians).  Recomputes the quadrature-point metric terms
 * G = w |det J| J^{-1} D J^{-T} (Eq. diffusiontensor evaluated at every
 * quadrature point, Section 4.2) of every precision in use. */
int sem_set_tissue(sem_ctx* ctx, const double* sigma_l, const double* sigma_t,
                   const double* theta, void* stream);

/* y = alpha M u + beta K u (Algorithm 1, cell loop with sum factorization).
 * precision SEM_PREC_FP64 or SEM_PREC_DF64: u, y are device double[ndofs].
 * precision SEM_PREC_FP32 / SEM_PREC_FP32_BF16 / SEM_PREC_BF16_TC: u, y are
 * device float[ndofs]; SEM_PREC_BF16_TC returns SEM_ERR_UNSUPPORTED outside
 * SEM-NI at p = 2..4.  y is overwritten; u and y must not overlap. */
int sem_apply(sem_ctx* ctx, double alpha, double beta, const void* u, void* y, int precision,
              void* stream);

/* Arithmetic of the operator inside sem_cg_solve / sem_step (the outer CG of
 * the multigrid PCG included): SEM_PREC_FP64 (default, FP64 instructions) or
 * SEM_PREC_DF64 (double-float on the FP32 pipe; vectors, residuals and inner
 * products stay FP64). */
int sem_set_operator_precision(sem_ctx* ctx, int precision);

/* Deterministic mode (enable = 1) or atomic scatter (0, the default).  The
 * element results of an operator apply (Algorithm 1's "compress" step) are
 * normally added into the global vector with atomic adds, whose order varies
 * from run to run, so results differ in the last bits.  In deterministic mode
 * every apply (sem_apply, sem_cg_solve, sem_step, the multigrid V-cycle and its
 * restrictions, the adjoint's solves) writes element-local results and a node
 * kernel adds each node's contributions in a fixed element order: the same
 * inputs give bitwise the same outputs, at the cost of an extra pass over
 * nelem (p+1)^3 values per apply.  The tensor-core smoother runs the scalar
 * bf16-metric kernel in this mode and sem_apply with SEM_PREC_BF16_TC returns
 * SEM_ERR_UNSUPPORTED; sem_apply_dot_static keeps atomic adds.  The first
 * enable allocates nelem (p+1)^3 doubles (owned by the context; SEM_ERR_NOMEM
 * when that fails).  Synchronises the device. */
int sem_set_deterministic(sem_ctx* ctx, int enable);

/* Diagonal of alpha M + beta K: device double d[ndofs]. */
int sem_diagonal(sem_ctx* ctx, double alpha, double beta, double* d, void* stream);

/* Solve (alpha M + K) x = b by preconditioned CG (Section 4), warm-started
 * from the x passed in.  Stops when ||r||_2 <= max(rtol ||b||_2, atol).
 * precond: SEM_PC_NONE, SEM_PC_JACOBI or SEM_PC_GMG (flexible PCG with one
 * V-cycle per iteration, see sem_set_gmg).  b, x: device double[ndofs].  iters / final_res may be NULL.
 * Returns SEM_ERR_NOT_CONVERGED after maxit iterations (x = last iterate) and
 * SEM_ERR_NONFINITE when an inner product is NaN or Inf.  Synchronises stream. */
int sem_cg_solve(sem_ctx* ctx, double alpha, const double* b, double* x, double rtol,
                 double atol, int maxit, int precond, int* iters, double* final_res,
                 void* stream);

/* Geometric multigrid preconditioner (Section 4.3), used by sem_cg_solve and
 * sem_step with precond = SEM_PC_GMG.  Levels: the fine Q_p level, p-coarsened
 * levels on the same mesh (p -> p/2 -> ... -> 1), then 2:1 h-coarsened Q_1
 * levels; coarsening stops at the first level (p- or h-) with at most
 * min_coarse_dofs nodes; operators are
 * rediscretised per level.  Smoother: Chebyshev-Jacobi of the given degree on
 * [0.08, 1.2] x lambda_max(D^{-1} A), lambda_max from 10 Lanczos (CG) steps;
 * coarse_degree Chebyshev steps on the coarsest level.  precision: the
 * V-cycle's arithmetic -- SEM_PREC_FP32 (FP32 metric), SEM_PREC_FP32_BF16
 * (bf16 metric), SEM_PREC_BF16_TC (bf16 metric, tensor-core contractions on
 * the SEM-NI levels of degree 2..4, the bf16-metric FP32 kernel on the others)
 * or SEM_PREC_FP64; the outer CG is flexible and stays FP64.
 * Defaults: degree 3, coarse_degree 10, min_coarse_dofs 2000, FP32.  The
 * hierarchy is (re)built on first use after this call or sem_set_tissue. */
int sem_set_gmg(sem_ctx* ctx, int degree, int coarse_degree, int min_coarse_dofs, int precision);

/* z = one V-cycle applied to r for the operator alpha M + K (device double[ndofs]). */
int sem_vcycle(sem_ctx* ctx, double alpha, const double* r, double* z, void* stream);

/* Hierarchy description for alpha (builds it if needed): number of levels, and
 * for the first max_levels levels their degree p, element counts dims[3 l ..
 * 3 l + 2], node counts and lambda_max estimates (any output may be NULL). */
int sem_gmg_info(sem_ctx* ctx, double alpha, int max_levels, int* nlevels, int* p, int* dims,
                 int64_t* ndofs, double* lambda_max, void* stream);

/* Ionic model parameters (copied). */
int sem_set_ionic(sem_ctx* ctx, const sem_ionic_params* prm);

/* Applied current I_app = amplitude on the nodes inside the region, for
 * t_on < t <= t_off (Section 5: a cuboid or a sphere of stimulation).
 * params: host double[6] (box) or double[4] (sphere). */
int sem_set_stimulus(sem_ctx* ctx, int region, const double* params, double amplitude,
                     double t_on, double t_off, void* stream);

/* Time-stepping state: u^n, u^{n-1}, h^n, h^{n-1} and the step counter n,
 * device memory owned by the state. */
int sem_state_create(sem_ctx* ctx, sem_state** out);
int sem_state_destroy(sem_state* st);

/* Set u^0 = u0 and h^0 = h0 (device double[ndofs]) and n = 0. */
int sem_state_set(sem_state* st, const double* u0, const double* h0, void* stream);

/* Copy the BDF2 state into device arrays: u^n -> u, u^{n-1} -> u_prev,
 * h^n -> h, h^{n-1} -> h_prev (each may be NULL); *n_out (may be NULL)
 * receives the number of steps taken.  With sem_state_restore this is a
 * checkpoint of the full time-stepping state. */
int sem_state_get(sem_state* st, double* u, double* u_prev, double* h, double* h_prev,
                  int64_t* n_out, void* stream);

/* Restore a full BDF2 state (device arrays of length ndofs) and its step count n
 * (n = 0 makes the next step BDF1 and ignores u_prev / h_prev). */
int sem_state_restore(sem_state* st, const double* u, const double* u_prev, const double* h,
                      const double* h_prev, int64_t n, void* stream);

/* Activation times (Section 5, Eq. tau): while enabled, every step of
 * sem_step records per node the largest |du/dt| met so far and the time of the
 * step that gave it; du/dt at t^{n+1} = (n+1) dt is the time scheme's own
 * derivative, (u^1 - u^0)/dt for the first step and
 * (3 u^{n+1} - 4 u^n + u^{n-1})/(2 dt) after; on a tie the earlier time stays.
 * Enabling (enable != 0) allocates the two arrays on first use (owned by the
 * state, freed by sem_state_destroy) and resets them (max -1, time NaN);
 * enable = 0 stops the updates and keeps the values.  SEM_ERR_NOMEM when the
 * arrays cannot be allocated. */
int sem_state_track_activation(sem_state* st, int enable, void* stream);

/* Copy the activation times (ms) and the max |du/dt| (mV/ms) into caller-owned
 * device double[ndofs] arrays (either may be NULL).  SEM_ERR_ARG when tracking
 * was never enabled or a pointer is not device memory. */
int sem_state_get_activation(sem_state* st, double* tau, double* dudt_max, void* stream);

/* Advance the state by nsteps time steps of size dt (ms): the first step from
 * n = 0 is BDF1 (u* = u^0, A = M/dt + K), the following ones BDF2
 * (u* = 2u^n - u^{n-1}, A = 3/(2 dt) M + K), each one
 *   gate update and I_ion per node (Eq. ionic_discr),
 *   b = M(history) - M I_ion + M I_app(t^{n+1})   (Eqs. algebraic_ionic, matrix_rhs),
 *   CG solve warm-started from u^n to ||r|| <= max(rtol ||b||, atol).
 * Consecutive steps of one state with the same operator take the initial
 * residual's A u^n from the previous step's solve (A u^n = b_prev - r_prev)
 * instead of applying the operator; every 50th step applies it, and any other
 * call that changes the context or the state ends this.
 * stats may be NULL.  Synchronises stream. */
int sem_step(sem_ctx* ctx, sem_state* st, double dt, int nsteps, double rtol, double atol,
             int maxit, int precond, sem_stats* stats, void* stream);

/* One time step on HOST arrays of length ndofs: the state (u^n, u^{n-1},
 * h^n, h^{n-1}, n) is copied to the device, advanced by one step as
 * sem_step does, and the new state is written back in place (u_prev <- u,
 * u <- u^{n+1}, h_prev <- h, h <- h^{n+1}).  Page-locked host memory makes
 * the copies asynchronous.  Synchronises stream. */
int sem_step_host(sem_ctx* ctx, double* u, double* u_prev, double* h, double* h_prev, int64_t n,
                  double dt, double rtol, double atol, int maxit, int precond, sem_stats* stats,
                  void* stream);

/* One time step on HOST arrays of length ndofs with inputs and outputs apart:
 * reads the state (u^n, u^{n-1}, h^n, h^{n-1}, n) from u, u_prev, h, h_prev
 * and writes u^{n+1}, h^{n+1} to u_next, h_next; the inputs are not modified.
 * The step is the one sem_step takes (Section 3, Algorithm 1).  A caller that
 * rotates three host arrays per field (u_prev <- u <- u_next) moves 4 vectors
 * to and 2 from the device per step, against 4 and 4 with sem_step_host.
 * With page-locked inputs the ionic update reads them over the host link
 * while it computes; pageable inputs are staged by copies.  h^{n+1} is copied
 * back on a second stream of the context while the linear solve runs, u^{n+1}
 * after the solve.  With the multigrid preconditioner, a call whose n follows
 * the previous call's and whose u equals, bit for bit, the u_next that call
 * returned takes the initial residual from that call's solve as sem_step
 * does; the device checks the equality while it reads u and otherwise applies
 * the operator (stats->carried_solves counts the carried solves).  The host
 * must not change the arrays during the call.  SEM_ERR_ARG when an array is
 * device memory or when u_next or h_next overlaps another array.
 * Synchronises stream. */
int sem_step_host_out(sem_ctx* ctx, const double* u, const double* u_prev, const double* h,
                      const double* h_prev, double* u_next, double* h_next, int64_t n, double dt,
                      double rtol, double atol, int maxit, int precond, sem_stats* stats, void* stream);

/* Run nsteps time steps from st as sem_step does, writing the traces
 * traces[k * nsens + s] = u^{n0+k+1}[sensors[s]] (device double[nsteps * nsens];
 * sensors: device int[nsens] node indices) and keeping a checkpoint of the full
 * BDF2 state every checkpoint_every steps in the context (device memory,
 * 4 ndofs doubles per checkpoint), for sem_adjoint_grad.  A new recording
 * replaces the previous one. */
int sem_forward_record(sem_ctx* ctx, sem_state* st, double dt, int nsteps, int checkpoint_every,
                       const int* sensors, int nsens, double* traces, double rtol, double atol,
                       int maxit, int precond, sem_stats* stats, void* stream);

/* Gradient of a loss L(traces) with respect to the per-element sigma_l, sigma_t
 * and theta of the recorded run, given trace_bar = dL/dtraces (device double,
 * same layout as the traces).  Discrete adjoint of the partitioned scheme
 * (Section 3): each checkpoint segment is recomputed forward, then reversed;
 * every reversed step solves A w = ubar with the same solver settings
 * (A is symmetric) and adds -w^T (dK/dparam) u^{n+1} per element.  The tissue
 * and stimulus must be those of the recording.  g_*: device double[nelem],
 * overwritten. */
int sem_adjoint_grad(sem_ctx* ctx, const double* trace_bar, double* g_sigma_l, double* g_sigma_t,
                     double* g_theta, double rtol, double atol, int maxit, int precond,
                     sem_stats* stats, void* stream);

/* y = alpha M u + beta K u and *dot = u . y (FP64), without allocating.
 * The paper has no counterpart: this is a variant of the operator apply for
 * callers that cannot let a library allocate device memory -- host frameworks
 * that own every device allocation through their own arena or a fixed budget,
 * and real-time loops that must not enter the allocator, whose calls can
 * synchronise the device (sem_cg_solve and sem_step allocate work vectors on
 * first use; this call never allocates).  u, y: device double[ndofs]; dot:
 * device double[1]; the caller passes all inputs and outputs, and none of the
 * three may overlap another (SEM_ERR_ARG).  beta must be finite and nonzero.
 * The grid reduction's scratch is one static device array of 65,536 per-CTA
 * partial sums (512 KiB in every CUDA context that loads libsem, held until
 * the process exits); meshes needing more CTAs (more than 65,536 x E
 * elements, E = 64, 28, 16, 10, 7, 5 for p = 1..6) are rejected with
 * SEM_ERR_ARG.  The calls made in one CUDA context share that array and it
 * keeps the last call's contents: calls that overlap on the GPU race on it,
 * so order them.  The first call on a context looks up the array's address
 * (the context's device current) and keeps it in ctx; make that first call
 * before any stream capture begins.  After a cudaDeviceReset the contexts of
 * that device, and the address, are invalid: create new ones.
 * Asynchronous on stream. */
int sem_apply_dot_static(sem_ctx* ctx, double alpha, double beta, const double* u, double* y,
                         double* dot, void* stream);

/* Fault injection for the SEM_DEBUG build (paper_2205_05136_gb300.build with
 * debug=True: -DSEM_DEBUG).  That build checks every node index the apply
 * and transfer kernels read from the element-to-DOF map (or compute from the
 * node lattice) against [0, ndofs); an index outside is not used (node 0 is
 * read or written instead), the first one is recorded in a device word, and
 * sem_apply, sem_cg_solve, sem_step and sem_vcycle then synchronise their
 * stream and return SEM_ERR_ARG naming it.  This entry point overwrites entry
 * `entry` (element e, local node a at e (p+1)^3 + a) of the context's fine
 * level map with `value` and returns the old value in *previous (may be
 * NULL), so a test can plant a bad index.  The normal build returns
 * SEM_ERR_UNSUPPORTED.  Synchronous. */
int sem_debug_set_map_entry(sem_ctx* ctx, int64_t entry, int value, int* previous);

/* SEM_DEBUG build only (the normal build returns SEM_ERR_UNSUPPORTED): the
 * pipelined FP32 apply of the fine level leaves out the metric copy of element
 * group `group` (its group index; -1: none), so that the warp's bounded wait
 * for that copy runs out.  That warp then sets the context's wait-timeout word,
 * lets its other copy in flight land and returns, and the next multigrid solve
 * returns SEM_ERR_TIMEOUT (its result is not used).  Exercises the timeout
 * path without any fault.  Drops the multigrid hierarchy (its captured graphs
 * hold the launch arguments); the next solve rebuilds it.  Synchronous. */
int sem_debug_hold_copy(sem_ctx* ctx, int group);

/* Enable (1) or disable (0) CUDA-event timing of the operator-apply kernels
 * inside sem_step / sem_cg_solve (reported in sem_stats).  One solve in ten
 * (the first after enabling, then every tenth) times the operator apply of its
 * first iteration, and with the multigrid preconditioner also the fine-level
 * residual apply of that iteration's V-cycle: the events that bracket them cost
 * a few microseconds each, so the other solves run without them. */
int sem_set_timing(sem_ctx* ctx, int enable);

#ifdef __cplusplus
}
#endif

#endif /* SEM_H */
