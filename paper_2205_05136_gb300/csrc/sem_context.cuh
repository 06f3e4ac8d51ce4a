// Context and state objects behind the opaque sem_ctx / sem_state handles.
#pragma once

#include <memory>
#include <string>
#include <vector>

#include "sem_internal.cuh"

namespace sem {

// Work vectors and device scalars of the solver (allocated on first use).
struct Workspace {
  bool ready = false;
  double *r = nullptr, *z = nullptr, *p = nullptr, *Ap = nullptr, *invdiag = nullptr;
  double *b = nullptr, *g = nullptr;
  double* Ax = nullptr;      // A x of the last time step's solution (its b - r), see sem_ctx::carry
  df_pair* p2 = nullptr;     // p split into float pairs for the double-float operator's gather
  double inv_alpha = -1.0;   // alpha for which invdiag holds 1 / diag(alpha M + K)
  CgScalars* cg = nullptr;   // device
  CgScalars* cg_host = nullptr;  // page-locked mirror
  double* vec_partials = nullptr;     // [kReduceSlots][kVecBlocksMax]
  unsigned int* tickets = nullptr;    // [4]: [0] the CG vector kernels' reductions, the rest spare
  double* apply_partials = nullptr;   // [apply grid]
  double* dot_result = nullptr;       // 1 double
  int* same = nullptr;        // device flag of sem_step_host_out's carry check (sem_ctx::carry)
  int* same_host = nullptr;   // page-locked copy, read after the call
  unsigned* fault_host = nullptr;  // page-locked copy of the level's wait-timeout word
};

struct Gmg;   // geometric multigrid hierarchy (sem_gmg.cu)
struct Tape;  // checkpoints of a recorded forward run (sem_adjoint.cu)

struct Timing {
  bool enabled = false;
  cudaEvent_t start = nullptr, stop = nullptr;
  double ms = 0.0;            // outer operator applies
  int64_t count = 0;
  double smoother_ms = 0.0;   // fine-level multigrid smoother applies (one per V-cycle timed)
  int64_t smoother_count = 0;
  int64_t solves = 0;         // multigrid solves since timing was enabled (every kTimingEvery-th is sampled)
};
// With timing on, the first PCG iteration of one multigrid solve in kTimingEvery
// runs the graph with event nodes (each costs a few microseconds of the step).
constexpr int kTimingEvery = 10;

}  // namespace sem

namespace sem {
// Time steps between true initial residuals when the residual is carried (sem_ctx::carry).
constexpr int kCarrySteps = 50;
}  // namespace sem

struct sem_ctx {
  int device = 0;
  sem::Level L;
  std::vector<double> vertices;  // host copy of the slab's vertex lattice
  double* sigma_l = nullptr;  // per element
  double* sigma_t = nullptr;
  double* theta = nullptr;
  int* d_flag = nullptr;      // setup error flag
  sem_ionic_params ionic{};
  double* stim_mask = nullptr;
  double stim_amp = 0.0, stim_on = 0.0, stim_off = -1.0;
  sem::Workspace ws;
  sem::Timing timing;
  int64_t launches = 0;             // libsem kernels launched so far
  sem::Gmg* gmg = nullptr;          // built on first use of the multigrid preconditioner
  sem::Tape* tape = nullptr;        // recorded forward run for the adjoint
  int gmg_degree = 3, gmg_coarse_degree = 10, gmg_min_coarse_dofs = 2000;
  int gmg_precision = SEM_PREC_FP32;
  int op_precision = SEM_PREC_FP64;  // operator of the CG iterations: FP64 or DF64
  sem_state* host_state = nullptr;  // device copy of the state for sem_step_host
  // deterministic mode: element-local results of every apply and restriction,
  // summed per node in a fixed order (scratch of nelem n^3 doubles, fine level)
  bool deterministic = false;
  double* det_scratch = nullptr;
  // device address of sem_apply_dot_static's static scratch array in the CUDA
  // context this sem_ctx was created in (looked up on that entry point's first call)
  double* static_scratch = nullptr;
  // Initial residual of the next time step without an operator apply: each
  // step's solve starts from x0 = u^n, the previous step's solution, with the
  // same A (alpha and tissue unchanged), and that solve ended with
  // r = b_prev - A u^n, so A x0 = b_prev - r (kept in ws.Ax) and
  // r0 = b - A x0.  Valid for the state `st` at step `n` while nothing but time
  // steps touched the context (every other mutating entry point clears it);
  // refreshed by a real apply every kCarrySteps steps, which bounds the drift of
  // the recursively updated residual.
  struct ResidualCarry {
    bool valid = false;
    const sem_state* st = nullptr;
    int64_t n = -1;
    double alpha = 0.0;
    int precond = -1;
    int age = 0;
    // sem_step_host_out: the state's u^n comes from the caller's host array, so
    // the carry holds only if it equals, bit for bit, the solution the last call
    // left in the state's solution buffer.  The ionic update compares the two
    // while it reads u^n and clears *same on a difference; the solve then
    // applies the operator after all (device-side choice, no host round trip).
    int* same = nullptr;
  } carry;
  // The carry left by the last sem_step_host_out call (step index of the next
  // call, operator and age); any other entry point that mutates clears it.
  struct HostCarry {
    bool valid = false;
    int64_t n = -1;
    double alpha = 0.0;
    int precond = -1;
    int age = 0;
  } host_carry;
  // sem_step_host_out: a second stream for the copy of h^{n+1} to the host,
  // which the ionic update writes first thing in the step and which then
  // overlaps the linear solve (time_steps issues it when h_dst is set)
  struct HostCopies {
    cudaStream_t side = nullptr;
    cudaEvent_t ev_ionic = nullptr, ev_h = nullptr;
    double* h_dst = nullptr;
  } host_copies;
  std::string err;
};

struct sem_state {
  sem_ctx* ctx = nullptr;
  double* U[3] = {nullptr, nullptr, nullptr};
  double* H[3] = {nullptr, nullptr, nullptr};
  int cur = 0, prev = 1, next = 2;
  int64_t n = 0;
  // activation times (Eq. tau): running max |du/dt| per node and its time
  double* act_dmax = nullptr;
  double* act_tau = nullptr;
  bool act_track = false;
};

namespace sem {

// Solver entry points (sem_solver.cu); return SEM_* codes and set ctx->err.
int ensure_workspace(sem_ctx* ctx);
int apply_fp64(sem_ctx* ctx, double alpha, double beta, const double* u, double* y,
               cudaStream_t s);
// ax0: when set, A x for the initial residual r = b - A x is taken from it (and it
// is overwritten) instead of an operator apply.  ax0_ok (multigrid PCG only): a
// device flag; where it reads zero at the set-up the operator is applied after all.
int cg_solve(sem_ctx* ctx, double alpha, const double* b, double* x, double rtol, double atol,
             int maxit, int precond, int* iters, double* final_res, sem_stats* stats,
             cudaStream_t s, double* ax0 = nullptr, const int* ax0_ok = nullptr);
int time_steps(sem_ctx* ctx, sem_state* st, double dt, int nsteps, double rtol, double atol,
               int maxit, int precond, sem_stats* stats, cudaStream_t s);
int fail(sem_ctx* ctx, int code, const std::string& msg);
int apply_fp32(sem_ctx* ctx, double alpha, double beta, const float* u, float* y, bool bf16,
               cudaStream_t s);
int apply_df64(sem_ctx* ctx, double alpha, double beta, const double* u, double* y,
               cudaStream_t s);
// FP32 vectors, bf16 metric, tensor-core contractions (SEM-NI, p = 2..4).
int apply_tc(sem_ctx* ctx, double alpha, double beta, const float* u, float* y, cudaStream_t s);
// The FP64-vector operator the solvers use (FP64 or df64 arithmetic per ctx->op_precision);
// prepare_operator makes its metric copy and must run before any stream capture.
cudaError_t prepare_operator(sem_ctx* ctx, cudaStream_t s);
// Activation-time arrays of a state to (max |du/dt| = -1, tau = NaN).
cudaError_t activation_reset(sem_state* st, cudaStream_t s);
cudaError_t launch_operator(sem_ctx* ctx, const ApplyArgs64& a, cudaStream_t s);

// Geometric multigrid (sem_gmg.cu).
void gmg_free(sem_ctx* ctx);
int gmg_vcycle(sem_ctx* ctx, double alpha, const double* r, double* z, cudaStream_t s);
int gmg_pcg(sem_ctx* ctx, double alpha, const double* b, double* x, double rtol, double atol,
            int maxit, int* iters, double* final_res, sem_stats* stats, cudaStream_t s,
            double* ax0 = nullptr, const int* ax0_ok = nullptr);
int gmg_info(sem_ctx* ctx, double alpha, int max_levels, int* nlevels, int* p, int* dims,
             int64_t* ndofs, double* lambda_max, cudaStream_t s);

// Adjoint (sem_adjoint.cu).
void tape_free(sem_ctx* ctx);
int forward_record(sem_ctx* ctx, sem_state* st, double dt, int nsteps, int every,
                   const int* sensors, int nsens, double* traces, double rtol, double atol,
                   int maxit, int precond, sem_stats* stats, cudaStream_t s);
int adjoint_grad(sem_ctx* ctx, const double* trace_bar, double* g_sl, double* g_st, double* g_th,
                 double rtol, double atol, int maxit, int precond, sem_stats* stats,
                 cudaStream_t s);
int cuda_fail(sem_ctx* ctx, cudaError_t e, const char* what);

}  // namespace sem
