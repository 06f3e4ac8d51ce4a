// C ABI of libsem (declared in include/sem.h): argument checking, context and
// state management, and dispatch to the setup, apply and solver layers.
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "sem_context.cuh"

using namespace sem;

namespace sem {
int apply_fp32(sem_ctx* ctx, double alpha, double beta, const float* u, float* y, bool bf16,
               cudaStream_t s);

bool pdl_enabled() {
  static const bool on = std::getenv("SEM_NO_PDL") == nullptr;
  return on;
}
}  // namespace sem

namespace {

thread_local std::string g_create_err;

// Entry points that change the operator, the preconditioner, a state or the CG
// workspace end the carried initial residual of consecutive time steps.
void invalidate_carry(sem_ctx* ctx) {
  if (ctx == nullptr) return;
  ctx->carry.valid = false;
  ctx->carry.same = nullptr;
  ctx->host_carry.valid = false;
}
// ... also on the way out, for entry points that step states of their own.
struct CarryScope {
  sem_ctx* ctx;
  ~CarryScope() { invalidate_carry(ctx); }
};
// sem_step_host_out: the state's own carry ends with the call, the one kept
// for the next call (host_carry) is set by the call itself.
struct StateCarryScope {
  sem_ctx* ctx;
  ~StateCarryScope() {
    ctx->carry.valid = false;
    ctx->carry.same = nullptr;
  }
};

struct DeviceGuard {
  int prev = -1;
  explicit DeviceGuard(int d) {
    if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
    if (prev != d) cudaSetDevice(d);
  }
  ~DeviceGuard() {
    if (prev >= 0) cudaSetDevice(prev);
  }
};

cudaStream_t as_stream(void* s) { return reinterpret_cast<cudaStream_t>(s); }

// Device memory of the context's device (or managed memory); host pointers are rejected.
bool is_device_ptr(const sem_ctx* ctx, const void* p) {
  if (p == nullptr) return false;
  cudaPointerAttributes at;
  if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  if (at.type == cudaMemoryTypeManaged) return true;
  return at.type == cudaMemoryTypeDevice && at.device == ctx->device;
}

bool is_host_ptr(const void* p) {
  if (p == nullptr) return false;
  cudaPointerAttributes at;
  if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
    cudaGetLastError();
    return true;  // unregistered host memory
  }
  return at.type == cudaMemoryTypeHost || at.type == cudaMemoryTypeUnregistered;
}

#define CK_CTX(ctx)                                      \
  do {                                                   \
    if ((ctx) == nullptr) return SEM_ERR_ARG;            \
  } while (0)

#define CK_DEV(ptr, name)                                                                 \
  do {                                                                                    \
    if (!is_device_ptr(ctx, (ptr)))                                                       \
      return fail(ctx, SEM_ERR_ARG, std::string(name) + " must be device memory of the context's device"); \
  } while (0)

#define SEM_CK(call)                                         \
  do {                                                       \
    cudaError_t e_ = (call);                                 \
    if (e_ != cudaSuccess) return cuda_fail(ctx, e_, #call); \
  } while (0)

void free_ctx(sem_ctx* ctx) {
  gmg_free(ctx);
  tape_free(ctx);
  cudaFree(ctx->L.dbg);  // shared with the multigrid levels, freed once here
  cudaFree(ctx->L.fault);  // the same
  level_free(ctx->L);
  cudaFree(ctx->sigma_l);
  cudaFree(ctx->sigma_t);
  cudaFree(ctx->theta);
  cudaFree(ctx->d_flag);
  cudaFree(ctx->stim_mask);
  Workspace& w = ctx->ws;
  cudaFree(w.r); cudaFree(w.z); cudaFree(w.p); cudaFree(w.Ap); cudaFree(w.invdiag);
  cudaFree(w.b); cudaFree(w.g); cudaFree(w.Ax); cudaFree(w.p2);
  cudaFree(ctx->det_scratch);
  cudaFree(w.cg);
  if (w.cg_host) cudaFreeHost(w.cg_host);
  cudaFree(w.vec_partials);
  cudaFree(w.tickets);
  cudaFree(w.apply_partials);
  cudaFree(w.dot_result);
  cudaFree(w.same);
  if (w.same_host) cudaFreeHost(w.same_host);
  if (w.fault_host) cudaFreeHost(w.fault_host);
}

__global__ void k_fill(int64_t n, double v, double* x) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    x[i] = v;
}

__global__ void k_axpby(int64_t n, double a, const double* __restrict__ x, double b,
                        const double* __restrict__ y, double* __restrict__ out) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    out[i] = a * x[i] + b * y[i];
}

int grid_for(int64_t n) {
  const int64_t g = (n + 255) / 256;
  return (int)std::max<int64_t>(1, std::min<int64_t>(g, 152 * 8));
}

// Builds the fine level (numbering, vertices, metric, node coordinates,
// diagonals) with the default tissue.
int build_level(sem_ctx* ctx, int nx, int ny, int nz, const double* vertices, int p, int quad,
                cudaStream_t s) {
  Level& L = ctx->L;
  ctx->vertices.assign(vertices, vertices + (size_t)(nx + 1) * (ny + 1) * (nz + 1) * 3);
  SEM_CK(level_create(L, nx, ny, nz, vertices, p, quad, true, s));
  SEM_CK(cudaMalloc(&ctx->sigma_l, sizeof(double) * L.nelem));
  SEM_CK(cudaMalloc(&ctx->sigma_t, sizeof(double) * L.nelem));
  SEM_CK(cudaMalloc(&ctx->theta, sizeof(double) * L.nelem));
  k_fill<<<grid_for(L.nelem), 256, 0, s>>>(L.nelem, 0.12, ctx->sigma_l);
  k_fill<<<grid_for(L.nelem), 256, 0, s>>>(L.nelem, 0.03, ctx->sigma_t);
  k_fill<<<grid_for(L.nelem), 256, 0, s>>>(L.nelem, 0.0, ctx->theta);
  SEM_CK(cudaGetLastError());
  SEM_CK(cudaMalloc(&ctx->d_flag, sizeof(int)));
  SEM_CK(cudaMemsetAsync(ctx->d_flag, 0, sizeof(int), s));
  SEM_CK(cudaMalloc(&L.fault, sizeof(unsigned)));
  SEM_CK(cudaMemsetAsync(L.fault, 0, sizeof(unsigned), s));
#ifdef SEM_DEBUG
  SEM_CK(cudaMalloc(&L.dbg, sizeof(unsigned long long)));
  SEM_CK(cudaMemsetAsync(L.dbg, 0, sizeof(unsigned long long), s));
#endif
  SEM_CK(setup_geometry(L, ctx->sigma_l, ctx->sigma_t, ctx->theta, ctx->d_flag, s));
  int bad = 0;
  SEM_CK(cudaMemcpyAsync(&bad, ctx->d_flag, sizeof(int), cudaMemcpyDeviceToHost, s));
  SEM_CK(cudaStreamSynchronize(s));
  if (bad) return fail(ctx, SEM_ERR_BAD_MESH, "non-positive Jacobian determinant at a quadrature point");
  SEM_CK(setup_node_coords(L, s));
  SEM_CK(setup_diagonals(L, s));
  SEM_CK(cudaStreamSynchronize(s));
  return SEM_OK;
}

}  // namespace

extern "C" {

// SEM_DEBUG build: after a call, the first out-of-range node index the kernels
// met (recorded instead of accessed) becomes SEM_ERR_ARG; the word is cleared.
// The normal build returns rc unchanged and does not synchronise.
int debug_check(sem_ctx* ctx, int rc, cudaStream_t s) {
#ifdef SEM_DEBUG
  if (ctx->L.dbg == nullptr) return rc;
  unsigned long long w = 0;
  if (cudaStreamSynchronize(s) != cudaSuccess ||
      cudaMemcpy(&w, ctx->L.dbg, sizeof(w), cudaMemcpyDeviceToHost) != cudaSuccess)
    return cuda_fail(ctx, cudaGetLastError(), "SEM_DEBUG index-error word");
  if (w == 0) return rc;
  cudaMemset(ctx->L.dbg, 0, sizeof(w));
  static const char* kinds[] = {"?", "gather", "scatter", "node line", "transfer"};
  const unsigned kind = (unsigned)(w >> 56);
  const int idx = (int)(uint32_t)(w & 0xffffffffull);
  return fail(ctx, SEM_ERR_ARG, std::string("SEM_DEBUG: ") + kinds[kind < 5 ? kind : 0] +
                                    " node index " + std::to_string(idx) + " outside [0, " +
                                    std::to_string(ctx->L.ndofs) + ") (access skipped)");
#else
  (void)ctx;
  (void)s;
  return rc;
#endif
}

#ifdef SEM_DEBUG
const char* sem_version(void) { return "libsem 0.2 (sm_103a, SEM_DEBUG index checks)"; }
#else
const char* sem_version(void) { return "libsem 0.2 (sm_103a)"; }
#endif

const char* sem_last_error(const sem_ctx* ctx) {
  if (ctx == nullptr) return g_create_err.c_str();
  return ctx->err.c_str();
}

int sem_create(sem_ctx** out, int nx, int ny, int nz, const double* vertices, int p, int quad,
               int device) {
  if (out == nullptr) { g_create_err = "out is NULL"; return SEM_ERR_ARG; }
  *out = nullptr;
  if (nx < 1 || ny < 1 || nz < 1) { g_create_err = "nx, ny, nz must be >= 1"; return SEM_ERR_ARG; }
  if (p < 1 || p > kMaxP) { g_create_err = "p must be in 1..6"; return SEM_ERR_ARG; }
  if (quad != SEM_QUAD_LG && quad != SEM_QUAD_LGL) { g_create_err = "bad quadrature"; return SEM_ERR_ARG; }
  if (vertices == nullptr) { g_create_err = "vertices is NULL"; return SEM_ERR_ARG; }
  const double ndofs = (double(p) * nx + 1) * (double(p) * ny + 1) * (double(p) * nz + 1);
  const double nel = double(nx) * ny * nz;
  if (ndofs >= 2147483647.0 || nel * (p + 1) * (p + 1) * (p + 1) >= 2147483647.0) {
    g_create_err = "mesh too large for 32-bit node indices";
    return SEM_ERR_ARG;
  }
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev) {
    cudaGetLastError();
    g_create_err = "invalid CUDA device";
    return SEM_ERR_ARG;
  }
  DeviceGuard guard(device);
  if (cudaError_t pe = prime_apply_kernels(); pe != cudaSuccess) {
    g_create_err = std::string("kernel attribute setup failed: ") + cudaGetErrorString(pe);
    return SEM_ERR_CUDA;
  }
  sem_ctx* ctx = new (std::nothrow) sem_ctx();
  if (!ctx) { g_create_err = "host allocation failed"; return SEM_ERR_NOMEM; }
  ctx->device = device;
  ctx->ionic = sem_ionic_params{-85.0, 100.0, 0.3, 6.0, 120.0, 150.0, 0.13, 0.01};
  cudaStream_t s = nullptr;
  if (cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) != cudaSuccess) {
    g_create_err = "cudaStreamCreate failed";
    delete ctx;
    return SEM_ERR_CUDA;
  }
  int rc = build_level(ctx, nx, ny, nz, vertices, p, quad, s);
  cudaStreamSynchronize(s);
  cudaStreamDestroy(s);
  if (rc != SEM_OK) {
    g_create_err = ctx->err;
    free_ctx(ctx);
    delete ctx;
    return rc;
  }
  *out = ctx;
  return SEM_OK;
}

int sem_destroy(sem_ctx* ctx) {
  if (ctx == nullptr) return SEM_OK;
  DeviceGuard guard(ctx->device);
  cudaDeviceSynchronize();
  if (ctx->host_state) sem_state_destroy(ctx->host_state);
  ctx->host_state = nullptr;
  auto& hc = ctx->host_copies;
  for (cudaEvent_t e : {hc.ev_ionic, hc.ev_h})
    if (e) cudaEventDestroy(e);
  if (hc.side) cudaStreamDestroy(hc.side);
  if (ctx->timing.start) cudaEventDestroy(ctx->timing.start);
  if (ctx->timing.stop) cudaEventDestroy(ctx->timing.stop);
  free_ctx(ctx);
  delete ctx;
  return SEM_OK;
}

int sem_num_dofs(const sem_ctx* ctx, int64_t* ndofs) {
  if (ctx == nullptr || ndofs == nullptr) return SEM_ERR_ARG;
  *ndofs = ctx->L.ndofs;
  return SEM_OK;
}

int sem_num_elements(const sem_ctx* ctx, int64_t* nelem) {
  if (ctx == nullptr || nelem == nullptr) return SEM_ERR_ARG;
  *nelem = ctx->L.nelem;
  return SEM_OK;
}

int sem_dof_coords(sem_ctx* ctx, double* xyz, void* stream) {
  CK_CTX(ctx);
  DeviceGuard guard(ctx->device);
  CK_DEV(xyz, "xyz");
  SEM_CK(cudaMemcpyAsync(xyz, ctx->L.xyz, sizeof(double) * 3 * ctx->L.ndofs,
                         cudaMemcpyDeviceToDevice, as_stream(stream)));
  return SEM_OK;
}

int sem_set_tissue(sem_ctx* ctx, const double* sigma_l, const double* sigma_t,
                   const double* theta, void* stream) {
  CK_CTX(ctx);
  invalidate_carry(ctx);
  DeviceGuard guard(ctx->device);
  CK_DEV(sigma_l, "sigma_l");
  CK_DEV(sigma_t, "sigma_t");
  CK_DEV(theta, "theta");
  cudaStream_t s = as_stream(stream);
  const size_t bytes = sizeof(double) * ctx->L.nelem;
  SEM_CK(cudaMemcpyAsync(ctx->sigma_l, sigma_l, bytes, cudaMemcpyDeviceToDevice, s));
  SEM_CK(cudaMemcpyAsync(ctx->sigma_t, sigma_t, bytes, cudaMemcpyDeviceToDevice, s));
  SEM_CK(cudaMemcpyAsync(ctx->theta, theta, bytes, cudaMemcpyDeviceToDevice, s));
  SEM_CK(setup_geometry(ctx->L, ctx->sigma_l, ctx->sigma_t, ctx->theta, ctx->d_flag, s));
  SEM_CK(setup_diagonals(ctx->L, s));
  ctx->ws.inv_alpha = -1.0;
  gmg_free(ctx);  // coarse levels inherit the tissue: rebuilt on next use
  return SEM_OK;
}

int sem_apply(sem_ctx* ctx, double alpha, double beta, const void* u, void* y, int precision,
              void* stream) {
  CK_CTX(ctx);
  DeviceGuard guard(ctx->device);
  CK_DEV(u, "u");
  CK_DEV(y, "y");
  if (u == y) return fail(ctx, SEM_ERR_ARG, "u and y must not overlap");
  if (!std::isfinite(alpha) || !std::isfinite(beta)) return fail(ctx, SEM_ERR_ARG, "alpha and beta must be finite");
  cudaStream_t s = as_stream(stream);
  int rc;
  switch (precision) {
    case SEM_PREC_FP64:
      rc = apply_fp64(ctx, alpha, beta, static_cast<const double*>(u), static_cast<double*>(y), s);
      break;
    case SEM_PREC_DF64:
      rc = apply_df64(ctx, alpha, beta, static_cast<const double*>(u), static_cast<double*>(y), s);
      break;
    case SEM_PREC_FP32:
      rc = apply_fp32(ctx, alpha, beta, static_cast<const float*>(u), static_cast<float*>(y), false, s);
      break;
    case SEM_PREC_FP32_BF16:
      rc = apply_fp32(ctx, alpha, beta, static_cast<const float*>(u), static_cast<float*>(y), true, s);
      break;
    case SEM_PREC_BF16_TC:
      rc = apply_tc(ctx, alpha, beta, static_cast<const float*>(u), static_cast<float*>(y), s);
      break;
    default:
      return fail(ctx, SEM_ERR_ARG, "unknown precision");
  }
  return debug_check(ctx, rc, s);
}

int sem_set_operator_precision(sem_ctx* ctx, int precision) {
  CK_CTX(ctx);
  invalidate_carry(ctx);
  if (precision != SEM_PREC_FP64 && precision != SEM_PREC_DF64)
    return fail(ctx, SEM_ERR_ARG, "operator precision must be SEM_PREC_FP64 or SEM_PREC_DF64");
  DeviceGuard guard(ctx->device);
  cudaDeviceSynchronize();
  ctx->op_precision = precision;
  gmg_free(ctx);  // captured graphs embed the operator kernel
  return SEM_OK;
}

int sem_set_deterministic(sem_ctx* ctx, int enable) {
  CK_CTX(ctx);
  invalidate_carry(ctx);
  DeviceGuard guard(ctx->device);
  cudaDeviceSynchronize();
  if (enable && ctx->det_scratch == nullptr) {
    const Level& L = ctx->L;
    const size_t n = (size_t)L.nelem * L.n * L.n * L.n;
    if (cudaMalloc(&ctx->det_scratch, sizeof(double) * n) != cudaSuccess) {
      cudaGetLastError();
      ctx->det_scratch = nullptr;
      return fail(ctx, SEM_ERR_NOMEM, "cannot allocate the element-local results of the deterministic mode");
    }
  }
  ctx->deterministic = enable != 0;
  gmg_free(ctx);  // captured graphs embed the apply and transfer kernels
  return SEM_OK;
}

int sem_diagonal(sem_ctx* ctx, double alpha, double beta, double* d, void* stream) {
  CK_CTX(ctx);
  DeviceGuard guard(ctx->device);
  CK_DEV(d, "d");
  const int64_t n = ctx->L.ndofs;
  k_axpby<<<grid_for(n), 256, 0, as_stream(stream)>>>(n, alpha, ctx->L.mdiag, beta, ctx->L.kdiag, d);
  SEM_CK(cudaGetLastError());
  return SEM_OK;
}

int sem_cg_solve(sem_ctx* ctx, double alpha, const double* b, double* x, double rtol,
                 double atol, int maxit, int precond, int* iters, double* final_res,
                 void* stream) {
  CK_CTX(ctx);
  invalidate_carry(ctx);
  DeviceGuard guard(ctx->device);
  CK_DEV(b, "b");
  CK_DEV(x, "x");
  if (b == x) return fail(ctx, SEM_ERR_ARG, "b and x must not overlap");
  if (maxit < 0 || !(rtol >= 0.0) || !(atol >= 0.0) || !std::isfinite(alpha))
    return fail(ctx, SEM_ERR_ARG, "bad solver parameters");
  const int rc = cg_solve(ctx, alpha, b, x, rtol, atol, maxit, precond, iters, final_res, nullptr,
                          as_stream(stream));
  return debug_check(ctx, rc, as_stream(stream));
}

int sem_set_ionic(sem_ctx* ctx, const sem_ionic_params* prm) {
  CK_CTX(ctx);
  if (prm == nullptr) return fail(ctx, SEM_ERR_ARG, "prm is NULL");
  if (!(prm->tau_in > 0) || !(prm->tau_out > 0) || !(prm->tau_open > 0) ||
      !(prm->tau_close > 0) || !(prm->kappa > 0) || !(prm->u_amp != 0))
    return fail(ctx, SEM_ERR_ARG, "time constants, kappa and u_amp must be positive");
  ctx->ionic = *prm;
  return SEM_OK;
}

int sem_set_stimulus(sem_ctx* ctx, int region, const double* params, double amplitude,
                     double t_on, double t_off, void* stream) {
  CK_CTX(ctx);
  DeviceGuard guard(ctx->device);
  if (params == nullptr) return fail(ctx, SEM_ERR_ARG, "params is NULL");
  if (region != SEM_REGION_BOX && region != SEM_REGION_SPHERE)
    return fail(ctx, SEM_ERR_ARG, "unknown region");
  if (!ctx->stim_mask) SEM_CK(cudaMalloc(&ctx->stim_mask, sizeof(double) * ctx->L.ndofs));
  SEM_CK(setup_region_mask(ctx->L, region, params, ctx->stim_mask, as_stream(stream)));
  ctx->stim_amp = amplitude;
  ctx->stim_on = t_on;
  ctx->stim_off = t_off;
  return SEM_OK;
}

int sem_state_create(sem_ctx* ctx, sem_state** out) {
  CK_CTX(ctx);
  if (out == nullptr) return fail(ctx, SEM_ERR_ARG, "out is NULL");
  *out = nullptr;
  DeviceGuard guard(ctx->device);
  sem_state* st = new (std::nothrow) sem_state();
  if (!st) return fail(ctx, SEM_ERR_NOMEM, "host allocation failed");
  st->ctx = ctx;
  for (int i = 0; i < 3; ++i) {
    if (cudaMalloc(&st->U[i], sizeof(double) * ctx->L.ndofs) != cudaSuccess ||
        cudaMalloc(&st->H[i], sizeof(double) * ctx->L.ndofs) != cudaSuccess) {
      cudaGetLastError();
      for (int j = 0; j < 3; ++j) { cudaFree(st->U[j]); cudaFree(st->H[j]); }
      delete st;
      return fail(ctx, SEM_ERR_NOMEM, "state allocation failed");
    }
  }
  *out = st;
  return SEM_OK;
}

int sem_state_destroy(sem_state* st) {
  if (st == nullptr) return SEM_OK;
  invalidate_carry(st->ctx);
  DeviceGuard guard(st->ctx->device);
  cudaDeviceSynchronize();
  for (int j = 0; j < 3; ++j) { cudaFree(st->U[j]); cudaFree(st->H[j]); }
  cudaFree(st->act_dmax);
  cudaFree(st->act_tau);
  delete st;
  return SEM_OK;
}

int sem_state_track_activation(sem_state* st, int enable, void* stream) {
  if (st == nullptr) return SEM_ERR_ARG;
  sem_ctx* ctx = st->ctx;
  DeviceGuard guard(ctx->device);
  if (!enable) {
    st->act_track = false;
    return SEM_OK;
  }
  const size_t bytes = sizeof(double) * ctx->L.ndofs;
  if (st->act_dmax == nullptr) {
    if (cudaMalloc(&st->act_dmax, bytes) != cudaSuccess || cudaMalloc(&st->act_tau, bytes) != cudaSuccess) {
      cudaGetLastError();
      cudaFree(st->act_dmax);
      cudaFree(st->act_tau);
      st->act_dmax = st->act_tau = nullptr;
      return fail(ctx, SEM_ERR_NOMEM, "activation arrays: allocation failed");
    }
  }
  SEM_CK(activation_reset(st, as_stream(stream)));
  st->act_track = true;
  return SEM_OK;
}

int sem_state_get_activation(sem_state* st, double* tau, double* dudt_max, void* stream) {
  if (st == nullptr) return SEM_ERR_ARG;
  sem_ctx* ctx = st->ctx;
  DeviceGuard guard(ctx->device);
  if (st->act_dmax == nullptr) return fail(ctx, SEM_ERR_ARG, "activation tracking was never enabled");
  const size_t bytes = sizeof(double) * ctx->L.ndofs;
  cudaStream_t s = as_stream(stream);
  if (tau != nullptr) {
    CK_DEV(tau, "tau");
    SEM_CK(cudaMemcpyAsync(tau, st->act_tau, bytes, cudaMemcpyDeviceToDevice, s));
  }
  if (dudt_max != nullptr) {
    CK_DEV(dudt_max, "dudt_max");
    SEM_CK(cudaMemcpyAsync(dudt_max, st->act_dmax, bytes, cudaMemcpyDeviceToDevice, s));
  }
  return SEM_OK;
}

int sem_state_set(sem_state* st, const double* u0, const double* h0, void* stream) {
  if (st == nullptr) return SEM_ERR_ARG;
  sem_ctx* ctx = st->ctx;
  invalidate_carry(ctx);
  DeviceGuard guard(ctx->device);
  CK_DEV(u0, "u0");
  CK_DEV(h0, "h0");
  cudaStream_t s = as_stream(stream);
  const size_t bytes = sizeof(double) * ctx->L.ndofs;
  st->cur = 0; st->prev = 1; st->next = 2; st->n = 0;
  SEM_CK(cudaMemcpyAsync(st->U[0], u0, bytes, cudaMemcpyDeviceToDevice, s));
  SEM_CK(cudaMemcpyAsync(st->U[1], u0, bytes, cudaMemcpyDeviceToDevice, s));
  SEM_CK(cudaMemcpyAsync(st->H[0], h0, bytes, cudaMemcpyDeviceToDevice, s));
  SEM_CK(cudaMemcpyAsync(st->H[1], h0, bytes, cudaMemcpyDeviceToDevice, s));
  return SEM_OK;
}

int sem_state_get(sem_state* st, double* u, double* u_prev, double* h, double* h_prev,
                  int64_t* n_out, void* stream) {
  if (st == nullptr) return SEM_ERR_ARG;
  sem_ctx* ctx = st->ctx;
  DeviceGuard guard(ctx->device);
  cudaStream_t s = as_stream(stream);
  const size_t bytes = sizeof(double) * ctx->L.ndofs;
  double* dst[4] = {u, u_prev, h, h_prev};
  const double* src[4] = {st->U[st->cur], st->U[st->prev], st->H[st->cur], st->H[st->prev]};
  const char* names[4] = {"u", "u_prev", "h", "h_prev"};
  for (int i = 0; i < 4; ++i) {
    if (dst[i] == nullptr) continue;
    CK_DEV(dst[i], names[i]);
    SEM_CK(cudaMemcpyAsync(dst[i], src[i], bytes, cudaMemcpyDeviceToDevice, s));
  }
  if (n_out) *n_out = st->n;
  return SEM_OK;
}

int sem_state_restore(sem_state* st, const double* u, const double* u_prev, const double* h,
                      const double* h_prev, int64_t n, void* stream) {
  if (st == nullptr) return SEM_ERR_ARG;
  sem_ctx* ctx = st->ctx;
  invalidate_carry(ctx);
  DeviceGuard guard(ctx->device);
  if (n < 0) return fail(ctx, SEM_ERR_ARG, "n must be >= 0");
  CK_DEV(u, "u");
  CK_DEV(h, "h");
  if (n > 0) {
    CK_DEV(u_prev, "u_prev");
    CK_DEV(h_prev, "h_prev");
  }
  cudaStream_t s = as_stream(stream);
  const size_t bytes = sizeof(double) * ctx->L.ndofs;
  st->cur = 0; st->prev = 1; st->next = 2; st->n = n;
  SEM_CK(cudaMemcpyAsync(st->U[0], u, bytes, cudaMemcpyDeviceToDevice, s));
  SEM_CK(cudaMemcpyAsync(st->U[1], n > 0 ? u_prev : u, bytes, cudaMemcpyDeviceToDevice, s));
  SEM_CK(cudaMemcpyAsync(st->H[0], h, bytes, cudaMemcpyDeviceToDevice, s));
  SEM_CK(cudaMemcpyAsync(st->H[1], n > 0 ? h_prev : h, bytes, cudaMemcpyDeviceToDevice, s));
  return SEM_OK;
}

int sem_step(sem_ctx* ctx, sem_state* st, double dt, int nsteps, double rtol, double atol,
             int maxit, int precond, sem_stats* stats, void* stream) {
  CK_CTX(ctx);
  if (st == nullptr || st->ctx != ctx) return fail(ctx, SEM_ERR_ARG, "state does not belong to ctx");
  if (!(dt > 0.0) || nsteps < 0 || maxit < 0 || !(rtol >= 0.0) || !(atol >= 0.0))
    return fail(ctx, SEM_ERR_ARG, "bad step parameters");
  DeviceGuard guard(ctx->device);
  sem_stats local{};
  sem_stats* sp = stats ? stats : &local;
  std::memset(sp, 0, sizeof(*sp));
  const double ms0 = ctx->timing.ms;
  const int64_t c0 = ctx->timing.count;
  const double sm0 = ctx->timing.smoother_ms;
  const int64_t sc0 = ctx->timing.smoother_count;
  const int64_t l0 = ctx->launches;
  const int rc = time_steps(ctx, st, dt, nsteps, rtol, atol, maxit, precond, sp, as_stream(stream));
  sp->apply_ms = ctx->timing.ms - ms0;
  sp->n_apply = ctx->timing.count - c0;
  sp->smoother_apply_ms = ctx->timing.smoother_ms - sm0;
  sp->n_smoother_apply = ctx->timing.smoother_count - sc0;
  sp->kernel_launches = ctx->launches - l0;
  return debug_check(ctx, rc, as_stream(stream));
}

int sem_step_host(sem_ctx* ctx, double* u, double* u_prev, double* h, double* h_prev, int64_t n,
                  double dt, double rtol, double atol, int maxit, int precond, sem_stats* stats,
                  void* stream) {
  CK_CTX(ctx);
  invalidate_carry(ctx);
  CarryScope carry_scope{ctx};
  DeviceGuard guard(ctx->device);
  if (!is_host_ptr(u) || !is_host_ptr(u_prev) || !is_host_ptr(h) || !is_host_ptr(h_prev))
    return fail(ctx, SEM_ERR_ARG, "u, u_prev, h, h_prev must be host memory");
  if (n < 0) return fail(ctx, SEM_ERR_ARG, "n must be >= 0");
  if (ctx->host_state == nullptr) {
    int rc = sem_state_create(ctx, &ctx->host_state);
    if (rc != SEM_OK) return rc;
  }
  sem_state* st = ctx->host_state;
  cudaStream_t s = as_stream(stream);
  const size_t bytes = sizeof(double) * ctx->L.ndofs;
  st->cur = 0; st->prev = 1; st->next = 2; st->n = n;
  SEM_CK(cudaMemcpyAsync(st->U[0], u, bytes, cudaMemcpyHostToDevice, s));
  SEM_CK(cudaMemcpyAsync(st->U[1], u_prev, bytes, cudaMemcpyHostToDevice, s));
  SEM_CK(cudaMemcpyAsync(st->H[0], h, bytes, cudaMemcpyHostToDevice, s));
  SEM_CK(cudaMemcpyAsync(st->H[1], h_prev, bytes, cudaMemcpyHostToDevice, s));
  int rc = sem_step(ctx, st, dt, 1, rtol, atol, maxit, precond, stats, stream);
  if (rc != SEM_OK) return rc;
  SEM_CK(cudaMemcpyAsync(u_prev, st->U[st->prev], bytes, cudaMemcpyDeviceToHost, s));
  SEM_CK(cudaMemcpyAsync(h_prev, st->H[st->prev], bytes, cudaMemcpyDeviceToHost, s));
  SEM_CK(cudaMemcpyAsync(u, st->U[st->cur], bytes, cudaMemcpyDeviceToHost, s));
  SEM_CK(cudaMemcpyAsync(h, st->H[st->cur], bytes, cudaMemcpyDeviceToHost, s));
  SEM_CK(cudaStreamSynchronize(s));
  return SEM_OK;
}

namespace {
// Device address of page-locked host memory (mapped into the device's address
// space), or nullptr for pageable memory.
double* mapped_ptr(const void* p) {
  cudaPointerAttributes at;
  if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
    cudaGetLastError();
    return nullptr;
  }
  return at.type == cudaMemoryTypeHost ? static_cast<double*>(at.devicePointer) : nullptr;
}

bool overlaps(const void* a, const void* b, size_t bytes) {
  const char* x = static_cast<const char*>(a);
  const char* y = static_cast<const char*>(b);
  return x < y + bytes && y < x + bytes;
}
}  // namespace

int sem_step_host_out(sem_ctx* ctx, const double* u, const double* u_prev, const double* h,
                      const double* h_prev, double* u_next, double* h_next, int64_t n, double dt,
                      double rtol, double atol, int maxit, int precond, sem_stats* stats, void* stream) {
  CK_CTX(ctx);
  const sem_ctx::HostCarry hcy = ctx->host_carry;
  invalidate_carry(ctx);
  StateCarryScope carry_scope{ctx};
  DeviceGuard guard(ctx->device);
  const void* all[6] = {u, u_prev, h, h_prev, u_next, h_next};
  for (const void* p : all)
    if (!is_host_ptr(p)) return fail(ctx, SEM_ERR_ARG, "u, u_prev, h, h_prev, u_next, h_next must be host memory");
  if (n < 0) return fail(ctx, SEM_ERR_ARG, "n must be >= 0");
  const size_t bytes = sizeof(double) * ctx->L.ndofs;
  for (int o = 4; o < 6; ++o)
    for (int i = 0; i < 6; ++i)
      if (i != o && overlaps(all[o], all[i], bytes))
        return fail(ctx, SEM_ERR_ARG, "u_next and h_next must not overlap any other array");
  if (ctx->host_state == nullptr) {
    int rc = sem_state_create(ctx, &ctx->host_state);
    if (rc != SEM_OK) return rc;
  }
  sem_state* st = ctx->host_state;
  cudaStream_t s = as_stream(stream);
  // Page-locked inputs are read in place by the ionic update, over the host
  // link while it computes (measured faster than copy-engine transfers of the
  // four inputs on two streams); pageable arrays are staged through the
  // state's device buffers.  h^{n+1} goes to the host on a second stream as
  // soon as the ionic update has written it (time_steps issues that copy), so
  // that it overlaps the linear solve; u^{n+1} follows the solve.
  auto& hc = ctx->host_copies;
  if (hc.side == nullptr) {
    SEM_CK(cudaStreamCreateWithFlags(&hc.side, cudaStreamNonBlocking));
    for (cudaEvent_t* e : {&hc.ev_ionic, &hc.ev_h}) SEM_CK(cudaEventCreateWithFlags(e, cudaEventDisableTiming));
  }
  sem_state view = *st;
  view.cur = 0; view.prev = 1; view.next = 2; view.n = n;
  const double* in[4] = {u, u_prev, h, h_prev};
  double* dev_in[4] = {st->U[0], st->U[1], st->H[0], st->H[1]};
  double* use[4];
  for (int i = 0; i < 4; ++i) {
    use[i] = mapped_ptr(in[i]);
    if (use[i] == nullptr) {
      SEM_CK(cudaMemcpyAsync(dev_in[i], in[i], bytes, cudaMemcpyHostToDevice, s));
      use[i] = dev_in[i];
    }
  }
  view.U[0] = use[0]; view.U[1] = use[1]; view.H[0] = use[2]; view.H[1] = use[3];
  view.U[2] = st->U[2];
  view.H[2] = st->H[2];
  // The last call left its u^{n+1} in U[2] and A u^{n+1} in the workspace.  If
  // this call continues it (n, operator) and its u is that u^{n+1}, the solve
  // takes the initial residual from there: the ionic update compares u with
  // U[2] as it overwrites U[2] by the warm start, and the set-up applies the
  // operator after all where they differ.
  int rc = ensure_workspace(ctx);
  if (rc != SEM_OK) return rc;
  const bool checked = hcy.valid && hcy.n == n && precond == SEM_PC_GMG;
  if (checked) {
    sem_ctx::ResidualCarry& cy = ctx->carry;
    cy.valid = true;
    cy.st = &view;
    cy.n = n;
    cy.alpha = hcy.alpha;
    cy.precond = hcy.precond;
    cy.age = hcy.age;
    cy.same = ctx->ws.same;
  }
  hc.h_dst = h_next;
  rc = sem_step(ctx, &view, dt, 1, rtol, atol, maxit, precond, stats, stream);
  hc.h_dst = nullptr;
  if (rc != SEM_OK) {
    cudaStreamSynchronize(hc.side);
    return rc;
  }
  // whether this call's solve used the carry (time_steps does not count checked ones)
  const bool used_check = ctx->carry.valid && ctx->carry.age > 0 && checked;
  if (used_check) SEM_CK(cudaMemcpyAsync(ctx->ws.same_host, ctx->ws.same, sizeof(int), cudaMemcpyDeviceToHost, s));
  SEM_CK(cudaMemcpyAsync(u_next, st->U[2], bytes, cudaMemcpyDeviceToHost, s));
  SEM_CK(cudaStreamWaitEvent(s, hc.ev_h, 0));
  SEM_CK(cudaStreamSynchronize(s));
  const bool carried = used_check && *ctx->ws.same_host != 0;
  if (stats && carried) stats->carried_solves += 1;
  // for the next call: its n, this solve's operator, and the carry's age
  const sem_ctx::ResidualCarry& cy = ctx->carry;
  if (cy.valid) {
    sem_ctx::HostCarry& next = ctx->host_carry;
    next.valid = true;
    next.n = n + 1;
    next.alpha = cy.alpha;
    next.precond = cy.precond;
    next.age = carried ? cy.age : 0;
  }
  return SEM_OK;
}

int sem_set_gmg(sem_ctx* ctx, int degree, int coarse_degree, int min_coarse_dofs, int precision) {
  CK_CTX(ctx);
  invalidate_carry(ctx);
  if (degree < 1 || degree > 20 || coarse_degree < 1 || coarse_degree > 200 || min_coarse_dofs < 1)
    return fail(ctx, SEM_ERR_ARG, "bad multigrid parameters");
  if (precision != SEM_PREC_FP64 && precision != SEM_PREC_FP32 && precision != SEM_PREC_FP32_BF16 &&
      precision != SEM_PREC_BF16_TC)
    return fail(ctx, SEM_ERR_ARG, "unknown precision");
  if (precision == SEM_PREC_BF16_TC && ctx->L.quad != SEM_QUAD_LGL)
    return fail(ctx, SEM_ERR_UNSUPPORTED, "tensor-core V-cycle needs SEM-NI (SEM_QUAD_LGL)");
  DeviceGuard guard(ctx->device);
  cudaDeviceSynchronize();
  gmg_free(ctx);
  ctx->gmg_degree = degree;
  ctx->gmg_coarse_degree = coarse_degree;
  ctx->gmg_min_coarse_dofs = min_coarse_dofs;
  ctx->gmg_precision = precision;
  return SEM_OK;
}

int sem_vcycle(sem_ctx* ctx, double alpha, const double* r, double* z, void* stream) {
  CK_CTX(ctx);
  invalidate_carry(ctx);
  DeviceGuard guard(ctx->device);
  CK_DEV(r, "r");
  CK_DEV(z, "z");
  if (!(alpha >= 0.0) || !std::isfinite(alpha)) return fail(ctx, SEM_ERR_ARG, "alpha must be finite and >= 0");
  return debug_check(ctx, gmg_vcycle(ctx, alpha, r, z, as_stream(stream)), as_stream(stream));
}

int sem_debug_set_map_entry(sem_ctx* ctx, int64_t entry, int value, int* previous) {
  CK_CTX(ctx);
  invalidate_carry(ctx);
#ifdef SEM_DEBUG
  const Level& L = ctx->L;
  if (entry < 0 || entry >= (int64_t)L.nelem * L.n * L.n * L.n)
    return fail(ctx, SEM_ERR_ARG, "entry outside the element-to-DOF map");
  DeviceGuard guard(ctx->device);
  int old = 0;
  if (cudaMemcpy(&old, L.map + entry, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess ||
      cudaMemcpy(L.map + entry, &value, sizeof(int), cudaMemcpyHostToDevice) != cudaSuccess)
    return cuda_fail(ctx, cudaGetLastError(), "map entry");
  if (previous != nullptr) *previous = old;
  return SEM_OK;
#else
  (void)entry;
  (void)value;
  (void)previous;
  return fail(ctx, SEM_ERR_UNSUPPORTED, "sem_debug_set_map_entry needs the SEM_DEBUG build");
#endif
}

int sem_debug_hold_copy(sem_ctx* ctx, int group) {
  CK_CTX(ctx);
#ifdef SEM_DEBUG
  if (group < -1) return fail(ctx, SEM_ERR_ARG, "group must be >= -1");
  invalidate_carry(ctx);
  DeviceGuard guard(ctx->device);
  cudaDeviceSynchronize();
  gmg_free(ctx);  // the multigrid graphs hold the launch arguments, this one included
  ctx->L.hold = group;
  return SEM_OK;
#else
  (void)group;
  return fail(ctx, SEM_ERR_UNSUPPORTED, "sem_debug_hold_copy needs the SEM_DEBUG build");
#endif
}

int sem_gmg_info(sem_ctx* ctx, double alpha, int max_levels, int* nlevels, int* p, int* dims,
                 int64_t* ndofs, double* lambda_max, void* stream) {
  CK_CTX(ctx);
  if (max_levels < 0) return fail(ctx, SEM_ERR_ARG, "max_levels must be >= 0");
  DeviceGuard guard(ctx->device);
  return gmg_info(ctx, alpha, max_levels, nlevels, p, dims, ndofs, lambda_max, as_stream(stream));
}

int sem_forward_record(sem_ctx* ctx, sem_state* st, double dt, int nsteps, int checkpoint_every,
                       const int* sensors, int nsens, double* traces, double rtol, double atol,
                       int maxit, int precond, sem_stats* stats, void* stream) {
  CK_CTX(ctx);
  invalidate_carry(ctx);
  if (st == nullptr || st->ctx != ctx) return fail(ctx, SEM_ERR_ARG, "state does not belong to ctx");
  if (!(dt > 0.0) || nsteps < 1 || checkpoint_every < 1 || nsens < 1 || maxit < 0 ||
      !(rtol >= 0.0) || !(atol >= 0.0))
    return fail(ctx, SEM_ERR_ARG, "bad recording parameters");
  DeviceGuard guard(ctx->device);
  CK_DEV(sensors, "sensors");
  CK_DEV(traces, "traces");
  {  // sensor indices must address nodes
    std::vector<int> h(nsens);
    SEM_CK(cudaMemcpy(h.data(), sensors, sizeof(int) * nsens, cudaMemcpyDeviceToHost));
    for (int v : h)
      if (v < 0 || v >= ctx->L.ndofs) return fail(ctx, SEM_ERR_ARG, "sensor index out of range");
  }
  sem_stats local{};
  sem_stats* sp = stats ? stats : &local;
  std::memset(sp, 0, sizeof(*sp));
  const int64_t l0 = ctx->launches;
  const int rc = forward_record(ctx, st, dt, nsteps, checkpoint_every, sensors, nsens, traces, rtol,
                                atol, maxit, precond, sp, as_stream(stream));
  sp->kernel_launches = ctx->launches - l0;
  return rc;
}

int sem_adjoint_grad(sem_ctx* ctx, const double* trace_bar, double* g_sigma_l, double* g_sigma_t,
                     double* g_theta, double rtol, double atol, int maxit, int precond,
                     sem_stats* stats, void* stream) {
  CK_CTX(ctx);
  invalidate_carry(ctx);
  CarryScope carry_scope{ctx};
  if (maxit < 0 || !(rtol >= 0.0) || !(atol >= 0.0)) return fail(ctx, SEM_ERR_ARG, "bad solver parameters");
  DeviceGuard guard(ctx->device);
  CK_DEV(trace_bar, "trace_bar");
  CK_DEV(g_sigma_l, "g_sigma_l");
  CK_DEV(g_sigma_t, "g_sigma_t");
  CK_DEV(g_theta, "g_theta");
  sem_stats local{};
  sem_stats* sp = stats ? stats : &local;
  std::memset(sp, 0, sizeof(*sp));
  const int64_t l0 = ctx->launches;
  const int rc = adjoint_grad(ctx, trace_bar, g_sigma_l, g_sigma_t, g_theta, rtol, atol, maxit,
                              precond, sp, as_stream(stream));
  sp->kernel_launches = ctx->launches - l0;
  return rc;
}

int sem_set_timing(sem_ctx* ctx, int enable) {
  CK_CTX(ctx);
  ctx->timing.enabled = enable != 0;
  ctx->timing.solves = 0;
  return SEM_OK;
}

}  // extern "C"
