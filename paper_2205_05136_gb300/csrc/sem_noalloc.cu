// sem_apply_dot_static: the FP64 operator apply fused with the inner product
// u . (A u), for callers that cannot allocate device memory.
//
// Why: sem_cg_solve and sem_step allocate their work vectors and reduction
// buffers on first use.  Some callers cannot do that -- code that runs while a
// CUDA stream capture is active (cudaMalloc is not permitted there), host
// frameworks that own every device allocation through their own arena or a
// fixed budget, and real-time loops that must not enter the allocator.  This
// entry point allocates nothing: the per-CTA partial sums of its inner product
// live in one file-scope static device array, and a one-CTA kernel launched
// after the apply adds them up.
//
// Limits and sharing:
//   * the array holds kStaticMaxCtas partial sums (512 KiB);
//     every GPU that loads libsem keeps it until the process exits;
//   * a mesh whose apply needs more CTAs than that is rejected (SEM_ERR_ARG);
//   * all calls share the array, and it keeps the last call's contents: calls
//     that overlap on the GPU (concurrent streams, or several contexts on one
//     device) race on it, so such calls must be ordered by the caller;
//   * the first call on a device looks up the array's device address with
//     cudaGetSymbolAddress (with that device current); make that first call
//     before any stream capture begins.
#include <cmath>
#include <mutex>
#include <string>

#include "sem_context.cuh"

namespace sem {
namespace {

constexpr int kStaticMaxCtas = 65536;
constexpr int kStaticMaxDevices = 64;

// Per-CTA partial sums of the inner product.
static __device__ __align__(256) double g_apply_dot_scratch[kStaticMaxCtas];

std::mutex g_scratch_mu;
double* g_scratch_addr[kStaticMaxDevices] = {};

// Device address of the static scratch on the current device (looked up once per device).
cudaError_t scratch_address(int device, double** out) {
  if (device < 0 || device >= kStaticMaxDevices) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(g_scratch_mu);
  if (g_scratch_addr[device] == nullptr) {
    void* p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_apply_dot_scratch);
    if (e != cudaSuccess) return e;
    g_scratch_addr[device] = static_cast<double*>(p);
  }
  *out = g_scratch_addr[device];
  return cudaSuccess;
}

bool on_device(const sem_ctx* ctx, const void* p) {
  if (p == nullptr) return false;
  cudaPointerAttributes at;
  if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  if (at.type == cudaMemoryTypeManaged) return true;
  return at.type == cudaMemoryTypeDevice && at.device == ctx->device;
}

}  // namespace
}  // namespace sem

using namespace sem;

extern "C" int sem_apply_dot_static(sem_ctx* ctx, double alpha, double beta, const double* u,
                                    double* y, double* dot, void* stream) {
  if (ctx == nullptr) return SEM_ERR_ARG;
  int prev = -1;
  if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
  if (prev != ctx->device) cudaSetDevice(ctx->device);
  struct Restore {
    int d;
    ~Restore() { if (d >= 0) cudaSetDevice(d); }
  } restore{prev};

  if (!on_device(ctx, u) || !on_device(ctx, y) || !on_device(ctx, dot))
    return fail(ctx, SEM_ERR_ARG, "u, y and dot must be device memory of the context's device");
  if (u == y) return fail(ctx, SEM_ERR_ARG, "u and y must not overlap");
  if (!std::isfinite(alpha) || !std::isfinite(beta) || beta == 0.0)
    return fail(ctx, SEM_ERR_ARG, "alpha must be finite and beta finite and nonzero");
  const Level& L = ctx->L;
  const int ctas = apply_grid_blocks(L);
  if (ctas > kStaticMaxCtas)
    return fail(ctx, SEM_ERR_ARG,
                "mesh needs " + std::to_string(ctas) + " CTAs; the static scratch of "
                "sem_apply_dot_static holds " + std::to_string(kStaticMaxCtas));
  double* scratch = nullptr;
  cudaError_t e = scratch_address(ctx->device, &scratch);
  if (e != cudaSuccess) return cuda_fail(ctx, e, "cudaGetSymbolAddress(static scratch)");
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  e = cudaMemsetAsync(y, 0, sizeof(double) * L.ndofs, s);
  if (e != cudaSuccess) return cuda_fail(ctx, e, "cudaMemsetAsync(y)");
  ApplyArgs64 a{};
  a.map = L.map;
  a.metric = L.metric;
  a.u = u;
  a.y = y;
  a.nelem = L.nelem;
  a.mass_coef = alpha / beta;
  a.out_scale = beta;
  a.scale_out = beta != 1.0;
  a.dot_partials = scratch;
  a.dot_out = dot;
  e = launch_apply_fp64(L, a, false, s);
  if (e != cudaSuccess) return cuda_fail(ctx, e, "apply kernel launch");
  return SEM_OK;
}
