// sem_apply_dot_static: the FP64 operator apply fused with the inner product
// u . (A u), for callers that cannot allocate device memory.
//
// Why: sem_cg_solve and sem_step allocate their work vectors and reduction
// buffers on first use.  Some callers cannot let a library do that: host
// frameworks that own every device allocation through their own arena or a
// fixed memory budget, and real-time loops that must not enter the allocator
// (cudaMalloc can synchronise the device and its latency is unbounded).  This
// entry point allocates nothing: the per-CTA partial sums of its inner product
// live in one file-scope static device array, and a one-CTA kernel launched
// after the apply adds them up.
//
// Limits and sharing:
//   * the array holds kStaticMaxCtas partial sums (512 KiB); every CUDA
//     context that loads libsem holds its own copy until the process exits;
//   * a mesh whose apply needs more CTAs than that is rejected (SEM_ERR_ARG);
//   * the calls made in one CUDA context share that context's array, and it
//     keeps the last call's contents: calls that overlap on the GPU
//     (concurrent streams, or several sem_ctx of one CUDA context) race on it,
//     so the caller must order them;
//   * the first call on a sem_ctx looks up the array's device address with
//     cudaGetSymbolAddress (the sem_ctx's device current) and keeps it in the
//     sem_ctx; make that first call before any stream capture begins.  A
//     cudaDeviceReset invalidates every sem_ctx of the device, this address
//     with them: create new contexts after a reset.
#include <cmath>
#include <string>

#include "sem_context.cuh"

namespace sem {
namespace {

constexpr int kStaticMaxCtas = 65536;

// Per-CTA partial sums of the inner product.
static __device__ __align__(256) double g_apply_dot_scratch[kStaticMaxCtas];

// Device address of the static scratch in the current CUDA context, kept in the
// sem_ctx after the first lookup.  Each CUDA context has its own copy of the
// array, so the address belongs to the context the sem_ctx's memory lives in.
cudaError_t scratch_address(sem_ctx* ctx, double** out) {
  if (ctx->static_scratch == nullptr) {
    void* p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_apply_dot_scratch);
    if (e != cudaSuccess) return e;
    ctx->static_scratch = static_cast<double*>(p);
  }
  *out = ctx->static_scratch;
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

// True when the byte ranges [a, a + na) and [b, b + nb) share a byte.
bool overlap(const void* a, size_t na, const void* b, size_t nb) {
  const uintptr_t a0 = reinterpret_cast<uintptr_t>(a), b0 = reinterpret_cast<uintptr_t>(b);
  return a0 < b0 + nb && b0 < a0 + na;
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
  const Level& L = ctx->L;
  const size_t vb = sizeof(double) * (size_t)L.ndofs;
  if (overlap(u, vb, y, vb) || overlap(dot, sizeof(double), u, vb) ||
      overlap(dot, sizeof(double), y, vb))
    return fail(ctx, SEM_ERR_ARG, "u, y and dot must not overlap");
  if (!std::isfinite(alpha) || !std::isfinite(beta) || beta == 0.0)
    return fail(ctx, SEM_ERR_ARG, "alpha must be finite and beta finite and nonzero");
  const int ctas = apply_grid_blocks(L);
  if (ctas > kStaticMaxCtas)
    return fail(ctx, SEM_ERR_ARG,
                "mesh needs " + std::to_string(ctas) + " CTAs; the static scratch of "
                "sem_apply_dot_static holds " + std::to_string(kStaticMaxCtas));
  double* scratch = nullptr;
  cudaError_t e = scratch_address(ctx, &scratch);
  if (e != cudaSuccess) return cuda_fail(ctx, e, "cudaGetSymbolAddress(static scratch)");
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  e = cudaMemsetAsync(y, 0, vb, s);
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
  ctx->launches += 2;  // the apply and the kernel that sums its partials
  return SEM_OK;
}
