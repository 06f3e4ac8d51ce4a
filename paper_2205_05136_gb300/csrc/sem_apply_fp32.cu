// FP32 instantiations of the matrix-free element kernel (float vectors and
// arithmetic; float or bfloat16 storage of the quadrature-point metric).
#include "sem_apply_kernel.cuh"

namespace sem {

cudaError_t launch_apply_fp32(const Level& L, const ApplyArgs<float, float>& a, bool mass_only,
                              cudaStream_t s) {
  return dispatch_apply<float, float>(L, a, mass_only, false, s);
}

cudaError_t launch_apply_bf16(const Level& L, const ApplyArgs<float, __nv_bfloat16>& a,
                              bool mass_only, cudaStream_t s) {
  return dispatch_apply<float, __nv_bfloat16>(L, a, mass_only, false, s);
}

cudaError_t prime_apply_kernels() {
  cudaError_t e = prime_all<float, float>();
  if (e != cudaSuccess) return e;
  if ((e = prime_all<float, __nv_bfloat16>()) != cudaSuccess) return e;
  return prime_apply_tc();
}

}  // namespace sem
