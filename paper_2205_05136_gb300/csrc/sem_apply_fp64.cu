// FP64 instantiations of the matrix-free element kernel.
#include "sem_apply_kernel.cuh"

namespace sem {

cudaError_t launch_apply_fp64(const Level& L, const ApplyArgs64& a, bool mass_only, cudaStream_t s) {
  return dispatch_apply<double, double>(L, a, mass_only, a.dot_partials != nullptr, s);
}

// One CTA of kApplyThreads threads: each thread adds the partials b = t,
// t + kApplyThreads, ... in order, then a fixed-shape tree (block_sum) adds
// the threads' sums, so the total does not depend on the order in which the
// apply's CTAs ran.  The stream order after the apply makes its partials visible.
__global__ void __launch_bounds__(kApplyThreads)
    k_apply_dot_finish(const double* __restrict__ partials, int n, CgScalars* cg, double* out,
                       const int* done) {
  __shared__ double red[32];
  if (done != nullptr && *done) return;
  double v = 0.0;
  for (int b = threadIdx.x; b < n; b += kApplyThreads) v += partials[b];
  v = block_sum(v, red);
  if (threadIdx.x == 0) {
    if (cg != nullptr) {
      cg->pAp = v;
      cg->alpha = cg->rz / v;
    } else if (out != nullptr) {
      *out = v;
    }
  }
}

cudaError_t launch_apply_dot_finish(const double* partials, int n, CgScalars* cg, double* out,
                                    const int* done, cudaStream_t s) {
  k_apply_dot_finish<<<1, kApplyThreads, 0, s>>>(partials, n, cg, out, done);
  return cudaGetLastError();
}

int apply_grid_blocks(const Level& L) {
  int E = 1;
  switch (L.p) {
    case 1: E = ApplyCfg<1>::E; break;
    case 2: E = ApplyCfg<2>::E; break;
    case 3: E = ApplyCfg<3>::E; break;
    case 4: E = ApplyCfg<4>::E; break;
    case 5: E = ApplyCfg<5>::E; break;
    case 6: E = ApplyCfg<6>::E; break;
    default: return 0;
  }
  return (L.nelem + E - 1) / E;
}

}  // namespace sem
