// df64 instantiations of the matrix-free element kernel: FP64 vectors, the FP64
// metric split into FP32 pairs, and double-float arithmetic (sem_df64.cuh) on
// the FP32 pipe.
#include "sem_apply_kernel.cuh"

namespace sem {

cudaError_t launch_apply_df64(const Level& L, const ApplyArgs<df, df_pair>& a, bool mass_only,
                              cudaStream_t s) {
  return dispatch_apply<df, df_pair>(L, a, mass_only, a.dot_partials != nullptr, s);
}

}  // namespace sem
