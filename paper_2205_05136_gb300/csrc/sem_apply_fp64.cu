// FP64 instantiations of the matrix-free element kernel.
#include "sem_apply_kernel.cuh"

namespace sem {

cudaError_t launch_apply_fp64(const Level& L, const ApplyArgs64& a, bool mass_only, cudaStream_t s) {
  return dispatch_apply<double, double>(L, a, mass_only, a.dot_partials != nullptr, s);
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
