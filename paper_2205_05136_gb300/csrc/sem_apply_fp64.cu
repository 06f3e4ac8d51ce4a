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
  pdl_entry();
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
  launch_k(k_apply_dot_finish, 1, kApplyThreads, 0, s, partials, n, cg, out, done);
  return cudaGetLastError();
}

// y[g] += sum of the element contributions of node g (I, J, K); the elements
// holding it are ex in [lo(I), hi(I)] (two when I is a multiple of p inside
// the lattice, else one), likewise ey and ez, summed in ez, ey, ex order.
template <typename V>
__global__ void __launch_bounds__(256)
    k_assemble(int nx, int ny, int nz, int p, const V* __restrict__ yloc, V* __restrict__ y,
               const int* done) {
  pdl_entry();
  if (done != nullptr && *done) return;
  const int n = p + 1, n2 = n * n, n3 = n2 * n;
  const int64_t NX = (int64_t)p * nx + 1, NY = (int64_t)p * ny + 1, nd = NX * NY * ((int64_t)p * nz + 1);
  for (int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; g < nd;
       g += (int64_t)gridDim.x * blockDim.x) {
    const int I = (int)(g % NX), J = (int)((g / NX) % NY), K = (int)(g / (NX * NY));
    auto range = [p](int idx, int ne, int& lo, int& hi) {
      hi = min(idx / p, ne - 1);
      lo = (idx % p == 0 && idx > 0 && idx / p <= ne - 1) ? idx / p - 1 : hi;
    };
    int x0, x1, y0, y1, z0, z1;
    range(I, nx, x0, x1);
    range(J, ny, y0, y1);
    range(K, nz, z0, z1);
    V acc = V(0);
    for (int ez = z0; ez <= z1; ++ez)
      for (int ey = y0; ey <= y1; ++ey)
        for (int ex = x0; ex <= x1; ++ex) {
          const int64_t e = ex + (int64_t)nx * (ey + (int64_t)ny * ez);
          acc += yloc[e * n3 + (I - p * ex) + n * (J - p * ey) + n2 * (K - p * ez)];
        }
    y[g] += acc;
  }
}

template <typename V>
cudaError_t assemble_t(const Level& L, const V* yloc, V* y, const int* done, cudaStream_t s) {
  const int64_t want = (L.ndofs + 255) / 256;
  const int grid = (int)std::max<int64_t>(1, std::min<int64_t>(want, 152 * 16));
  launch_k(k_assemble<V>, grid, 256, 0, s, L.nx, L.ny, L.nz, L.p, yloc, y, done);
  return cudaGetLastError();
}

cudaError_t launch_assemble(const Level& L, const double* yloc, double* y, const int* done, cudaStream_t s) {
  return assemble_t(L, yloc, y, done, s);
}
cudaError_t launch_assemble(const Level& L, const float* yloc, float* y, const int* done, cudaStream_t s) {
  return assemble_t(L, yloc, y, done, s);
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
