// p-multigrid transfers between Q_pf and Q_pc on the same mesh, by sum
// factorization (Section 4.3: transfers are matrix-vector products).
//
//   prolongation  x_f += P x_c:  per element, coarse nodal values -> fine nodes
//                 through the 1-D interpolation matrix P[i_f][a_c] = l^c_a(x^f_i)
//                 applied along x, y, z; each fine node is written by one
//                 element (the highest-index element holding it), which also
//                 clears the fine work vector t there;
//   restriction   b_c += P^T (b_f - t_f): the fine residual, divided by the
//                 number of elements sharing each node, goes through P^T along
//                 x, y, z and is scatter-added to the coarse nodes.
// Mapping as in the operator kernel: E elements per CTA in shared memory, one
// 1-D line per thread and sweep, the matrix in the kernel-parameter bank.
#include "sem_apply_kernel.cuh"
#include "sem_context.cuh"

namespace sem {
namespace {

constexpr int kTThreads = 256;

template <int NF, int NC, typename T>
struct PMat {
  T P[NF][NC];
};

template <int NF> struct TransferCfg { static constexpr int E = (256 + NF * NF - 1) / (NF * NF); };

// out[i] = sum_a P[i][a] in[a]  (NC -> NF)
template <int NF, int NC, typename T>
__device__ __forceinline__ void up_line(const T (&P)[NF][NC], const T (&in)[NC], T (&out)[NF]) {
#pragma unroll
  for (int i = 0; i < NF; ++i) {
    T acc = P[i][0] * in[0];
#pragma unroll
    for (int a = 1; a < NC; ++a) acc = fma(P[i][a], in[a], acc);
    out[i] = acc;
  }
}

// out[a] = sum_i P[i][a] in[i]  (NF -> NC)
template <int NF, int NC, typename T>
__device__ __forceinline__ void down_line(const T (&P)[NF][NC], const T (&in)[NF], T (&out)[NC]) {
#pragma unroll
  for (int a = 0; a < NC; ++a) {
    T acc = P[0][a] * in[0];
#pragma unroll
    for (int i = 1; i < NF; ++i) acc = fma(P[i][a], in[i], acc);
    out[a] = acc;
  }
}

// Position flags of the CTA's elements, computed once per element (the slab
// coordinates need divisions by the runtime mesh sizes): bit 0 ex > 0, bit 1
// ex < nx - 1, bit 2 ey > 0, bit 3 ey < ny - 1, bit 4 ez > 0, bit 5
// ez < nz - 1, bit 6 the element exists.  The caller synchronises.
template <int E>
__device__ __forceinline__ void element_flags(int e0, int nelem, int nx, int ny, int nz,
                                              unsigned char (&fl)[E]) {
  if (threadIdx.x < E) {
    const int e = e0 + threadIdx.x;
    unsigned f = 0;
    if (e < nelem) {
      const int ex = e % nx, ey = (e / nx) % ny, ez = e / (nx * ny);
      f = (ex > 0 ? 1u : 0u) | (ex < nx - 1 ? 2u : 0u) | (ey > 0 ? 4u : 0u) | (ey < ny - 1 ? 8u : 0u) |
          (ez > 0 ? 16u : 0u) | (ez < nz - 1 ? 32u : 0u) | 64u;
    }
    fl[threadIdx.x] = (unsigned char)f;
  }
}

// Loops of the transfer kernels run over compile-time trip counts
// (kTThreads threads per CTA in every launch), so the per-node index
// arithmetic divides by constants only and the gathers of all iterations are
// in flight together.
template <int NF, int NC, typename T>
__global__ void __launch_bounds__(kTThreads)
    k_prolong_sf(int nelem, int nx, int ny, int nz, const int* __restrict__ map_c,
                 const int* __restrict__ map_f, const __grid_constant__ PMat<NF, NC, T> pm,
                 const T* __restrict__ xc, T* __restrict__ xf, T* __restrict__ tf, int64_t ndf,
                 int64_t ndc, unsigned long long* dbg, const int* done) {
  pdl_entry();
  if (done != nullptr && *done) return;
  constexpr int E = TransferCfg<NF>::E;
  constexpr int NF3 = NF * NF * NF, NC3 = NC * NC * NC;
  __shared__ T c0[E * NC3];
  __shared__ T s1[E * NC * NC * NF];  // [k_c][j_c][i_f]
  __shared__ T s2[E * NC * NF * NF];  // [k_c][j_f][i_f]
  __shared__ unsigned char fl[E];
  const int e0 = blockIdx.x * E;
  element_flags<E>(e0, nelem, nx, ny, nz, fl);
  {
    const int nv = min(E, nelem - e0) * NC3;  // coarse values of the CTA's elements
    const int* gm = map_c + (size_t)e0 * NC3;
    constexpr int IT = (E * NC3 + kTThreads - 1) / kTThreads;
#pragma unroll
    for (int it = 0; it < IT; ++it) {
      const int idx = threadIdx.x + it * kTThreads;
      if (IT * kTThreads == E * NC3 || idx < E * NC3)
        c0[idx] = idx < nv ? xc[SEM_IDX(__ldg(gm + idx), ndc, dbg, kDbgTransfer)] : T(0);
    }
  }
  __syncthreads();
  for (int w = threadIdx.x; w < E * NC * NC; w += kTThreads) {  // x-lines (j_c, k_c)
    const int s = w / (NC * NC), l = w - s * NC * NC;
    T in[NC], out[NF];
#pragma unroll
    for (int a = 0; a < NC; ++a) in[a] = c0[s * NC3 + l * NC + a];
    up_line<NF, NC>(pm.P, in, out);
#pragma unroll
    for (int i = 0; i < NF; ++i) s1[s * NC * NC * NF + l * NF + i] = out[i];
  }
  __syncthreads();
  for (int w = threadIdx.x; w < E * NC * NF; w += kTThreads) {  // y-lines (i_f, k_c)
    const int s = w / (NC * NF), l = w - s * NC * NF, i = l % NF, k = l / NF;
    T in[NC], out[NF];
#pragma unroll
    for (int b = 0; b < NC; ++b) in[b] = s1[s * NC * NC * NF + (k * NC + b) * NF + i];
    up_line<NF, NC>(pm.P, in, out);
#pragma unroll
    for (int j = 0; j < NF; ++j) s2[s * NC * NF * NF + (k * NF + j) * NF + i] = out[j];
  }
  __syncthreads();
  for (int w = threadIdx.x; w < E * NF * NF; w += kTThreads) {  // z-lines (i_f, j_f)
    const int s = w / (NF * NF), l = w - s * NF * NF, i = l % NF, j = l / NF;
    const unsigned f = fl[s];
    if (!(f & 64u)) continue;
    T in[NC], out[NF];
#pragma unroll
    for (int c = 0; c < NC; ++c) in[c] = s2[s * NC * NF * NF + (c * NF + j) * NF + i];
    up_line<NF, NC>(pm.P, in, out);
    // the element owns its nodes except those on its upper faces that a next
    // element shares (ex < nx - 1 at i = NF - 1, and likewise in y and z)
    const bool own_xy = (i < NF - 1 || !(f & 2u)) && (j < NF - 1 || !(f & 8u));
    if (!own_xy) continue;
    const int* gm = map_f + (size_t)(e0 + s) * NF3 + j * NF + i;
#pragma unroll
    for (int k = 0; k < NF; ++k) {
      if (k == NF - 1 && (f & 32u)) continue;
      const int64_t g = SEM_IDX(__ldg(gm + k * NF * NF), ndf, dbg, kDbgTransfer);
      xf[g] += out[k];
      tf[g] = T(0);
    }
  }
}

template <int NF, int NC, typename T>
__global__ void __launch_bounds__(kTThreads)
    k_restrict_sf(int nelem, int nx, int ny, int nz, const int* __restrict__ map_c,
                  const int* __restrict__ map_f, const __grid_constant__ PMat<NF, NC, T> pm,
                  const T* __restrict__ bf, const T* __restrict__ tf, T* __restrict__ bc,
                  T* __restrict__ bloc, int64_t ndf, int64_t ndc, unsigned long long* dbg,
                  const int* done) {
  pdl_entry();
  if (done != nullptr && *done) return;
  constexpr int E = TransferCfg<NF>::E;
  constexpr int NF3 = NF * NF * NF, NC3 = NC * NC * NC;
  __shared__ T f0[E * NF3];
  __shared__ T s1[E * NF * NF * NC];  // [k_f][j_f][a]
  __shared__ T s2[E * NF * NC * NC];  // [k_f][b][a]
  __shared__ unsigned char fl[E];
  const int e0 = blockIdx.x * E;
  element_flags<E>(e0, nelem, nx, ny, nz, fl);
  __syncthreads();
  {
    const int* gm = map_f + (size_t)e0 * NF3;
    constexpr int IT = (E * NF3 + kTThreads - 1) / kTThreads;
#pragma unroll
    for (int it = 0; it < IT; ++it) {
      const int idx = threadIdx.x + it * kTThreads;
      if (IT * kTThreads == E * NF3 || idx < E * NF3) {
        const int s = idx / NF3, loc = idx - s * NF3;
        const unsigned f = fl[s];
        T v = T(0);
        if (f & 64u) {
          const int i = loc % NF, j = (loc / NF) % NF, k = loc / (NF * NF);
          // 1 / multiplicity of the node (elements sharing it): a power of two, exact
          const T w = (((i == 0 && (f & 1u)) || (i == NF - 1 && (f & 2u))) ? T(0.5) : T(1)) *
                      (((j == 0 && (f & 4u)) || (j == NF - 1 && (f & 8u))) ? T(0.5) : T(1)) *
                      (((k == 0 && (f & 16u)) || (k == NF - 1 && (f & 32u))) ? T(0.5) : T(1));
          const int64_t g = SEM_IDX(__ldg(gm + idx), ndf, dbg, kDbgTransfer);
          v = (bf[g] - tf[g]) * w;
        }
        f0[idx] = v;
      }
    }
  }
  __syncthreads();
  for (int w = threadIdx.x; w < E * NF * NF; w += kTThreads) {  // x-lines (j_f, k_f)
    const int s = w / (NF * NF), l = w - s * NF * NF;
    T in[NF], out[NC];
#pragma unroll
    for (int i = 0; i < NF; ++i) in[i] = f0[s * NF3 + l * NF + i];
    down_line<NF, NC>(pm.P, in, out);
#pragma unroll
    for (int a = 0; a < NC; ++a) s1[s * NF * NF * NC + l * NC + a] = out[a];
  }
  __syncthreads();
  for (int w = threadIdx.x; w < E * NF * NC; w += kTThreads) {  // y-lines (a, k_f)
    const int s = w / (NF * NC), l = w - s * NF * NC, a = l % NC, k = l / NC;
    T in[NF], out[NC];
#pragma unroll
    for (int j = 0; j < NF; ++j) in[j] = s1[s * NF * NF * NC + (k * NF + j) * NC + a];
    down_line<NF, NC>(pm.P, in, out);
#pragma unroll
    for (int b = 0; b < NC; ++b) s2[s * NF * NC * NC + (k * NC + b) * NC + a] = out[b];
  }
  __syncthreads();
  for (int w = threadIdx.x; w < E * NC * NC; w += kTThreads) {  // z-lines (a, b)
    const int s = w / (NC * NC), l = w - s * NC * NC, a = l % NC, b = l / NC;
    if (!(fl[s] & 64u)) continue;
    T in[NF], out[NC];
#pragma unroll
    for (int k = 0; k < NF; ++k) in[k] = s2[s * NF * NC * NC + (k * NC + b) * NC + a];
    down_line<NF, NC>(pm.P, in, out);
    if (bloc != nullptr) {  // deterministic mode: coarse-element results, assembled afterwards
#pragma unroll
      for (int c = 0; c < NC; ++c) bloc[(size_t)(e0 + s) * NC3 + c * NC * NC + b * NC + a] = out[c];
      continue;
    }
    const int* gm = map_c + (size_t)(e0 + s) * NC3 + b * NC + a;
#pragma unroll
    for (int c = 0; c < NC; ++c) atomicAdd(bc + SEM_IDX(__ldg(gm + c * NC * NC), ndc, dbg, kDbgTransfer), out[c]);
  }
}

template <int NF, int NC, typename T>
cudaError_t launch_pair(bool prolong, const Level& F, const Level& C, const double (*P)[kMaxN],
                        const T* src_b, const T* src_t, T* dst, T* dst_t, T* loc, const int* done,
                        cudaStream_t s) {
  PMat<NF, NC, T> pm;
  for (int i = 0; i < NF; ++i)
    for (int a = 0; a < NC; ++a) pm.P[i][a] = (T)P[i][a];
  const int E = TransferCfg<NF>::E;
  const int grid = (F.nelem + E - 1) / E;
  if (prolong)
    launch_k(k_prolong_sf<NF, NC, T>, grid, kTThreads, 0, s, F.nelem, F.nx, F.ny, F.nz, C.map, F.map, pm,
                                                       src_b, dst, dst_t, F.ndofs, C.ndofs, F.dbg, done);
  else
    launch_k(k_restrict_sf<NF, NC, T>, grid, kTThreads, 0, s, F.nelem, F.nx, F.ny, F.nz, C.map, F.map, pm,
                                                        src_b, src_t, dst, loc, F.ndofs, C.ndofs, F.dbg,
                                                        done);
  const cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess || prolong || loc == nullptr) return e;
  return launch_assemble(C, loc, dst, done, s);
}

}  // namespace

// prolong: dst (fine x) += P src_b (coarse x), dst_t (fine t) cleared.
// restrict: dst (coarse b) += P^T (src_b - src_t) (fine b, fine t); with loc set
// (deterministic mode) through coarse-element results in loc and the
// fixed-order node sums instead of atomic adds.
template <typename T>
cudaError_t p_transfer(bool prolong, const Level& F, const Level& C, const double (*P)[kMaxN],
                       const T* src_b, const T* src_t, T* dst, T* dst_t, T* loc, const int* done,
                       cudaStream_t s) {
  const int nf = F.n, nc = C.n;
#define SEM_PAIR(A, B) \
  if (nf == A && nc == B) return launch_pair<A, B, T>(prolong, F, C, P, src_b, src_t, dst, dst_t, loc, done, s);
  SEM_PAIR(7, 4)
  SEM_PAIR(6, 3)
  SEM_PAIR(5, 3)
  SEM_PAIR(4, 2)
  SEM_PAIR(3, 2)
  SEM_PAIR(7, 2)
  SEM_PAIR(6, 2)
  SEM_PAIR(5, 2)
#undef SEM_PAIR
  return cudaErrorInvalidValue;
}

template cudaError_t p_transfer<float>(bool, const Level&, const Level&, const double (*)[kMaxN],
                                       const float*, const float*, float*, float*, float*, const int*,
                                       cudaStream_t);
template cudaError_t p_transfer<double>(bool, const Level&, const Level&, const double (*)[kMaxN],
                                        const double*, const double*, double*, double*, double*,
                                        const int*, cudaStream_t);

}  // namespace sem
