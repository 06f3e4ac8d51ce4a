// Matrix-free element kernel of the SEM / SEM-NI operator (Algorithm 1's
// vectorized cell loop, Section 4) with sum factorization (Section 4.1):
//
//   y += sum_e  P_e^T (mass_coef M_e + K_e) P_e u          (P_e: gather through the map)
//
// per element, with n = p + 1 points per direction:
//   SEM-NI (LGL quadrature on the nodes):
//     g_d   = D along direction d of u_e                    3 sweeps
//     q     = G g,  m = mass_coef W u                       per quadrature point
//     y_e   = m + sum_d D^T along d of q_d                  3 sweeps
//   SEM (LG quadrature):
//     u_q   = Bi (x) Bi (x) Bi u_e                          3 sweeps to the Gauss points
//     g_d   = Dg along d of u_q  (collocation derivative on the Gauss points)
//     q, m  as above at the Gauss points
//     y_e   = Bi^T (x) Bi^T (x) Bi^T (m + sum_d Dg^T along d of q_d)
//
// GPU mapping: one CTA holds E elements in shared memory (three n^3 tiles per
// element).  A sweep along x or y gives each thread one 1-D line of n values
// (n^2 FMAs on registers, matrix entries read from the kernel-parameter bank);
// the z-sweep, the quadrature-point stage and the transposed z-sweep run on
// the (i, j) columns in registers.  The result is scatter-added with
// atomicAdd (RED) through the element-to-DOF map.
#pragma once

#include "sem_internal.cuh"

namespace sem {

constexpr int kApplyThreads = 256;

// Elements per CTA: E * n^2 close to the 256 threads of the CTA.
template <int P> struct ApplyCfg;
template <> struct ApplyCfg<1> { static constexpr int E = 64; };
template <> struct ApplyCfg<2> { static constexpr int E = 28; };
template <> struct ApplyCfg<3> { static constexpr int E = 16; };
template <> struct ApplyCfg<4> { static constexpr int E = 10; };
template <> struct ApplyCfg<5> { static constexpr int E = 7; };
template <> struct ApplyCfg<6> { static constexpr int E = 5; };

__device__ __forceinline__ double ldmetric(const double* p) { return __ldg(p); }
__device__ __forceinline__ float ldmetric(const float* p) { return __ldg(p); }
__device__ __forceinline__ float ldmetric(const __nv_bfloat16* p) {
  return __bfloat162float(__ldg(p));
}
__device__ __forceinline__ df ldmetric(const df_pair* p) {
  const float2 v = __ldg(reinterpret_cast<const float2*>(p));
  return df(v.x, v.y);
}

// Scatter-add of one element result; exact-match overloads so that no value is
// converted between precisions.
__device__ __forceinline__ void scatter_add(double* p, double v) { atomicAdd(p, v); }
__device__ __forceinline__ void scatter_add(float* p, float v) { atomicAdd(p, v); }
__device__ __forceinline__ void scatter_add(double* p, df v) { atomicAdd(p, (double)v); }

// Base offset and stride of line l of an n^3 tile along direction DIR
// (0: x-line (j,k), l = j + n k; 1: y-line (i,k), l = i + n k; 2: z-line (i,j), l = i + n j).
template <int N, int DIR>
__device__ __forceinline__ void line_geom(int l, int& base, int& stride) {
  if (DIR == 0) { base = l * N; stride = 1; }
  else if (DIR == 1) { const int i = l % N, k = l / N; base = k * N * N + i; stride = N; }
  else { base = l; stride = N * N; }
}

// out[q] = sum_l M[q][l] in[l]
template <int N, typename T>
__device__ __forceinline__ void mat_line(const T (&M)[N][N], const T (&in)[N], T (&out)[N]) {
#pragma unroll
  for (int q = 0; q < N; ++q) {
    T acc = M[q][0] * in[0];
#pragma unroll
    for (int l = 1; l < N; ++l) acc = fma(M[q][l], in[l], acc);
    out[q] = acc;
  }
}

// out[l] = sum_q M[q][l] in[q]  (ACC: out[l] += ...)
template <int N, bool ACC, typename T>
__device__ __forceinline__ void matT_line(const T (&M)[N][N], const T (&in)[N], T (&out)[N]) {
#pragma unroll
  for (int l = 0; l < N; ++l) {
    T acc;
    if (ACC) {
      acc = out[l];
#pragma unroll
      for (int q = 0; q < N; ++q) acc = fma(M[q][l], in[q], acc);
    } else {
      acc = M[0][l] * in[0];
#pragma unroll
      for (int q = 1; q < N; ++q) acc = fma(M[q][l], in[q], acc);
    }
    out[l] = acc;
  }
}

// dst = M along DIR of src, for every line of the E element tiles (thread tid
// of a group of nth threads).
template <int N, int E, int DIR, typename T>
__device__ __forceinline__ void sweep(const T (&M)[N][N], const T* src, T* dst, int tid, int nth) {
  constexpr int N2 = N * N, N3 = N2 * N;
  for (int w = tid; w < E * N2; w += nth) {
    const int s = w / N2, l = w - s * N2;
    int base, stride;
    line_geom<N, DIR>(l, base, stride);
    const T* ps = src + s * N3 + base;
    T* pd = dst + s * N3 + base;
    T in[N], out[N];
#pragma unroll
    for (int t = 0; t < N; ++t) in[t] = ps[t * stride];
    mat_line<N>(M, in, out);
#pragma unroll
    for (int t = 0; t < N; ++t) pd[t * stride] = out[t];
  }
}

// dst = M^T along DIR of src (ACC: dst += M^T src).  src may equal dst.
template <int N, int E, int DIR, bool ACC, typename T>
__device__ __forceinline__ void sweepT(const T (&M)[N][N], const T* src, T* dst, int tid, int nth) {
  constexpr int N2 = N * N, N3 = N2 * N;
  for (int w = tid; w < E * N2; w += nth) {
    const int s = w / N2, l = w - s * N2;
    int base, stride;
    line_geom<N, DIR>(l, base, stride);
    const T* ps = src + s * N3 + base;
    T* pd = dst + s * N3 + base;
    T in[N], out[N];
#pragma unroll
    for (int t = 0; t < N; ++t) in[t] = ps[t * stride];
    if (ACC) {
#pragma unroll
      for (int t = 0; t < N; ++t) out[t] = pd[t * stride];
    }
    matT_line<N, ACC>(M, in, out);
#pragma unroll
    for (int t = 0; t < N; ++t) pd[t * stride] = out[t];
  }
}

// Block-wide sum of v (all threads must call); result valid in thread 0.
__device__ __forceinline__ double block_sum(double v, double* red) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (lane == 0) red[warp] = v;
  __syncthreads();
  v = 0.0;
  if (warp == 0) {
    const int nw = (blockDim.x + 31) >> 5;
    v = (lane < nw) ? red[lane] : 0.0;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  }
  return v;
}

// Writes this block's partial; the last block to arrive sums all partials in
// block order (deterministic) and returns true in its thread 0 with *total set.
__device__ __forceinline__ bool finish_reduction(double partial, double* partials,
                                                 unsigned int* ticket, double* total,
                                                 double* red) {
  __shared__ bool is_last;
  if (threadIdx.x == 0) {
    partials[blockIdx.x] = partial;
    __threadfence();
    const unsigned int t = atomicAdd(ticket, 1u);
    is_last = (t == gridDim.x - 1);
  }
  __syncthreads();
  if (!is_last) return false;
  __threadfence();
  double v = 0.0;
  // fixed assignment of partials to threads, then a fixed-shape tree
  for (int b = threadIdx.x; b < (int)gridDim.x; b += blockDim.x)
    v += ((volatile double*)partials)[b];
  v = block_sum(v, red);
  if (threadIdx.x == 0) {
    *total = v;
    *ticket = 0u;
  }
  return threadIdx.x == 0;
}

// Shared-memory bytes of one CTA: three n^3 tiles per element, plus, when
// StageMetric is set, the CTA's metric block staged by cp.async at kernel entry
// (16-byte aligned thanks to the padded metric layout).  Staging is off: on
// GB300 the extra 36 KB per CTA halves the resident CTAs of the FP32 kernel and
// measured slower (p = 4: 63 us against 58 us per launch), because the gather
// and scatter latencies then overlap less.
template <typename T> struct StageMetric { static constexpr bool value = false; };

template <int P, typename T, typename MT>
__host__ __device__ constexpr size_t apply_tile_bytes() {
  return ((size_t)3 * ApplyCfg<P>::E * (P + 1) * (P + 1) * (P + 1) * sizeof(T) + 15) / 16 * 16;
}
template <int P, typename T>
__host__ __device__ constexpr size_t apply_warp_tile_bytes();
template <int P, typename T, typename MT>
__host__ __device__ constexpr size_t apply_smem_bytes() {
  return apply_tile_bytes<P, T, MT>() +
         (StageMetric<T>::value ? (size_t)ApplyCfg<P>::E * kMetricComps * padded_n3(P + 1) * sizeof(MT) : 0);
}

__device__ __forceinline__ float ldsmetric(const float* p) { return *p; }
__device__ __forceinline__ float ldsmetric(const __nv_bfloat16* p) { return __bfloat162float(*p); }
__device__ __forceinline__ double ldsmetric(const double* p) { return *p; }
__device__ __forceinline__ df ldsmetric(const df_pair* p) { return df(p->h, p->l); }

// Warp-per-element mode (WARP): each warp of the CTA owns one element and
// synchronises with __syncwarp only, so the warps of an SM run their gather,
// sweep, metric and scatter phases independently.  Used for the FP32 kernels,
// which are bound by memory latency rather than by arithmetic.
constexpr int kWarpsPerCta = kApplyThreads / 32;

// Elements per warp in warp mode: G n^2 lines close to 32 lanes (p <= 4).
template <int P> struct WarpCfg { static constexpr int G = 1; };
template <> struct WarpCfg<1> { static constexpr int G = 8; };
template <> struct WarpCfg<2> { static constexpr int G = 3; };
template <> struct WarpCfg<3> { static constexpr int G = 2; };

template <int P, typename T>
__host__ __device__ constexpr size_t apply_warp_tile_bytes() {
  return (size_t)3 * kWarpsPerCta * WarpCfg<P>::G * (P + 1) * (P + 1) * (P + 1) * sizeof(T);
}

template <int P, int QUAD, typename T, typename MT, bool DOT, bool MASS_ONLY, bool WARP = false>
__global__ void __launch_bounds__(kApplyThreads)
    sem_apply_kernel(const ApplyArgs<T, MT> a, const __grid_constant__ KTab<P + 1, T> tab) {
  static_assert(!(WARP && DOT), "the fused inner product needs the CTA-wide mode");
  constexpr int N = P + 1, N2 = N * N, N3 = N2 * N, N3P = padded_n3(N);
  constexpr int E = WARP ? WarpCfg<P>::G : ApplyCfg<P>::E;
  constexpr bool STAGE = StageMetric<T>::value && !MASS_ONLY && !WARP;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int warp = threadIdx.x >> 5;
  const int tid = WARP ? (threadIdx.x & 31) : threadIdx.x;
  const int nth = WARP ? 32 : blockDim.x;
  T* sA = reinterpret_cast<T*>(smem_raw) + (WARP ? warp * 3 * E * N3 : 0);
  T* sB = sA + E * N3;
  T* sC = sB + E * N3;
  MT* sM = reinterpret_cast<MT*>(smem_raw + apply_tile_bytes<P, T, MT>());
  __shared__ double red[32];
  auto group_sync = [] {
    if (WARP) __syncwarp(); else __syncthreads();
  };

  if (a.done != nullptr && *a.done) return;
  const int e0 = WARP ? (blockIdx.x * kWarpsPerCta + warp) * E : blockIdx.x * E;
  if (WARP && e0 >= a.nelem) return;  // no CTA-wide barrier follows in this mode

  if (STAGE) {  // the CTA's metric block: contiguous, 16-byte aligned, a multiple of 16 bytes
    const int ne = min(E, a.nelem - e0);
    const size_t bytes = (size_t)ne * kMetricComps * N3P * sizeof(MT);
    const char* src = reinterpret_cast<const char*>(a.metric + (size_t)e0 * kMetricComps * N3P);
    const unsigned dst = (unsigned)__cvta_generic_to_shared(sM);
    for (size_t off = (size_t)threadIdx.x * 16; off < bytes; off += (size_t)blockDim.x * 16)
      asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(dst + (unsigned)off),
                   "l"(src + off)
                   : "memory");
    asm volatile("cp.async.commit_group;\n" ::: "memory");
  }

  // gather u_e = P_e u
  for (int idx = tid; idx < E * N3; idx += nth) {
    const int s = idx / N3, loc = idx - s * N3, e = e0 + s;
    sA[idx] = (e < a.nelem) ? T(a.u[__ldg(a.map + (size_t)e * N3 + loc)]) : T(0);
  }
  group_sync();

  if (QUAD == SEM_QUAD_LG) {  // values at the Gauss points
    sweep<N, E, 0>(tab.Bi, sA, sB, tid, nth);
    group_sync();
    sweep<N, E, 1>(tab.Bi, sB, sC, tid, nth);
    group_sync();
    sweep<N, E, 2>(tab.Bi, sC, sA, tid, nth);
    group_sync();
  }

  if (MASS_ONLY) {
    for (int idx = tid; idx < E * N3; idx += nth) {
      const int s = idx / N3, loc = idx - s * N3, e = e0 + s;
      if (e < a.nelem) {
        const T W = ldmetric(a.metric + ((size_t)e * kMetricComps + 6) * N3P + loc);
        sA[idx] = (a.mass_coef * W) * sA[idx];
      }
    }
    group_sync();
  } else {
    // reference gradient along x and y (into sB, sC)
    sweep<N, E, 0>(tab.D, sA, sB, tid, nth);
    sweep<N, E, 1>(tab.D, sA, sC, tid, nth);
    if (STAGE) asm volatile("cp.async.wait_all;\n" ::: "memory");
    group_sync();
    // z-gradient, quadrature-point stage and transposed z-sweep on the columns
    for (int w = tid; w < E * N2; w += nth) {
      const int s = w / N2, c = w - s * N2, e = e0 + s;
      if (e >= a.nelem) continue;
      T* pa = sA + s * N3 + c;
      T* pb = sB + s * N3 + c;
      T* pc = sC + s * N3 + c;
      T uz[N], g3[N], q3[N], m[N];
#pragma unroll
      for (int k = 0; k < N; ++k) uz[k] = pa[k * N2];
      mat_line<N>(tab.D, uz, g3);
      const MT* mp = STAGE ? sM + (size_t)s * kMetricComps * N3P + c
                           : a.metric + (size_t)e * kMetricComps * N3P + c;
#pragma unroll
      for (int k = 0; k < N; ++k) {
        const T g1 = pb[k * N2], g2 = pc[k * N2];
        T G00, G01, G02, G11, G12, G22, W;
        if (STAGE) {
          G00 = ldsmetric(mp + 0 * N3P + k * N2);
          G01 = ldsmetric(mp + 1 * N3P + k * N2);
          G02 = ldsmetric(mp + 2 * N3P + k * N2);
          G11 = ldsmetric(mp + 3 * N3P + k * N2);
          G12 = ldsmetric(mp + 4 * N3P + k * N2);
          G22 = ldsmetric(mp + 5 * N3P + k * N2);
          W = ldsmetric(mp + 6 * N3P + k * N2);
        } else {
          G00 = ldmetric(mp + 0 * N3P + k * N2);
          G01 = ldmetric(mp + 1 * N3P + k * N2);
          G02 = ldmetric(mp + 2 * N3P + k * N2);
          G11 = ldmetric(mp + 3 * N3P + k * N2);
          G12 = ldmetric(mp + 4 * N3P + k * N2);
          G22 = ldmetric(mp + 5 * N3P + k * N2);
          W = ldmetric(mp + 6 * N3P + k * N2);
        }
        pb[k * N2] = fma(G02, g3[k], fma(G01, g2, G00 * g1));
        pc[k * N2] = fma(G12, g3[k], fma(G11, g2, G01 * g1));
        q3[k] = fma(G22, g3[k], fma(G12, g2, G02 * g1));
        m[k] = (a.mass_coef * W) * uz[k];
      }
      matT_line<N, true>(tab.D, q3, m);
#pragma unroll
      for (int k = 0; k < N; ++k) pa[k * N2] = m[k];
    }
    group_sync();
    sweepT<N, E, 1, true>(tab.D, sC, sA, tid, nth);
    group_sync();
    sweepT<N, E, 0, true>(tab.D, sB, sA, tid, nth);
    group_sync();
  }

  if (QUAD == SEM_QUAD_LG) {  // back from the Gauss points to the nodes
    sweepT<N, E, 0, false>(tab.Bi, sA, sB, tid, nth);
    group_sync();
    sweepT<N, E, 1, false>(tab.Bi, sB, sC, tid, nth);
    group_sync();
    sweepT<N, E, 2, false>(tab.Bi, sC, sA, tid, nth);
    group_sync();
  }

  // scatter-add y += P_e^T y_e
  double dot = 0.0;
  for (int idx = tid; idx < E * N3; idx += nth) {
    const int s = idx / N3, loc = idx - s * N3, e = e0 + s;
    if (e < a.nelem) {
      const int g = __ldg(a.map + (size_t)e * N3 + loc);
      T v = sA[idx];
      if (a.scale_out) v *= a.out_scale;
      scatter_add(a.y + g, v);
      if (DOT) dot = fma((double)a.u[g], (double)v, dot);
    }
  }
  if (DOT) {
    double bs = block_sum(dot, red);
    double total;
    if (finish_reduction(bs, a.dot_partials, a.dot_ticket, &total, red)) {
      if (a.cg != nullptr) {
        a.cg->pAp = total;
        a.cg->alpha = a.cg->rz / total;
      } else if (a.dot_out != nullptr) {
        *a.dot_out = total;
      }
    }
  }
}

// Launch helper shared by the precision-specific translation units.
template <int P, int QUAD, typename T, typename MT>
cudaError_t launch_apply_t(const Level& L, const ApplyArgs<T, MT>& a, bool mass_only, bool dot,
                           cudaStream_t s) {
  constexpr int N = P + 1;
  KTab<N, T> tab;
  for (int q = 0; q < N; ++q)
    for (int l = 0; l < N; ++l) {
      tab.D[q][l] = (T)(QUAD == SEM_QUAD_LG ? L.tab.Dg[q][l] : L.tab.D[q][l]);
      tab.Bi[q][l] = (T)L.tab.Bi[q][l];
    }
  const int E = ApplyCfg<P>::E;
  const int grid = (L.nelem + E - 1) / E;
  if (grid == 0) return cudaSuccess;
  constexpr size_t tiles = apply_tile_bytes<P, T, MT>();
  constexpr size_t full = apply_smem_bytes<P, T, MT>();
  // FP32 kernels at p <= 4: elements owned by warps (measured faster; at p = 5, 6
  // the n^2 = 36, 49 lines fill warps poorly and the CTA-wide mode is faster)
  constexpr bool warp_mode = sizeof(T) == 4 && P <= 4;
  if (warp_mode && !dot) {
    constexpr int per_cta = kWarpsPerCta * WarpCfg<P>::G;
    const int wgrid = (L.nelem + per_cta - 1) / per_cta;
    constexpr size_t wbytes = apply_warp_tile_bytes<P, T>();
    if (mass_only)
      sem_apply_kernel<P, QUAD, T, MT, false, true, true><<<wgrid, kApplyThreads, wbytes, s>>>(a, tab);
    else
      sem_apply_kernel<P, QUAD, T, MT, false, false, true><<<wgrid, kApplyThreads, wbytes, s>>>(a, tab);
    return cudaGetLastError();
  }
  if (mass_only) {
    sem_apply_kernel<P, QUAD, T, MT, false, true><<<grid, kApplyThreads, tiles, s>>>(a, tab);
  } else if (dot) {
    sem_apply_kernel<P, QUAD, T, MT, true, false><<<grid, kApplyThreads, full, s>>>(a, tab);
  } else {
    sem_apply_kernel<P, QUAD, T, MT, false, false><<<grid, kApplyThreads, full, s>>>(a, tab);
  }
  return cudaGetLastError();
}

// Dynamic shared-memory limits of the three variants of one instantiation.
template <int P, int QUAD, typename T, typename MT>
cudaError_t prime_t() {
  constexpr int full = (int)apply_smem_bytes<P, T, MT>();
  cudaError_t e;
  if ((e = cudaFuncSetAttribute(sem_apply_kernel<P, QUAD, T, MT, false, false>,
                                cudaFuncAttributeMaxDynamicSharedMemorySize, full)) != cudaSuccess) return e;
  if ((e = cudaFuncSetAttribute(sem_apply_kernel<P, QUAD, T, MT, true, false>,
                                cudaFuncAttributeMaxDynamicSharedMemorySize, full)) != cudaSuccess) return e;
  return cudaFuncSetAttribute(sem_apply_kernel<P, QUAD, T, MT, false, true>,
                              cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (int)apply_tile_bytes<P, T, MT>());
}

template <typename T, typename MT>
cudaError_t prime_all() {
  cudaError_t e;
#define SEM_PRIME(PP)                                                                   \
  if ((e = prime_t<PP, SEM_QUAD_LG, T, MT>()) != cudaSuccess) return e;                \
  if ((e = prime_t<PP, SEM_QUAD_LGL, T, MT>()) != cudaSuccess) return e;
  SEM_PRIME(1) SEM_PRIME(2) SEM_PRIME(3) SEM_PRIME(4) SEM_PRIME(5) SEM_PRIME(6)
#undef SEM_PRIME
  return cudaSuccess;
}

template <typename T, typename MT>
cudaError_t dispatch_apply(const Level& L, const ApplyArgs<T, MT>& a, bool mass_only, bool dot,
                           cudaStream_t s) {
#define SEM_CASE(PP)                                                                  \
  case PP:                                                                            \
    return L.quad == SEM_QUAD_LG ? launch_apply_t<PP, SEM_QUAD_LG, T, MT>(L, a, mass_only, dot, s) \
                                 : launch_apply_t<PP, SEM_QUAD_LGL, T, MT>(L, a, mass_only, dot, s);
  switch (L.p) {
    SEM_CASE(1)
    SEM_CASE(2)
    SEM_CASE(3)
    SEM_CASE(4)
    SEM_CASE(5)
    SEM_CASE(6)
    default:
      return cudaErrorInvalidValue;
  }
#undef SEM_CASE
}

}  // namespace sem
