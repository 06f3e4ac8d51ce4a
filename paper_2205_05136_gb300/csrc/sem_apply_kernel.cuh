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

#include <algorithm>
#include <type_traits>

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
// the pair's halves widened by integer operations: one FP64 instruction per node
// instead of three (measured 0.2 % on the mixed step)
__device__ __forceinline__ void scatter_add(double* p, df v) { atomicAdd(p, df_to_double(v)); }
// Element-local store of one element result (deterministic mode).
__device__ __forceinline__ void store_loc(double* p, double v) { *p = v; }
__device__ __forceinline__ void store_loc(float* p, float v) { *p = v; }
__device__ __forceinline__ void store_loc(double* p, df v) { *p = (double)v; }

// Base offset and stride of line l of an n^3 tile along direction DIR
// (0: x-line (j,k), l = j + n k; 1: y-line (i,k), l = i + n k; 2: z-line (i,j), l = i + n j).
template <int N, int DIR>
__device__ __forceinline__ void line_geom(int l, int& base, int& stride) {
  if (DIR == 0) { base = l * N; stride = 1; }
  else if (DIR == 1) { const int i = l % N, k = l / N; base = k * N * N + i; stride = N; }
  else { base = l; stride = N * N; }
}

// out = M in (ACC: out += M in) for M in even-odd form (EoMat), ANTI for
// s = -1.  With e_l = in_l + in_{n-1-l}, o_l = in_l - in_{n-1-l} (l < H):
//   se_q = sum_l a[q][l] e_l (+ a[q][H] in_H),  so_q = sum_l b[q][l] o_l,
//   out_q = se_q + so_q,  out_{n-1-q} = (ANTI ? so_q - se_q : se_q - so_q)   (q < H),
//   odd n: out_H = ANTI ? sum_l c[l] o_l : sum_l c[l] e_l + c[H] in_H.
// At n = 5 that is 12 multiply-adds and 8 additions instead of 25 multiply-adds.
template <int N, bool ANTI, bool ACC, typename T>
__device__ __forceinline__ void eo_line(const EoMat<N, T>& M, const T (&in)[N], T (&out)[N]) {
  if constexpr (EoMat<N, T>::kDirect) {  // out_q (+)= sum_l m[q][l] in_l
#pragma unroll
    for (int q = 0; q < N; ++q) {
      T acc = ACC ? fma(M.m[q][0], in[0], out[q]) : M.m[q][0] * in[0];
#pragma unroll
      for (int l = 1; l < N; ++l) acc = fma(M.m[q][l], in[l], acc);
      out[q] = acc;
    }
    return;
  }
  constexpr int H = N / 2;
  constexpr bool ODD = (N & 1) != 0;
  T e[H], o[H];
#pragma unroll
  for (int l = 0; l < H; ++l) {
    e[l] = in[l] + in[N - 1 - l];
    o[l] = in[l] - in[N - 1 - l];
  }
#pragma unroll
  for (int q = 0; q < H; ++q) {
    T se = M.a[q][0] * e[0];
#pragma unroll
    for (int l = 1; l < H; ++l) se = fma(M.a[q][l], e[l], se);
    if (ODD) se = fma(M.a[q][H], in[H], se);
    T so = M.b[q][0] * o[0];
#pragma unroll
    for (int l = 1; l < H; ++l) so = fma(M.b[q][l], o[l], so);
    const T y0 = se + so;
    const T y1 = ANTI ? so - se : se - so;
    if (ACC) {
      out[q] = out[q] + y0;
      out[N - 1 - q] = out[N - 1 - q] + y1;
    } else {
      out[q] = y0;
      out[N - 1 - q] = y1;
    }
  }
  if (ODD) {
    T ym;
    if (ANTI) {
      ym = M.c[0] * o[0];
#pragma unroll
      for (int l = 1; l < H; ++l) ym = fma(M.c[l], o[l], ym);
    } else {
      ym = M.c[0] * e[0];
#pragma unroll
      for (int l = 1; l < H; ++l) ym = fma(M.c[l], e[l], ym);
      ym = fma(M.c[H], in[H], ym);
    }
    out[H] = ACC ? out[H] + ym : ym;
  }
}

// dst = M along DIR of src (ACC: dst += ...), for every line of the E element
// tiles (thread tid of a group of nth threads).  src may equal dst.
template <int N, int E, int DIR, bool ANTI, bool ACC, typename T>
__device__ __forceinline__ void sweep(const EoMat<N, T>& M, const T* src, T* dst, int tid, int nth) {
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
    eo_line<N, ANTI, ACC>(M, in, out);
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
         (StageMetric<T>::value ? (size_t)ApplyCfg<P>::E * MetricLayout<MT>::block(P + 1) * sizeof(MT) : 0);
}

__device__ __forceinline__ float ldsmetric(const float* p) { return *p; }
__device__ __forceinline__ float ldsmetric(const __nv_bfloat16* p) { return __bfloat162float(*p); }
__device__ __forceinline__ double ldsmetric(const double* p) { return *p; }
__device__ __forceinline__ df ldsmetric(const df_pair* p) { return df(p->h, p->l); }

// The 7 metric values G00 G01 G02 G11 G12 G22 W of the quadrature points of
// one column (i, j) of an element, level by level: MetricColumn(block, c) then
// point(k, g).  SHARED: the block is in shared memory.  The bf16 column is read
// once, with 64-bit loads, into registers; the other layouts are read point by
// point.
__device__ __forceinline__ float bf16_lo(unsigned w) { return __uint_as_float(w << 16); }
__device__ __forceinline__ float bf16_hi(unsigned w) { return __uint_as_float(w & 0xffff0000u); }
template <int N, typename MT, bool SHARED>
struct MetricColumn {  // component-major layouts: point by point
  using ML = MetricLayout<MT>;
  const MT* p;
  __device__ __forceinline__ MetricColumn(const MT* block, int c) : p(block + ML::at(N, c, 0, 0)) {}
  template <typename T>
  __device__ __forceinline__ void point(int k, T (&g)[kMetricComps]) const {
#pragma unroll
    for (int comp = 0; comp < kMetricComps; ++comp) {
      const MT* q = p + ML::at(N, 0, k, comp);
      g[comp] = SHARED ? ldsmetric(q) : ldmetric(q);
    }
  }
};
template <int N, bool SHARED>
struct MetricColumn<N, __nv_bfloat16, SHARED> {
  using ML = MetricLayout<__nv_bfloat16>;
  static constexpr int NW = ML::col_width(N) / 4;  // 64-bit words of a column
  uint2 w[NW];
  __device__ __forceinline__ MetricColumn(const __nv_bfloat16* block, int c) {
    const uint2* q = reinterpret_cast<const uint2*>(block + ML::at(N, c, 0, 0));
#pragma unroll
    for (int t = 0; t < NW; ++t) w[t] = SHARED ? q[t] : __ldg(q + t);
  }
  // k is a compile-time constant after unrolling: the selects below resolve to registers
  __device__ __forceinline__ void point(int k, float (&g)[kMetricComps]) const {
#pragma unroll
    for (int comp = 0; comp < kMetricComps; ++comp) {
      const int v = kMetricComps * k + comp, h = v >> 1;
      const unsigned u = (h & 1) ? w[h >> 1].y : w[h >> 1].x;
      g[comp] = (v & 1) ? bf16_hi(u) : bf16_lo(u);
    }
  }
};

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

// The double-float kernel at p = 4 (the outer operator of the benchmark's mixed
// step) is bound by issue and memory latency: 5 CTAs per SM at 48 registers, with
// small spills, measured faster than 4 at 62 (at p = 3, 5, 6 it would spill far more).
template <int P, int QUAD, typename T, typename MT, bool DOT, bool MASS_ONLY, bool WARP = false>
__global__ void __launch_bounds__(kApplyThreads, (std::is_same<T, df>::value && P == 4) ? 5 : 1)
    sem_apply_kernel(const ApplyArgs<T, MT> a, const __grid_constant__ KTab<P + 1, T> tab) {
  pdl_trigger();
  static_assert(!(WARP && DOT), "the fused inner product needs the CTA-wide mode");
  constexpr int N = P + 1, N2 = N * N, N3 = N2 * N;
  using ML = MetricLayout<MT>;
  constexpr int BLK = ML::block(N);
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

  const int e0 = WARP ? (blockIdx.x * kWarpsPerCta + warp) * E : blockIdx.x * E;
  if (WARP && e0 >= a.nelem) return;  // no CTA-wide barrier follows in this mode
  // while the previous kernel drains: the group's map entries into L2
  prefetch_l2_lines(a.map + (size_t)e0 * N3, (size_t)min(E, a.nelem - e0) * N3 * sizeof(int), tid, nth);
  pdl_wait();
  if (a.done != nullptr && *a.done) return;

  if (STAGE) {  // the CTA's metric block: contiguous, 16-byte aligned, a multiple of 16 bytes
    const int ne = min(E, a.nelem - e0);
    const size_t bytes = (size_t)ne * BLK * sizeof(MT);
    const char* src = reinterpret_cast<const char*>(a.metric + (size_t)e0 * BLK);
    const unsigned dst = (unsigned)__cvta_generic_to_shared(sM);
    for (size_t off = (size_t)threadIdx.x * 16; off < bytes; off += (size_t)blockDim.x * 16)
      asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(dst + (unsigned)off),
                   "l"(src + off)
                   : "memory");
    asm volatile("cp.async.commit_group;\n" ::: "memory");
  }
  if (std::is_same<T, df>::value && !STAGE && !MASS_ONLY) {
    // Bulk prefetch of the group's metric block (contiguous, 16-byte aligned, a
    // multiple of 16 bytes) into L2, in 16 KB pieces: the quadrature-point stage
    // reads it after the gather and two sweeps, and then hits L2.  Measured
    // faster for the memory-latency-bound double-float kernel only (the FP64
    // kernel is bound by the FP64 pipe, the FP32 ones stage the metric).
    const int ne = min(E, a.nelem - e0);
    const unsigned bytes = (unsigned)((size_t)ne * BLK * sizeof(MT));
    const char* src = reinterpret_cast<const char*>(a.metric + (size_t)e0 * BLK);
    for (unsigned off = (unsigned)tid * 16384u; off < bytes; off += (unsigned)nth * 16384u)
      asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;\n" ::"l"(src + off),
                   "r"(min(16384u, bytes - off))
                   : "memory");
  }

  // Gather and scatter loops.  Every launch of this kernel has kApplyThreads
  // threads per CTA (a warp per element group in warp mode), so the loops of
  // the plain apply have compile-time trip counts: they unroll and keep the
  // loads of all their iterations in flight at once.  The apply with the fused
  // inner product keeps the rolled loops (both measured faster that way).
  constexpr int NTH = WARP ? 32 : kApplyThreads;
  constexpr int IT = (E * N3 + NTH - 1) / NTH;

  // gather u_e = P_e u
  if constexpr (DOT) {
    // the double-float operator with the fused inner product gathers u as the
    // float pairs the CG kernel that formed u wrote (a.u2), converting nothing
    for (int idx = tid; idx < E * N3; idx += nth) {
      const int s = idx / N3, loc = idx - s * N3, e = e0 + s;
      if (e < a.nelem) {
        const int gi = (int)SEM_IDX(__ldg(a.map + (size_t)e * N3 + loc), a.ndofs, a.dbg, kDbgGather);
        if constexpr (std::is_same<T, df>::value) {
          const float2 v = __ldg(reinterpret_cast<const float2*>(a.u2) + gi);
          sA[idx] = df(v.x, v.y);
        } else {
          sA[idx] = T(a.u[gi]);
        }
      } else {
        sA[idx] = T(0);
      }
    }
  } else {
    const int nv = min(E, a.nelem - e0) * N3;  // nodal values of the group's elements
    const int* gmap = a.map + (size_t)e0 * N3;
#pragma unroll
    for (int it = 0; it < IT; ++it) {
      const int idx = tid + it * NTH;
      if (IT * NTH == E * N3 || idx < E * N3)
        sA[idx] = idx < nv ? T(a.u[SEM_IDX(__ldg(gmap + idx), a.ndofs, a.dbg, kDbgGather)]) : T(0);
    }
  }
  group_sync();

  if (QUAD == SEM_QUAD_LG) {  // values at the Gauss points
    sweep<N, E, 0, false, false>(tab.Bi, sA, sB, tid, nth);
    group_sync();
    sweep<N, E, 1, false, false>(tab.Bi, sB, sC, tid, nth);
    group_sync();
    sweep<N, E, 2, false, false>(tab.Bi, sC, sA, tid, nth);
    group_sync();
  }

  if (MASS_ONLY) {
    for (int idx = tid; idx < E * N3; idx += nth) {
      const int s = idx / N3, loc = idx - s * N3, e = e0 + s;
      if (e < a.nelem) {
        const T W = ldmetric(a.metric + (size_t)e * BLK + ML::at(N, loc % N2, loc / N2, 6));
        sA[idx] = (a.mass_coef * W) * sA[idx];
      }
    }
    group_sync();
  } else {
    // reference gradient along x and y (into sB, sC)
    sweep<N, E, 0, true, false>(tab.D, sA, sB, tid, nth);
    sweep<N, E, 1, true, false>(tab.D, sA, sC, tid, nth);
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
      eo_line<N, true, false>(tab.D, uz, g3);
      // bf16: the column's values into registers by 64-bit loads (MetricColumn);
      // the component-major layouts point by point from the column's first value
      // (measured 17 % faster for the double-float kernel than through MetricColumn)
      const MT* mblk = STAGE ? sM + (size_t)s * BLK : a.metric + (size_t)e * BLK;
      const MetricColumn<N, MT, STAGE> mcol(mblk, ML::kColumnMajor ? c : 0);
      const MT* mp = mblk + c;
#pragma unroll
      for (int k = 0; k < N; ++k) {
        const T g1 = pb[k * N2], g2 = pc[k * N2];
        T gm[kMetricComps];
        if constexpr (ML::kColumnMajor) {
          mcol.point(k, gm);
        } else {
#pragma unroll
          for (int cc = 0; cc < kMetricComps; ++cc) {
            const MT* q = mp + k * N2 + cc * padded_n3(N);
            gm[cc] = STAGE ? ldsmetric(q) : ldmetric(q);
          }
        }
        const T G00 = gm[0], G01 = gm[1], G02 = gm[2], G11 = gm[3], G12 = gm[4], G22 = gm[5], W = gm[6];
        pb[k * N2] = fma(G02, g3[k], fma(G01, g2, G00 * g1));
        pc[k * N2] = fma(G12, g3[k], fma(G11, g2, G01 * g1));
        q3[k] = fma(G22, g3[k], fma(G12, g2, G02 * g1));
        m[k] = (a.mass_coef * W) * uz[k];
      }
      eo_line<N, true, true>(tab.Dt, q3, m);
#pragma unroll
      for (int k = 0; k < N; ++k) pa[k * N2] = m[k];
    }
    group_sync();
    sweep<N, E, 1, true, true>(tab.Dt, sC, sA, tid, nth);
    group_sync();
    sweep<N, E, 0, true, true>(tab.Dt, sB, sA, tid, nth);
    group_sync();
  }

  if (QUAD == SEM_QUAD_LG) {  // back from the Gauss points to the nodes
    sweep<N, E, 0, false, false>(tab.Bit, sA, sB, tid, nth);
    group_sync();
    sweep<N, E, 1, false, false>(tab.Bit, sB, sC, tid, nth);
    group_sync();
    sweep<N, E, 2, false, false>(tab.Bit, sC, sA, tid, nth);
    group_sync();
  }

  // scatter-add y += P_e^T y_e, and with DOT the partial u_e . y_e
  double dot = 0.0;
  if constexpr (DOT) {
    if constexpr (std::is_same<T, df>::value) {
      // the partial u_e . y_e in double-float arithmetic from the float pairs of u
      // (in L1 since the gather)
      df dd(0);
      for (int idx = tid; idx < E * N3; idx += nth) {
        const int s = idx / N3, loc = idx - s * N3, e = e0 + s;
        if (e < a.nelem) {
          const int g = (int)SEM_IDX(__ldg(a.map + (size_t)e * N3 + loc), a.ndofs, a.dbg, kDbgScatter);
          T v = sA[idx];
          if (a.scale_out) v *= a.out_scale;
          if (a.yloc != nullptr) store_loc(a.yloc + (size_t)e * N3 + loc, v);
          else scatter_add(a.y + g, v);
          const float2 uu = __ldg(reinterpret_cast<const float2*>(a.u2) + g);
          dd = fma(df(uu.x, uu.y), v, dd);
        }
      }
      dot = (double)dd;
    } else {
      for (int idx = tid; idx < E * N3; idx += nth) {
        const int s = idx / N3, loc = idx - s * N3, e = e0 + s;
        if (e < a.nelem) {
          const int g = (int)SEM_IDX(__ldg(a.map + (size_t)e * N3 + loc), a.ndofs, a.dbg, kDbgScatter);
          T v = sA[idx];
          if (a.scale_out) v *= a.out_scale;
          if (a.yloc != nullptr) store_loc(a.yloc + (size_t)e * N3 + loc, v);
          else scatter_add(a.y + g, v);
          dot = fma((double)a.u[g], (double)v, dot);
        }
      }
    }
  } else {
    const int nv = min(E, a.nelem - e0) * N3;
    const int* gmap = a.map + (size_t)e0 * N3;
#pragma unroll
    for (int it = 0; it < IT; ++it) {
      const int idx = tid + it * NTH;
      if ((IT * NTH == E * N3 || idx < E * N3) && idx < nv) {
        T v = sA[idx];
        if (a.scale_out) v *= a.out_scale;
        if (a.yloc != nullptr) store_loc(a.yloc + (size_t)e0 * N3 + idx, v);
        else scatter_add(a.y + SEM_IDX(__ldg(gmap + idx), a.ndofs, a.dbg, kDbgScatter), v);
      }
    }
  }
  if (DOT) {  // this CTA's partial; k_apply_dot_finish sums them after the launch
    const double bs = block_sum(dot, red);
    if (threadIdx.x == 0) a.dot_partials[blockIdx.x] = bs;
  }
}

// ---------------------------------------------------------------------------
// Pipelined warp kernel of the FP32 operator (p <= 4, stiffness and mass).
//
// A warp that owns one element at a time waits for the map, then for the
// gathered values, then for the metric, and has nothing in flight while it
// computes.  Here each warp loops over "units" of G consecutive elements
// (unit j of the warp is unit w + j W, W warps in the grid) and keeps the
// copies of unit j+1 in flight while it computes unit j:
//   - the unit's metric block, contiguous in the element-blocked layout
//     (16-byte aligned), by one bulk copy (cp.async.bulk) that lane 0 issues;
//   - the unit's nodal values, gathered by plain loads into registers from the
//     map entries (loaded one unit earlier still) and stored to the stage after
//     this unit's sweeps.  Each lane gathers (and later scatters) the n nodes of
//     its z-column: for each level the lanes read consecutive map entries.
// Two stage buffers per warp; a stage's metric is complete when its mbarrier's
// phase completes (every lane waits on it), its nodal values after __syncwarp.
// The grid is persistent
// (the CTAs that are resident at once, 3 per SM), so the pipeline runs over
// several units.
//
// Every lane owns one line of each sweep (G n^2 <= 32 for p <= 4).  Lanes
// beyond the unit's G n^2 lines run the same instructions on the line of lane
// (lane - (32 - G n^2)): their loads are broadcasts of that lane's, their
// stores are predicated off, so no sweep needs a divergent branch.  The unit
// tiles use the bank-skewed placement of pipe_word, so that no x-, y- or z-line
// access conflicts; each lane keeps the tile words of its three lines in
// registers (80 registers, 3 CTAs per SM: at p = 4 it cut shared-memory
// wavefronts 14 % and the mixed time step 2.7 % against the plain [k][j][i]
// tile with 64 registers and 4 CTAs per SM).
template <int P, typename MT>
struct PipeCfg {
  static constexpr int N = P + 1, N2 = N * N, N3 = N2 * N;
  static constexpr int BLK = MetricLayout<MT>::block(N);  // metric values of an element
  static constexpr int G = WarpCfg<P>::G;
  static constexpr int NL = G * N2;                  // lines per sweep direction
  static constexpr int UT = G * N3;                  // nodal values of a unit
  static constexpr int TW = 32 * N;                  // words of a unit tile (pipe_word)
  static constexpr int MV = G * BLK;                 // metric values of a unit
  static constexpr int CH = (int)(MV * sizeof(MT) / 16);  // 16-byte chunks of a unit's metric
  // two metric stages, two nodal stages, the two work tiles of the sweeps and the
  // two metric stages' mbarriers
  static constexpr size_t bar_offset = 2 * (size_t)MV * sizeof(MT) + 4 * (size_t)TW * sizeof(float);
  static constexpr size_t warp_bytes = bar_offset + 2 * sizeof(uint64_t);
  static constexpr size_t cta_bytes = kWarpsPerCta * warp_bytes;
  static_assert(NL <= 32, "a unit must have at most 32 lines per direction");
  static_assert((MV * sizeof(MT)) % 16 == 0, "stage buffers must stay 16-byte aligned");
  static_assert(bar_offset % 16 == 0 && warp_bytes % 16 == 0, "mbarriers and warp regions stay aligned");
};

// Word of node (i, j, k) of element slot s in a unit tile: row i of 32 words,
// bank s n^2 + n ((j - i) mod n) + ((k - i) mod n).  For every sweep pattern the
// warp's lanes run over the slots and two of (i, j, k) with the third fixed, and
// the banks (i, j, k) -> ((j - i) mod n, (k - i) mod n) are distinct on each such
// plane (a Latin-square placement), so no line access has a bank conflict; no
// affine layout of the 5^3 tile does that for x-, y- and z-lines at once.
template <int N>
__device__ __forceinline__ int pipe_word(int s, int i, int j, int k) {
  const int jj = j - i + (j < i ? N : 0), kk = k - i + (k < i ? N : 0);
  return 32 * i + s * N * N + N * jj + kk;
}

// The metric block of a unit reaches shared memory by one bulk copy (the TMA
// engine, cp.async.bulk) that lane 0 issues; 16-byte cp.async copies from every
// lane took four load instructions of the warp and about 11 more L1 tag-stage
// wavefronts per element, in a kernel bound by the L1 pipes and by issue.  Each
// of a warp's two stages has an mbarrier of count 1: lane 0 arrives with the
// expected byte count and the copy's completion ends the phase.
// Shared-memory addresses are passed as 32-bit shared-window offsets.
__device__ __forceinline__ unsigned smem_u32(const void* p) { return (unsigned)__cvta_generic_to_shared(p); }
__device__ __forceinline__ void mbar_init(unsigned bar) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(bar) : "memory");
}
__device__ __forceinline__ void bulk_copy(unsigned dst, const void* src, unsigned bytes, unsigned bar) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(bar), "r"(bytes) : "memory");
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];\n" ::"r"(dst),
      "l"(src), "r"(bytes), "r"(bar)
      : "memory");
}
// Waits for the phase of the given parity to complete; false when it has not
// within kMbarTimeoutNs of the global timer (the copy takes microseconds: the
// bound only turns a copy that never completes into an error status).
#ifdef SEM_DEBUG
constexpr unsigned long long kMbarTimeoutNs = 20000000ull;  // 20 ms: a test of the timeout path ends quickly
#else
constexpr unsigned long long kMbarTimeoutNs = 1000000000ull;  // 1 s
#endif
__device__ __forceinline__ bool mbar_try(unsigned a, unsigned parity) {
  unsigned ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(a), "r"(parity)
      : "memory");
  return ok != 0;
}
__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;\n" : "=l"(t));
  return t;
}
// (the polling loop out of line: it keeps the hot loop's registers free)
static __device__ __noinline__ bool mbar_wait_timed(unsigned a, unsigned parity) {
  const unsigned long long t0 = global_ns();
  while (true) {
    for (int i = 0; i < 64; ++i)
      if (mbar_try(a, parity)) return true;
    if (global_ns() - t0 > kMbarTimeoutNs) return false;
  }
}
__device__ __forceinline__ bool mbar_wait(unsigned a, unsigned parity) {
  return mbar_try(a, parity) || mbar_wait_timed(a, parity);
}

// Map entries of the lane's z-column of unit `unit`: node zc + n^2 t of the unit
// for t < n (zc = slot s n^3 + column (i + n j)); 0 for elements past the mesh.
template <int P, typename MT>
__device__ __forceinline__ void pipe_load_map(const ApplyArgs<float, MT>& a, int unit, int nunits, int slot, int zc,
                                              int (&m)[P + 1]) {
  using C = PipeCfg<P, MT>;
  const bool present = unit < nunits && unit * C::G + slot < a.nelem;
  const int* src = a.map + (size_t)unit * C::UT + zc;
#pragma unroll
  for (int t = 0; t < C::N; ++t)
    m[t] = present ? (int)SEM_IDX(__ldg(src + t * C::N2), a.ndofs, a.dbg, kDbgGather) : 0;
}

// Lane 0 issues the bulk copy of one unit's metric block (the elements of the unit
// inside the mesh: a multiple of 16 bytes from a 16-byte aligned address) into a
// stage.
template <int P, typename MT>
__device__ __forceinline__ void pipe_issue_metric(const ApplyArgs<float, MT>& a, int unit, int lane,
                                                  unsigned sM, unsigned bar) {
  using C = PipeCfg<P, MT>;
  const int e0 = unit * C::G;
  if (lane == 0 && !SEM_HOLD(a, unit))
    bulk_copy(sM, a.metric + (size_t)e0 * C::BLK, (unsigned)(min(C::G, a.nelem - e0) * C::BLK * (int)sizeof(MT)),
              bar);
}

// One 1-D line of n values at tile words off[]: dst = M src (ACC: dst += M src),
// M in even-odd form.  src may equal dst.
template <int N, bool ANTI, bool ACC, typename T>
__device__ __forceinline__ void lane_line(const EoMat<N, T>& M, const T* src, T* dst, const int (&off)[N],
                                          bool store) {
  T in[N], out[N];
#pragma unroll
  for (int t = 0; t < N; ++t) in[t] = src[off[t]];
  if (ACC) {
#pragma unroll
    for (int t = 0; t < N; ++t) out[t] = dst[off[t]];
  }
  eo_line<N, ANTI, ACC>(M, in, out);
#pragma unroll
  for (int t = 0; t < N; ++t)
    if (store) dst[off[t]] = out[t];
}

// 3 CTAs per SM (80 registers) at p = 3, 4; 4 at p <= 2, whose 64 registers hold
// the shorter lines' offsets without spills (more warps for the small, latency-bound
// coarse levels: mixed step -0.2 %).
template <int P, int QUAD, typename MT>
__global__ void __launch_bounds__(kApplyThreads, P <= 2 ? 4 : 3)
    sem_apply_pipe_kernel(const ApplyArgs<float, MT> a, const __grid_constant__ KTab<P + 1, float> tab,
                          int nunits) {
  pdl_trigger();
  using C = PipeCfg<P, MT>;
  using T = float;
  constexpr int N = C::N, N2 = C::N2, N3 = C::N3, G = C::G, NL = C::NL;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  int unit = blockIdx.x * kWarpsPerCta + warp;
  if (unit >= nunits) return;  // no CTA-wide barrier in this kernel
  {  // while the previous kernel drains: the first unit's map entries and metric into L2
    const int ne = min(G, a.nelem - unit * G);
    prefetch_l2_lines(a.map + (size_t)unit * C::UT, (size_t)ne * N3 * sizeof(int), lane, 32);
    prefetch_l2_lines(a.metric + (size_t)unit * G * C::BLK, (size_t)ne * C::BLK * sizeof(MT), lane, 32);
  }
  pdl_wait();
  if (a.done != nullptr && *a.done) return;
  const int tw = gridDim.x * kWarpsPerCta;
  unsigned char* wb = smem_raw + (size_t)warp * C::warp_bytes;
  MT* sM0 = reinterpret_cast<MT*>(wb);
  T* sU0 = reinterpret_cast<T*>(wb + 2 * (size_t)C::MV * sizeof(MT));
  T* sB = sU0 + 2 * C::TW;
  T* sC = sB + C::TW;
  // the two metric stages and their mbarriers, as shared-window offsets
  const unsigned sm_s = smem_u32(sM0), bar_s = smem_u32(wb + C::bar_offset);
  constexpr unsigned kStageBytes = (unsigned)(C::MV * sizeof(MT));
  if (lane == 0) {
    mbar_init(bar_s);
    mbar_init(bar_s + 8);
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
  }
  __syncwarp();
  unsigned phase = 0;  // bit s: parity of stage s's next completion

  // The lane's lines (those of lane - (32 - NL) for the lanes >= NL, a lane of the
  // same half-warp, so that the 64-bit metric loads of the idle lanes are
  // broadcasts within their phase): element slot ls, line ll = r + n q, which is
  // the x-line (j, k) = (r, q), the y-line (i, k) = (r, q) and the z-line
  // (i, j) = (r, q); their tile words for t = 0..n-1.
  static_assert(NL >= 24, "idle lanes must replay a lane of their half-warp");
  const bool act = lane < NL;
  const int lw = act ? lane : lane - (32 - NL);
  const int ls = lw / N2, ll = lw - ls * N2, r = ll % N, q = ll / N;
  int ox[N], oy[N], oz[N];
#pragma unroll
  for (int t = 0; t < N; ++t) {
    ox[t] = pipe_word<N>(ls, t, r, q);
    oy[t] = pipe_word<N>(ls, r, t, q);
    oz[t] = pipe_word<N>(ls, r, q, t);
  }
  const int zc = ls * N3 + ll;  // first node of the lane's z-column in the unit

  int mc[N], mn[N], mnn[N];  // map entries of the lane's z-column in units j, j+1, j+2
  pipe_load_map<P>(a, unit, nunits, ls, zc, mc);
  float gv[N];  // the next unit's gathered values, in flight during this unit's sweeps
  pipe_issue_metric<P>(a, unit, lane, sm_s, bar_s);
  {
    const bool present = unit * G + ls < a.nelem;
#pragma unroll
    for (int t = 0; t < N; ++t) gv[t] = present ? __ldg(a.u + mc[t]) : 0.f;
#pragma unroll
    for (int t = 0; t < N; ++t)
      if (act) sU0[oz[t]] = gv[t];
  }
  pipe_load_map<P>(a, unit + tw, nunits, ls, zc, mn);
  int b = 0;
  for (; unit < nunits; unit += tw) {
    const int nxt = unit + tw;
    if (nxt < nunits) {
      pipe_issue_metric<P>(a, nxt, lane, sm_s + (b ^ 1) * kStageBytes, bar_s + 8 * (b ^ 1));
      const bool present = nxt * G + ls < a.nelem;
#pragma unroll
      for (int t = 0; t < N; ++t) gv[t] = present ? __ldg(a.u + mn[t]) : 0.f;
    }
    pipe_load_map<P>(a, nxt + tw, nunits, ls, zc, mnn);
    if (!mbar_wait(bar_s + 8 * b, (phase >> b) & 1u)) {
      // the copy did not complete: report it, let the other stage's copy land, stop
      if (lane == 0 && a.fault != nullptr) atomicOr(a.fault, 1u);
      if (nxt < nunits) mbar_wait(bar_s + 8 * (b ^ 1), (phase >> (b ^ 1)) & 1u);
      return;
    }
    phase ^= 1u << b;
    __syncwarp();

    T* sA = sU0 + b * C::TW;
    const MT* sM = sM0 + b * C::MV;
    const int e = unit * G + ls;  // the lane's element
    if (QUAD == SEM_QUAD_LG) {  // values at the Gauss points
      lane_line<N, false, false>(tab.Bi, sA, sB, ox, act);
      __syncwarp();
      lane_line<N, false, false>(tab.Bi, sB, sC, oy, act);
      __syncwarp();
      lane_line<N, false, false>(tab.Bi, sC, sA, oz, act);
      __syncwarp();
    }
    // reference gradient along x and y (into sB, sC)
    lane_line<N, true, false>(tab.D, sA, sB, ox, act);
    lane_line<N, true, false>(tab.D, sA, sC, oy, act);
    __syncwarp();
    // z-gradient, quadrature-point stage and transposed z-sweep on the lane's column
    {
      T uz[N], g3[N], q3[N], m[N];
#pragma unroll
      for (int k = 0; k < N; ++k) uz[k] = sA[oz[k]];
      eo_line<N, true, false>(tab.D, uz, g3);
      const MetricColumn<N, MT, true> mcol(sM + ls * C::BLK, ll);
#pragma unroll
      for (int k = 0; k < N; ++k) {
        const T g1 = sB[oz[k]], g2 = sC[oz[k]];
        T gm[kMetricComps];
        mcol.point(k, gm);
        const T G00 = gm[0], G01 = gm[1], G02 = gm[2], G11 = gm[3], G12 = gm[4], G22 = gm[5], W = gm[6];
        const T q1 = fma(G02, g3[k], fma(G01, g2, G00 * g1));
        const T q2 = fma(G12, g3[k], fma(G11, g2, G01 * g1));
        if (act) {
          sB[oz[k]] = q1;
          sC[oz[k]] = q2;
        }
        q3[k] = fma(G22, g3[k], fma(G12, g2, G02 * g1));
        m[k] = (a.mass_coef * W) * uz[k];
      }
      eo_line<N, true, true>(tab.Dt, q3, m);
#pragma unroll
      for (int k = 0; k < N; ++k)
        if (act) sA[oz[k]] = m[k];
    }
    __syncwarp();
    lane_line<N, true, true>(tab.Dt, sC, sA, oy, act);
    __syncwarp();
    lane_line<N, true, true>(tab.Dt, sB, sA, ox, act);
    __syncwarp();
    if (QUAD == SEM_QUAD_LG) {  // back from the Gauss points to the nodes
      lane_line<N, false, false>(tab.Bit, sA, sB, ox, act);
      __syncwarp();
      lane_line<N, false, false>(tab.Bit, sB, sC, oy, act);
      __syncwarp();
      lane_line<N, false, false>(tab.Bit, sC, sA, oz, act);
      __syncwarp();
    }
    // scatter-add y += P_e^T y_e along the lane's z-column
    const T sc = a.scale_out ? a.out_scale : T(1);
    if (act && e < a.nelem) {
      if (a.yloc != nullptr) {  // deterministic mode: element-local results
#pragma unroll
        for (int t = 0; t < N; ++t) a.yloc[(size_t)unit * C::UT + zc + t * N2] = sA[oz[t]] * sc;
      } else {
#pragma unroll
        for (int t = 0; t < N; ++t) atomicAdd(a.y + mc[t], sA[oz[t]] * sc);
      }
    }
    if (nxt < nunits) {
#pragma unroll
      for (int t = 0; t < N; ++t)
        if (act) sU0[(b ^ 1) * C::TW + oz[t]] = gv[t];
    }
    __syncwarp();  // stage b is refilled by the next iteration's issue
#pragma unroll
    for (int t = 0; t < N; ++t) {
      mc[t] = mn[t];
      mn[t] = mnn[t];
    }
    b ^= 1;
  }
}

// Persistent grid of the pipelined kernel: the CTAs resident on the device at
// once (set by prime_t, before any stream capture), at most one warp per unit.
template <int P, int QUAD, typename MT>
struct PipeGrid {
  static inline int resident = 0;
};

template <int P, int QUAD, typename MT>
cudaError_t pipe_prime() {
  using C = PipeCfg<P, MT>;
  cudaError_t e = cudaFuncSetAttribute(sem_apply_pipe_kernel<P, QUAD, MT>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)C::cta_bytes);
  int dev = 0, sms = 0, per_sm = 0;
  if (e == cudaSuccess) e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e == cudaSuccess)
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, sem_apply_pipe_kernel<P, QUAD, MT>,
                                                      kApplyThreads, C::cta_bytes);
  if (e != cudaSuccess) return e;
  if (per_sm < 1) return cudaErrorInvalidConfiguration;
  PipeGrid<P, QUAD, MT>::resident = sms * per_sm;
  return cudaSuccess;
}

template <int P, int QUAD, typename MT>
cudaError_t launch_apply_pipe(const Level& L, const ApplyArgs<float, MT>& a, const KTab<P + 1, float>& tab,
                              cudaStream_t s) {
  using C = PipeCfg<P, MT>;
  const int resident = PipeGrid<P, QUAD, MT>::resident;
  if (resident < 1) return cudaErrorInitializationError;  // prime_apply_kernels was not called
  const int nunits = (L.nelem + C::G - 1) / C::G;
  const int grid = std::min(resident, (nunits + kWarpsPerCta - 1) / kWarpsPerCta);
  if (grid == 0) return cudaSuccess;
  launch_k(sem_apply_pipe_kernel<P, QUAD, MT>, grid, kApplyThreads, C::cta_bytes, s, a, tab, nunits);
  return cudaGetLastError();
}

// Even-odd form (EoMat) of the n x n matrix M (or of its transpose), from the
// host tables; the mirrored rows are implied by the symmetry of M.
template <int N, typename T>
void make_eo(EoMat<N, T>& E, const double (&M)[kMaxN][kMaxN], bool transpose) {
  constexpr int H = N / 2;
  auto m = [&](int q, int l) { return transpose ? M[l][q] : M[q][l]; };
  for (int q = 0; q < H; ++q) {
    for (int l = 0; l < H; ++l) {
      E.a[q][l] = (T)(0.5 * (m(q, l) + m(q, N - 1 - l)));
      E.b[q][l] = (T)(0.5 * (m(q, l) - m(q, N - 1 - l)));
    }
    E.a[q][H] = (T)((N & 1) ? m(q, H) : 0.0);
  }
  for (int l = 0; l <= H; ++l) E.c[l] = (T)((N & 1) ? m(H, l) : 0.0);
  if constexpr (EoMat<N, T>::kDirect)
    for (int q = 0; q < N; ++q)
      for (int l = 0; l < N; ++l) E.m[q][l] = (T)m(q, l);
}

// The apply kernels of one degree, quadrature and precision (atomic adds into
// y, or element-local results into a.yloc).
template <int P, int QUAD, typename T, typename MT>
cudaError_t launch_apply_kernels(const Level& L, const ApplyArgs<T, MT>& a, const KTab<P + 1, T>& tab,
                                 bool mass_only, bool dot, cudaStream_t s) {
  constexpr int E = ApplyCfg<P>::E;
  const int grid = (L.nelem + E - 1) / E;
  if (grid == 0) return cudaSuccess;
  constexpr size_t tiles = apply_tile_bytes<P, T, MT>();
  constexpr size_t full = apply_smem_bytes<P, T, MT>();
  // FP32 kernels at p <= 4: elements owned by warps (measured faster; at p = 5, 6
  // the n^2 = 36, 49 lines fill warps poorly and the CTA-wide mode is faster)
  constexpr bool warp_mode = sizeof(T) == 4 && P <= 4;
  if constexpr (std::is_same<T, float>::value && P <= 4) {
    if (!mass_only && !dot) return launch_apply_pipe<P, QUAD, MT>(L, a, tab, s);
  }
  if (warp_mode && !dot) {
    constexpr int per_cta = kWarpsPerCta * WarpCfg<P>::G;
    const int wgrid = (L.nelem + per_cta - 1) / per_cta;
    constexpr size_t wbytes = apply_warp_tile_bytes<P, T>();
    if (mass_only)
      launch_k(sem_apply_kernel<P, QUAD, T, MT, false, true, true>, wgrid, kApplyThreads, wbytes, s, a, tab);
    else
      launch_k(sem_apply_kernel<P, QUAD, T, MT, false, false, true>, wgrid, kApplyThreads, wbytes, s, a, tab);
    return cudaGetLastError();
  }
  if (mass_only) {
    launch_k(sem_apply_kernel<P, QUAD, T, MT, false, true>, grid, kApplyThreads, tiles, s, a, tab);
  } else if (dot) {
    launch_k(sem_apply_kernel<P, QUAD, T, MT, true, false>, grid, kApplyThreads, full, s, a, tab);
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    return launch_apply_dot_finish(a.dot_partials, grid, a.cg, a.dot_out, a.done, s);
  } else {
    launch_k(sem_apply_kernel<P, QUAD, T, MT, false, false>, grid, kApplyThreads, full, s, a, tab);
  }
  return cudaGetLastError();
}

// Launch helper shared by the precision-specific translation units.  With
// a.yloc set (deterministic mode) the kernels write element results and the
// node sums follow in a fixed order.
template <int P, int QUAD, typename T, typename MT>
cudaError_t launch_apply_t(const Level& L, const ApplyArgs<T, MT>& a, bool mass_only, bool dot,
                           cudaStream_t s) {
  constexpr int N = P + 1;
  KTab<N, T> tab;
  make_eo(tab.D, QUAD == SEM_QUAD_LG ? L.tab.Dg : L.tab.D, false);
  make_eo(tab.Dt, QUAD == SEM_QUAD_LG ? L.tab.Dg : L.tab.D, true);
  make_eo(tab.Bi, L.tab.Bi, false);
  make_eo(tab.Bit, L.tab.Bi, true);
  ApplyArgs<T, MT> b = a;
  b.ndofs = L.ndofs;
  b.dbg = L.dbg;
  b.fault = L.fault;
  b.hold = L.hold;
  const cudaError_t e = launch_apply_kernels<P, QUAD, T, MT>(L, b, tab, mass_only, dot, s);
  if (e != cudaSuccess || a.yloc == nullptr) return e;
  return launch_assemble(L, a.yloc, a.y, a.done, s);
}

// Dynamic shared-memory limits of the three variants of one instantiation.
template <int P, int QUAD, typename T, typename MT>
cudaError_t prime_t() {
  constexpr int full = (int)apply_smem_bytes<P, T, MT>();
  cudaError_t e;
  if constexpr (std::is_same<T, float>::value && P <= 4) {
    if ((e = pipe_prime<P, QUAD, MT>()) != cudaSuccess) return e;
  }
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
