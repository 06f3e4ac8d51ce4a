// Tensor-core form of the FP32 SEM-NI operator apply (Section 4.1's sum
// factorization written as small dense contractions, Algorithm 1's cell loop):
//
//   y += sum_e P_e^T (mass_coef M_e + K_e) P_e u,   LGL quadrature on the nodes,
//
// for the multigrid smoother (float vectors, bf16 metric).  The contractions
// run as mma.sync m16n8k16 with bf16 operands and FP32 accumulation.
//
// Rows.  An MMA tile has 16 rows.  Row r of a tile is the plane k = r % n of
// element r / n of the tile; a tile holds EPT = floor(16 / n) whole elements
// (3 at p = 4; rows from EPT n on are padding).  A row holds the n^2 nodal
// values of its plane, column i + n j.
//
//   in-plane gradient   [gx | gy](row, :) = u(row, :) Pxy        Pxy: n^2 x 2n^2 (D along i, D along j)
//   z-gradient          gz = Z u                                 Z = blockdiag(D, ..., D) over the tile's rows
//   quadrature stage    q = G (gx, gy, gz),  m = mass_coef W u   per point, FP32
//   transposed          y = [qx | qy] Pxy^T + Z^T qz + m
//
// Column orders are chosen so that every one of these values of a point sits
// in the same thread: the in-plane output's column block 2m holds gx of
// points 8m..8m+7 and block 2m+1 their gy; the z output's block m and the
// transposed outputs' block m hold points 8m..8m+7.  Then the FP32
// accumulators of the in-plane gradient, rounded to bf16 pairs, are the A
// operand of the transposed in-plane product, the mass term adds to the
// transposed accumulators, and only qz goes through shared memory (the
// z-contraction mixes rows, which a thread does not hold).
//
// Precision.  A multigrid smoother whose operator is off by a relative 1e-3
// already costs outer iterations (three PCG iterations to 1e-10 mean a V-cycle
// contraction near 5e-4), so the contractions here are as accurate as FP32:
// u, the derivative matrix D and q each enter as a pair of bf16 numbers (hi +
// lo, hi = bf16(v), lo = bf16(v - hi), together about 2^-16 relative), and
// each product takes the three terms hi hi, hi lo, lo hi.  The remaining error
// is the bf16 metric's, as in the FP32 kernel with the bf16 metric; the mass
// term and all accumulation are FP32.
//
// Units.  A warp processes units of MTU tiles: G = MTU EPT elements that are
// consecutive along x in one row of the slab.  Their nodes form n^2 lines of
// p G + 1 consecutive global nodes: the gather reads and the scatter adds whole
// lines (coalesced), and the node indices follow from the slab's lexicographic
// numbering (the one the element-to-DOF map holds), so no map is read.  The
// gathered values land element by element in shared memory ([e][k][j][i], a
// node shared by two elements of the unit twice), which is the tiles' row
// layout; each element's results overwrite its own values there, and the
// scatter adds the two copies of a shared node.  The next unit's nodes are
// gathered by cp.async while the current one is computed, and its metric,
// stored in the order the threads read it (setup_metric_tc), is prefetched
// into L2.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "sem_internal.cuh"

namespace sem {

template <int P>
struct TcCfg {
  static constexpr int N = P + 1, NP = N * N, N3 = NP * N;
  static constexpr int EPT = 16 / N;              // elements per 16-row tile
  static constexpr int ROWS = EPT * N;            // rows of a tile that hold element planes
  static constexpr int NG = (NP + 7) / 8;         // groups of 8 points
  static constexpr int KS1 = (NG + 1) / 2;        // k-steps of the in-plane gradient (K = n^2 padded)
  static constexpr int NT1 = 2 * NG;              // n-tiles of the in-plane gradient (gx, gy per group)
  static constexpr int KS2 = NG;                  // k-steps of the transposed in-plane product
  static constexpr int NT2 = NG;                  // n-tiles of outputs per row (points)
  static constexpr int MTU = 2;                   // tiles per unit
  static constexpr int G = MTU * EPT;             // elements per unit
  static constexpr int L = P * G + 1;             // nodes per line of a unit
  static constexpr int QPITCH = 16 * KS1 + 8;     // bf16 qz tile row pitch (halves): conflict-free ldmatrix
  // element-by-element stage: rows e n + k of n^2 values; the reads of a tile's
  // padding rows and columns run past the unit's last row into a zeroed tail
  static constexpr int STAGE = ((MTU * ROWS + 16 - ROWS) * NP + 16 * KS1 + 3) / 4 * 4;  // floats
  static constexpr int NB1 = KS1 * NT1, NB2 = KS2 * NT2;  // B fragments (hi and lo pairs) per lane
  static constexpr int NFRAG = 4 * NB1 + 4 * NB2 + 16;  // constant fragment words per lane
  static constexpr int WARPS = 4;                       // independent warps per CTA
  // metric records of a tile: point group m, half h (rows g / g + 8); per valid
  // lane the 7 bf16 pairs as [lane][4] (components 0-3), [lane][2] (4-5), [lane] (6)
  __host__ __device__ static constexpr int tmax(int m) {
    return (NP - 8 * m) >= 8 ? 4 : (NP - 8 * m + 1) / 2;
  }
  __host__ __device__ static constexpr int gmax(int h) {
    return ROWS - 8 * h >= 8 ? 8 : (ROWS - 8 * h > 0 ? ROWS - 8 * h : 0);
  }
  __host__ __device__ static constexpr int cnt(int m, int h) { return gmax(h) * tmax(m); }
  __host__ __device__ static constexpr int rec_words(int m, int h) { return (7 * cnt(m, h) + 3) / 4 * 4; }
  __host__ __device__ static constexpr int rec_base(int m, int h) {
    int o = 0;
    for (int mm = 0; mm < NG; ++mm)
      for (int hh = 0; hh < 2; ++hh) {
        if (mm == m && hh == h) return o;
        o += rec_words(mm, hh);
      }
    return o;
  }
  static constexpr int MT_WORDS = rec_base(NG, 0);            // words of one tile's metric
  static constexpr int UNIT_WORDS = MTU * MT_WORDS;            // a multiple of 4: 16-byte aligned units
  // per warp: two element stages (the second use of a stage is the scatter
  // staging) and the bf16 qz tiles (hi, lo); per CTA the constant B fragments
  static constexpr size_t warp_bytes = (2 * (size_t)STAGE * 4 + (size_t)2 * 16 * QPITCH * 2 + 15) / 16 * 16;
  static constexpr size_t const_bytes = (size_t)(NB1 + NB2) * 32 * 16;
  static constexpr size_t cta_bytes = const_bytes + WARPS * warp_bytes;
  static_assert(L <= 32, "a unit line must fit one warp");
  static_assert(EPT >= 1 && ROWS <= 16, "tile rows");
  static_assert(UNIT_WORDS % 4 == 0, "16-byte aligned metric blocks");
};

struct TcArgs {
  const float* u;
  float* y;
  const uint32_t* metric;  // setup_metric_tc layout
  const uint32_t* frag;    // constant MMA fragments [NFRAG][32]
  int nx, ny, nz;          // elements per direction
  int NX, NY;              // nodes per direction (x, y)
  int upr;                 // units per element row
  int nunits;
  float mass_coef, out_scale;
  int scale_out;
  const int* done;
  int64_t ndofs;             // SEM_DEBUG index checks
  unsigned long long* dbg;
};

namespace {

__device__ __forceinline__ void mma16816(float (&c)[4], const uint32_t (&a)[4], uint32_t b0, uint32_t b1) {
  asm(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
      "{%0,%1,%2,%3};\n"
      : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

__device__ __forceinline__ void ldsm_x2_t(uint32_t& r0, uint32_t& r1, unsigned addr) {
  asm volatile("ldmatrix.sync.aligned.m8n8.x2.trans.shared.b16 {%0,%1}, [%2];\n"
               : "=r"(r0), "=r"(r1)
               : "r"(addr));
}

// Two floats as a bf16 pair (round to nearest even): lo in the low half.
__device__ __forceinline__ uint32_t pack_bf16(float lo, float hi) {
  uint32_t d;
  asm("cvt.rn.bf16x2.f32 %0, %1, %2;\n" : "=r"(d) : "f"(hi), "f"(lo));
  return d;
}
__device__ __forceinline__ float bf_lo(uint32_t w) { return __uint_as_float(w << 16); }
__device__ __forceinline__ float bf_hi(uint32_t w) { return __uint_as_float(w & 0xffff0000u); }
// hi and lo bf16 pairs of two floats: v = hi + lo to about 2^-16 relative
__device__ __forceinline__ void split_bf16(float v0, float v1, uint32_t& hi, uint32_t& lo) {
  hi = pack_bf16(v0, v1);
  lo = pack_bf16(v0 - bf_lo(hi), v1 - bf_hi(hi));
}

// Packed pair arithmetic (two FP32 lanes in one 64-bit register pair).
__device__ __forceinline__ unsigned long long f2(float lo, float hi) {
  unsigned long long d;
  asm("mov.b64 %0, {%1, %2};\n" : "=l"(d) : "f"(lo), "f"(hi));
  return d;
}
__device__ __forceinline__ void f2split(unsigned long long v, float& lo, float& hi) {
  asm("mov.b64 {%0, %1}, %2;\n" : "=f"(lo), "=f"(hi) : "l"(v));
}
__device__ __forceinline__ unsigned long long fma2(unsigned long long a, unsigned long long b,
                                                   unsigned long long c) {
  unsigned long long d;
  asm("fma.rn.f32x2 %0, %1, %2, %3;\n" : "=l"(d) : "l"(a), "l"(b), "l"(c));
  return d;
}
__device__ __forceinline__ unsigned long long mul2(unsigned long long a, unsigned long long b) {
  unsigned long long d;
  asm("mul.rn.f32x2 %0, %1, %2;\n" : "=l"(d) : "l"(a), "l"(b));
  return d;
}
__device__ __forceinline__ unsigned long long bf2(uint32_t w) { return f2(bf_lo(w), bf_hi(w)); }
__device__ __forceinline__ uint32_t pack2(unsigned long long v) {
  float lo, hi;
  f2split(v, lo, hi);
  return pack_bf16(lo, hi);
}

__device__ __forceinline__ void cp4(void* dst, const void* src) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"((unsigned)__cvta_generic_to_shared(dst)),
               "l"(src)
               : "memory");
}

// Position of unit `unit` in the slab: first element (ex0, ey, ez) and its
// number of elements.
struct UnitPos {
  int ex0, ey, ez, gv;
};
template <int P>
__device__ __forceinline__ UnitPos unit_pos(const TcArgs& a, int unit) {
  using C = TcCfg<P>;
  const int r = unit / a.upr, s = unit - r * a.upr;
  UnitPos q;
  q.ey = r % a.ny;
  q.ez = r / a.ny;
  q.ex0 = s * C::G;
  q.gv = min(C::G, a.nx - q.ex0);
  return q;
}

// Global index of node x of line (k, j) of a unit.
__device__ __forceinline__ int64_t line_base(const TcArgs& a, const UnitPos& q, int P, int k, int j) {
  return ((int64_t)(P * q.ez + k) * a.NY + (P * q.ey + j)) * a.NX + (int64_t)P * q.ex0;
}

}  // namespace

template <int P>
__global__ void __launch_bounds__(TcCfg<P>::WARPS * 32, 3) sem_apply_tc_kernel(const TcArgs a) {
  pdl_entry();
  using C = TcCfg<P>;
  constexpr int N = C::N, NP = C::NP, N3 = C::N3, EPT = C::EPT, ROWS = C::ROWS, NG = C::NG;
  constexpr int KS1 = C::KS1, NT1 = C::NT1, NT2 = C::NT2, MTU = C::MTU;
  constexpr int QPITCH = C::QPITCH, STAGE = C::STAGE, UW = C::UNIT_WORDS;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  if (a.done != nullptr && *a.done) return;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int g = lane >> 2, t = lane & 3;

  // constant fragments of the CTA: (hi0, hi1, lo0, lo1) of B1 per (ks, nt), then of B2
  uint4* sB = reinterpret_cast<uint4*>(smem_raw);
  for (int i = threadIdx.x; i < (C::NB1 + C::NB2) * 32; i += blockDim.x) {
    const int f = i >> 5, ln = i & 31;
    sB[i] = make_uint4(__ldg(a.frag + (4 * f) * 32 + ln), __ldg(a.frag + (4 * f + 1) * 32 + ln),
                       __ldg(a.frag + (4 * f + 2) * 32 + ln), __ldg(a.frag + (4 * f + 3) * 32 + ln));
  }
  uint32_t azh[4], azl[4], azth[4], aztl[4];
  {
    const uint32_t* fz = a.frag + 4 * (C::NB1 + C::NB2) * 32 + lane;
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      azh[i] = __ldg(fz + 32 * i);
      azl[i] = __ldg(fz + 32 * (4 + i));
      azth[i] = __ldg(fz + 32 * (8 + i));
      aztl[i] = __ldg(fz + 32 * (12 + i));
    }
  }
  __syncthreads();  // the only CTA-wide barrier: the warps run independently from here

  unsigned char* wb = smem_raw + C::const_bytes + (size_t)warp * C::warp_bytes;
  float* sSt = reinterpret_cast<float*>(wb);                                 // [2][STAGE]
  unsigned short* sQz = reinterpret_cast<unsigned short*>(sSt + 2 * STAGE);  // [2][16][QPITCH] (hi, lo)
  const uint4* pB1 = sB + lane;
  const uint4* pB2 = sB + 32 * C::NB1 + lane;

  int unit = blockIdx.x * C::WARPS + warp;
  if (unit >= a.nunits) return;  // no CTA-wide barrier follows
  const int stride = gridDim.x * C::WARPS;

  // zero both stages (the tails past the last element stay zero) and the qz tiles
  for (int i = lane; i < 2 * STAGE + 16 * QPITCH; i += 32) sSt[i] = 0.f;
  __syncwarp();

  const unsigned sQz_addr = (unsigned)__cvta_generic_to_shared(sQz);
  const int lq = lane >> 3, lr = lane & 7;

  // the unit's nodes into stage `buf` element by element (4-byte cp.async; a node on
  // the face between elements e - 1 and e of the unit goes to both), and an L2
  // prefetch of its metric block
  auto issue = [&](int un, int buf) {
    const UnitPos q = unit_pos<P>(a, un);
    const int x = lane, lv = P * q.gv;
    float* dst = sSt + buf * STAGE;
    if (x <= lv) {
      const int e = min(x / P, q.gv - 1), i = x - P * e;
      const bool dup = i == 0 && e > 0;
      const int o1 = e * N3 + i, o2 = dup ? (e - 1) * N3 + P : 0;
#pragma unroll
      for (int rr = 0; rr < NP; ++rr) {
        const int k = rr / N, j = rr - k * N;
        const float* src = a.u + SEM_IDX(line_base(a, q, P, k, j) + x, a.ndofs, a.dbg, kDbgLine);
        cp4(dst + o1 + k * NP + j * N, src);
        if (dup) cp4(dst + o2 + k * NP + j * N, src);
      }
    }
    if (lane == 0)
      asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;\n" ::"l"(a.metric + (size_t)un * UW),
                   "r"((unsigned)(UW * 4))
                   : "memory");
  };

  issue(unit, 0);
  asm volatile("cp.async.commit_group;\n" ::: "memory");
  int b = 0;
  for (; unit < a.nunits; unit += stride) {
    const int nxt = unit + stride;
    if (nxt < a.nunits) issue(nxt, b ^ 1);
    asm volatile("cp.async.commit_group;\n" ::: "memory");
    asm volatile("cp.async.wait_group 1;\n" ::: "memory");
    __syncwarp();
    const UnitPos q = unit_pos<P>(a, unit);
    float* st = sSt + b * STAGE;
    const uint32_t* gmet = a.metric + (size_t)unit * UW;

#pragma unroll 1
    for (int mt = 0; mt < MTU; ++mt) {
      const float* tu = st + mt * ROWS * NP;  // row r of the tile at tu + r NP
      // in-plane gradient: u (hi, lo) as the A operand, the derivative (hi, lo) as B
      float c1[NT1][4];
#pragma unroll
      for (int nt = 0; nt < NT1; ++nt) c1[nt][0] = c1[nt][1] = c1[nt][2] = c1[nt][3] = 0.f;
#pragma unroll
      for (int ks = 0; ks < KS1; ++ks) {
        uint32_t ah[4], al[4];
#pragma unroll
        for (int rg = 0; rg < 4; ++rg) {  // (row g + 8 (rg & 1), columns 16 ks + 8 (rg >> 1) + 2t, +1)
          const float* pu = tu + (g + 8 * (rg & 1)) * NP + 16 * ks + 8 * (rg >> 1) + 2 * t;
          split_bf16(pu[0], pu[1], ah[rg], al[rg]);
        }
        // consecutive products go to different accumulators (no dependent MMA pairs)
        uint4 bb[NT1];
#pragma unroll
        for (int nt = 0; nt < NT1; ++nt) bb[nt] = pB1[32 * (ks * NT1 + nt)];
#pragma unroll
        for (int nt = 0; nt < NT1; ++nt) mma16816(c1[nt], ah, bb[nt].x, bb[nt].y);
#pragma unroll
        for (int nt = 0; nt < NT1; ++nt) mma16816(c1[nt], ah, bb[nt].z, bb[nt].w);
#pragma unroll
        for (int nt = 0; nt < NT1; ++nt) mma16816(c1[nt], al, bb[nt].x, bb[nt].y);
      }
      // z-gradient: Z (rows) times u (columns = points): u read transposed as the B operand
      float cz[NT2][4];
      uint32_t bzh[NT2][2], bzl[NT2][2];
#pragma unroll
      for (int nt = 0; nt < NT2; ++nt) {
        const float* pu = tu + 2 * t * NP + 8 * nt + g;
        split_bf16(pu[0], pu[NP], bzh[nt][0], bzl[nt][0]);
        split_bf16(pu[8 * NP], pu[9 * NP], bzh[nt][1], bzl[nt][1]);
        cz[nt][0] = cz[nt][1] = cz[nt][2] = cz[nt][3] = 0.f;
      }
#pragma unroll
      for (int nt = 0; nt < NT2; ++nt) mma16816(cz[nt], azh, bzh[nt][0], bzh[nt][1]);
#pragma unroll
      for (int nt = 0; nt < NT2; ++nt) mma16816(cz[nt], azl, bzh[nt][0], bzh[nt][1]);
#pragma unroll
      for (int nt = 0; nt < NT2; ++nt) mma16816(cz[nt], azh, bzl[nt][0], bzl[nt][1]);
      // quadrature-point stage, point group by point group; the thread's points are
      // (row g + 8h, point 8m + 2t + s)
      float yc[NT2][4];
#pragma unroll
      for (int nt = 0; nt < NT2; ++nt) yc[nt][0] = yc[nt][1] = yc[nt][2] = yc[nt][3] = 0.f;
      const uint32_t* mtm = gmet + mt * C::MT_WORDS;
      const unsigned long long mc2 = f2(a.mass_coef, a.mass_coef);
#pragma unroll
      for (int m = 0; m < NG; ++m) {
        uint32_t aqh[4], aql[4];
#pragma unroll
        for (int h = 0; h < 2; ++h) {
          const int tm = C::tmax(m), cn = C::cnt(m, h);
          const bool ok = g < C::gmax(h) && t < tm;
          const int idx = ok ? g * tm + t : 0;
          const uint32_t* rec = mtm + C::rec_base(m, h);
          uint4 w03 = make_uint4(0u, 0u, 0u, 0u);
          uint2 w45 = make_uint2(0u, 0u);
          uint32_t w6 = 0u;
          if (ok) {
            w03 = __ldg(reinterpret_cast<const uint4*>(rec) + idx);
            w45 = __ldg(reinterpret_cast<const uint2*>(rec + 4 * cn) + idx);
            w6 = __ldg(rec + 6 * cn + idx);
          }
          const float* pu = tu + (g + 8 * h) * NP + 8 * m + 2 * t;
          const unsigned long long uu = f2(pu[0], pu[1]);
          const unsigned long long gx = f2(c1[2 * m][2 * h], c1[2 * m][2 * h + 1]);
          const unsigned long long gy = f2(c1[2 * m + 1][2 * h], c1[2 * m + 1][2 * h + 1]);
          const unsigned long long gz = f2(cz[m][2 * h], cz[m][2 * h + 1]);
          const unsigned long long G00 = bf2(w03.x), G01 = bf2(w03.y), G02 = bf2(w03.z);
          const unsigned long long G11 = bf2(w03.w), G12 = bf2(w45.x), G22 = bf2(w45.y), Wq = bf2(w6);
          const unsigned long long qx = fma2(G02, gz, fma2(G01, gy, mul2(G00, gx)));
          const unsigned long long qy = fma2(G12, gz, fma2(G11, gy, mul2(G01, gx)));
          const unsigned long long qz = fma2(G22, gz, fma2(G12, gy, mul2(G02, gx)));
          float m0, m1;
          f2split(mul2(mul2(mc2, Wq), uu), m0, m1);
          yc[m][2 * h] += m0;
          yc[m][2 * h + 1] += m1;
          float v0, v1;
          f2split(qx, v0, v1);
          split_bf16(v0, v1, aqh[h], aql[h]);
          f2split(qy, v0, v1);
          split_bf16(v0, v1, aqh[2 + h], aql[2 + h]);
          f2split(qz, v0, v1);
          uint32_t zh, zl;
          split_bf16(v0, v1, zh, zl);
          const int wq = ((g + 8 * h) * QPITCH + 8 * m + 2 * t) / 2;
          reinterpret_cast<uint32_t*>(sQz)[wq] = zh;
          reinterpret_cast<uint32_t*>(sQz)[8 * QPITCH + wq] = zl;
        }
        // this group's share of the transposed in-plane product
        uint4 bb[NT2];
#pragma unroll
        for (int nt = 0; nt < NT2; ++nt) bb[nt] = pB2[32 * (m * NT2 + nt)];
#pragma unroll
        for (int nt = 0; nt < NT2; ++nt) mma16816(yc[nt], aqh, bb[nt].x, bb[nt].y);
#pragma unroll
        for (int nt = 0; nt < NT2; ++nt) mma16816(yc[nt], aqh, bb[nt].z, bb[nt].w);
#pragma unroll
        for (int nt = 0; nt < NT2; ++nt) mma16816(yc[nt], aql, bb[nt].x, bb[nt].y);
      }
      __syncwarp();
      // transposed z-contraction
      uint32_t qh[NT2][2], ql[NT2][2];
#pragma unroll
      for (int nt = 0; nt < NT2; ++nt) {
        const unsigned ad = sQz_addr + (unsigned)(((lr + 8 * (lq & 1)) * QPITCH + 8 * nt) * 2);
        ldsm_x2_t(qh[nt][0], qh[nt][1], ad);
        ldsm_x2_t(ql[nt][0], ql[nt][1], ad + (unsigned)(16 * QPITCH * 2));
      }
#pragma unroll
      for (int nt = 0; nt < NT2; ++nt) mma16816(yc[nt], azth, qh[nt][0], qh[nt][1]);
#pragma unroll
      for (int nt = 0; nt < NT2; ++nt) mma16816(yc[nt], aztl, qh[nt][0], qh[nt][1]);
#pragma unroll
      for (int nt = 0; nt < NT2; ++nt) mma16816(yc[nt], azth, ql[nt][0], ql[nt][1]);
      // the tile's element results over its own nodal values in the stage (the
      // other tile of the unit reads and writes other rows)
      const bool rows_ok0 = g < ROWS && mt * EPT + g / N < q.gv;
      const bool rows_ok1 = g + 8 < ROWS && mt * EPT + (g + 8) / N < q.gv;
      float* ty = st + mt * ROWS * NP;
#pragma unroll
      for (int nt = 0; nt < NT2; ++nt) {
#pragma unroll
        for (int s2 = 0; s2 < 2; ++s2) {
          const int pt = 8 * nt + 2 * t + s2;
          if (pt < NP) {
            if (rows_ok0) ty[g * NP + pt] = yc[nt][s2];
            if (rows_ok1) ty[(g + 8) * NP + pt] = yc[nt][2 + s2];
          }
        }
      }
      __syncwarp();  // the qz tiles are rewritten by the next tile
    }
    // scatter-add the unit's lines: node x = P e + i is (e, i) of the stage, and
    // x = P e (0 < e) also (e - 1, P)
    {
      const float sc = a.scale_out ? a.out_scale : 1.f;
      const int x = lane;
      const int lv = P * q.gv;
      if (x <= lv) {
        const int e = x / P, i = x - P * e;
        const bool own = x < lv, face = i == 0 && e > 0;
        const int o1 = own ? e * N3 + i : 0, o2 = face ? (e - 1) * N3 + P : 0;
#pragma unroll 5
        for (int rr = 0; rr < NP; ++rr) {
          const int k = rr / N, j = rr - k * N;
          float v = own ? st[o1 + k * NP + j * N] : 0.f;
          if (face) v += st[o2 + k * NP + j * N];
          atomicAdd(a.y + SEM_IDX(line_base(a, q, P, k, j) + x, a.ndofs, a.dbg, kDbgLine), v * sc);
        }
      }
    }
    __syncwarp();  // this stage is refilled two units later
    b ^= 1;
  }
  asm volatile("cp.async.wait_group 0;\n" ::: "memory");
}

// ---------------------------------------------------------------------------
// Host side: constant fragments, the metric layout and the launcher.

namespace {

uint16_t bf16_host(float f) {
  uint32_t u;
  std::memcpy(&u, &f, 4);
  const uint32_t lsb = (u >> 16) & 1u;
  u += 0x7fffu + lsb;  // round to nearest even (finite inputs)
  return (uint16_t)(u >> 16);
}
double bf16_value(uint16_t h) {
  const uint32_t u = (uint32_t)h << 16;
  float f;
  std::memcpy(&f, &u, 4);
  return f;
}
uint32_t pack_host(double lo, double hi) {
  return (uint32_t)bf16_host((float)lo) | ((uint32_t)bf16_host((float)hi) << 16);
}

// bf16 pair of the residuals v - bf16(v)
uint32_t pack_host_lo(double lo, double hi) {
  const double rl = lo - bf16_value(bf16_host((float)lo));
  const double rh = hi - bf16_value(bf16_host((float)hi));
  return pack_host(rl, rh);
}

// Fragments [NFRAG][32] of one degree: per (ks, nt) of B1 (in-plane gradient:
// D along i for gx, D along j for gy) the hi pair and the lo pair, the same for
// B2 (transposed in-plane product), then Z hi, Z lo, Z^T hi, Z^T lo as A
// operands (4 words each).
template <int P>
bool tc_fragments(const Tables1D& tab, std::vector<uint32_t>& f) {
  using C = TcCfg<P>;
  constexpr int N = C::N, NP = C::NP;
  auto Dx = [&](int pt, int q) {  // d/dxi of basis q at point pt (same j)
    if (pt >= NP || q >= NP) return 0.0;
    const int ip = pt % N, jp = pt / N, i = q % N, j = q / N;
    return j == jp ? tab.D[ip][i] : 0.0;
  };
  auto Dy = [&](int pt, int q) {
    if (pt >= NP || q >= NP) return 0.0;
    const int ip = pt % N, jp = pt / N, i = q % N, j = q / N;
    return i == ip ? tab.D[jp][j] : 0.0;
  };
  auto B1 = [&](int kk, int col) {  // K: basis q = kk; column block 2m + d, point 8m + col % 8
    const int nt = col / 8, m = nt / 2, d = nt % 2, pt = 8 * m + col % 8;
    return d == 0 ? Dx(pt, kk) : Dy(pt, kk);
  };
  auto B2 = [&](int kk, int col) {  // K: (qx or qy of point 8 ks + c % 8); column: basis q
    const int ks = kk / 16, c = kk % 16, pt = 8 * ks + c % 8;
    return c < 8 ? Dx(pt, col) : Dy(pt, col);
  };
  auto Z = [&](int r, int c) {  // rows (element, k'), columns (element, k): D[k'][k]
    if (r >= C::ROWS || c >= C::ROWS || r / N != c / N) return 0.0;
    return tab.D[r % N][c % N];
  };
  auto ZT = [&](int r, int c) {  // rows (element, k), columns (element, k'): D[k'][k]
    if (r >= C::ROWS || c >= C::ROWS || r / N != c / N) return 0.0;
    return tab.D[c % N][r % N];
  };
  f.assign((size_t)C::NFRAG * 32, 0u);
  for (int lane = 0; lane < 32; ++lane) {
    const int g = lane >> 2, t = lane & 3;
    int r = 0;
    for (int which = 0; which < 2; ++which)
      for (int ks = 0; ks < (which ? C::KS2 : C::KS1); ++ks)
        for (int nt = 0; nt < (which ? C::NT2 : C::NT1); ++nt) {
          const int col = 8 * nt + g, k0 = 16 * ks + 2 * t;
          auto B = [&](int kk) { return which ? B2(kk, col) : B1(kk, col); };
          f[32 * r++ + lane] = pack_host(B(k0), B(k0 + 1));
          f[32 * r++ + lane] = pack_host(B(k0 + 8), B(k0 + 9));
          f[32 * r++ + lane] = pack_host_lo(B(k0), B(k0 + 1));
          f[32 * r++ + lane] = pack_host_lo(B(k0 + 8), B(k0 + 9));
        }
    for (int which = 0; which < 4; ++which) {
      auto A = [&](int rr, int cc) { return which < 2 ? Z(rr, cc) : ZT(rr, cc); };
      auto pk = (which & 1) ? pack_host_lo : pack_host;
      f[32 * r++ + lane] = pk(A(g, 2 * t), A(g, 2 * t + 1));
      f[32 * r++ + lane] = pk(A(g + 8, 2 * t), A(g + 8, 2 * t + 1));
      f[32 * r++ + lane] = pk(A(g, 2 * t + 8), A(g, 2 * t + 9));
      f[32 * r++ + lane] = pk(A(g + 8, 2 * t + 8), A(g + 8, 2 * t + 9));
    }
  }
  return true;
}

// One thread per 32-bit word of the tensor-core metric: the bf16 pair of
// component c at the two points (row g + 8h, points 8m + 2t, 8m + 2t + 1) of
// tile mt of unit u, zero for points, rows and elements outside the mesh.
template <int P>
__global__ void k_metric_tc(int64_t nwords, int nx, int ny, int upr, const double* __restrict__ metric,
                            uint32_t* __restrict__ out) {
  pdl_entry();
  using C = TcCfg<P>;
  constexpr int N = C::N, NP = C::NP, N3P = padded_n3(N);
  for (int64_t w = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; w < nwords;
       w += (int64_t)gridDim.x * blockDim.x) {
    const int64_t un = w / C::UNIT_WORDS;
    const int rem = (int)(w - un * C::UNIT_WORDS);
    const int mt = rem / C::MT_WORDS;
    int off = rem - mt * C::MT_WORDS;
    int m = 0, h = 0;
    for (int mm = 0; mm < C::NG; ++mm)
      for (int hh = 0; hh < 2; ++hh) {
        const int rb = C::rec_base(mm, hh), rw = C::rec_words(mm, hh);
        if (off >= rb && off < rb + rw) { m = mm; h = hh; }
      }
    off -= C::rec_base(m, h);
    const int cn = C::cnt(m, h), tm = C::tmax(m);
    int c = -1, idx = 0;
    if (off < 4 * cn) { c = off % 4; idx = off / 4; }
    else if (off < 6 * cn) { c = 4 + (off - 4 * cn) % 2; idx = (off - 4 * cn) / 2; }
    else if (off < 7 * cn) { c = 6; idx = off - 6 * cn; }
    uint32_t val = 0u;
    if (c >= 0) {
      const int g = idx / tm, t = idx - g * tm;
      const int row = g + 8 * h;
      const int el = row / N, k = row - el * N;
      const int r = (int)(un / upr), s = (int)(un - (int64_t)r * upr);
      const int ey = r % ny, ez = r / ny, ex0 = s * C::G;
      const int e = mt * C::EPT + el;
      if (row < C::ROWS && ex0 + e < nx) {
        const int64_t elem = (int64_t)(ex0 + e) + (int64_t)nx * (ey + (int64_t)ny * ez);
        const double* blk = metric + elem * 7 * N3P + (int64_t)c * N3P;
        double v[2] = {0.0, 0.0};
        for (int sb = 0; sb < 2; ++sb) {
          const int pt = 8 * m + 2 * t + sb;
          if (pt < NP) {
            const int j = pt / N, i = pt - j * N;
            v[sb] = blk[i + N * j + N * N * k];
          }
        }
        const uint32_t lo = __bfloat16_as_ushort(__float2bfloat16_rn((float)v[0]));
        const uint32_t hi = __bfloat16_as_ushort(__float2bfloat16_rn((float)v[1]));
        val = lo | (hi << 16);
      }
    }
    out[w] = val;
  }
}

template <int P>
struct TcGrid {
  static inline int resident = 0;
};

template <int P>
cudaError_t tc_prime_p() {
  using C = TcCfg<P>;
  cudaError_t e = cudaFuncSetAttribute(sem_apply_tc_kernel<P>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)C::cta_bytes);
  int dev = 0, sms = 0, per_sm = 0;
  if (e == cudaSuccess) e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e == cudaSuccess)
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, sem_apply_tc_kernel<P>, C::WARPS * 32,
                                                      C::cta_bytes);
  if (e != cudaSuccess) return e;
  if (per_sm < 1) return cudaErrorInvalidConfiguration;
  TcGrid<P>::resident = sms * per_sm;
  return cudaSuccess;
}

template <int P>
int units_per_row(const Level& L) {
  return (L.nx + TcCfg<P>::G - 1) / TcCfg<P>::G;
}

template <int P>
size_t tc_metric_words_p(const Level& L) {
  return (size_t)units_per_row<P>(L) * L.ny * L.nz * TcCfg<P>::UNIT_WORDS;
}

template <int P>
cudaError_t setup_tc_p(Level& L, cudaStream_t s) {
  std::vector<uint32_t> f;
  if (!tc_fragments<P>(L.tab, f)) return cudaErrorInvalidValue;
  cudaError_t e;
  if (!L.tc_frag && (e = cudaMalloc(&L.tc_frag, sizeof(uint32_t) * f.size())) != cudaSuccess) return e;
  if ((e = cudaMemcpyAsync(L.tc_frag, f.data(), sizeof(uint32_t) * f.size(), cudaMemcpyHostToDevice, s)) !=
      cudaSuccess)
    return e;
  const int64_t nw = (int64_t)tc_metric_words_p<P>(L);
  const int threads = 256;
  const int blocks = (int)std::min<int64_t>((nw + threads - 1) / threads, 152 * 16);
  launch_k(k_metric_tc<P>, blocks, threads, 0, s, nw, L.nx, L.ny, units_per_row<P>(L), L.metric, L.metric_tc);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  // the fragments' host vector must outlive the copy
  return cudaStreamSynchronize(s);
}

template <int P>
cudaError_t launch_tc_p(const Level& L, const ApplyArgs<float, __nv_bfloat16>& a, cudaStream_t s) {
  using C = TcCfg<P>;
  const int resident = TcGrid<P>::resident;
  if (resident < 1) return cudaErrorInitializationError;  // prime_apply_kernels was not called
  TcArgs t{};
  t.u = a.u;
  t.y = a.y;
  t.metric = L.metric_tc;
  t.frag = L.tc_frag;
  t.nx = L.nx; t.ny = L.ny; t.nz = L.nz;
  t.NX = L.p * L.nx + 1;
  t.NY = L.p * L.ny + 1;
  t.upr = units_per_row<P>(L);
  t.nunits = t.upr * L.ny * L.nz;
  t.mass_coef = a.mass_coef;
  t.out_scale = a.out_scale;
  t.scale_out = a.scale_out;
  t.done = a.done;
  t.ndofs = L.ndofs;
  t.dbg = L.dbg;
  const int grid = std::min(resident, (t.nunits + C::WARPS - 1) / C::WARPS);
  if (grid == 0) return cudaSuccess;
  launch_k(sem_apply_tc_kernel<P>, grid, C::WARPS * 32, C::cta_bytes, s, t);
  return cudaGetLastError();
}

}  // namespace

bool tc_supported(const Level& L) { return L.quad == SEM_QUAD_LGL && L.p >= 2 && L.p <= 4; }

size_t tc_metric_words(const Level& L) {
  switch (L.p) {
    case 2: return tc_metric_words_p<2>(L);
    case 3: return tc_metric_words_p<3>(L);
    case 4: return tc_metric_words_p<4>(L);
    default: return 0;
  }
}

cudaError_t setup_metric_tc(Level& L, cudaStream_t s) {
  if (!tc_supported(L)) return cudaErrorInvalidValue;
  cudaError_t e = cudaSuccess;
  if (!L.metric_tc && (e = cudaMalloc(&L.metric_tc, sizeof(uint32_t) * tc_metric_words(L))) != cudaSuccess)
    return e;
  switch (L.p) {
    case 2: e = setup_tc_p<2>(L, s); break;
    case 3: e = setup_tc_p<3>(L, s); break;
    case 4: e = setup_tc_p<4>(L, s); break;
    default: return cudaErrorInvalidValue;
  }
  if (e == cudaSuccess) L.metric_tc_valid = true;
  return e;
}

cudaError_t launch_apply_tc(const Level& L, const ApplyArgs<float, __nv_bfloat16>& a, cudaStream_t s) {
  if (!tc_supported(L) || !L.metric_tc_valid) return cudaErrorInvalidValue;
  switch (L.p) {
    case 2: return launch_tc_p<2>(L, a, s);
    case 3: return launch_tc_p<3>(L, a, s);
    case 4: return launch_tc_p<4>(L, a, s);
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t prime_apply_tc() {
  cudaError_t e;
  if ((e = tc_prime_p<2>()) != cudaSuccess) return e;
  if ((e = tc_prime_p<3>()) != cudaSuccess) return e;
  return tc_prime_p<4>();
}

}  // namespace sem
