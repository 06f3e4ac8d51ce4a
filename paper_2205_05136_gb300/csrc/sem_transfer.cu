// p-multigrid transfers between Q_pf and Q_pc on the same slab mesh
// (Section 4.3: transfers are matrix-vector products).
//
// On the structured slab lattice the global prolongation is the tensor product
// P = Pz Py Px of 1-D global prolongations: along x, fine node I of element
// e = min(I / pf, nx - 1) takes sum_a P[I - pf e][a] x_c[pc e + a], with
// P[i][a] = l^c_a(x^f_i) the 1-D interpolation matrix.  A node on an element
// boundary gets the same value from either element, because the interpolation
// is exact at the shared end points (rows 0 and pf of P are unit rows).  So
//   prolongation  x_f += P x_c, t_f = 0: three 1-D passes, coarse lattice ->
//                 (NXc, NYc, NZf) -> (NXc, NYf, NZf) -> fine lattice;
//   restriction   b_c = P^T (b_f - t_f): three 1-D passes the other way,
//                 coarse node A summing P1[I][A] over the fine nodes I of the
//                 elements that hold it, each fine node once.
// Each pass is one thread per output node reading a short run along one
// lattice axis: no shared memory, no barriers and no atomics, so the result is
// the same in every run (the deterministic mode needs no variant).  A CTA
// covers a 32 x 8 patch of a lattice plane and steps through the planes
// (stride gridDim.z): the grid stays within one wave of CTAs, because a grid of
// thousands of short CTAs costs more in block launches than its memory traffic.
#include <algorithm>

#include "sem_apply_kernel.cuh"
#include "sem_context.cuh"

namespace sem {
namespace {

constexpr int kTThreads = 256;

template <int NF, int NC, typename T>
struct PMat {
  T P[NF][NC];
};

enum { kProlong = 0, kProlongAdd = 1, kRestrict = 2, kRestrictDiff = 3 };
constexpr int kPassX = 32, kPassY = kTThreads / kPassX;  // CTA of a pass: 32 x 8 output nodes

// One 1-D pass along lattice axis AX (0 x, 1 y, 2 z) between degree pf = NF - 1
// and pc = NC - 1 on ne elements along that axis.  Output lattice d[0..2]; the
// input lattice is the same except along AX.
//   kProlong:      out = P in;           kProlongAdd:   out += P in, out2 = 0;
//   kRestrict:     out = P^T in;         kRestrictDiff: out = P^T (in - in2).
template <int NF, int NC, int AX, int MODE, typename T>
__global__ void __launch_bounds__(kTThreads)
    k_ptransfer_pass(int ne, int d0, int d1, int d2, const T* __restrict__ in, const T* __restrict__ in2,
                     T* __restrict__ out, T* __restrict__ out2, const __grid_constant__ PMat<NF, NC, T> pm,
                     const int* done) {
  pdl_entry();
  if (done != nullptr && *done) return;
  constexpr int PF = NF - 1, PC = NC - 1;
  constexpr bool PRO = MODE == kProlong || MODE == kProlongAdd;
  // output node (c0, c1, c2) from the grid: no index divisions
  const int c0 = blockIdx.x * kPassX + threadIdx.x;
  const int c1 = blockIdx.y * kPassY + threadIdx.y;
  if (c0 >= d0 || c1 >= d1) return;
  // input extent along AX and input strides
  const int nin = PRO ? PC * ne + 1 : PF * ne + 1;
  const int i0 = AX == 0 ? nin : d0, i1 = AX == 1 ? nin : d1;
  const int64_t stride = AX == 0 ? 1 : (AX == 1 ? (int64_t)i0 : (int64_t)i0 * i1);
#pragma unroll 1
  for (int c2 = blockIdx.z; c2 < d2; c2 += gridDim.z) {
    const int q = AX == 0 ? c0 : (AX == 1 ? c1 : c2);
    // input offset of the output's position with the AX coordinate at 0
    const int64_t base = AX == 0 ? (int64_t)i0 * ((int64_t)i1 * c2 + c1)
                                 : (AX == 1 ? c0 + (int64_t)i0 * i1 * c2 : c0 + (int64_t)i0 * c1);
    const int64_t o = c0 + (int64_t)d0 * (c1 + (int64_t)d1 * c2);
    T acc = T(0);
    if constexpr (PRO) {
      const int e = min(q / PF, ne - 1), i = q - PF * e;
      const T* src = in + base + (int64_t)(PC * e) * stride;
#pragma unroll
      for (int a = 0; a < NC; ++a) acc = fma(pm.P[i][a], src[a * stride], acc);
      if constexpr (MODE == kProlongAdd) {
        out[o] += acc;
        out2[o] = T(0);
      } else {
        out[o] = acc;
      }
    } else {
      auto val = [&](int I) {
        const int64_t k = base + (int64_t)I * stride;
        return MODE == kRestrictDiff ? in[k] - in2[k] : in[k];
      };
      const int e = min(q / PC, ne - 1), a = q - PC * e;
#pragma unroll
      for (int i = 0; i < NF; ++i) acc = fma(pm.P[i][a], val(PF * e + i), acc);
      if (a == 0 && e > 0) {  // a vertex of the element before too; its last fine node is counted above
#pragma unroll
        for (int i = 0; i < NF - 1; ++i) acc = fma(pm.P[i][PC], val(PF * (e - 1) + i), acc);
      }
      out[o] = acc;
    }
  }
}

// 32 x 8 patches of a plane in x and y; along z as many CTAs as keep the grid
// within 8 CTAs per SM (at least one plane each).
dim3 pass_grid(int d0, int d1, int d2) {
  const int gx = (d0 + kPassX - 1) / kPassX, gy = (d1 + kPassY - 1) / kPassY;
  const int gz = std::max(1, std::min(d2, (152 * 8) / std::max(1, gx * gy)));
  return dim3((unsigned)gx, (unsigned)gy, (unsigned)gz);
}

template <int NF, int NC, typename T>
cudaError_t launch_passes(bool prolong, const Level& F, const Level& C, const double (*P)[kMaxN],
                          const T* src_b, const T* src_t, T* dst, T* dst_t, T* w1, T* w2,
                          const int* done, cudaStream_t s) {
  PMat<NF, NC, T> pm;
  for (int i = 0; i < NF; ++i)
    for (int a = 0; a < NC; ++a) pm.P[i][a] = (T)P[i][a];
  const int nx = F.nx, ny = F.ny, nz = F.nz;
  const int xf = F.p * nx + 1, yf = F.p * ny + 1, zf = F.p * nz + 1;
  const int xc = C.p * nx + 1, yc = C.p * ny + 1, zc = C.p * nz + 1;
  if ((std::max(yf, yc) + kPassY - 1) / kPassY > 65535) return cudaErrorInvalidValue;  // grid y limit
  cudaError_t e;
  if (prolong) {  // coarse -> (xc, yc, zf) -> (xc, yf, zf) -> fine
    e = launch_k(k_ptransfer_pass<NF, NC, 2, kProlong, T>, pass_grid(xc, yc, zf), dim3(kPassX, kPassY), 0, s,
                 nz, xc, yc, zf, src_b, nullptr, w2, nullptr, pm, done);
    if (e == cudaSuccess)
      e = launch_k(k_ptransfer_pass<NF, NC, 1, kProlong, T>, pass_grid(xc, yf, zf), dim3(kPassX, kPassY), 0,
                   s, ny, xc, yf, zf, w2, nullptr, w1, nullptr, pm, done);
    if (e == cudaSuccess)
      e = launch_k(k_ptransfer_pass<NF, NC, 0, kProlongAdd, T>, pass_grid(xf, yf, zf), dim3(kPassX, kPassY),
                   0, s, nx, xf, yf, zf, w1, nullptr, dst, dst_t, pm, done);
  } else {  // fine -> (xc, yf, zf) -> (xc, yc, zf) -> coarse
    e = launch_k(k_ptransfer_pass<NF, NC, 0, kRestrictDiff, T>, pass_grid(xc, yf, zf), dim3(kPassX, kPassY),
                 0, s, nx, xc, yf, zf, src_b, src_t, w1, nullptr, pm, done);
    if (e == cudaSuccess)
      e = launch_k(k_ptransfer_pass<NF, NC, 1, kRestrict, T>, pass_grid(xc, yc, zf), dim3(kPassX, kPassY), 0,
                   s, ny, xc, yc, zf, w1, nullptr, w2, nullptr, pm, done);
    if (e == cudaSuccess)
      e = launch_k(k_ptransfer_pass<NF, NC, 2, kRestrict, T>, pass_grid(xc, yc, zc), dim3(kPassX, kPassY), 0,
                   s, nz, xc, yc, zc, w2, nullptr, dst, nullptr, pm, done);
  }
  return e;
}

}  // namespace

// prolong: dst (fine x) += P src_b (coarse x), dst_t (fine t) cleared.
// restrict: dst (coarse b) = P^T (src_b - src_t) (fine b, fine t).
// w1, w2: scratch of (NXc NYf NZf) and (NXc NYc NZf) entries.
template <typename T>
cudaError_t p_transfer(bool prolong, const Level& F, const Level& C, const double (*P)[kMaxN],
                       const T* src_b, const T* src_t, T* dst, T* dst_t, T* w1, T* w2, const int* done,
                       cudaStream_t s) {
  const int nf = F.n, nc = C.n;
#define SEM_PAIR(A, B) \
  if (nf == A && nc == B) return launch_passes<A, B, T>(prolong, F, C, P, src_b, src_t, dst, dst_t, w1, w2, done, s);
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

// Scratch entries of p_transfer between F and C.
size_t p_transfer_scratch(const Level& F, const Level& C, int which) {
  const size_t xc = (size_t)C.p * F.nx + 1, yf = (size_t)F.p * F.ny + 1, yc = (size_t)C.p * F.ny + 1,
               zf = (size_t)F.p * F.nz + 1;
  return which == 1 ? xc * yf * zf : xc * yc * zf;
}

template cudaError_t p_transfer<float>(bool, const Level&, const Level&, const double (*)[kMaxN],
                                       const float*, const float*, float*, float*, float*, float*,
                                       const int*, cudaStream_t);
template cudaError_t p_transfer<double>(bool, const Level&, const Level&, const double (*)[kMaxN],
                                        const double*, const double*, double*, double*, double*, double*,
                                        const int*, cudaStream_t);

}  // namespace sem
