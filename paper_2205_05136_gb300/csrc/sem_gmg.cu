// Geometric multigrid preconditioner (Section 4.3) and the flexible PCG it drives.
//
// Levels: the fine Q_p level, then p-coarsened levels on the same mesh
// (p -> max(1, p/2) -> ... -> 1), then 2:1 h-coarsened Q_1 levels (each
// direction's n elements -> ceil(n/2) elements built from every other vertex)
// until a level has at most `min_coarse_dofs` nodes.  Every level
// rediscretises alpha M + K with its own metric; a coarse element takes the
// tissue of its first fine child.
//
// Transfers (matrix-vector products, Section 4.3):
//   p-levels: per element, nodal interpolation Q_pc -> Q_pf by three 1-D
//     sweeps; restriction is its transpose, with each fine node's residual
//     divided by the number of elements sharing it so that the element-wise
//     sum equals P^T r;
//   h-levels: per fine vertex, the coarse trilinear function evaluated at the
//     reference coordinates -1, 0, +1 of the coarse element (a trailing odd
//     element spans one fine element: -1, +1); restriction by the transpose.
// Smoother: Chebyshev semi-iteration with point-Jacobi on [0.08, 1.2] x the
//   largest eigenvalue of D^{-1} A, estimated by 10 preconditioned CG
//   (Lanczos) steps from a fixed start vector; degree `degree` before and after
//   the coarse correction, degree `coarse_degree` on the coarsest level.
// Precision: the V-cycle runs in FP32 with an FP32 or bf16 metric, or in FP64;
//   the outer CG, its inner products and residual stay in FP64.  A V-cycle in
//   FP32 is not exactly symmetric, so the outer iteration is the flexible
//   (Polak-Ribiere) PCG: beta = r_{k+1} . (z_{k+1} - z_k) / (r_k . z_k).
#include <algorithm>
#include <cmath>
#include <string>
#include <vector>

#include "sem_apply_kernel.cuh"
#include "sem_context.cuh"
#include "sem_dfmath.cuh"

namespace sem {

// Separable p-transfers on the slab lattice (sem_transfer.cu); w1, w2 scratch of
// p_transfer_scratch(F, C, 1) and (F, C, 2) entries.
template <typename T>
cudaError_t p_transfer(bool prolong, const Level& F, const Level& C, const double (*P)[kMaxN],
                       const T* src_b, const T* src_t, T* dst, T* dst_t, T* w1, T* w2, const int* done,
                       cudaStream_t s);
size_t p_transfer_scratch(const Level& F, const Level& C, int which);

struct GmgLevel {
  Level* L = nullptr;
  bool owned = false;
  int to_next = 0;  // 0: p-transfer to the next level, 1: h-transfer
  double *sl = nullptr, *st = nullptr, *th = nullptr;
  bool owns_tissue = false;
  void *b = nullptr, *x = nullptr, *t = nullptr, *d = nullptr, *invd = nullptr;
  void *pw1 = nullptr, *pw2 = nullptr;  // p-transfer scratch towards the next level
  double* dinv64 = nullptr;
  double lam = 0.0;
};

struct Gmg {
  std::vector<GmgLevel> lv;
  double alpha = -1.0;
  int precision = SEM_PREC_FP32;
  int degree = 3, coarse_degree = 10;
  double* z = nullptr;                                 // outer PCG preconditioned residual
  // CUDA graphs of the PCG set-up and of one PCG iteration (V-cycle included),
  // keyed by the solution pointer and alpha; captured on a private stream.
  struct Graphs {
    const double* x = nullptr;
    const double* b = nullptr;
    double alpha = 0.0;
    double rtol = 0.0, atol = 0.0;
    cudaGraphExec_t init = nullptr, iter = nullptr;
    cudaGraphExec_t init_carried = nullptr;  // set-up from the carried A x (ws.Ax)
    cudaGraphExec_t init_checked = nullptr;  // the same where ws.same reads nonzero, else applied
    cudaGraphExec_t iter_timed = nullptr;    // an iteration with event nodes around two applies
    int64_t init_kernels = 0, iter_kernels = 0, init_carried_kernels = 0, init_checked_kernels = 0;
    int64_t iter_timed_kernels = 0;
    int last_iters = 0;  // iterations the previous solve with these graphs took
    // the set-up (variant v: applied, carried, checked) and its first `n` iterations
    // (the first one timed when t = 1) as one graph: one launch where five were
    struct Combo {
      cudaGraphExec_t exec = nullptr;
      int n = 0;
      int64_t kernels = 0;
    } combo[3][2];
  };
  Graphs graphs[16];
  int next_graph = 0;
  cudaStream_t capture = nullptr;
  cudaEvent_t ev0 = nullptr, ev1 = nullptr;           // recorded around the outer operator apply
  cudaEvent_t ev2 = nullptr, ev3 = nullptr;           // around the fine-level smoother apply
  double *lr = nullptr, *lz = nullptr, *lp = nullptr, *lAp = nullptr;  // Lanczos
  double* dots = nullptr;                              // device scalars
  double* partials = nullptr;
  unsigned int* tickets = nullptr;
  int partial_len = 0;
};

namespace {

constexpr int kThreads = 256;

int grid1d(int64_t n) {
  const int64_t g = (n + kThreads - 1) / kThreads;
  return (int)std::max<int64_t>(1, std::min<int64_t>(g, 152 * 8));
}

// Grid of a kernel that moves K entries per thread and iteration (16-byte
// chunks): one thread per chunk up to 8 CTAs per SM.  On a small level a grid
// sized by entries would launch 4x the CTAs, most of them without work.
template <typename T>
int grid_chunks(int64_t n) {
  constexpr int K = 16 / (int)sizeof(T);
  const int64_t g = (n / K + kThreads - 1) / kThreads;
  return (int)std::max<int64_t>(1, std::min<int64_t>(g, 152 * 8));
}

#define GRID_LOOP(i, n)                                                          \
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < (n); \
       i += (int64_t)gridDim.x * blockDim.x)

__device__ __forceinline__ bool skip(const int* done) { return done != nullptr && *done; }

inline bool aligned16(const void* p) { return (reinterpret_cast<uintptr_t>(p) & 15u) == 0; }

// ---------------------------------------------------------------- vectors
// Streaming vector kernels: consecutive entries are handled in 16-byte groups
// (4 floats or 2 doubles) by vector loads and stores, which keeps enough bytes
// in flight per thread to stream at HBM speed; the remaining n % K entries go
// one by one.  Level and workspace vectors come from cudaMalloc (256-byte
// aligned); kernels that also touch a caller's vector take a VEC flag that the
// host sets from the pointers' alignment.
template <typename T, int K>
struct alignas(K * sizeof(T)) Pk {
  T e[K];
};
template <typename T>
__host__ __device__ constexpr int k16() { return 16 / (int)sizeof(T); }

// Grid-stride loops over 16-byte chunks and over the scalar tail.  They stay
// rolled: with grids of 8 CTAs per SM a thread runs only a few iterations, and
// an unrolled body would only raise the register count (to 56-72 registers a
// thread, which halves the resident CTAs) without ever running.
#define GRID_CHUNKS(c, nc)                                                         \
  _Pragma("unroll 1")                                                              \
  for (int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; c < (nc);     \
       c += (int64_t)gridDim.x * blockDim.x)
#define GRID_TAIL(i, start, n)                                                     \
  _Pragma("unroll 1")                                                              \
  for (int64_t i = (start) + blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < (n); \
       i += (int64_t)gridDim.x * blockDim.x)

template <typename T>
__global__ void k_zero(int64_t n, T* x, const int* done) {
  pdl_entry();
  if (skip(done)) return;
  constexpr int K = k16<T>();
  const int64_t nc = n / K;
  GRID_CHUNKS(c, nc) reinterpret_cast<Pk<T, K>*>(x)[c] = Pk<T, K>{};
  GRID_TAIL(i, nc * K, n) x[i] = T(0);
}

template <typename T>
__global__ void k_level_inv_diag(int64_t n, double alpha, const double* m, const double* k,
                                 T* inv, double* inv64) {
  pdl_entry();
  GRID_LOOP(i, n) {
    const double v = 1.0 / fma(alpha, m[i], k[i]);
    inv[i] = (T)v;
    inv64[i] = v;
  }
}

// Chebyshev step 0 from a zero start: d = D^{-1} b / theta, x = d, t = 0.
template <typename T>
__global__ void k_cheb_zero_start(int64_t n, const T* __restrict__ b, const T* __restrict__ invd,
                                  T* __restrict__ x, T* __restrict__ d, T* __restrict__ t,
                                  T inv_theta, const int* done) {
  pdl_entry();
  if (skip(done)) return;
  constexpr int K = k16<T>();
  using V = Pk<T, K>;
  const int64_t nc = n / K;
  GRID_CHUNKS(c, nc) {
    const V bb = reinterpret_cast<const V*>(b)[c], ii = reinterpret_cast<const V*>(invd)[c];
    V dd;
#pragma unroll
    for (int k = 0; k < K; ++k) dd.e[k] = ii.e[k] * bb.e[k] * inv_theta;
    reinterpret_cast<V*>(d)[c] = dd;
    reinterpret_cast<V*>(x)[c] = dd;
    reinterpret_cast<V*>(t)[c] = V{};
  }
  GRID_TAIL(i, nc * K, n) {
    const T di = invd[i] * b[i] * inv_theta;
    d[i] = di;
    x[i] = di;
    t[i] = T(0);
  }
}

// Chebyshev step with t = A x: d = c1 d + c2 D^{-1}(b - t), x += d, t = 0
// (first: d = c2 D^{-1}(b - t)).
template <typename T>
__device__ __forceinline__ T cheb_d(T b, T t, T invd, T d, T c1, T c2, bool first) {
  const T ri = b - t;
  return first ? c2 * invd * ri : fma(c1, d, c2 * invd * ri);
}

template <typename T>
__global__ void k_cheb_step(int64_t n, const T* __restrict__ b, const T* __restrict__ invd,
                            T* __restrict__ x, T* __restrict__ d, T* __restrict__ t, T c1, T c2,
                            int first, const int* done) {
  pdl_entry();
  if (skip(done)) return;
  constexpr int K = k16<T>();
  using V = Pk<T, K>;
  const int64_t nc = n / K;
  GRID_CHUNKS(c, nc) {
    const V bb = reinterpret_cast<const V*>(b)[c], tt = reinterpret_cast<const V*>(t)[c];
    const V ii = reinterpret_cast<const V*>(invd)[c];
    V xx = reinterpret_cast<const V*>(x)[c];
    V dd = first ? V{} : reinterpret_cast<const V*>(d)[c];
#pragma unroll
    for (int k = 0; k < K; ++k) {
      dd.e[k] = cheb_d(bb.e[k], tt.e[k], ii.e[k], dd.e[k], c1, c2, first != 0);
      xx.e[k] += dd.e[k];
    }
    reinterpret_cast<V*>(d)[c] = dd;
    reinterpret_cast<V*>(x)[c] = xx;
    reinterpret_cast<V*>(t)[c] = V{};
  }
  GRID_TAIL(i, nc * K, n) {
    const T di = cheb_d(b[i], t[i], invd[i], first ? T(0) : d[i], c1, c2, first != 0);
    d[i] = di;
    x[i] += di;
    t[i] = T(0);
  }
}

// ---------------------------------------------------------------- transfers
struct PTab {
  int nf, nc;
  double P[kMaxN][kMaxN];  // P[i][a] = l^c_a(x^f_i)
};

// Coarse vertex k (and k+1) and weights of fine vertex I along one direction.
__device__ __forceinline__ void hweights(int I, int nf, int nc, int& k, double& w0, double& w1) {
  k = min(I / 2, nc - 1);
  const int t = I - 2 * k;
  if (2 * k + 2 <= nf) {  // coarse element made of two fine elements
    w0 = t == 0 ? 1.0 : (t == 1 ? 0.5 : 0.0);
  } else {                // trailing single fine element
    w0 = t == 0 ? 1.0 : 0.0;
  }
  w1 = 1.0 - w0;
}

template <typename T>
__global__ void k_prolong_h(int nfx, int nfy, int nfz, int ncx, int ncy, int ncz,
                            const T* __restrict__ xc, T* __restrict__ xf, T* __restrict__ tf,
                            const int* done) {
  pdl_entry();
  if (skip(done)) return;
  const int64_t NX = nfx + 1, NY = nfy + 1, n = NX * NY * (nfz + 1);
  const int64_t CX = ncx + 1, CY = ncy + 1;
  GRID_LOOP(g, n) {
    const int I = (int)(g % NX), J = (int)((g / NX) % NY), K = (int)(g / (NX * NY));
    int kx, ky, kz;
    double wx[2], wy[2], wz[2];
    hweights(I, nfx, ncx, kx, wx[0], wx[1]);
    hweights(J, nfy, ncy, ky, wy[0], wy[1]);
    hweights(K, nfz, ncz, kz, wz[0], wz[1]);
    T s = T(0);
    for (int c = 0; c < 2; ++c)
      for (int b = 0; b < 2; ++b)
        for (int a = 0; a < 2; ++a) {
          const double w = wx[a] * wy[b] * wz[c];
          if (w != 0.0) s += (T)w * xc[(kx + a) + CX * ((ky + b) + CY * (kz + c))];
        }
    xf[g] += s;
    tf[g] = T(0);
  }
}

template <typename T>
__global__ void k_restrict_h(int nfx, int nfy, int nfz, int ncx, int ncy, int ncz,
                             const T* __restrict__ bf, const T* __restrict__ tf,
                             T* __restrict__ bc, const int* done) {
  pdl_entry();
  if (skip(done)) return;
  const int64_t NX = nfx + 1, NY = nfy + 1, n = NX * NY * (nfz + 1);
  const int64_t CX = ncx + 1, CY = ncy + 1;
  GRID_LOOP(g, n) {
    const int I = (int)(g % NX), J = (int)((g / NX) % NY), K = (int)(g / (NX * NY));
    int kx, ky, kz;
    double wx[2], wy[2], wz[2];
    hweights(I, nfx, ncx, kx, wx[0], wx[1]);
    hweights(J, nfy, ncy, ky, wy[0], wy[1]);
    hweights(K, nfz, ncz, kz, wz[0], wz[1]);
    const T r = bf[g] - tf[g];
    for (int c = 0; c < 2; ++c)
      for (int b = 0; b < 2; ++b)
        for (int a = 0; a < 2; ++a) {
          const double w = wx[a] * wy[b] * wz[c];
          if (w != 0.0) atomicAdd(bc + (kx + a) + CX * ((ky + b) + CY * (kz + c)), (T)w * r);
        }
  }
}

// The same restriction gathered per coarse node (deterministic mode): the fine
// nodes within 3 of 2 C in each direction, in a fixed order, weighted by the
// trilinear prolongation's weight of that coarse node.
template <typename T>
__global__ void k_restrict_h_det(int nfx, int nfy, int nfz, int ncx, int ncy, int ncz,
                                 const T* __restrict__ bf, const T* __restrict__ tf,
                                 T* __restrict__ bc, const int* done) {
  pdl_entry();
  if (skip(done)) return;
  const int64_t NX = nfx + 1, NY = nfy + 1;
  const int64_t CX = ncx + 1, CY = ncy + 1, nc = CX * CY * (ncz + 1);
  GRID_LOOP(c, nc) {
    const int CI = (int)(c % CX), CJ = (int)((c / CX) % CY), CK = (int)(c / (CX * CY));
    auto wt = [](int I, int nf, int ncoarse, int C) {
      int k;
      double w0, w1;
      hweights(I, nf, ncoarse, k, w0, w1);
      return k == C ? w0 : (k + 1 == C ? w1 : 0.0);
    };
    T acc = T(0);
    for (int K = max(0, 2 * CK - 3); K <= min(nfz, 2 * CK + 3); ++K) {
      const double wz = wt(K, nfz, ncz, CK);
      if (wz == 0.0) continue;
      for (int J = max(0, 2 * CJ - 3); J <= min(nfy, 2 * CJ + 3); ++J) {
        const double wy = wt(J, nfy, ncy, CJ);
        if (wy == 0.0) continue;
        for (int I = max(0, 2 * CI - 3); I <= min(nfx, 2 * CI + 3); ++I) {
          const double wx = wt(I, nfx, ncx, CI);
          if (wx == 0.0) continue;
          const int64_t g = I + NX * (J + NY * (int64_t)K);
          acc += (T)(wx * wy * wz) * (bf[g] - tf[g]);
        }
      }
    }
    bc[c] += acc;
  }
}

__global__ void k_coarse_tissue(int ncx, int ncy, int ncz, int nfx, int nfy, const double* sl,
                                const double* st, const double* th, double* csl, double* cst,
                                double* cth) {
  pdl_entry();
  const int64_t n = (int64_t)ncx * ncy * ncz;
  GRID_LOOP(e, n) {
    const int kx = (int)(e % ncx), ky = (int)((e / ncx) % ncy), kz = (int)(e / ((int64_t)ncx * ncy));
    const int64_t f = 2 * kx + (int64_t)nfx * (2 * ky + (int64_t)nfy * 2 * kz);
    csl[e] = sl[f];
    cst[e] = st[f];
    cth[e] = th[f];
  }
}

// ---------------------------------------------------------------- reductions
// Deterministic dot product; the last CTA writes the total to *out.
__global__ void k_dot(int64_t n, const double* __restrict__ a, const double* __restrict__ b,
                      double* partials, unsigned int* ticket, double* out) {
  pdl_entry();
  __shared__ double red[32];
  double v = 0.0;
  GRID_LOOP(i, n) v = fma(a[i], b[i], v);
  v = block_sum(v, red);
  double total;
  if (finish_reduction(v, partials, ticket, &total, red)) *out = total;
}

__global__ void k_fill_start(int64_t n, double* v) {
  pdl_entry();
  GRID_LOOP(i, n) {
    const unsigned long long h = ((unsigned long long)i * 2654435761ull) & 0xffffffffull;
    v[i] = (double)h / 4294967296.0 - 0.5;
  }
}

__global__ void k_lanczos_z(int64_t n, const double* dinv, const double* r, double* z) {
  pdl_entry();
  GRID_LOOP(i, n) z[i] = dinv[i] * r[i];
}

__global__ void k_lanczos_update(int64_t n, double alpha, const double* Ap, double* r,
                                 const double* dinv, double* z) {
  pdl_entry();
  GRID_LOOP(i, n) {
    const double ri = fma(-alpha, Ap[i], r[i]);
    r[i] = ri;
    z[i] = dinv[i] * ri;
  }
}

__global__ void k_lanczos_p(int64_t n, double beta, const double* z, double* p, double* Ap) {
  pdl_entry();
  GRID_LOOP(i, n) {
    p[i] = fma(beta, p[i], z[i]);
    Ap[i] = 0.0;
  }
}

// ---------------------------------------------------------------- outer flexible PCG
template <int K>
__device__ __forceinline__ bool grid_sums_k(double (&v)[K], double* partials, int stride,
                                            unsigned int* ticket, double (&tot)[K]) {
  __shared__ double red[K][32];
  __shared__ bool is_last;
  double bs[K];
#pragma unroll
  for (int k = 0; k < K; ++k) bs[k] = block_sum(v[k], red[k]);
  if (threadIdx.x == 0) {
#pragma unroll
    for (int k = 0; k < K; ++k) partials[k * stride + blockIdx.x] = bs[k];
    __threadfence();
    const unsigned int t = atomicAdd(ticket, 1u);
    is_last = (t == gridDim.x - 1);
  }
  __syncthreads();
  if (!is_last) return false;
  __threadfence();
#pragma unroll
  for (int k = 0; k < K; ++k) {
    double s = 0.0;
    for (int b = threadIdx.x; b < (int)gridDim.x; b += blockDim.x)
      s += ((volatile double*)partials)[k * stride + b];
    tot[k] = block_sum(s, red[k]);
    __syncthreads();
  }
  if (threadIdx.x == 0) *ticket = 0u;
  return threadIdx.x == 0;
}

// r = b - Ap, Ap = 0, b0 = (T) r; r.r, b.b; stopping threshold.  VEC: b is
// 16-byte aligned (pairs of entries by 16-byte accesses).
template <typename T, bool VEC>
__global__ void k_fpcg_init(int64_t n, const double* __restrict__ b, double* Ap_main, double* Ap_alt,
                            const int* use_main, double* __restrict__ r, T* __restrict__ b0, CgScalars* cg,
                            double* partials, int stride, unsigned int* ticket, double rtol,
                            double atol) {
  pdl_entry();
  // A x: Ap_main, or Ap_alt where the flag use_main reads zero
  double* __restrict__ Ap = (use_main == nullptr || *use_main != 0) ? Ap_main : Ap_alt;
  double v[2] = {0.0, 0.0};
  const int64_t nc = VEC ? n / 2 : 0;
  GRID_CHUNKS(c, nc) {
    const Pk<double, 2> bb = reinterpret_cast<const Pk<double, 2>*>(b)[c];
    const Pk<double, 2> aa = reinterpret_cast<const Pk<double, 2>*>(Ap)[c];
    Pk<double, 2> rr;
    Pk<T, 2> rb;
#pragma unroll
    for (int k = 0; k < 2; ++k) {
      rr.e[k] = bb.e[k] - aa.e[k];
      rb.e[k] = (T)rr.e[k];
      v[0] = fma(rr.e[k], rr.e[k], v[0]);
      v[1] = fma(bb.e[k], bb.e[k], v[1]);
    }
    reinterpret_cast<Pk<double, 2>*>(r)[c] = rr;
    reinterpret_cast<Pk<double, 2>*>(Ap)[c] = Pk<double, 2>{};
    reinterpret_cast<Pk<T, 2>*>(b0)[c] = rb;
  }
  GRID_TAIL(i, nc * 2, n) {
    const double bi = b[i];
    const double ri = bi - Ap[i];
    r[i] = ri;
    Ap[i] = 0.0;
    b0[i] = (T)ri;
    v[0] = fma(ri, ri, v[0]);
    v[1] = fma(bi, bi, v[1]);
  }
  double tot[2];
  if (grid_sums_k<2>(v, partials, stride, ticket, tot)) {
    cg->rr = tot[0];
    cg->bb = tot[1];
    cg->tol2 = fmax(rtol * rtol * tot[1], atol * atol);
    cg->iters = 0;
    cg->status = 0;
    const bool finite = isfinite(tot[0]) && isfinite(tot[1]);
    if (!finite) cg->status = SEM_ERR_NONFINITE;
    cg->done = (!finite || tot[0] <= cg->tol2) ? 1 : 0;
  }
}

// z_new = (double) x0; first iteration (no iteration finished yet): p = z_new,
// rz = r.z_new; else beta = (r.z_new - r.z_old) / rz, rz = r.z_new (z holds
// z_old on entry).  Pairs of entries by 16-byte (8-byte for float x0) accesses.
// With p2 set, p is also written there as float pairs.
template <typename T>
__global__ void k_fpcg_z(int64_t n, const T* __restrict__ x0, double* __restrict__ z,
                         const double* __restrict__ r, double* __restrict__ p, df_pair* __restrict__ p2,
                         CgScalars* cg, double* partials, int stride, unsigned int* ticket) {
  pdl_entry();
  if (cg->done) return;
  const bool first = cg->iters == 0;
  double v[2] = {0.0, 0.0};
  using D2 = Pk<double, 2>;
  const int64_t nc = n / 2;
  GRID_CHUNKS(c, nc) {
    const Pk<T, 2> xx = reinterpret_cast<const Pk<T, 2>*>(x0)[c];
    const D2 rr = reinterpret_cast<const D2*>(r)[c];
    const D2 zo = first ? D2{} : reinterpret_cast<const D2*>(z)[c];
    D2 zn;
#pragma unroll
    for (int k = 0; k < 2; ++k) {
      zn.e[k] = (double)xx.e[k];
      if (!first) v[1] = fma(rr.e[k], zo.e[k], v[1]);
      v[0] = fma(rr.e[k], zn.e[k], v[0]);
    }
    if (first) {
      reinterpret_cast<D2*>(p)[c] = zn;
      if (p2 != nullptr) {
        const df_pair a0 = split_pair(zn.e[0]), a1 = split_pair(zn.e[1]);
        reinterpret_cast<float4*>(p2)[c] = make_float4(a0.h, a0.l, a1.h, a1.l);
      }
    }
    reinterpret_cast<D2*>(z)[c] = zn;
  }
  GRID_TAIL(i, nc * 2, n) {
    const double zi = (double)x0[i];
    const double ri = r[i];
    if (first) {
      p[i] = zi;
      if (p2 != nullptr) p2[i] = split_pair(zi);
    } else {
      v[1] = fma(ri, z[i], v[1]);
    }
    z[i] = zi;
    v[0] = fma(ri, zi, v[0]);
  }
  double tot[2];
  if (grid_sums_k<2>(v, partials, stride, ticket, tot)) {
    if (first) {
      cg->beta = 0.0;
    } else {
      cg->beta = (tot[0] - tot[1]) / cg->rz;
    }
    cg->rz = tot[0];
    if (!isfinite(tot[0]) || !isfinite(tot[1])) {
      cg->status = SEM_ERR_NONFINITE;
      cg->done = 1;
    }
  }
}

__global__ void k_fpcg_p(int64_t n, const double* __restrict__ z, double* __restrict__ p,
                         df_pair* __restrict__ p2, const CgScalars* cg) {
  pdl_entry();
  if (cg->done || cg->iters == 0) return;  // first iteration: k_fpcg_z set p = z
  const double beta = cg->beta;
  using D2 = Pk<double, 2>;
  const int64_t nc = n / 2;
  GRID_CHUNKS(c, nc) {
    const D2 zz = reinterpret_cast<const D2*>(z)[c];
    D2 pp = reinterpret_cast<const D2*>(p)[c];
#pragma unroll
    for (int k = 0; k < 2; ++k) pp.e[k] = fma(beta, pp.e[k], zz.e[k]);
    reinterpret_cast<D2*>(p)[c] = pp;
    if (p2 != nullptr) {
      const df_pair a0 = split_pair(pp.e[0]), a1 = split_pair(pp.e[1]);
      reinterpret_cast<float4*>(p2)[c] = make_float4(a0.h, a0.l, a1.h, a1.l);
    }
  }
  GRID_TAIL(i, nc * 2, n) {
    const double pi = fma(beta, p[i], z[i]);
    p[i] = pi;
    if (p2 != nullptr) p2[i] = split_pair(pi);
  }
}

// x += alpha p, r -= alpha Ap, Ap = 0, b0 = (T) r; r.r; convergence.  VEC: x is
// 16-byte aligned.
template <typename T, bool VEC>
__global__ void k_fpcg_xr(int64_t n, double* __restrict__ x, const double* __restrict__ p,
                          double* __restrict__ Ap, double* __restrict__ r, T* __restrict__ b0,
                          CgScalars* cg, double* partials, int stride, unsigned int* ticket) {
  pdl_entry();
  if (cg->done) return;
  const double alpha = cg->alpha;
  double v[1] = {0.0};
  using D2 = Pk<double, 2>;
  const int64_t nc = VEC ? n / 2 : 0;
  GRID_CHUNKS(c, nc) {
    D2 xx = reinterpret_cast<const D2*>(x)[c];
    const D2 pp = reinterpret_cast<const D2*>(p)[c];
    const D2 aa = reinterpret_cast<const D2*>(Ap)[c];
    D2 rr = reinterpret_cast<const D2*>(r)[c];
    Pk<T, 2> rb;
#pragma unroll
    for (int k = 0; k < 2; ++k) {
      xx.e[k] = fma(alpha, pp.e[k], xx.e[k]);
      rr.e[k] = fma(-alpha, aa.e[k], rr.e[k]);
      rb.e[k] = (T)rr.e[k];
      v[0] = fma(rr.e[k], rr.e[k], v[0]);
    }
    reinterpret_cast<D2*>(x)[c] = xx;
    reinterpret_cast<D2*>(r)[c] = rr;
    reinterpret_cast<D2*>(Ap)[c] = D2{};
    reinterpret_cast<Pk<T, 2>*>(b0)[c] = rb;
  }
  GRID_TAIL(i, nc * 2, n) {
    x[i] = fma(alpha, p[i], x[i]);
    const double ri = fma(-alpha, Ap[i], r[i]);
    r[i] = ri;
    Ap[i] = 0.0;
    b0[i] = (T)ri;
    v[0] = fma(ri, ri, v[0]);
  }
  double tot[1];
  if (grid_sums_k<1>(v, partials, stride, ticket, tot)) {
    cg->rr = tot[0];
    cg->iters += 1;
    if (!isfinite(tot[0]) || !isfinite(alpha)) {
      cg->status = SEM_ERR_NONFINITE;
      cg->done = 1;
    } else if (tot[0] <= cg->tol2) {
      cg->done = 1;
    }
  }
}

// ---- the same flexible PCG with the double-float operator: r and p are kept
// as float pairs, z as the V-cycle's own values (type T), and their updates and
// inner products run in double-float arithmetic on the FP32 pipe; only x, the
// caller's FP64 solution, is updated by FP64 instructions (one DFMA and one
// addition per entry).  GB300 issues two FP64 operations per clock per SM, which
// bound the FP64 forms of these kernels (FP64 pipe 76 % busy).

// double-float value of a T (exact for float)
__device__ __forceinline__ df df_of(float v) { return df(v, 0.f); }
__device__ __forceinline__ df df_of(double v) { return dfd(v); }
// T-rounded high part for the V-cycle's right-hand side
template <typename T> __device__ __forceinline__ T t_of(df v);
template <> __device__ __forceinline__ float t_of<float>(df v) { return v.h; }
template <> __device__ __forceinline__ double t_of<double>(df v) { return df_to_double(v); }

// Block sum of double-float values: the warps add in double-float (FP32
// shuffles), each warp's sum becomes a double once, and warp 0 adds those.
__device__ __forceinline__ double block_sum_df(df v, double* red) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const float h = __shfl_down_sync(0xffffffffu, v.h, o), l = __shfl_down_sync(0xffffffffu, v.l, o);
    v = v + df(h, l);
  }
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (lane == 0) red[warp] = (double)v.h + (double)v.l;
  __syncthreads();
  double d = 0.0;
  if (warp == 0) {
    const int nw = (blockDim.x + 31) >> 5;
    d = (lane < nw) ? red[lane] : 0.0;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) d += __shfl_down_sync(0xffffffffu, d, o);
  }
  return d;
}

// grid_sums_k with double-float per-thread values.
template <int K>
__device__ __forceinline__ bool grid_sums_df(df (&v)[K], double* partials, int stride, unsigned int* ticket,
                                             double (&tot)[K]) {
  __shared__ double red[K][32];
  __shared__ bool is_last;
  double bs[K];
#pragma unroll
  for (int k = 0; k < K; ++k) bs[k] = block_sum_df(v[k], red[k]);
  if (threadIdx.x == 0) {
#pragma unroll
    for (int k = 0; k < K; ++k) partials[k * stride + blockIdx.x] = bs[k];
    __threadfence();
    const unsigned int t = atomicAdd(ticket, 1u);
    is_last = (t == gridDim.x - 1);
  }
  __syncthreads();
  if (!is_last) return false;
  __threadfence();
#pragma unroll
  for (int k = 0; k < K; ++k) {
    double s = 0.0;
    for (int b = threadIdx.x; b < (int)gridDim.x; b += blockDim.x)
      s += ((volatile double*)partials)[k * stride + b];
    tot[k] = block_sum(s, red[k]);
    __syncthreads();
  }
  if (threadIdx.x == 0) *ticket = 0u;
  return threadIdx.x == 0;
}

// The double-float PCG kernels move two entries per thread and iteration
// (16-byte accesses to FP64 and float-pair vectors) and the odd last entry
// alone.  Workspace and level vectors come from cudaMalloc; VEC is false when a
// caller's FP64 vector is not 16-byte aligned (then every entry goes the scalar
// way).  8 CTAs of 256 threads per SM stay resident (32 registers); 6 for
// k_dfpcg_xr (40 registers: at 32 it spills), whose grid is sized to match.
template <typename T> using C2 = Pk<T, 2>;
constexpr int kXrCtasPerSm = 6;

// one entry of the set-up: r = b - A x (pairs), b0 = r rounded to T
template <typename T>
__device__ __forceinline__ void init_entry(double bi, df ax, df_pair& r2, T& b0, df (&v)[2]) {
  const df bd = dfd(bi);
  const df r = dfnorm(bd - ax);
  r2 = df_pair{r.h, r.l};
  b0 = t_of<T>(r);
  v[0] = fma(r, r, v[0]);
  v[1] = fma(bd, bd, v[1]);
}

// r = b - A x, b0 = r; r.r, b.b; stopping threshold.  A x is the FP64 result of
// an apply in Ap (zeroed here), or the carried float pairs in ax2_in (Ap is then
// already zero).
template <typename T, bool VEC>
__global__ void __launch_bounds__(kThreads, 8)
    k_dfpcg_init(int64_t n, const double* __restrict__ b, double* __restrict__ Ap,
                 const df_pair* __restrict__ ax2_in, const int* ax2_ok, df_pair* __restrict__ r2,
                 T* __restrict__ b0, CgScalars* cg, double* partials, int stride, unsigned int* ticket,
                 double rtol, double atol) {
  pdl_entry();
  // the carried pairs, unless the flag ax2_ok reads zero (then A x is in Ap)
  const df_pair* __restrict__ ax2 = (ax2_ok == nullptr || *ax2_ok != 0) ? ax2_in : nullptr;
  df v[2] = {df(0.f, 0.f), df(0.f, 0.f)};
  const int64_t nc = VEC ? n / 2 : 0;
  GRID_CHUNKS(c, nc) {
    const C2<double> bb = reinterpret_cast<const C2<double>*>(b)[c];
    C2<df_pair> ax, rr;
    C2<double> aa;
    if (ax2 != nullptr) {
      ax = reinterpret_cast<const C2<df_pair>*>(ax2)[c];
    } else {
      aa = reinterpret_cast<const C2<double>*>(Ap)[c];
      reinterpret_cast<C2<double>*>(Ap)[c] = C2<double>{};
    }
    C2<T> rb;
#pragma unroll
    for (int k = 0; k < 2; ++k)
      init_entry(bb.e[k], ax2 != nullptr ? df(ax.e[k].h, ax.e[k].l) : dfd(aa.e[k]), rr.e[k], rb.e[k], v);
    reinterpret_cast<C2<df_pair>*>(r2)[c] = rr;
    reinterpret_cast<C2<T>*>(b0)[c] = rb;
  }
  GRID_TAIL(i, nc * 2, n) {
    df ax;
    if (ax2 != nullptr) {
      ax = df(ax2[i].h, ax2[i].l);
    } else {
      ax = dfd(Ap[i]);
      Ap[i] = 0.0;
    }
    init_entry(b[i], ax, r2[i], b0[i], v);
  }
  double tot[2];
  if (grid_sums_df<2>(v, partials, stride, ticket, tot)) {
    cg->rr = tot[0];
    cg->bb = tot[1];
    cg->tol2 = fmax(rtol * rtol * tot[1], atol * atol);
    cg->iters = 0;
    cg->status = 0;
    const bool finite = isfinite(tot[0]) && isfinite(tot[1]);
    if (!finite) cg->status = SEM_ERR_NONFINITE;
    cg->done = (!finite || tot[0] <= cg->tol2) ? 1 : 0;
  }
}

// z_new = the V-cycle's result (kept in zs, which holds z_old on entry); first
// iteration: p = z_new, rz = r.z_new; else beta = (r.z_new - r.z_old) / rz, rz = r.z_new.
template <typename T>
__device__ __forceinline__ void z_entry(T z, T& zs, df_pair rp, df_pair& p2, bool first, df (&v)[2]) {
  const df r(rp.h, rp.l), zd = df_of(z);
  v[0] = fma(r, zd, v[0]);
  if (first) p2 = df_pair{zd.h, zd.l};
  else v[1] = fma(r, df_of(zs), v[1]);
  zs = z;
}

template <typename T>
__global__ void __launch_bounds__(kThreads, 8)
    k_dfpcg_z(int64_t n, const T* __restrict__ x0, T* __restrict__ zs, const df_pair* __restrict__ r2,
              df_pair* __restrict__ p2, CgScalars* cg, double* partials, int stride, unsigned int* ticket) {
  pdl_entry();
  if (cg->done) return;
  const bool first = cg->iters == 0;
  df v[2] = {df(0.f, 0.f), df(0.f, 0.f)};
  const int64_t nc = n / 2;
  GRID_CHUNKS(c, nc) {
    const C2<T> z = reinterpret_cast<const C2<T>*>(x0)[c];
    C2<T> zz = reinterpret_cast<const C2<T>*>(zs)[c];
    const C2<df_pair> rr = reinterpret_cast<const C2<df_pair>*>(r2)[c];
    C2<df_pair> pp;
#pragma unroll
    for (int k = 0; k < 2; ++k) z_entry(z.e[k], zz.e[k], rr.e[k], pp.e[k], first, v);
    reinterpret_cast<C2<T>*>(zs)[c] = zz;
    if (first) reinterpret_cast<C2<df_pair>*>(p2)[c] = pp;
  }
  GRID_TAIL(i, nc * 2, n) {
    df_pair pp;
    z_entry(x0[i], zs[i], r2[i], pp, first, v);
    if (first) p2[i] = pp;
  }
  double tot[2];
  if (grid_sums_df<2>(v, partials, stride, ticket, tot)) {
    cg->beta = first ? 0.0 : (tot[0] - tot[1]) / cg->rz;
    cg->rz = tot[0];
    if (!isfinite(tot[0]) || !isfinite(tot[1])) {
      cg->status = SEM_ERR_NONFINITE;
      cg->done = 1;
    }
  }
}

// p = z + beta p (float pairs)
template <typename T>
__device__ __forceinline__ df_pair p_entry(df beta, df_pair pp, T z) {
  const df pn = dfnorm(fma(beta, df(pp.h, pp.l), df_of(z)));
  return df_pair{pn.h, pn.l};
}

template <typename T>
__global__ void __launch_bounds__(kThreads, 8)
    k_dfpcg_p(int64_t n, const T* __restrict__ zs, df_pair* __restrict__ p2, const CgScalars* cg) {
  pdl_entry();
  if (cg->done || cg->iters == 0) return;  // first iteration: k_dfpcg_z set p = z
  const df beta = dfd(cg->beta);
  const int64_t nc = n / 2;
  GRID_CHUNKS(c, nc) {
    const C2<T> zz = reinterpret_cast<const C2<T>*>(zs)[c];
    C2<df_pair> pp = reinterpret_cast<const C2<df_pair>*>(p2)[c];
#pragma unroll
    for (int k = 0; k < 2; ++k) pp.e[k] = p_entry(beta, pp.e[k], zz.e[k]);
    reinterpret_cast<C2<df_pair>*>(p2)[c] = pp;
  }
  GRID_TAIL(i, nc * 2, n) p2[i] = p_entry(beta, p2[i], zs[i]);
}

// x += alpha p (FP64), r -= alpha Ap, Ap = 0, b0 = r; r.r; convergence.
template <typename T>
__device__ __forceinline__ T xr_entry(double alpha, df nalpha, df_pair pp, double& x, double& ap, df_pair& r2,
                                      df (&v)[1]) {
  x = fma(alpha, df_to_double(df(pp.h, pp.l)), x);
  const df r = dfnorm(fma(nalpha, dfd(ap), df(r2.h, r2.l)));
  r2 = df_pair{r.h, r.l};
  ap = 0.0;
  v[0] = fma(r, r, v[0]);
  return t_of<T>(r);
}

template <typename T, bool VEC>
__global__ void __launch_bounds__(kThreads, kXrCtasPerSm)
    k_dfpcg_xr(int64_t n, double* __restrict__ x, const df_pair* __restrict__ p2, double* __restrict__ Ap,
               df_pair* __restrict__ r2, T* __restrict__ b0, CgScalars* cg, double* partials, int stride,
               unsigned int* ticket) {
  pdl_entry();
  if (cg->done) return;
  const double alpha = cg->alpha;
  const df nalpha = dfneg(dfd(alpha));
  df v[1] = {df(0.f, 0.f)};
  const int64_t nc = VEC ? n / 2 : 0;
  GRID_CHUNKS(c, nc) {
    const C2<df_pair> pp = reinterpret_cast<const C2<df_pair>*>(p2)[c];
    C2<double> xx = reinterpret_cast<const C2<double>*>(x)[c];
    C2<double> aa = reinterpret_cast<const C2<double>*>(Ap)[c];
    C2<df_pair> rr = reinterpret_cast<const C2<df_pair>*>(r2)[c];
    C2<T> rb;
#pragma unroll
    for (int k = 0; k < 2; ++k) rb.e[k] = xr_entry<T>(alpha, nalpha, pp.e[k], xx.e[k], aa.e[k], rr.e[k], v);
    reinterpret_cast<C2<double>*>(x)[c] = xx;
    reinterpret_cast<C2<df_pair>*>(r2)[c] = rr;
    reinterpret_cast<C2<double>*>(Ap)[c] = aa;
    reinterpret_cast<C2<T>*>(b0)[c] = rb;
  }
  GRID_TAIL(i, nc * 2, n) {
    b0[i] = xr_entry<T>(alpha, nalpha, p2[i], x[i], Ap[i], r2[i], v);
  }
  double tot[1];
  if (grid_sums_df<1>(v, partials, stride, ticket, tot)) {
    cg->rr = tot[0];
    cg->iters += 1;
    if (!isfinite(tot[0]) || !isfinite(alpha)) {
      cg->status = SEM_ERR_NONFINITE;
      cg->done = 1;
    } else if (tot[0] <= cg->tol2) {
      cg->done = 1;
    }
  }
}

template <typename T>
__global__ void k_to_level0(int64_t n, const double* __restrict__ r, T* __restrict__ b0) {
  pdl_entry();
  GRID_LOOP(i, n) b0[i] = (T)r[i];
}

template <typename T>
__global__ void k_from_level0(int64_t n, const T* __restrict__ x0, double* __restrict__ z) {
  pdl_entry();
  GRID_LOOP(i, n) z[i] = (double)x0[i];
}

// ---------------------------------------------------------------- host helpers
#define GMG_CK(call)                                          \
  do {                                                        \
    cudaError_t e_ = (call);                                  \
    if (e_ != cudaSuccess) return cuda_fail(ctx, e_, #call);  \
  } while (0)

size_t elem_size(int precision) { return precision == SEM_PREC_FP64 ? sizeof(double) : sizeof(float); }

// Largest eigenvalue of the symmetric tridiagonal matrix (diag a, off-diagonal e) by bisection.
double tridiag_max_eig(const std::vector<double>& a, const std::vector<double>& e) {
  const int m = (int)a.size();
  double lo = 1e300, hi = -1e300;
  for (int i = 0; i < m; ++i) {
    const double r = (i > 0 ? std::fabs(e[i - 1]) : 0.0) + (i + 1 < m ? std::fabs(e[i]) : 0.0);
    lo = std::min(lo, a[i] - r);
    hi = std::max(hi, a[i] + r);
  }
  auto count_below = [&](double x) {
    int c = 0;
    double d = 1.0;
    for (int i = 0; i < m; ++i) {
      d = a[i] - x - (i > 0 ? e[i - 1] * e[i - 1] / d : 0.0);
      if (d == 0.0) d = -1e-300;
      if (d < 0.0) ++c;
    }
    return c;
  };
  for (int it = 0; it < 200; ++it) {
    const double mid = 0.5 * (lo + hi);
    if (mid <= lo || mid >= hi) break;
    if (count_below(mid) >= m) hi = mid; else lo = mid;
  }
  return 0.5 * (lo + hi);
}

// y += (alpha M + K) x on one level in the V-cycle's precision.
int level_apply(sem_ctx* ctx, const Level& L, int precision, double alpha, const void* x, void* y,
                const int* done, cudaStream_t s) {
  cudaError_t e;
  // deterministic mode: element-local results and fixed-order node sums (scalar kernels)
  void* loc = ctx->deterministic ? ctx->det_scratch : nullptr;
  if (precision == SEM_PREC_FP64) {
    ApplyArgs64 a{};
    a.map = L.map; a.metric = L.metric; a.u = (const double*)x; a.y = (double*)y;
    a.nelem = L.nelem; a.mass_coef = alpha; a.out_scale = 1.0; a.scale_out = 0; a.done = done;
    a.yloc = (double*)loc;
    e = launch_apply_fp64(L, a, false, s);
  } else if (precision == SEM_PREC_FP32_BF16 || precision == SEM_PREC_BF16_TC) {
    ApplyArgs<float, __nv_bfloat16> a{};
    a.map = L.map; a.metric = L.metric16; a.u = (const float*)x; a.y = (float*)y;
    a.nelem = L.nelem; a.mass_coef = (float)alpha; a.out_scale = 1.f; a.scale_out = 0; a.done = done;
    a.yloc = (float*)loc;
    e = (precision == SEM_PREC_BF16_TC && tc_supported(L) && loc == nullptr) ? launch_apply_tc(L, a, s)
                                                                             : launch_apply_bf16(L, a, false, s);
  } else {
    ApplyArgs<float, float> a{};
    a.map = L.map; a.metric = L.metric32; a.u = (const float*)x; a.y = (float*)y;
    a.nelem = L.nelem; a.mass_coef = (float)alpha; a.out_scale = 1.f; a.scale_out = 0; a.done = done;
    a.yloc = (float*)loc;
    e = launch_apply_fp32(L, a, false, s);
  }
  if (e != cudaSuccess) return cuda_fail(ctx, e, "level apply");
  ctx->launches += 1;
  return SEM_OK;
}

PTab make_ptab(const Level& fine, const Level& coarse) {
  PTab t{};
  t.nf = fine.n;
  t.nc = coarse.n;
  // l^c_a(x^f_i) by the barycentric formula on the coarse LGL nodes
  const double* xc = coarse.tab.xg;
  const double* xf = fine.tab.xg;
  double lam[kMaxN];
  for (int a = 0; a < t.nc; ++a) {
    double prod = 1.0;
    for (int b = 0; b < t.nc; ++b) if (b != a) prod *= (xc[a] - xc[b]);
    lam[a] = 1.0 / prod;
  }
  for (int i = 0; i < t.nf; ++i) {
    int hit = -1;
    for (int a = 0; a < t.nc; ++a) if (std::fabs(xf[i] - xc[a]) < 1e-15) hit = a;
    if (hit >= 0) {
      for (int a = 0; a < t.nc; ++a) t.P[i][a] = (a == hit) ? 1.0 : 0.0;
      continue;
    }
    double den = 0.0;
    for (int a = 0; a < t.nc; ++a) den += lam[a] / (xf[i] - xc[a]);
    for (int a = 0; a < t.nc; ++a) t.P[i][a] = (lam[a] / (xf[i] - xc[a])) / den;
  }
  return t;
}

// Restrict (b_l - t_l) into b_{l+1}.
template <typename T>
int restrict_to(sem_ctx* ctx, Gmg& g, int l, const int* done, cudaStream_t s) {
  GmgLevel& F = g.lv[l];
  GmgLevel& C = g.lv[l + 1];
  if (F.to_next == 0) {  // three passes that write b_{l+1}
    const PTab tab = make_ptab(*F.L, *C.L);
    GMG_CK(p_transfer<T>(false, *F.L, *C.L, tab.P, (const T*)F.b, (const T*)F.t, (T*)C.b, nullptr,
                         (T*)F.pw1, (T*)F.pw2, done, s));
    ctx->launches += 3;
    return SEM_OK;
  }
  launch_k(k_zero<T>, grid_chunks<T>(C.L->ndofs), kThreads, 0, s, C.L->ndofs, (T*)C.b, done);
  T* loc = ctx->deterministic ? reinterpret_cast<T*>(ctx->det_scratch) : nullptr;
  if (loc != nullptr) {
    launch_k(k_restrict_h_det<T>, grid1d(C.L->ndofs), kThreads, 0, s,
        F.L->nx, F.L->ny, F.L->nz, C.L->nx, C.L->ny, C.L->nz, (const T*)F.b, (const T*)F.t,
        (T*)C.b, done);
  } else {
    launch_k(k_restrict_h<T>, grid1d(F.L->ndofs), kThreads, 0, s,
        F.L->nx, F.L->ny, F.L->nz, C.L->nx, C.L->ny, C.L->nz, (const T*)F.b, (const T*)F.t,
        (T*)C.b, done);
  }
  GMG_CK(cudaGetLastError());
  ctx->launches += 2;
  return SEM_OK;
}

template <typename T>
int prolong_from(sem_ctx* ctx, Gmg& g, int l, const int* done, cudaStream_t s) {
  GmgLevel& F = g.lv[l];
  GmgLevel& C = g.lv[l + 1];
  if (F.to_next == 0) {
    const PTab tab = make_ptab(*F.L, *C.L);
    GMG_CK(p_transfer<T>(true, *F.L, *C.L, tab.P, (const T*)C.x, nullptr, (T*)F.x, (T*)F.t, (T*)F.pw1,
                         (T*)F.pw2, done, s));
    ctx->launches += 3;
    return SEM_OK;
  } else {
    launch_k(k_prolong_h<T>, grid1d(F.L->ndofs), kThreads, 0, s,
        F.L->nx, F.L->ny, F.L->nz, C.L->nx, C.L->ny, C.L->nz, (const T*)C.x, (T*)F.x, (T*)F.t,
        done);
  }
  GMG_CK(cudaGetLastError());
  ctx->launches += 1;
  return SEM_OK;
}

// `degree` Chebyshev steps on level l for A x = b (zero start, or from the current x
// with t = 0).
template <typename T>
int chebyshev(sem_ctx* ctx, Gmg& g, int l, int degree, bool zero_start, const int* done,
              cudaStream_t s) {
  GmgLevel& V = g.lv[l];
  const Level& L = *V.L;
  const int64_t n = L.ndofs;
  const double lo = 0.08 * V.lam, hi = 1.2 * V.lam;
  const double theta = 0.5 * (hi + lo), delta = 0.5 * (hi - lo), sigma = theta / delta;
  double rho_old = 1.0 / sigma;
  T* b = (T*)V.b; T* x = (T*)V.x; T* t = (T*)V.t; T* d = (T*)V.d; const T* invd = (const T*)V.invd;
  int k0 = 0;
  if (zero_start) {
    launch_k(k_cheb_zero_start<T>, grid_chunks<T>(n), kThreads, 0, s, n, b, invd, x, d, t, (T)(1.0 / theta), done);
    GMG_CK(cudaGetLastError());
    ctx->launches += 1;
    k0 = 1;
  }
  for (int k = k0; k < degree; ++k) {
    int rc = level_apply(ctx, L, g.precision, g.alpha, x, t, done, s);
    if (rc != SEM_OK) return rc;
    if (k == 0) {
      launch_k(k_cheb_step<T>, grid_chunks<T>(n), kThreads, 0, s, n, b, invd, x, d, t, (T)0, (T)(1.0 / theta), 1,
                                                           done);
    } else {
      const double rho = 1.0 / (2.0 * sigma - rho_old);
      launch_k(k_cheb_step<T>, grid_chunks<T>(n), kThreads, 0, s, n, b, invd, x, d, t, (T)(rho * rho_old),
                                                           (T)(2.0 * rho / delta), 0, done);
      rho_old = rho;
    }
    GMG_CK(cudaGetLastError());
    ctx->launches += 1;
  }
  return SEM_OK;
}

template <typename T>
int vcycle_level(sem_ctx* ctx, Gmg& g, int l, const int* done, cudaStream_t s, bool record) {
  const int last = (int)g.lv.size() - 1;
  int rc;
  if (l == last) return chebyshev<T>(ctx, g, l, g.coarse_degree, true, done, s);
  if ((rc = chebyshev<T>(ctx, g, l, g.degree, true, done, s)) != SEM_OK) return rc;
  GmgLevel& V = g.lv[l];
  // t = A x (t is zero after the smoother), then b_{l+1} = R (b - t)
  // the fine-level residual apply is bracketed by event nodes when `record`
  if (record && l == 0) GMG_CK(cudaEventRecordWithFlags(g.ev2, s, cudaEventRecordExternal));
  if ((rc = level_apply(ctx, *V.L, g.precision, g.alpha, V.x, V.t, done, s)) != SEM_OK) return rc;
  if (record && l == 0) GMG_CK(cudaEventRecordWithFlags(g.ev3, s, cudaEventRecordExternal));
  if ((rc = restrict_to<T>(ctx, g, l, done, s)) != SEM_OK) return rc;
  if ((rc = vcycle_level<T>(ctx, g, l + 1, done, s, false)) != SEM_OK) return rc;
  if ((rc = prolong_from<T>(ctx, g, l, done, s)) != SEM_OK) return rc;  // also clears t
  return chebyshev<T>(ctx, g, l, g.degree, false, done, s);
}

int vcycle(sem_ctx* ctx, Gmg& g, const int* done, cudaStream_t s, bool record = false) {
  if (g.precision == SEM_PREC_FP64) return vcycle_level<double>(ctx, g, 0, done, s, record);
  return vcycle_level<float>(ctx, g, 0, done, s, record);
}

// 10 Jacobi-PCG steps on level V from the fixed start vector; largest Lanczos eigenvalue.
int estimate_lambda(sem_ctx* ctx, Gmg& g, GmgLevel& V, double alpha, cudaStream_t s) {
  const Level& L = *V.L;
  const int64_t n = L.ndofs;
  const int gr = grid1d(n);
  launch_k(k_fill_start, gr, kThreads, 0, s, n, g.lr);
  launch_k(k_lanczos_z, gr, kThreads, 0, s, n, V.dinv64, g.lr, g.lz);
  GMG_CK(cudaMemcpyAsync(g.lp, g.lz, sizeof(double) * n, cudaMemcpyDeviceToDevice, s));
  GMG_CK(cudaMemsetAsync(g.lAp, 0, sizeof(double) * n, s));
  launch_k(k_dot, gr, kThreads, 0, s, n, g.lr, g.lz, g.partials, g.tickets, g.dots + 0);
  GMG_CK(cudaGetLastError());
  double h[2];
  GMG_CK(cudaMemcpyAsync(h, g.dots, sizeof(double), cudaMemcpyDeviceToHost, s));
  GMG_CK(cudaStreamSynchronize(s));
  double rz = h[0];
  std::vector<double> alphas, betas;
  const int iters = (int)std::min<int64_t>(10, n);
  for (int it = 0; it < iters; ++it) {
    ApplyArgs64 a{};
    a.map = L.map; a.metric = L.metric; a.u = g.lp; a.y = g.lAp; a.nelem = L.nelem;
    a.mass_coef = alpha; a.out_scale = 1.0; a.scale_out = 0;
    a.yloc = ctx->deterministic ? ctx->det_scratch : nullptr;
    GMG_CK(launch_apply_fp64(L, a, false, s));
    launch_k(k_dot, gr, kThreads, 0, s, n, g.lp, g.lAp, g.partials, g.tickets, g.dots + 1);
    GMG_CK(cudaMemcpyAsync(h, g.dots + 1, sizeof(double), cudaMemcpyDeviceToHost, s));
    GMG_CK(cudaStreamSynchronize(s));
    const double pAp = h[0];
    if (!(pAp > 0.0) || !(rz > 0.0)) break;
    const double al = rz / pAp;
    launch_k(k_lanczos_update, gr, kThreads, 0, s, n, al, g.lAp, g.lr, V.dinv64, g.lz);
    launch_k(k_dot, gr, kThreads, 0, s, n, g.lr, g.lz, g.partials, g.tickets, g.dots + 2);
    GMG_CK(cudaMemcpyAsync(h, g.dots + 2, sizeof(double), cudaMemcpyDeviceToHost, s));
    GMG_CK(cudaStreamSynchronize(s));
    const double rz_new = h[0];
    const double be = rz_new / rz;
    alphas.push_back(al);
    betas.push_back(be);
    rz = rz_new;
    launch_k(k_lanczos_p, gr, kThreads, 0, s, n, be, g.lz, g.lp, g.lAp);
    GMG_CK(cudaGetLastError());
    if (!(rz > 0.0)) break;
  }
  const int m = (int)alphas.size();
  if (m == 0) return fail(ctx, SEM_ERR_NONFINITE, "eigenvalue estimate failed on a multigrid level");
  std::vector<double> d(m), e(std::max(0, m - 1));
  for (int j = 0; j < m; ++j) {
    d[j] = 1.0 / alphas[j] + (j > 0 ? betas[j - 1] / alphas[j - 1] : 0.0);
    if (j + 1 < m) e[j] = std::sqrt(betas[j]) / alphas[j];
  }
  V.lam = tridiag_max_eig(d, e);
  return SEM_OK;
}

int set_alpha(sem_ctx* ctx, Gmg& g, double alpha, cudaStream_t s) {
  if (g.alpha == alpha) return SEM_OK;
  for (GmgLevel& V : g.lv) {
    const Level& L = *V.L;
    if (g.precision == SEM_PREC_FP64)
      launch_k(k_level_inv_diag<double>, grid1d(L.ndofs), kThreads, 0, s, L.ndofs, alpha, L.mdiag, L.kdiag,
                                                                   (double*)V.invd, V.dinv64);
    else
      launch_k(k_level_inv_diag<float>, grid1d(L.ndofs), kThreads, 0, s, L.ndofs, alpha, L.mdiag, L.kdiag,
                                                                  (float*)V.invd, V.dinv64);
    GMG_CK(cudaGetLastError());
    int rc = estimate_lambda(ctx, g, V, alpha, s);
    if (rc != SEM_OK) return rc;
  }
  g.alpha = alpha;
  return SEM_OK;
}

void free_gmg_struct(Gmg* g) {
  if (!g) return;
  for (GmgLevel& V : g->lv) {
    if (V.owned && V.L) {
      level_free(*V.L);
      delete V.L;
    }
    if (V.owns_tissue) {
      cudaFree(V.sl); cudaFree(V.st); cudaFree(V.th);
    }
    cudaFree(V.b); cudaFree(V.x); cudaFree(V.t); cudaFree(V.d); cudaFree(V.invd);
    cudaFree(V.pw1); cudaFree(V.pw2);
    cudaFree(V.dinv64);
  }
  cudaFree(g->z);
  for (auto& gr : g->graphs) {
    if (gr.init) cudaGraphExecDestroy(gr.init);
    if (gr.iter) cudaGraphExecDestroy(gr.iter);
    if (gr.init_carried) cudaGraphExecDestroy(gr.init_carried);
    if (gr.init_checked) cudaGraphExecDestroy(gr.init_checked);
    if (gr.iter_timed) cudaGraphExecDestroy(gr.iter_timed);
    for (auto& cv : gr.combo)
      for (auto& c : cv)
        if (c.exec) cudaGraphExecDestroy(c.exec);
  }
  if (g->capture) cudaStreamDestroy(g->capture);
  if (g->ev0) cudaEventDestroy(g->ev0);
  if (g->ev1) cudaEventDestroy(g->ev1);
  if (g->ev2) cudaEventDestroy(g->ev2);
  if (g->ev3) cudaEventDestroy(g->ev3);
  cudaFree(g->lr); cudaFree(g->lz); cudaFree(g->lp); cudaFree(g->lAp);
  cudaFree(g->dots); cudaFree(g->partials); cudaFree(g->tickets);
  delete g;
}

int build(sem_ctx* ctx, cudaStream_t s) {
  if (ctx->gmg) return SEM_OK;
  Gmg* g = new Gmg();
  g->precision = ctx->gmg_precision;
  g->degree = ctx->gmg_degree;
  g->coarse_degree = ctx->gmg_coarse_degree;
  struct Guard {
    Gmg*& g;
    ~Guard() { if (g) free_gmg_struct(g); }
  } guard{g};
  GmgLevel top;
  top.L = &ctx->L;
  top.sl = ctx->sigma_l; top.st = ctx->sigma_t; top.th = ctx->theta;
  g->lv.push_back(top);
  std::vector<double> verts = ctx->vertices;
  int nx = ctx->L.nx, ny = ctx->L.ny, nz = ctx->L.nz, p = ctx->L.p;
  const int quad = ctx->L.quad;
  GMG_CK(cudaMemsetAsync(ctx->d_flag, 0, sizeof(int), s));
  // p-coarsening on the fine mesh, then h-coarsening, while the level is larger
  // than min_coarse_dofs (a p-level may be the coarsest)
  while (p > 1 && g->lv.back().L->ndofs > ctx->gmg_min_coarse_dofs) {
    const int pc = std::max(1, p / 2);
    GmgLevel V;
    V.L = new Level();
    V.owned = true;
    V.sl = ctx->sigma_l; V.st = ctx->sigma_t; V.th = ctx->theta;
    g->lv.back().to_next = 0;
    g->lv.push_back(V);
    GMG_CK(level_create(*g->lv.back().L, nx, ny, nz, verts.data(), pc, quad, false, s));
    g->lv.back().L->dbg = ctx->L.dbg;
    g->lv.back().L->fault = ctx->L.fault;
    GMG_CK(setup_geometry(*g->lv.back().L, V.sl, V.st, V.th, ctx->d_flag, s));
    GMG_CK(setup_diagonals(*g->lv.back().L, s));
    p = pc;
  }
  while (g->lv.back().L->ndofs > ctx->gmg_min_coarse_dofs && std::max(nx, std::max(ny, nz)) > 1) {
    const int cx = (nx + 1) / 2, cy = (ny + 1) / 2, cz = (nz + 1) / 2;
    std::vector<double> cv((size_t)(cx + 1) * (cy + 1) * (cz + 1) * 3);
    for (int K = 0; K <= cz; ++K)
      for (int J = 0; J <= cy; ++J)
        for (int I = 0; I <= cx; ++I) {
          const size_t f = (size_t)std::min(2 * I, nx) +
                           (size_t)(nx + 1) * (std::min(2 * J, ny) + (size_t)(ny + 1) * std::min(2 * K, nz));
          const size_t c = (size_t)I + (size_t)(cx + 1) * (J + (size_t)(cy + 1) * K);
          for (int d = 0; d < 3; ++d) cv[c * 3 + d] = verts[f * 3 + d];
        }
    GmgLevel& F = g->lv.back();
    GmgLevel V;
    V.L = new Level();
    V.owned = true;
    V.owns_tissue = true;
    const size_t ne = (size_t)cx * cy * cz;
    GMG_CK(cudaMalloc(&V.sl, sizeof(double) * ne));
    GMG_CK(cudaMalloc(&V.st, sizeof(double) * ne));
    GMG_CK(cudaMalloc(&V.th, sizeof(double) * ne));
    launch_k(k_coarse_tissue, grid1d((int64_t)ne), kThreads, 0, s, cx, cy, cz, nx, ny, F.sl, F.st, F.th,
                                                              V.sl, V.st, V.th);
    GMG_CK(cudaGetLastError());
    F.to_next = 1;
    g->lv.push_back(V);
    GMG_CK(level_create(*g->lv.back().L, cx, cy, cz, cv.data(), 1, quad, false, s));
    g->lv.back().L->dbg = ctx->L.dbg;
    g->lv.back().L->fault = ctx->L.fault;
    GMG_CK(setup_geometry(*g->lv.back().L, V.sl, V.st, V.th, ctx->d_flag, s));
    GMG_CK(setup_diagonals(*g->lv.back().L, s));
    verts.swap(cv);
    nx = cx; ny = cy; nz = cz;
  }
  int bad = 0;
  GMG_CK(cudaMemcpyAsync(&bad, ctx->d_flag, sizeof(int), cudaMemcpyDeviceToHost, s));
  GMG_CK(cudaStreamSynchronize(s));
  if (bad) return fail(ctx, SEM_ERR_BAD_MESH, "a coarsened multigrid level has an inverted element");
  const size_t es = elem_size(g->precision);
  int64_t nmax = 0;
  for (GmgLevel& V : g->lv) {
    Level& L = *V.L;
    nmax = std::max(nmax, L.ndofs);
    if (g->precision == SEM_PREC_FP32 && !L.metric32_valid) {
      if (!L.metric32) GMG_CK(cudaMalloc(&L.metric32, sizeof(float) * metric_count(L)));
      GMG_CK(setup_metric_lowp(L, false, s));
    }
    const bool tc = g->precision == SEM_PREC_BF16_TC && tc_supported(L) && !ctx->deterministic;
    if ((g->precision == SEM_PREC_FP32_BF16 || (g->precision == SEM_PREC_BF16_TC && !tc)) &&
        !L.metric16_valid) {
      if (!L.metric16) GMG_CK(cudaMalloc(&L.metric16, sizeof(__nv_bfloat16) * metric16_count(L)));
      GMG_CK(setup_metric_lowp(L, true, s));
    }
    if (tc && !L.metric_tc_valid) GMG_CK(setup_metric_tc(L, s));
    void** vecs[] = {&V.b, &V.x, &V.t, &V.d, &V.invd};
    for (void** v : vecs) GMG_CK(cudaMalloc(v, es * L.ndofs));
    GMG_CK(cudaMemsetAsync(V.t, 0, es * L.ndofs, s));
    GMG_CK(cudaMalloc(&V.dinv64, sizeof(double) * L.ndofs));
  }
  for (size_t l = 0; l + 1 < g->lv.size(); ++l) {
    GmgLevel& V = g->lv[l];
    if (V.to_next != 0) continue;
    GMG_CK(cudaMalloc(&V.pw1, es * p_transfer_scratch(*V.L, *g->lv[l + 1].L, 1)));
    GMG_CK(cudaMalloc(&V.pw2, es * p_transfer_scratch(*V.L, *g->lv[l + 1].L, 2)));
  }
  const int64_t nf = ctx->L.ndofs;
  GMG_CK(cudaMalloc(&g->z, sizeof(double) * nf));
  GMG_CK(cudaStreamCreateWithFlags(&g->capture, cudaStreamNonBlocking));
  GMG_CK(cudaEventCreate(&g->ev0));
  GMG_CK(cudaEventCreate(&g->ev1));
  GMG_CK(cudaEventCreate(&g->ev2));
  GMG_CK(cudaEventCreate(&g->ev3));
  double** lv4[] = {&g->lr, &g->lz, &g->lp, &g->lAp};
  for (double** v : lv4) GMG_CK(cudaMalloc(v, sizeof(double) * nmax));
  GMG_CK(cudaMalloc(&g->dots, sizeof(double) * 8));
  g->partial_len = 2048;
  GMG_CK(cudaMalloc(&g->partials, sizeof(double) * 4 * g->partial_len));
  GMG_CK(cudaMalloc(&g->tickets, sizeof(unsigned int) * 4));
  GMG_CK(cudaMemsetAsync(g->tickets, 0, sizeof(unsigned int) * 4, s));
  GMG_CK(cudaStreamSynchronize(s));
  ctx->gmg = g;
  g = nullptr;  // ownership moved to the context
  return SEM_OK;
}

// Kernel nodes of an instantiated graph's source graph.
int64_t count_kernels(cudaGraph_t graph) {
  size_t n = 0;
  if (cudaGraphGetNodes(graph, nullptr, &n) != cudaSuccess) return 0;
  std::vector<cudaGraphNode_t> nodes(n);
  if (cudaGraphGetNodes(graph, nodes.data(), &n) != cudaSuccess) return 0;
  int64_t k = 0;
  for (auto nd : nodes) {
    cudaGraphNodeType t;
    if (cudaGraphNodeGetType(nd, &t) == cudaSuccess && t == cudaGraphNodeTypeKernel) ++k;
  }
  return k;
}

// The PCG launch sequences, issued on stream s (a capture stream when graphs are built).
// Set-up: r = b - A x, stopping threshold, convergence test.  One iteration:
// z = V(r), beta, p = z + beta p, A p with alpha = r.z / p.Ap, x and r updated,
// convergence test.  The iteration ends with the test, so the host launches no
// V-cycle after convergence.
// carried: A x is read from ws.Ax (the last time step's b - r) instead of
// applied; ws.Ap is then already zero (every PCG iteration leaves it zero).
// checked (with carried): a device flag; the zeroing of ws.Ap and the apply run
// only where it reads zero (they return at once otherwise), and the residual
// kernel reads ws.Ax or ws.Ap accordingly.
template <typename T>
int pcg_init_seq(sem_ctx* ctx, Gmg& g, double alpha, const double* b, const double* x, double rtol,
                 double atol, bool carried, const int* checked, cudaStream_t s) {
  Workspace& w = ctx->ws;
  Level& L = ctx->L;
  const int64_t n = L.ndofs;
  const int gr = grid1d(n);
  T* b0 = (T*)g.lv[0].b;
  const int stride = g.partial_len;
  if (!carried || checked != nullptr) {
    launch_k(k_zero<double>, gr, kThreads, 0, s, n, w.Ap, checked);
    ApplyArgs64 a{};
    a.map = L.map; a.metric = L.metric; a.u = x; a.y = w.Ap; a.nelem = L.nelem;
    a.mass_coef = alpha; a.out_scale = 1.0; a.scale_out = 0; a.done = checked;
    a.yloc = ctx->deterministic ? ctx->det_scratch : nullptr;
    GMG_CK(launch_operator(ctx, a, s));
  }
  if (ctx->op_precision == SEM_PREC_DF64) {  // r kept as float pairs in ws.r, carried A x as pairs in ws.Ax
    auto kern = aligned16(b) ? k_dfpcg_init<T, true> : k_dfpcg_init<T, false>;
    launch_k(kern, gr, kThreads, 0, s, n, b, w.Ap, carried ? reinterpret_cast<const df_pair*>(w.Ax) : nullptr,
             checked, reinterpret_cast<df_pair*>(w.r), b0, w.cg, g.partials, stride, g.tickets, rtol, atol);
  } else {
    auto kern = aligned16(b) ? k_fpcg_init<T, true> : k_fpcg_init<T, false>;
    launch_k(kern, gr, kThreads, 0, s, n, b, carried ? w.Ax : w.Ap, w.Ap, checked, w.r, b0, w.cg, g.partials,
             stride, g.tickets, rtol, atol);
  }
  GMG_CK(cudaGetLastError());
  return SEM_OK;
}

// timed: external event nodes around the fine-level residual apply of the V-cycle
// (ev2, ev3) and the outer operator apply (ev0, ev1).  Each event node costs a few
// microseconds of the step (it breaks the programmatic dependent launch around it),
// so only the sampled iterations use the timed graph.
template <typename T>
int pcg_iter_seq(sem_ctx* ctx, Gmg& g, double alpha, double* x, bool timed, cudaStream_t s) {
  Workspace& w = ctx->ws;
  Level& L = ctx->L;
  const int64_t n = L.ndofs;
  const int gr = grid1d(n);
  const int stride = g.partial_len;
  const int* done = &w.cg->done;
  int rc = vcycle(ctx, g, done, s, timed);
  if (rc != SEM_OK) return rc;
  // the double-float operator gathers p as the float pairs the p kernels write
  const bool dfop = ctx->op_precision == SEM_PREC_DF64;
  df_pair* p2 = dfop ? w.p2 : nullptr;
  df_pair* r2 = reinterpret_cast<df_pair*>(w.r);
  if (dfop) {
    launch_k(k_dfpcg_z<T>, gr, kThreads, 0, s, n, (const T*)g.lv[0].x, reinterpret_cast<T*>(g.z), r2, p2, w.cg,
             g.partials, stride, g.tickets + 1);
    launch_k(k_dfpcg_p<T>, gr, kThreads, 0, s, n, reinterpret_cast<const T*>(g.z), p2, w.cg);
  } else {
    launch_k(k_fpcg_z<T>, gr, kThreads, 0, s, n, (const T*)g.lv[0].x, g.z, w.r, w.p, p2, w.cg, g.partials,
             stride, g.tickets + 1);
    launch_k(k_fpcg_p, gr, kThreads, 0, s, n, g.z, w.p, p2, w.cg);
  }
  GMG_CK(cudaGetLastError());
  ApplyArgs64 ap{};
  ap.map = L.map; ap.metric = L.metric; ap.u = w.p; ap.y = w.Ap; ap.nelem = L.nelem;
  ap.mass_coef = alpha; ap.out_scale = 1.0; ap.scale_out = 0; ap.done = done;
  ap.dot_partials = w.apply_partials; ap.cg = w.cg; ap.u2 = p2;
  ap.yloc = ctx->deterministic ? ctx->det_scratch : nullptr;
  // external records become event nodes of the captured graph (timing of the outer apply)
  if (timed) GMG_CK(cudaEventRecordWithFlags(g.ev0, s, cudaEventRecordExternal));
  GMG_CK(launch_operator(ctx, ap, s));
  if (timed) GMG_CK(cudaEventRecordWithFlags(g.ev1, s, cudaEventRecordExternal));
  if (dfop)
    launch_k(aligned16(x) ? k_dfpcg_xr<T, true> : k_dfpcg_xr<T, false>, std::min(gr, 152 * kXrCtasPerSm),
             kThreads, 0, s, n, x, p2, w.Ap, r2, (T*)g.lv[0].b, w.cg, g.partials, stride, g.tickets + 2);
  else if (aligned16(x))
    launch_k(k_fpcg_xr<T, true>, gr, kThreads, 0, s, n, x, w.p, w.Ap, w.r, (T*)g.lv[0].b, w.cg, g.partials,
                                             stride, g.tickets + 2);
  else
    launch_k(k_fpcg_xr<T, false>, gr, kThreads, 0, s, n, x, w.p, w.Ap, w.r, (T*)g.lv[0].b, w.cg, g.partials,
                                              stride, g.tickets + 2);
  GMG_CK(cudaGetLastError());
  return SEM_OK;
}

// Captures (once per solution pointer, right-hand side, alpha and tolerances) the
// set-up and iteration sequences as CUDA graphs; sixteen are cached.
template <typename T>
int get_graphs(sem_ctx* ctx, Gmg& g, double alpha, const double* b, double* x, double rtol,
               double atol, Gmg::Graphs** out) {
  for (auto& gr : g.graphs)
    if (gr.iter && gr.x == x && gr.b == b && gr.alpha == alpha && gr.rtol == rtol && gr.atol == atol) {
      *out = &gr;
      return SEM_OK;
    }
  Gmg::Graphs& gr = g.graphs[g.next_graph];
  g.next_graph = (g.next_graph + 1) % 16;
  if (gr.init) { cudaGraphExecDestroy(gr.init); gr.init = nullptr; }
  if (gr.iter) { cudaGraphExecDestroy(gr.iter); gr.iter = nullptr; }
  if (gr.init_carried) { cudaGraphExecDestroy(gr.init_carried); gr.init_carried = nullptr; }
  if (gr.init_checked) { cudaGraphExecDestroy(gr.init_checked); gr.init_checked = nullptr; }
  if (gr.iter_timed) { cudaGraphExecDestroy(gr.iter_timed); gr.iter_timed = nullptr; }
  for (auto& cv : gr.combo)
    for (auto& c : cv) {
      if (c.exec) cudaGraphExecDestroy(c.exec);
      c = Gmg::Graphs::Combo();
    }
  cudaStream_t cs = g.capture;
  const int64_t l0 = ctx->launches;
  for (int which = 0; which < 5; ++which) {
    GMG_CK(cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal));
    int rc = (which == 1 || which == 4) ? pcg_iter_seq<T>(ctx, g, alpha, x, which == 4, cs)
                                        : pcg_init_seq<T>(ctx, g, alpha, b, x, rtol, atol, which >= 2,
                                                          which == 3 ? ctx->ws.same : nullptr, cs);
    cudaGraph_t graph = nullptr;
    const cudaError_t ec = cudaStreamEndCapture(cs, &graph);
    if (rc != SEM_OK) {
      if (graph) cudaGraphDestroy(graph);
      return rc;
    }
    if (ec != cudaSuccess) return cuda_fail(ctx, ec, "cudaStreamEndCapture");
    cudaGraphExec_t exec = nullptr;
    const cudaError_t ei = cudaGraphInstantiate(&exec, graph, 0);
    const int64_t nk = count_kernels(graph);
    cudaGraphDestroy(graph);
    if (ei != cudaSuccess) return cuda_fail(ctx, ei, "cudaGraphInstantiate");
    if (which == 0) { gr.init = exec; gr.init_kernels = nk; }
    else if (which == 1) { gr.iter = exec; gr.iter_kernels = nk; }
    else if (which == 2) { gr.init_carried = exec; gr.init_carried_kernels = nk; }
    else if (which == 3) { gr.init_checked = exec; gr.init_checked_kernels = nk; }
    else { gr.iter_timed = exec; gr.iter_timed_kernels = nk; }
  }
  ctx->launches = l0;  // capture launched nothing; replays are counted
  gr.x = x;
  gr.b = b;
  gr.alpha = alpha;
  gr.rtol = rtol;  // the stopping tolerances are baked into the set-up graph
  gr.atol = atol;
  *out = &gr;
  return SEM_OK;
}

// The combined graph of set-up variant v and n iterations (the first timed when
// timed), captured on first use and again when n changes.
template <typename T>
int get_combo(sem_ctx* ctx, Gmg& g, Gmg::Graphs& gr, int v, bool timed, int n, double alpha, const double* b,
              double* x, double rtol, double atol, Gmg::Graphs::Combo** out) {
  Gmg::Graphs::Combo& c = gr.combo[v][timed ? 1 : 0];
  if (c.exec == nullptr || c.n != n) {
    if (c.exec) { cudaGraphExecDestroy(c.exec); c = Gmg::Graphs::Combo(); }
    cudaStream_t cs = g.capture;
    const int64_t l0 = ctx->launches;
    GMG_CK(cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal));
    int rc = pcg_init_seq<T>(ctx, g, alpha, b, x, rtol, atol, v >= 1, v == 2 ? ctx->ws.same : nullptr, cs);
    for (int i = 0; i < n && rc == SEM_OK; ++i) rc = pcg_iter_seq<T>(ctx, g, alpha, x, timed && i == 0, cs);
    cudaGraph_t graph = nullptr;
    const cudaError_t ec = cudaStreamEndCapture(cs, &graph);
    ctx->launches = l0;
    if (rc != SEM_OK) {
      if (graph) cudaGraphDestroy(graph);
      return rc;
    }
    if (ec != cudaSuccess) return cuda_fail(ctx, ec, "cudaStreamEndCapture");
    const cudaError_t ei = cudaGraphInstantiate(&c.exec, graph, 0);
    c.kernels = count_kernels(graph);
    cudaGraphDestroy(graph);
    if (ei != cudaSuccess) {
      c.exec = nullptr;
      return cuda_fail(ctx, ei, "cudaGraphInstantiate");
    }
    c.n = n;
  }
  *out = &c;
  return SEM_OK;
}

template <typename T>
int pcg_t(sem_ctx* ctx, Gmg& g, double alpha, const double* b, double* x, double rtol,
          double atol, int maxit, int* iters, double* final_res, sem_stats* stats, bool carried,
          bool checked, cudaStream_t s) {
  Workspace& w = ctx->ws;
  Gmg::Graphs* gr = nullptr;
  int rc = get_graphs<T>(ctx, g, alpha, b, x, rtol, atol, &gr);
  if (rc != SEM_OK) return rc;
  Timing& tm = ctx->timing;
  bool done_h = false;
  int launched = 0;
  // with timing on, the first iteration of one solve in kTimingEvery is the timed one
  bool sample = tm.enabled && (tm.solves++ % kTimingEvery) == 0;
  auto launch_iter = [&]() -> cudaError_t {
    const bool timed = sample && launched == 0;
    const cudaError_t e = cudaGraphLaunch(timed ? gr->iter_timed : gr->iter, s);
    ctx->launches += timed ? gr->iter_timed_kernels : gr->iter_kernels;
    return e;
  };
  // Successive solves (time steps) take about the same number of iterations:
  // the set-up and the previous count go out as one graph before the scalars are
  // read, so that a solve that needs no more costs one launch and one host round
  // trip.  An iteration launched after convergence runs kernels that return at once.
  const int ahead = std::min(maxit, std::max(0, gr->last_iters));
  const int variant = !carried ? 0 : (checked ? 2 : 1);
  if (ahead > 0) {
    Gmg::Graphs::Combo* c = nullptr;
    if ((rc = get_combo<T>(ctx, g, *gr, variant, sample, ahead, alpha, b, x, rtol, atol, &c)) != SEM_OK) return rc;
    GMG_CK(cudaGraphLaunch(c->exec, s));
    ctx->launches += c->kernels;
    launched = ahead;
  } else {
    GMG_CK(cudaGraphLaunch(variant == 0 ? gr->init : (variant == 2 ? gr->init_checked : gr->init_carried), s));
    ctx->launches += variant == 0 ? gr->init_kernels : (variant == 2 ? gr->init_checked_kernels : gr->init_carried_kernels);
  }
  while (true) {
    GMG_CK(cudaMemcpyAsync(w.cg_host, w.cg, sizeof(CgScalars), cudaMemcpyDeviceToHost, s));
    GMG_CK(cudaMemcpyAsync(w.fault_host, ctx->L.fault, sizeof(unsigned), cudaMemcpyDeviceToHost, s));
    GMG_CK(cudaStreamSynchronize(s));
    if (*w.fault_host != 0u) {  // an apply kernel gave up waiting for its metric copy
      *w.fault_host = 0u;
      GMG_CK(cudaMemsetAsync(ctx->L.fault, 0, sizeof(unsigned), s));
      GMG_CK(cudaStreamSynchronize(s));
      return fail(ctx, SEM_ERR_TIMEOUT, "an apply kernel's wait for its metric copy timed out");
    }
    if (sample && launched > 0 && w.cg_host->iters >= 1) {  // the timed first iteration ran
      sample = false;
      float ms = 0.f;
      if (cudaEventElapsedTime(&ms, g.ev0, g.ev1) == cudaSuccess) {
        tm.ms += ms;
        tm.count += 1;
      } else {
        cudaGetLastError();  // timing unavailable for these event nodes: not an error
      }
      if (cudaEventElapsedTime(&ms, g.ev2, g.ev3) == cudaSuccess) {
        tm.smoother_ms += ms;
        tm.smoother_count += 1;
      } else {
        cudaGetLastError();
      }
    }
    if (w.cg_host->done) { done_h = true; break; }
    if (launched >= maxit) break;
    GMG_CK(launch_iter());
    ++launched;
  }
  const CgScalars& h = *w.cg_host;
  gr->last_iters = h.iters;
  if (iters) *iters = h.iters;
  if (final_res) *final_res = std::sqrt(h.rr);
  if (stats) {
    stats->cg_iters += h.iters;
    stats->last_residual = std::sqrt(h.rr);
  }
  if (h.status == SEM_ERR_NONFINITE)
    return fail(ctx, SEM_ERR_NONFINITE, "non-finite value in a CG inner product");
  if (!done_h)
    return fail(ctx, SEM_ERR_NOT_CONVERGED,
                "multigrid PCG did not converge in " + std::to_string(maxit) + " iterations");
  return SEM_OK;
}

}  // namespace

void gmg_free(sem_ctx* ctx) {
  if (ctx->gmg) {
    free_gmg_struct(ctx->gmg);
    ctx->gmg = nullptr;
  }
}

int gmg_pcg(sem_ctx* ctx, double alpha, const double* b, double* x, double rtol, double atol,
            int maxit, int* iters, double* final_res, sem_stats* stats, cudaStream_t s, double* ax0,
            const int* ax0_ok) {
  int rc = ensure_workspace(ctx);
  if (rc != SEM_OK) return rc;
  // the carried A x and its check flag are always the workspace's (captured into the set-up graphs)
  if (ax0 != nullptr && ax0 != ctx->ws.Ax) return fail(ctx, SEM_ERR_ARG, "carried A x must be the workspace's");
  if (ax0_ok != nullptr && ax0_ok != ctx->ws.same) return fail(ctx, SEM_ERR_ARG, "carry check must be the workspace's");
  if (rc != SEM_OK) return rc;
  if ((rc = build(ctx, s)) != SEM_OK) return rc;
  GMG_CK(prepare_operator(ctx, s));
  Gmg& g = *ctx->gmg;
  if ((rc = set_alpha(ctx, g, alpha, s)) != SEM_OK) return rc;
  if (g.precision == SEM_PREC_FP64)
    return pcg_t<double>(ctx, g, alpha, b, x, rtol, atol, maxit, iters, final_res, stats, ax0 != nullptr,
                         ax0_ok != nullptr, s);
  return pcg_t<float>(ctx, g, alpha, b, x, rtol, atol, maxit, iters, final_res, stats, ax0 != nullptr,
                      ax0_ok != nullptr, s);
}

int gmg_vcycle(sem_ctx* ctx, double alpha, const double* r, double* z, cudaStream_t s) {
  int rc = build(ctx, s);
  if (rc != SEM_OK) return rc;
  Gmg& g = *ctx->gmg;
  if ((rc = set_alpha(ctx, g, alpha, s)) != SEM_OK) return rc;
  const int64_t n = ctx->L.ndofs;
  if (g.precision == SEM_PREC_FP64)
    launch_k(k_to_level0<double>, grid1d(n), kThreads, 0, s, n, r, (double*)g.lv[0].b);
  else
    launch_k(k_to_level0<float>, grid1d(n), kThreads, 0, s, n, r, (float*)g.lv[0].b);
  GMG_CK(cudaGetLastError());
  if ((rc = vcycle(ctx, g, nullptr, s)) != SEM_OK) return rc;
  if (g.precision == SEM_PREC_FP64)
    launch_k(k_from_level0<double>, grid1d(n), kThreads, 0, s, n, (const double*)g.lv[0].x, z);
  else
    launch_k(k_from_level0<float>, grid1d(n), kThreads, 0, s, n, (const float*)g.lv[0].x, z);
  GMG_CK(cudaGetLastError());
  return SEM_OK;
}

int gmg_info(sem_ctx* ctx, double alpha, int max_levels, int* nlevels, int* p, int* dims,
             int64_t* ndofs, double* lambda_max, cudaStream_t s) {
  int rc = build(ctx, s);
  if (rc != SEM_OK) return rc;
  Gmg& g = *ctx->gmg;
  if ((rc = set_alpha(ctx, g, alpha, s)) != SEM_OK) return rc;
  const int nl = (int)g.lv.size();
  if (nlevels) *nlevels = nl;
  for (int l = 0; l < std::min(nl, max_levels); ++l) {
    const Level& L = *g.lv[l].L;
    if (p) p[l] = L.p;
    if (dims) { dims[3 * l] = L.nx; dims[3 * l + 1] = L.ny; dims[3 * l + 2] = L.nz; }
    if (ndofs) ndofs[l] = L.ndofs;
    if (lambda_max) lambda_max[l] = g.lv[l].lam;
  }
  return SEM_OK;
}

}  // namespace sem
