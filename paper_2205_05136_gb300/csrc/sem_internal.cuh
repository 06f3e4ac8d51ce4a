// Internal declarations of libsem (not part of the C ABI).
//
// Layout of the data in HBM (one context = one slab, one device):
//   map      int32  [nelem][n^3]   local node a = i + n j + n^2 k -> global node
//   metric   double [nelem][7][n3p] per quadrature point: G00 G01 G02 G11 G12 G22 W,
//            n3p = n^3 rounded up to a multiple of 8 (16-byte aligned blocks),
//            G = w |det J| J^{-1} D J^{-T}, W = w |det J|  (element-blocked SoA)
//   metric32 float [nelem][7][n3p] copy of the same array (mixed-precision applies)
//   metric16 bf16  [nelem][n^2][CW] column-major copy: the 7 n values of the
//            quadrature points of column (i, j) in CW = 7 n rounded up to 4
//            (p = 4: 36 values, 72 bytes), read by 64-bit loads
//   mdiag    double [ndofs]  diagonal of the assembled mass matrix
//   kdiag    double [ndofs]  diagonal of the assembled stiffness matrix
//   xyz      double [3][ndofs] node coordinates
#pragma once

#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <stdint.h>

#include <string>
#include <utility>

#include "sem.h"
#include "sem_df64.cuh"

namespace sem {

// Index checks of the SEM_DEBUG build.  dbg_index returns a node index read
// from an element-to-DOF map (or computed from the lattice) when it lies in
// [0, n); otherwise it records the first offender in *word as
// (kind << 56) | (32-bit index) and returns 0, so no access leaves the vector.
// The host reads and clears the word after the call (debug_check) and returns
// SEM_ERR_ARG with the index.  In the normal build SEM_IDX is the index itself.
constexpr unsigned kDbgGather = 1, kDbgScatter = 2, kDbgLine = 3, kDbgTransfer = 4;
#if defined(SEM_DEBUG) && defined(__CUDACC__)
__device__ __forceinline__ int64_t dbg_index(int64_t g, int64_t n, unsigned long long* word, unsigned kind) {
  if (g >= 0 && g < n) return g;
  if (word != nullptr)
    atomicCAS(word, 0ull, ((unsigned long long)kind << 56) | (unsigned long long)(uint32_t)g);
  return 0;
}
#define SEM_IDX(g, n, word, kind) dbg_index((g), (n), (word), (kind))
// a copy the SEM_DEBUG build leaves out on request (sem_debug_hold_copy), so that
// the wait for it runs out and the timeout path runs
#define SEM_HOLD(a, unit) ((unit) == (a).hold)
#else
#define SEM_IDX(g, n, word, kind) (g)
#define SEM_HOLD(a, unit) false
#endif

// Programmatic dependent launch (PDL).  A kernel launched by launch_k may be
// scheduled while the kernel before it in the stream is still draining, and
// then runs its blocks up to pdl_entry().  pdl_entry() first lets the next
// kernel of the stream launch in turn (griddepcontrol.launch_dependents), then
// waits until the previous grid has completed and its writes are visible
// (griddepcontrol.wait).  Every kernel launched by launch_k calls pdl_entry()
// in every block before it reads or writes memory that another kernel writes
// or reads, so that grids still complete in stream order and each kernel sees
// all earlier results.  In a kernel launched without the attribute both
// instructions return at once.  Inside a CUDA graph the attribute becomes a
// programmatic edge between the two kernel nodes.
// Kernels that can start useful independent work (L2 prefetches of the map and
// metric, which no kernel of a solve writes) call pdl_trigger(), issue it, then
// pdl_wait(); a prefetch only warms L2, the point of coherence, so nothing read
// before the wait is used.
#ifdef __CUDACC__
__device__ __forceinline__ void pdl_trigger() { asm volatile("griddepcontrol.launch_dependents;\n" ::: "memory"); }
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;\n" ::: "memory"); }
__device__ __forceinline__ void pdl_entry() {
  pdl_trigger();
  pdl_wait();
}
// L2 prefetch of the 128-byte lines of [p, p + bytes), line `first` and every
// `step`-th after it by this thread.
__device__ __forceinline__ void prefetch_l2_lines(const void* p, size_t bytes, int first, int step) {
  const uintptr_t a0 = reinterpret_cast<uintptr_t>(p) & ~(uintptr_t)127;
  const uintptr_t end = reinterpret_cast<uintptr_t>(p) + bytes;
  for (uintptr_t a = a0 + (uintptr_t)first * 128u; a < end; a += (uintptr_t)step * 128u)
    asm volatile("prefetch.global.L2 [%0];\n" ::"l"(a));
}
#endif
bool pdl_enabled();  // false when the environment sets SEM_NO_PDL (read once)
template <typename... P, typename... A>
cudaError_t launch_k(void (*kernel)(P...), dim3 grid, dim3 block, size_t smem, cudaStream_t s,
                     A&&... args) {
  cudaLaunchConfig_t cfg{};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  at[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = at;
  cfg.numAttrs = pdl_enabled() ? 1 : 0;
  return cudaLaunchKernelEx(&cfg, kernel, std::forward<A>(args)...);
}

// Storage type of the vectors an operator kernel reads and writes: the df64
// operator works on FP64 vectors.
template <typename T> struct VecOf { using type = T; };
template <> struct VecOf<df> { using type = double; };

constexpr int kMaxP = 6;
constexpr int kMaxN = kMaxP + 1;
constexpr int kMetricComps = 7;

// Quadrature points per element rounded up to a multiple of 8: every element's
// metric block and each of its 7 components then start on a 16-byte boundary
// in every storage precision (bf16, float, double, float pairs).
__host__ __device__ constexpr int padded_n3(int n) { return ((n * n * n + 7) / 8) * 8; }

// 1-D tables of one degree p and one quadrature kind (host side, double).
struct Tables1D {
  int p = 0, n = 0, quad = 0;
  double xg[kMaxN] = {}, wg[kMaxN] = {};  // LGL nodes / weights
  double xq[kMaxN] = {}, wq[kMaxN] = {};  // quadrature nodes / weights
  double D[kMaxN][kMaxN] = {};   // D[q][l] = l_l'(xg_q)  (GLL collocation derivative)
  double Bi[kMaxN][kMaxN] = {};  // Bi[q][l] = l_l(xq_q)   (GLL basis at quadrature points)
  double Dg[kMaxN][kMaxN] = {};  // Dg[q][m] = g_m'(xq_q)  (collocation derivative on the quadrature points)
};

// Builds the tables of degree p (1..kMaxP) for quad SEM_QUAD_LG / SEM_QUAD_LGL.
void build_tables(int p, int quad, Tables1D* t);

// Even-odd form of an n x n matrix M with M[n-1-q][n-1-l] = s M[q][l]: s = -1
// for a derivative matrix on points symmetric about 0 (and its transpose),
// s = +1 for interpolation between two symmetric point sets.  With H = n / 2,
// for q, l < H:
//   a[q][l] = (M[q][l] + M[q][n-1-l]) / 2,   b[q][l] = (M[q][l] - M[q][n-1-l]) / 2,
// and for odd n the middle column a[q][H] = M[q][H] and the middle row
// c[l] = M[H][l] (l <= H).  A product y = M x then takes about half the
// multiplications (see eo_line).  For n = 2 and 4 the split saves no
// multiplication, so the matrix itself (m) is kept and multiplied directly.
template <int N, typename T>
struct EoMat {
  static constexpr int H = N / 2;
  static constexpr bool kDirect = (N == 2 || N == 4);
  static constexpr int NM = kDirect ? N : 1;
  T a[H][H + 1];
  T b[H][H];
  T c[H + 1];
  T m[NM][NM];
};

// Tables in the kernel's arithmetic type, passed to kernels by value (kernel
// parameter space): accesses with compile-time indices become constant-bank
// operands of the FMA instructions.
template <int N, typename T>
struct KTab {
  EoMat<N, T> D, Dt;    // derivative matrix of the gradient (D for SEM-NI, Dg for SEM), its transpose
  EoMat<N, T> Bi, Bit;  // interpolation GLL -> quadrature points (SEM only), its transpose
};

// Deterministic grid reductions: every block writes a partial, the last block
// to finish (atomic ticket) sums the partials in block order.
// Partials of the vector kernels: kVecBlocksMax per reduction slot.
constexpr int kVecBlocksMax = 2048;
constexpr int kReduceSlots = 4;

// Device scalars of one CG solve.
struct CgScalars {
  double rz;      // r . z of the current iterate
  double rr;      // r . r
  double bb;      // b . b
  double pAp;     // p . A p
  double alpha;   // step length
  double beta;    // conjugation coefficient
  double tol2;    // squared stopping threshold on ||r||
  int done;       // 1 when converged or failed
  int iters;      // iterations taken
  int status;     // 0 ok, SEM_ERR_NONFINITE
  int pad;
};

struct Level {
  int p = 0, quad = 0, n = 0;
  int nx = 0, ny = 0, nz = 0;
  int nelem = 0;
  int64_t ndofs = 0;
  Tables1D tab;
  int* map = nullptr;
  double* evert = nullptr;   // [nelem][8][3] element vertices
  double* metric = nullptr;  // [nelem][7][n^3]
  float* metric32 = nullptr;
  __nv_bfloat16* metric16 = nullptr;
  df_pair* metric2 = nullptr;  // FP64 metric split into FP32 pairs (df64 operator)
  uint32_t* metric_tc = nullptr;  // bf16 metric in the tensor-core kernel's order (sem_apply_tc.cu)
  uint32_t* tc_frag = nullptr;    // constant MMA fragments of the tensor-core kernel
  bool metric32_valid = false, metric16_valid = false, metric2_valid = false, metric_tc_valid = false;
  unsigned long long* dbg = nullptr;  // SEM_DEBUG build: the context's index-error word
  unsigned* fault = nullptr;  // the context's wait-timeout word (nonzero: a kernel gave up a wait)
  int hold = -1;  // SEM_DEBUG build: element group whose metric copy the pipelined apply skips
  double* mdiag = nullptr;
  double* kdiag = nullptr;
  double* xyz = nullptr;
};

// Number of metric values of a level (7 components x padded points per element).
inline size_t metric_count(const Level& L) {
  return (size_t)L.nelem * kMetricComps * padded_n3(L.n);
}

// Offset of component `comp` of the quadrature point on column c = i + n j at
// level k inside one element's metric block.
//   double, float, float pairs: component-major [7][padded n^3], point c + n^2 k;
//   bf16: column-major, the 7 values of level k at 7 k .. 7 k + 6 of the
//   column's CW = 7 n (rounded up to a multiple of 4) values, so that a lane
//   reads its whole column with CW / 4 aligned 64-bit loads and no point is
//   padded; the block is rounded up to 16 bytes (cp.async / TMA granularity).
template <typename MT>
struct MetricLayout {
  static constexpr bool kColumnMajor = false;
  __host__ __device__ static constexpr int block(int n) { return kMetricComps * padded_n3(n); }
  __host__ __device__ static constexpr int at(int n, int c, int k, int comp) {
    return comp * padded_n3(n) + c + k * n * n;
  }
};
template <>
struct MetricLayout<__nv_bfloat16> {
  static constexpr bool kColumnMajor = true;
  __host__ __device__ static constexpr int col_width(int n) { return (kMetricComps * n + 3) / 4 * 4; }
  __host__ __device__ static constexpr int block(int n) { return (n * n * col_width(n) + 7) / 8 * 8; }
  __host__ __device__ static constexpr int at(int n, int c, int k, int comp) {
    return c * col_width(n) + kMetricComps * k + comp;
  }
};

// Number of values of the bf16 metric of a level.
inline size_t metric16_count(const Level& L) {
  return (size_t)L.nelem * MetricLayout<__nv_bfloat16>::block(L.n);
}

// Arguments of the element kernel y += A_e u_e (scatter-add into y).
template <typename T, typename MT>
struct ApplyArgs {
  const int* map;
  const MT* metric;
  const typename VecOf<T>::type* u;
  typename VecOf<T>::type* y;
  int nelem;
  T mass_coef;        // coefficient of the mass term inside the element kernel
  T out_scale;        // factor applied to the element result before the scatter
  int scale_out;      // out_scale != 1
  const int* done;    // optional: skip all work when *done != 0
  // optional fused u . (A u) (CG's p . A p): every CTA writes its partial sum
  // to dot_partials (one double per CTA of the launch) and a one-CTA kernel
  // launched after the apply adds them up
  double* dot_partials;
  CgScalars* cg;      // when set, the sum goes to pAp, and alpha = rz / pAp
  double* dot_out;    // otherwise the sum goes here
  // optional (double-float operator with the fused inner product): u split into
  // float pairs by the kernel that formed u; the gather then reads the pairs and
  // converts nothing
  const df_pair* u2;
  // optional (deterministic mode): element results go to yloc[e][n^3] instead of
  // atomic adds, and a node kernel then adds each node's contributions to y in a
  // fixed order
  typename VecOf<T>::type* yloc;
  // set by the launcher: the vectors' length, the SEM_DEBUG index-error word and
  // the wait-timeout word
  int64_t ndofs;
  unsigned long long* dbg;
  unsigned* fault;
  int hold;  // SEM_DEBUG build: Level::hold
};
using ApplyArgs64 = ApplyArgs<double, double>;

// Kernel launchers (sem_apply_fp64.cu, sem_apply_fp32.cu).
cudaError_t launch_apply_fp64(const Level& L, const ApplyArgs64& a, bool mass_only, cudaStream_t s);
cudaError_t launch_apply_fp32(const Level& L, const ApplyArgs<float, float>& a, bool mass_only,
                              cudaStream_t s);
cudaError_t launch_apply_bf16(const Level& L, const ApplyArgs<float, __nv_bfloat16>& a,
                              bool mass_only, cudaStream_t s);
cudaError_t launch_apply_df64(const Level& L, const ApplyArgs<df, df_pair>& a, bool mass_only,
                              cudaStream_t s);
int apply_grid_blocks(const Level& L);
// y[g] += the element contributions yloc[e][n^3] of node g, elements in a fixed
// order (ez, ey, ex ascending): the deterministic assembly of the apply kernels'
// element results (and of the p-restriction's coarse-element results).
cudaError_t launch_assemble(const Level& L, const double* yloc, double* y, const int* done, cudaStream_t s);
cudaError_t launch_assemble(const Level& L, const float* yloc, float* y, const int* done, cudaStream_t s);
// Sum, in a fixed order, of the n per-CTA partials of a fused inner product:
// to cg (pAp and alpha = rz / pAp) when set, else to *out; nothing when *done.
cudaError_t launch_apply_dot_finish(const double* partials, int n, CgScalars* cg, double* out,
                                    const int* done, cudaStream_t s);
// Raises the dynamic shared-memory limit of the kernels that stage the metric in
// shared memory; call once per device before any stream capture.
cudaError_t prime_apply_kernels();

// Tensor-core FP32 operator with the bf16 metric (sem_apply_tc.cu): SEM-NI, p = 2..4.
bool tc_supported(const Level& L);
size_t tc_metric_words(const Level& L);
// Builds the level's metric_tc (from the FP64 metric) and constant fragments.
cudaError_t setup_metric_tc(Level& L, cudaStream_t s);
// y += (mass_coef M + K) u with a.u, a.y float vectors (a.map, a.metric unused).
cudaError_t launch_apply_tc(const Level& L, const ApplyArgs<float, __nv_bfloat16>& a, cudaStream_t s);
cudaError_t prime_apply_tc();

// Level construction (sem_setup.cu): structured numbering of an nx x ny x nz
// slab with host vertices, device allocation of map, element vertices, metric,
// diagonals (and node coordinates when `coords`).  Metric and diagonals are
// filled by setup_geometry / setup_diagonals.
cudaError_t level_create(Level& L, int nx, int ny, int nz, const double* vertices, int p, int quad,
                         bool coords, cudaStream_t s);
void level_free(Level& L);

// Setup kernels (sem_setup.cu).
cudaError_t setup_geometry(Level& L, const double* sigma_l, const double* sigma_t,
                           const double* theta, int* d_bad, cudaStream_t s);
cudaError_t setup_diagonals(Level& L, cudaStream_t s);
cudaError_t setup_metric_lowp(Level& L, bool bf16, cudaStream_t s);
cudaError_t setup_metric_df(Level& L, cudaStream_t s);
cudaError_t setup_node_coords(Level& L, cudaStream_t s);
cudaError_t setup_region_mask(const Level& L, int region, const double* prm, double* mask,
                              cudaStream_t s);

// Vector kernels (sem_solver.cu).
int vec_blocks(int64_t n);
cudaError_t vec_axpby_diag(int64_t n, double a, const double* x, double b, const double* y,
                           double* out, cudaStream_t s);  // out = a x + b y
cudaError_t vec_inv_diag(int64_t n, double alpha, const double* mdiag, const double* kdiag,
                         double* inv, cudaStream_t s);     // inv = 1/(alpha m + k)
cudaError_t vec_scale_mul(int64_t n, double a, const double* d, const double* x, double* y,
                          cudaStream_t s);                 // y = a d x

}  // namespace sem
