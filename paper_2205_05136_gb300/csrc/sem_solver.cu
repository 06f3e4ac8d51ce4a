// Solver layer: fused CG vector kernels, the preconditioned CG driver
// (Section 4: A is SPD, CG / PCG; one matrix-free apply per iteration), and
// the partitioned BDF time step (Section 3, Eqs. ionic_discr - matrix_rhs,
// Algorithm 1).
//
// One CG iteration is three kernels on the caller's stream:
//   apply   Ap += A p (element kernel) and p . Ap; its last CTA sets
//           alpha = (r . z) / (p . Ap)
//   xr      x += alpha p, r -= alpha Ap, z = Jacobi(r), r . z, r . r; its last
//           CTA sets beta, the iteration count and the convergence flag
//   p       p = z + beta p, Ap = 0
// Every reduction is deterministic (per-CTA partials summed in CTA order by
// the last CTA).  Scalars stay on the device; the host reads them once per
// chunk of iterations, and kernels of a finished solve return at once.
#include <algorithm>
#include <cmath>
#include <limits>
#include <vector>

#include "sem_apply_kernel.cuh"
#include "sem_context.cuh"
#include "sem_dfmath.cuh"

namespace sem {
namespace {

constexpr int kVecThreads = 256;

int vec_grid(int64_t n) {
  const int64_t want = (n + kVecThreads - 1) / kVecThreads;
  return (int)std::max<int64_t>(1, std::min<int64_t>(want, 152 * 8));
}

// Sum K values over the grid; the last CTA gets the totals (thread 0 returns true).
template <int K>
__device__ __forceinline__ bool grid_sums(double (&v)[K], double* partials, unsigned int* ticket,
                                          double (&tot)[K]) {
  __shared__ double red[K][32];
  __shared__ bool is_last;
  double bs[K];
#pragma unroll
  for (int k = 0; k < K; ++k) {
    bs[k] = block_sum(v[k], red[k]);
  }
  if (threadIdx.x == 0) {
#pragma unroll
    for (int k = 0; k < K; ++k) partials[k * kVecBlocksMax + blockIdx.x] = bs[k];
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
      s += ((volatile double*)partials)[k * kVecBlocksMax + b];
    tot[k] = block_sum(s, red[k]);
    __syncthreads();
  }
  if (threadIdx.x == 0) *ticket = 0u;
  return threadIdx.x == 0;
}

__global__ void k_inv_diag(int64_t n, double alpha, const double* __restrict__ m,
                           const double* __restrict__ k, double* __restrict__ inv) {
  pdl_entry();
#pragma unroll 1
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    inv[i] = 1.0 / fma(alpha, m[i], k[i]);
}

__global__ void k_scale_mul(int64_t n, double a, const double* __restrict__ d,
                            const double* __restrict__ x, double* __restrict__ y) {
  pdl_entry();
#pragma unroll 1
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    y[i] = a * d[i] * x[i];
}

__global__ void k_scale_mul32(int64_t n, float a, const double* __restrict__ d,
                              const float* __restrict__ x, float* __restrict__ y) {
  pdl_entry();
#pragma unroll 1
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    y[i] = a * (float)d[i] * x[i];
}

// r = b - Ap, z = Jacobi(r), p = z, Ap = 0; r.z, r.r, b.b; convergence test.
__global__ void __launch_bounds__(kVecThreads)
    k_cg_init(int64_t n, const double* __restrict__ b, double* __restrict__ Ap,
              const double* __restrict__ inv, double* __restrict__ r, double* __restrict__ z,
              double* __restrict__ p, df_pair* __restrict__ p2, CgScalars* cg, double* partials,
              unsigned int* ticket, double rtol, double atol) {
  pdl_entry();
  double v[3] = {0.0, 0.0, 0.0};
#pragma unroll 1
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const double bi = b[i];
    const double ri = bi - Ap[i];
    const double zi = inv ? inv[i] * ri : ri;
    r[i] = ri;
    z[i] = zi;
    p[i] = zi;
    if (p2 != nullptr) p2[i] = split_pair(zi);
    Ap[i] = 0.0;
    v[0] = fma(ri, zi, v[0]);
    v[1] = fma(ri, ri, v[1]);
    v[2] = fma(bi, bi, v[2]);
  }
  double tot[3];
  if (grid_sums<3>(v, partials, ticket, tot)) {
    cg->rz = tot[0];
    cg->rr = tot[1];
    cg->bb = tot[2];
    cg->tol2 = fmax(rtol * rtol * tot[2], atol * atol);
    cg->iters = 0;
    cg->status = 0;
    cg->beta = 0.0;
    const bool finite = isfinite(tot[0]) && isfinite(tot[1]) && isfinite(tot[2]);
    if (!finite) cg->status = SEM_ERR_NONFINITE;
    cg->done = (!finite || tot[1] <= cg->tol2) ? 1 : 0;
  }
}

// Pairs of consecutive entries as one 16-byte access (the workspace vectors come
// from cudaMalloc; a caller's x is checked for alignment on the host: VEC).
struct alignas(16) D2 {
  double e[2];
};

// x += alpha p, r -= alpha Ap, z = Jacobi(r); r.z, r.r; beta, convergence.
template <bool VEC>
__global__ void __launch_bounds__(kVecThreads)
    k_cg_xr(int64_t n, double* __restrict__ x, const double* __restrict__ p,
            const double* __restrict__ Ap, double* __restrict__ r, const double* __restrict__ inv,
            double* __restrict__ z, CgScalars* cg, double* partials, unsigned int* ticket) {
  pdl_entry();
  if (cg->done) return;
  const double alpha = cg->alpha;
  double v[2] = {0.0, 0.0};
  const int64_t g0 = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const int64_t gs = (int64_t)gridDim.x * blockDim.x;
  const int64_t nc = VEC ? n / 2 : 0;
#pragma unroll 1
  for (int64_t c = g0; c < nc; c += gs) {
    D2 xx = reinterpret_cast<const D2*>(x)[c];
    const D2 pp = reinterpret_cast<const D2*>(p)[c];
    const D2 aa = reinterpret_cast<const D2*>(Ap)[c];
    D2 rr = reinterpret_cast<const D2*>(r)[c];
    D2 ii;
    if (inv) ii = reinterpret_cast<const D2*>(inv)[c];
    D2 zz;
#pragma unroll
    for (int k = 0; k < 2; ++k) {
      xx.e[k] = fma(alpha, pp.e[k], xx.e[k]);
      rr.e[k] = fma(-alpha, aa.e[k], rr.e[k]);
      zz.e[k] = inv ? ii.e[k] * rr.e[k] : rr.e[k];
      v[0] = fma(rr.e[k], zz.e[k], v[0]);
      v[1] = fma(rr.e[k], rr.e[k], v[1]);
    }
    reinterpret_cast<D2*>(x)[c] = xx;
    reinterpret_cast<D2*>(r)[c] = rr;
    reinterpret_cast<D2*>(z)[c] = zz;
  }
#pragma unroll 1
  for (int64_t i = nc * 2 + g0; i < n; i += gs) {
    x[i] = fma(alpha, p[i], x[i]);
    const double ri = fma(-alpha, Ap[i], r[i]);
    const double zi = inv ? inv[i] * ri : ri;
    r[i] = ri;
    z[i] = zi;
    v[0] = fma(ri, zi, v[0]);
    v[1] = fma(ri, ri, v[1]);
  }
  double tot[2];
  if (grid_sums<2>(v, partials, ticket, tot)) {
    cg->beta = tot[0] / cg->rz;
    cg->rz = tot[0];
    cg->rr = tot[1];
    cg->iters += 1;
    const bool finite = isfinite(tot[0]) && isfinite(tot[1]) && isfinite(alpha);
    if (!finite) {
      cg->status = SEM_ERR_NONFINITE;
      cg->done = 1;
    } else if (tot[1] <= cg->tol2) {
      cg->done = 1;
    }
  }
}

// p = z + beta p, Ap = 0; with p2 set, p also as float pairs (split_pair).
__global__ void __launch_bounds__(kVecThreads)
    k_cg_p(int64_t n, const double* __restrict__ z, double* __restrict__ p, df_pair* __restrict__ p2,
           double* __restrict__ Ap, const CgScalars* cg) {
  pdl_entry();
  if (cg->done) return;
  const double beta = cg->beta;
  const int64_t g0 = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const int64_t gs = (int64_t)gridDim.x * blockDim.x;
  const int64_t nc = n / 2;
#pragma unroll 1
  for (int64_t c = g0; c < nc; c += gs) {
    const D2 zz = reinterpret_cast<const D2*>(z)[c];
    D2 pp = reinterpret_cast<const D2*>(p)[c];
#pragma unroll
    for (int k = 0; k < 2; ++k) pp.e[k] = fma(beta, pp.e[k], zz.e[k]);
    reinterpret_cast<D2*>(p)[c] = pp;
    reinterpret_cast<D2*>(Ap)[c] = D2{};
    if (p2 != nullptr) {
      const df_pair a0 = split_pair(pp.e[0]), a1 = split_pair(pp.e[1]);
      reinterpret_cast<float4*>(p2)[c] = make_float4(a0.h, a0.l, a1.h, a1.l);
    }
  }
#pragma unroll 1
  for (int64_t i = nc * 2 + g0; i < n; i += gs) {
    const double pi = fma(beta, p[i], z[i]);
    p[i] = pi;
    Ap[i] = 0.0;
    if (p2 != nullptr) p2[i] = split_pair(pi);
  }
}

// With `same` set (sem_step_host_out), x0 still holds the solution the last call
// left there: a value that differs from the incoming u^n, bit for bit, clears *same.
__device__ __forceinline__ void check_same(int* same, double old, double u) {
  if (same != nullptr && __double_as_longlong(old) != __double_as_longlong(u)) *same = 0;
}

// Ionic parameters folded into the constants of the per-node arithmetic (host side):
//   v = u* inv_amp + v_off            (v_off = -u_rest / u_amp)
//   exponent = x_off - v inv_kappa    (x_off = v_gate / kappa)
//   I_ion = i_in h v^2 (1 - v) + i_out v   (i_in = -u_amp / tau_in, i_out = u_amp / tau_out)
struct IonicArgs {
  double inv_amp, v_off, inv_kappa, x_off, inv_tau_open, inv_tau_close, i_in, i_out;
};

// Per node (Algorithm 1, DOF loop; Eq. ionic_discr):
//   u* = u^n (first step) or 2 u^n - u^{n-1}
//   gate: BDF1 / BDF2 equation, affine in h^{n+1}, solved in closed form
//   I_ion(u*, h^{n+1}); g = history/dt terms - I_ion + I_app
//   out = mdiag * g (SEM-NI: M diagonal) or g (SEM: M g applied afterwards)
//   x0 = u^n (warm start of CG)
// With the switch s = 1 / (1 + E), E = exp(-(v - v_gate) / kappa), the opening
// and closing rates are a = E / ((1 + E) tau_open) and b = 1 / ((1 + E) tau_close);
// multiplying the gate update through by (1 + E) leaves one FP64 division:
//   BDF2: h = (H (1 + E) + 2 dt E / tau_open) / (3 (1 + E) + 2 dt (E / tau_open + 1 / tau_close)),
//         H = 4 h^n - h^{n-1}
//   BDF1: h = (h^n (1 + E) + dt E / tau_open) / ((1 + E) + dt (E / tau_open + 1 / tau_close)).
// The exponent is capped at 80 (v more than 0.8 below v_gate): s < 2e-35 there,
// below the rounding of h.  The FP64 pipe bounds this kernel, so the constant
// parts of the terms are folded on the host (IonicArgs) and the history term
// enters g by one multiply-add.
__global__ void __launch_bounds__(kVecThreads)
    k_ionic_rhs(int64_t n, const double* __restrict__ un, const double* __restrict__ unm1,
                const double* __restrict__ hn, const double* __restrict__ hnm1,
                double* __restrict__ hnext, double* __restrict__ x0, double* __restrict__ out,
                const double* __restrict__ mdiag, const double* __restrict__ mask, double iapp,
                const IonicArgs prm, double dt, int first, int* same) {
  pdl_entry();
  const double inv_dt = 1.0 / dt, inv_2dt = 0.5 / dt;
  const double c_open = (first ? dt : 2.0 * dt) * prm.inv_tau_open;
  const double c_close = (first ? dt : 2.0 * dt) * prm.inv_tau_close;
  const double c_den = first ? 1.0 : 3.0;
#pragma unroll 1
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const double u0 = un[i];
    const double u1 = first ? u0 : unm1[i];
    const double us = first ? u0 : 2.0 * u0 - u1;
    const double v = fma(us, prm.inv_amp, prm.v_off);
    const double E = exp(fmin(fma(v, -prm.inv_kappa, prm.x_off), 80.0));
    const double ope = 1.0 + E;
    const double H = first ? hn[i] : fma(4.0, hn[i], -hnm1[i]);
    const double h = fma(H, ope, c_open * E) / fma(c_den, ope, fma(c_open, E, c_close));
    const double v2 = v * v;
    const double iion = fma(prm.i_in * h, fma(-v, v2, v2), prm.i_out * v);
    double g = first ? fma(u0, inv_dt, -iion) : fma(fma(4.0, u0, -u1), inv_2dt, -iion);
    if (mask != nullptr) g += iapp * mask[i];
    hnext[i] = h;
    if (same != nullptr) check_same(same, x0[i], u0);
    x0[i] = u0;
    out[i] = mdiag ? mdiag[i] * g : g;
  }
}

// The same per-node update in double-float arithmetic on the FP32 pipe (the
// operator precision SEM_PREC_DF64): inputs split into float pairs and results
// joined by integer operations, exp and the division from sem_dfmath.cuh.
// Agrees with the FP64 kernel to about 1e-14 relative.
struct IonicDfArgs {
  df inv_amp, v_off, neg_inv_kappa, x_off, i_in, i_out;
  df c_open, c_close, c_den, inv_dt, inv_2dt, iapp;
  DfExpConst ex;
};

// One node: h^{n+1} and the right-hand side from u^n, u^{n-1}, h^n, h^{n-1}
// (the mass diagonal md and the stimulus mask value mk, 0 or 1, when present).
__device__ __forceinline__ void ionic_df_node(double u0d, double u1d, double h0d, double h1d, double md,
                                              bool use_md, bool stim, const IonicDfArgs& P, int first,
                                              double& h_out, double& rhs_out) {
  const df u0 = dfd(u0d);
  const df u1 = first ? u0 : dfd(u1d);
  const df us = first ? u0 : (u0 + u0) - u1;
  const df v = dfnorm(fma(us, P.inv_amp, P.v_off));
  df xe = fma(v, P.neg_inv_kappa, P.x_off);
  if (xe.h > 80.f) xe = df(80.f, 0.f);
  const df E = dfexp(xe, P.ex);
  const df ope = df(1.f, 0.f) + E;
  const df H = first ? dfd(h0d) : fma(df(4.f, 0.f), dfd(h0d), dfneg(dfd(h1d)));
  const df num = fma(H, ope, P.c_open * E);
  const df den = fma(P.c_den, ope, fma(P.c_open, E, P.c_close));
  const df h = dfdiv(num, den);
  const df v2 = v * v;
  const df iion = fma(P.i_in * h, v2 - v * v2, P.i_out * v);
  df g = first ? fma(u0, P.inv_dt, dfneg(iion)) : fma((u0 + u0 + u0 + u0) - u1, P.inv_2dt, dfneg(iion));
  if (stim) g = g + P.iapp;
  h_out = df_to_double(h);
  rhs_out = df_to_double(use_md ? dfnorm(dfd(md) * g) : dfnorm(g));
}

__global__ void __launch_bounds__(kVecThreads)
    k_ionic_rhs_df(int64_t n, const double* __restrict__ un, const double* __restrict__ unm1,
                   const double* __restrict__ hn, const double* __restrict__ hnm1,
                   double* __restrict__ hnext, double* __restrict__ x0, double* __restrict__ out,
                   const double* __restrict__ mdiag, const double* __restrict__ mask,
                   const IonicDfArgs P, int first, int* same) {
  pdl_entry();
#pragma unroll 1
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const double u0d = un[i];
    if (same != nullptr) check_same(same, x0[i], u0d);
    // the stimulus mask holds 0 or 1
    const bool stim = mask != nullptr && __double2hiint(mask[i]) != 0;
    ionic_df_node(u0d, first ? 0.0 : unm1[i], hn[i], first ? 0.0 : hnm1[i], mdiag ? mdiag[i] : 0.0,
                  mdiag != nullptr, stim, P, first, hnext[i], out[i]);
    x0[i] = u0d;
  }
}

// The same on two consecutive nodes per thread with 16-byte loads and stores
// (all arrays 16-byte aligned): twice the bytes in flight per load, which
// matters when the inputs are page-locked host memory read over the host link.
// The last node of an odd n is done by thread 0 of block 0.
__global__ void __launch_bounds__(kVecThreads)
    k_ionic_rhs_df2(int64_t n, const double2* __restrict__ un, const double2* __restrict__ unm1,
                    const double2* __restrict__ hn, const double2* __restrict__ hnm1,
                    double2* __restrict__ hnext, double2* __restrict__ x0, double2* __restrict__ out,
                    const double2* __restrict__ mdiag, const double2* __restrict__ mask,
                    const IonicDfArgs P, int first, int* same) {
  pdl_entry();
  if ((n & 1) && blockIdx.x == 0 && threadIdx.x == 0) {
    const int64_t t = n - 1;
    auto r = [](const double2* q, int64_t i) { return reinterpret_cast<const double*>(q)[i]; };
    const double u0 = r(un, t);
    if (same != nullptr) check_same(same, reinterpret_cast<const double*>(x0)[t], u0);
    ionic_df_node(u0, first ? 0.0 : r(unm1, t), r(hn, t), first ? 0.0 : r(hnm1, t),
                  mdiag ? r(mdiag, t) : 0.0, mdiag != nullptr, mask != nullptr && __double2hiint(r(mask, t)) != 0,
                  P, first, reinterpret_cast<double*>(hnext)[t], reinterpret_cast<double*>(out)[t]);
    reinterpret_cast<double*>(x0)[t] = u0;
  }
  const int64_t n2 = n / 2;
#pragma unroll 1
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n2;
       i += (int64_t)gridDim.x * blockDim.x) {
    const double2 u0 = un[i];
    const double2 u1 = first ? make_double2(0.0, 0.0) : unm1[i];
    const double2 h0 = hn[i];
    const double2 h1 = first ? make_double2(0.0, 0.0) : hnm1[i];
    const double2 md = mdiag ? mdiag[i] : make_double2(0.0, 0.0);
    const double2 mk = mask ? mask[i] : make_double2(0.0, 0.0);
    double2 hh, rr;
    ionic_df_node(u0.x, u1.x, h0.x, h1.x, md.x, mdiag != nullptr, __double2hiint(mk.x) != 0, P, first, hh.x,
                  rr.x);
    ionic_df_node(u0.y, u1.y, h0.y, h1.y, md.y, mdiag != nullptr, __double2hiint(mk.y) != 0, P, first, hh.y,
                  rr.y);
    hnext[i] = hh;
    out[i] = rr;
    if (same != nullptr) {
      const double2 old = x0[i];
      check_same(same, old.x, u0.x);
      check_same(same, old.y, u0.y);
    }
    x0[i] = u0;
  }
}

// c = a - b
__global__ void __launch_bounds__(kVecThreads)
    k_sub(int64_t n, const double* __restrict__ a, const double* __restrict__ b, double* __restrict__ c) {
  pdl_entry();
#pragma unroll 1
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    c[i] = a[i] - b[i];
}

// c = a - b in double-float, b and c float pairs
__global__ void __launch_bounds__(kVecThreads)
    k_sub_pairs(int64_t n, const double* __restrict__ a, const df_pair* __restrict__ b, df_pair* __restrict__ c) {
  pdl_entry();
#pragma unroll 1
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const df_pair v = b[i];
    const df d = dfnorm(dfd(a[i]) - df(v.h, v.l));
    c[i] = df_pair{d.h, d.l};
  }
}

__global__ void k_fill_pair(int64_t n, double* a, double va, double* b, double vb) {
  pdl_entry();
#pragma unroll 1
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    a[i] = va;
    b[i] = vb;
  }
}

// Activation time (Eq. tau): du/dt at t1 by the time scheme (BDF1 for the first
// step, BDF2 after), and where |du/dt| exceeds the node's running maximum the
// maximum and t1 are replaced (ties keep the earlier time).
__global__ void __launch_bounds__(kVecThreads)
    k_activation(int64_t n, const double* __restrict__ u1, const double* __restrict__ u0,
                 const double* __restrict__ um1, int first, double dt, double t1,
                 double* __restrict__ dmax, double* __restrict__ tau) {
  pdl_entry();
  const double inv_dt = 1.0 / dt, inv_2dt = 0.5 / dt;
#pragma unroll 1
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const double d = first ? (u1[i] - u0[i]) * inv_dt : (3.0 * u1[i] - 4.0 * u0[i] + um1[i]) * inv_2dt;
    const double ad = fabs(d);
    if (ad > dmax[i]) {
      dmax[i] = ad;
      tau[i] = t1;
    }
  }
}

}  // namespace

cudaError_t activation_reset(sem_state* st, cudaStream_t s) {
  const int64_t n = st->ctx->L.ndofs;
  launch_k(k_fill_pair, vec_grid(n), kVecThreads, 0, s, n, st->act_dmax, -1.0, st->act_tau,
                                                  std::numeric_limits<double>::quiet_NaN());
  return cudaGetLastError();
}

int vec_blocks(int64_t n) { return vec_grid(n); }

int fail(sem_ctx* ctx, int code, const std::string& msg) {
  if (ctx) ctx->err = msg;
  return code;
}

int cuda_fail(sem_ctx* ctx, cudaError_t e, const char* what) {
  return fail(ctx, e == cudaErrorMemoryAllocation ? SEM_ERR_NOMEM : SEM_ERR_CUDA,
              std::string(what) + ": " + cudaGetErrorString(e));
}

#define SEM_CK(call)                                      \
  do {                                                    \
    cudaError_t e_ = (call);                              \
    if (e_ != cudaSuccess) return cuda_fail(ctx, e_, #call); \
  } while (0)

int ensure_workspace(sem_ctx* ctx) {
  Workspace& w = ctx->ws;
  if (w.ready) return SEM_OK;
  const size_t n = (size_t)ctx->L.ndofs;
  double** vecs[] = {&w.r, &w.z, &w.p, &w.Ap, &w.invdiag, &w.b, &w.g, &w.Ax};
  for (double** v : vecs) SEM_CK(cudaMalloc(v, sizeof(double) * n));
  SEM_CK(cudaMalloc(&w.p2, sizeof(df_pair) * n));
  SEM_CK(cudaMalloc(&w.cg, sizeof(CgScalars)));
  SEM_CK(cudaMemset(w.cg, 0, sizeof(CgScalars)));
  SEM_CK(cudaMallocHost(&w.cg_host, sizeof(CgScalars)));
  SEM_CK(cudaMalloc(&w.vec_partials, sizeof(double) * kReduceSlots * kVecBlocksMax));
  SEM_CK(cudaMalloc(&w.tickets, sizeof(unsigned int) * 4));
  SEM_CK(cudaMemset(w.tickets, 0, sizeof(unsigned int) * 4));
  const int ag = std::max(1, apply_grid_blocks(ctx->L));
  SEM_CK(cudaMalloc(&w.apply_partials, sizeof(double) * ag));
  SEM_CK(cudaMalloc(&w.dot_result, sizeof(double)));
  SEM_CK(cudaMalloc(&w.same, sizeof(int)));
  SEM_CK(cudaMallocHost(&w.same_host, sizeof(int)));
  SEM_CK(cudaMallocHost(&w.fault_host, sizeof(unsigned)));
  *w.fault_host = 0u;
  w.inv_alpha = -1.0;
  w.ready = true;
  return SEM_OK;
}

namespace {

ApplyArgs64 base_args(sem_ctx* ctx, double alpha, double beta, const double* u, double* y) {
  ApplyArgs64 a{};
  a.map = ctx->L.map;
  a.metric = ctx->L.metric;
  a.u = u;
  a.y = y;
  a.nelem = ctx->L.nelem;
  a.mass_coef = alpha / beta;
  a.out_scale = beta;
  a.scale_out = beta != 1.0;
  a.yloc = ctx->deterministic ? ctx->det_scratch : nullptr;
  return a;
}

}  // namespace

int apply_fp64(sem_ctx* ctx, double alpha, double beta, const double* u, double* y,
               cudaStream_t s) {
  const Level& L = ctx->L;
  if (beta == 0.0) {
    if (L.quad == SEM_QUAD_LGL) {
      launch_k(k_scale_mul, vec_grid(L.ndofs), kVecThreads, 0, s, L.ndofs, alpha, L.mdiag, u, y);
      ctx->launches += 1;
      SEM_CK(cudaGetLastError());
      return SEM_OK;
    }
    SEM_CK(cudaMemsetAsync(y, 0, sizeof(double) * L.ndofs, s));
    ApplyArgs64 a = base_args(ctx, alpha, 1.0, u, y);
    SEM_CK(launch_apply_fp64(L, a, true, s));
    ctx->launches += 1;
    return SEM_OK;
  }
  SEM_CK(cudaMemsetAsync(y, 0, sizeof(double) * L.ndofs, s));
  ApplyArgs64 a = base_args(ctx, alpha, beta, u, y);
  SEM_CK(launch_apply_fp64(L, a, false, s));
  ctx->launches += 1;
  return SEM_OK;
}

cudaError_t prepare_operator(sem_ctx* ctx, cudaStream_t s) {
  Level& L = ctx->L;
  if (ctx->op_precision != SEM_PREC_DF64 || L.metric2_valid) return cudaSuccess;
  cudaError_t e;
  if (!L.metric2 &&
      (e = cudaMalloc(&L.metric2, sizeof(df_pair) * metric_count(L))) != cudaSuccess)
    return e;
  return setup_metric_df(L, s);
}

cudaError_t launch_operator(sem_ctx* ctx, const ApplyArgs64& a, cudaStream_t s) {
  Level& L = ctx->L;
  if (ctx->op_precision != SEM_PREC_DF64) return launch_apply_fp64(L, a, false, s);
  if (!L.metric2_valid) return cudaErrorNotReady;  // prepare_operator was not called
  // the fused inner product of the double-float operator reads u as float pairs
  if (a.dot_partials != nullptr && a.u2 == nullptr) return cudaErrorInvalidValue;
  ApplyArgs<df, df_pair> d{};
  d.map = a.map; d.metric = L.metric2; d.u = a.u; d.y = a.y; d.nelem = a.nelem;
  d.mass_coef = df(a.mass_coef); d.out_scale = df(a.out_scale); d.scale_out = a.scale_out;
  d.done = a.done; d.dot_partials = a.dot_partials; d.cg = a.cg;
  d.dot_out = a.dot_out;
  d.u2 = a.u2;
  d.yloc = a.yloc;
  return launch_apply_df64(L, d, false, s);
}

int apply_df64(sem_ctx* ctx, double alpha, double beta, const double* u, double* y,
               cudaStream_t s) {
  const Level& L = ctx->L;
  if (beta == 0.0) return apply_fp64(ctx, alpha, beta, u, y, s);  // the mass operator is FP64 either way
  SEM_CK(cudaMemsetAsync(y, 0, sizeof(double) * L.ndofs, s));
  ApplyArgs64 a = base_args(ctx, alpha, beta, u, y);
  const int saved = ctx->op_precision;
  ctx->op_precision = SEM_PREC_DF64;
  cudaError_t e = prepare_operator(ctx, s);
  if (e == cudaSuccess) e = launch_operator(ctx, a, s);
  ctx->op_precision = saved;
  SEM_CK(e);
  ctx->launches += 1;
  return SEM_OK;
}

int apply_fp32(sem_ctx* ctx, double alpha, double beta, const float* u, float* y, bool bf16,
               cudaStream_t s) {
  Level& L = ctx->L;
  if (bf16 && !L.metric16_valid) {
    if (!L.metric16)
      SEM_CK(cudaMalloc(&L.metric16, sizeof(__nv_bfloat16) * metric16_count(L)));
    SEM_CK(setup_metric_lowp(L, true, s));
  }
  if (!bf16 && !L.metric32_valid) {
    if (!L.metric32)
      SEM_CK(cudaMalloc(&L.metric32, sizeof(float) * metric_count(L)));
    SEM_CK(setup_metric_lowp(L, false, s));
  }
  if (beta == 0.0 && L.quad == SEM_QUAD_LGL) {
    launch_k(k_scale_mul32, vec_grid(L.ndofs), kVecThreads, 0, s, L.ndofs, (float)alpha, L.mdiag, u, y);
    SEM_CK(cudaGetLastError());
    return SEM_OK;
  }
  SEM_CK(cudaMemsetAsync(y, 0, sizeof(float) * L.ndofs, s));
  const bool mass_only = beta == 0.0;
  const double bb = mass_only ? 1.0 : beta;
  if (bf16) {
    ApplyArgs<float, __nv_bfloat16> a{};
    a.map = L.map; a.metric = L.metric16; a.u = u; a.y = y; a.nelem = L.nelem;
    a.mass_coef = (float)(alpha / bb); a.out_scale = (float)bb; a.scale_out = bb != 1.0;
    a.yloc = ctx->deterministic ? (float*)ctx->det_scratch : nullptr;
    SEM_CK(launch_apply_bf16(L, a, mass_only, s));
  } else {
    ApplyArgs<float, float> a{};
    a.map = L.map; a.metric = L.metric32; a.u = u; a.y = y; a.nelem = L.nelem;
    a.mass_coef = (float)(alpha / bb); a.out_scale = (float)bb; a.scale_out = bb != 1.0;
    a.yloc = ctx->deterministic ? (float*)ctx->det_scratch : nullptr;
    SEM_CK(launch_apply_fp32(L, a, mass_only, s));
  }
  return SEM_OK;
}

int apply_tc(sem_ctx* ctx, double alpha, double beta, const float* u, float* y, cudaStream_t s) {
  Level& L = ctx->L;
  if (!tc_supported(L))
    return fail(ctx, SEM_ERR_UNSUPPORTED, "the tensor-core apply covers SEM-NI at p = 2..4");
  if (ctx->deterministic)
    return fail(ctx, SEM_ERR_UNSUPPORTED, "the tensor-core apply has no deterministic mode");
  if (beta == 0.0) {  // SEM-NI mass: diagonal
    launch_k(k_scale_mul32, vec_grid(L.ndofs), kVecThreads, 0, s, L.ndofs, (float)alpha, L.mdiag, u, y);
    SEM_CK(cudaGetLastError());
    return SEM_OK;
  }
  if (!L.metric_tc_valid) SEM_CK(setup_metric_tc(L, s));
  SEM_CK(cudaMemsetAsync(y, 0, sizeof(float) * L.ndofs, s));
  ApplyArgs<float, __nv_bfloat16> a{};
  a.u = u; a.y = y; a.nelem = L.nelem;
  a.mass_coef = (float)(alpha / beta); a.out_scale = (float)beta; a.scale_out = beta != 1.0;
  SEM_CK(launch_apply_tc(L, a, s));
  ctx->launches += 1;
  return SEM_OK;
}

int cg_solve(sem_ctx* ctx, double alpha, const double* b, double* x, double rtol, double atol,
             int maxit, int precond, int* iters, double* final_res, sem_stats* stats,
             cudaStream_t s, double* ax0, const int* ax0_ok) {
  int rc = ensure_workspace(ctx);
  if (rc != SEM_OK) return rc;
  SEM_CK(prepare_operator(ctx, s));
  Level& L = ctx->L;
  Workspace& w = ctx->ws;
  const int64_t n = L.ndofs;
  const int vg = vec_grid(n);
  const double* inv = nullptr;
  if (precond == SEM_PC_JACOBI) {
    if (w.inv_alpha != alpha) {
      launch_k(k_inv_diag, vg, kVecThreads, 0, s, n, alpha, L.mdiag, L.kdiag, w.invdiag);
      ctx->launches += 1;
      SEM_CK(cudaGetLastError());
      w.inv_alpha = alpha;
    }
    inv = w.invdiag;
  } else if (precond == SEM_PC_GMG) {
    return gmg_pcg(ctx, alpha, b, x, rtol, atol, maxit, iters, final_res, stats, s, ax0, ax0_ok);
  } else if (precond != SEM_PC_NONE) {
    return fail(ctx, SEM_ERR_ARG, "unknown preconditioner");
  }
  if (ax0_ok != nullptr) ax0 = nullptr;  // no device-side choice here: apply the operator
  // Ap = A x (or the carried ax0), then the initial residual; Ap is zero for the iterations
  SEM_CK(cudaMemsetAsync(w.Ap, 0, sizeof(double) * n, s));
  if (ax0 == nullptr) {
    ApplyArgs64 a = base_args(ctx, alpha, 1.0, x, w.Ap);
    SEM_CK(launch_operator(ctx, a, s));
    ctx->launches += 1;
  }
  ctx->launches += 1;
  // the double-float operator gathers p as the float pairs the p kernels write
  df_pair* p2 = ctx->op_precision == SEM_PREC_DF64 ? w.p2 : nullptr;
  launch_k(k_cg_init, vg, kVecThreads, 0, s, n, b, ax0 ? ax0 : w.Ap, inv, w.r, w.z, w.p, p2, w.cg,
           w.vec_partials, w.tickets + 0, rtol, atol);
  SEM_CK(cudaGetLastError());

  ApplyArgs64 ap = base_args(ctx, alpha, 1.0, w.p, w.Ap);
  ap.done = &w.cg->done;
  ap.dot_partials = w.apply_partials;
  ap.cg = w.cg;
  ap.u2 = p2;

  Timing& tm = ctx->timing;
  constexpr int kChunkMax = 16;
  // with timing on, the apply of the first iteration of one solve in kTimingEvery
  // is bracketed by events (they interrupt the programmatic dependent launch)
  bool sample = tm.enabled && (tm.solves++ % kTimingEvery) == 0;
  if (sample && (tm.start == nullptr || tm.stop == nullptr)) {
    if (tm.start == nullptr) SEM_CK(cudaEventCreate(&tm.start));
    if (tm.stop == nullptr) SEM_CK(cudaEventCreate(&tm.stop));
  }
  int launched = 0;
  int chunk = 4;
  bool done = false;
  int rc_out = SEM_OK;
  while (true) {
    const int this_chunk = std::min(chunk, maxit - launched);
    if (this_chunk > 0) {
      for (int c = 0; c < this_chunk; ++c) {
        const bool timed = sample && launched == 0 && c == 0;
        if (timed) SEM_CK(cudaEventRecord(tm.start, s));
        SEM_CK(launch_operator(ctx, ap, s));
        if (timed) SEM_CK(cudaEventRecord(tm.stop, s));
        if ((reinterpret_cast<uintptr_t>(x) & 15u) == 0)
          launch_k(k_cg_xr<true>, vg, kVecThreads, 0, s, n, x, w.p, w.Ap, w.r, inv, w.z, w.cg, w.vec_partials,
                                                   w.tickets + 0);
        else
          launch_k(k_cg_xr<false>, vg, kVecThreads, 0, s, n, x, w.p, w.Ap, w.r, inv, w.z, w.cg, w.vec_partials,
                                                    w.tickets + 0);
        launch_k(k_cg_p, vg, kVecThreads, 0, s, n, w.z, w.p, p2, w.Ap, w.cg);
      }
      SEM_CK(cudaGetLastError());
      launched += this_chunk;
      ctx->launches += 4 * this_chunk;  // apply, its inner-product sum, x/r update, p update
    }
    SEM_CK(cudaMemcpyAsync(w.cg_host, w.cg, sizeof(CgScalars), cudaMemcpyDeviceToHost, s));
    SEM_CK(cudaStreamSynchronize(s));
    const CgScalars& h = *w.cg_host;
    if (sample && h.iters >= 1) {  // the timed first iteration ran
      sample = false;
      float ms = 0.f;
      SEM_CK(cudaEventElapsedTime(&ms, tm.start, tm.stop));
      tm.ms += ms;
      tm.count += 1;
    }
    if (h.done) { done = true; break; }
    if (launched >= maxit) break;
    chunk = std::min(kChunkMax, chunk * 2);
  }
  const CgScalars& h = *w.cg_host;
  if (iters) *iters = h.iters;
  if (final_res) *final_res = std::sqrt(h.rr);
  if (stats) {
    stats->cg_iters += h.iters;
    stats->last_residual = std::sqrt(h.rr);
  }
  if (h.status == SEM_ERR_NONFINITE)
    rc_out = fail(ctx, SEM_ERR_NONFINITE, "non-finite value in a CG inner product");
  else if (!done)
    rc_out = fail(ctx, SEM_ERR_NOT_CONVERGED,
                  "CG did not converge in " + std::to_string(maxit) + " iterations (|r| = " +
                      std::to_string(std::sqrt(h.rr)) + ")");
  return rc_out;
}

// Constants of dfexp: ln2 split for Cody and Waite's reduction (c1, c2 with 16
// significant bits, so k c1 and k c2 are exact floats for |k| < 128; c3 the
// rest), and the Taylor coefficients 1 / j! as float pairs.
DfExpConst dfexp_constants() {
  DfExpConst K{};
  const long double ln2 = 0.6931471805599453094172321214581765680755L;
  const long double c1 = std::ldexp(std::floor(std::ldexp(ln2, 16)), -16);
  const long double rem = ln2 - c1;
  const int e = std::ilogb(rem);
  const long double c2 = std::ldexp(std::floor(std::ldexp(rem, 15 - e)), e - 15);
  K.inv_ln2 = (float)(1.0L / ln2);
  K.c1 = (float)c1;
  K.c2 = (float)c2;
  K.c3 = (float)(rem - c2);
  long double f = 1.0L;
  for (int j = 0; j < 14; ++j) {
    if (j > 0) f /= (long double)j;
    K.th[j] = (float)f;
    K.tl[j] = (float)(f - (long double)K.th[j]);
  }
  return K;
}

int time_steps(sem_ctx* ctx, sem_state* st, double dt, int nsteps, double rtol, double atol,
               int maxit, int precond, sem_stats* stats, cudaStream_t s) {
  int rc = ensure_workspace(ctx);
  if (rc != SEM_OK) return rc;
  Level& L = ctx->L;
  Workspace& w = ctx->ws;
  const int64_t n = L.ndofs;
  const int vg = vec_grid(n);
  const sem_ionic_params& ip = ctx->ionic;
  IonicArgs ia;
  ia.inv_amp = 1.0 / ip.u_amp;
  ia.v_off = -ip.u_rest / ip.u_amp;
  ia.inv_kappa = 1.0 / ip.kappa;
  ia.x_off = ip.v_gate / ip.kappa;
  ia.inv_tau_open = 1.0 / ip.tau_open;
  ia.inv_tau_close = 1.0 / ip.tau_close;
  ia.i_in = -ip.u_amp / ip.tau_in;
  ia.i_out = ip.u_amp / ip.tau_out;
  // double-float update with the double-float operator
  const bool ionic_df = ctx->op_precision == SEM_PREC_DF64;
  IonicDfArgs idf{};
  if (ionic_df) {
    idf.inv_amp = df(ia.inv_amp);
    idf.v_off = df(ia.v_off);
    idf.neg_inv_kappa = df(-ia.inv_kappa);
    idf.x_off = df(ia.x_off);
    idf.i_in = df(ia.i_in);
    idf.i_out = df(ia.i_out);
    idf.ex = dfexp_constants();
  }
  for (int k = 0; k < nsteps; ++k) {
    const int first = st->n == 0 ? 1 : 0;
    const double alpha = first ? 1.0 / dt : 1.5 / dt;
    sem_ctx::ResidualCarry& cy = ctx->carry;
    const bool carried = cy.valid && cy.st == st && cy.n == st->n && cy.alpha == alpha &&
                         cy.precond == precond && cy.age < kCarrySteps;
    // a carry that depends on the caller's u^n: checked by the ionic update
    int* same = carried ? cy.same : nullptr;
    if (same != nullptr) SEM_CK(cudaMemsetAsync(same, 0x01, sizeof(int), s));
    const double t1 = (double)(st->n + 1) * dt;
    const bool on = ctx->stim_mask != nullptr && t1 > ctx->stim_on && t1 <= ctx->stim_off;
    double* out = L.quad == SEM_QUAD_LGL ? w.b : w.g;
    if (ionic_df) {
      idf.c_open = df((first ? dt : 2.0 * dt) * ia.inv_tau_open);
      idf.c_close = df((first ? dt : 2.0 * dt) * ia.inv_tau_close);
      idf.c_den = df(first ? 1.0 : 3.0);
      idf.inv_dt = df(1.0 / dt);
      idf.inv_2dt = df(0.5 / dt);
      idf.iapp = df(on ? ctx->stim_amp : 0.0);
      const double* ptrs[9] = {st->U[st->cur], st->U[st->prev], st->H[st->cur], st->H[st->prev],
                               st->H[st->next], st->U[st->next], out, L.mdiag, ctx->stim_mask};
      bool a16 = true;
      for (const double* q : ptrs) a16 = a16 && (q == nullptr || (reinterpret_cast<uintptr_t>(q) & 15u) == 0);
      const double* md = L.quad == SEM_QUAD_LGL ? L.mdiag : nullptr;
      const double* mk = on ? ctx->stim_mask : nullptr;
      if (a16) {
        auto d2 = [](const double* q) { return reinterpret_cast<const double2*>(q); };
        auto w2 = [](double* q) { return reinterpret_cast<double2*>(q); };
        launch_k(k_ionic_rhs_df2, vec_grid(n / 2 + 1), kVecThreads, 0, s, n, d2(st->U[st->cur]),
                 d2(st->U[st->prev]), d2(st->H[st->cur]), d2(st->H[st->prev]), w2(st->H[st->next]),
                 w2(st->U[st->next]), w2(out), d2(md), d2(mk), idf, first, same);
      } else {
        launch_k(k_ionic_rhs_df, vg, kVecThreads, 0, s, n, st->U[st->cur], st->U[st->prev], st->H[st->cur],
                 st->H[st->prev], st->H[st->next], st->U[st->next], out, md, mk, idf, first, same);
      }
    } else {
      launch_k(k_ionic_rhs, vg, kVecThreads, 0, s,
          n, st->U[st->cur], st->U[st->prev], st->H[st->cur], st->H[st->prev], st->H[st->next],
          st->U[st->next], out, L.quad == SEM_QUAD_LGL ? L.mdiag : nullptr,
          on ? ctx->stim_mask : nullptr, on ? ctx->stim_amp : 0.0, ia, dt, first, same);
    }
    SEM_CK(cudaGetLastError());
    ctx->launches += 1;
    auto& hc = ctx->host_copies;
    if (hc.h_dst != nullptr && k == 0) {  // h^{n+1} to the host while the solve runs
      SEM_CK(cudaEventRecord(hc.ev_ionic, s));
      SEM_CK(cudaStreamWaitEvent(hc.side, hc.ev_ionic, 0));
      SEM_CK(cudaMemcpyAsync(hc.h_dst, st->H[st->next], sizeof(double) * n, cudaMemcpyDeviceToHost,
                             hc.side));
      SEM_CK(cudaEventRecord(hc.ev_h, hc.side));
    }
    if (L.quad == SEM_QUAD_LG) {
      rc = apply_fp64(ctx, 1.0, 0.0, w.g, w.b, s);
      if (rc != SEM_OK) return rc;
    }
    cy.valid = false;
    rc = cg_solve(ctx, alpha, w.b, st->U[st->next], rtol, atol, maxit, precond, nullptr, nullptr,
                  stats, s, carried ? w.Ax : nullptr, same);
    if (rc != SEM_OK) return rc;
    if (stats && carried && same == nullptr) stats->carried_solves += 1;  // checked ones: by the caller
    // A u^{n+1} = b - r for the next step's initial residual (the multigrid PCG with
    // the double-float operator keeps r as float pairs)
    if (precond == SEM_PC_GMG && ctx->op_precision == SEM_PREC_DF64)  // kept as float pairs too
      launch_k(k_sub_pairs, vg, kVecThreads, 0, s, n, w.b, reinterpret_cast<const df_pair*>(w.r),
               reinterpret_cast<df_pair*>(w.Ax));
    else
      launch_k(k_sub, vg, kVecThreads, 0, s, n, w.b, w.r, w.Ax);
    SEM_CK(cudaGetLastError());
    ctx->launches += 1;
    const int old_prev = st->prev;
    st->prev = st->cur;
    st->cur = st->next;
    st->next = old_prev;
    st->n += 1;
    cy.valid = true;
    cy.st = st;
    cy.n = st->n;
    cy.alpha = alpha;
    cy.precond = precond;
    cy.age = carried ? cy.age + 1 : 0;
    if (st->act_track) {  // u^{n+1}, u^n, u^{n-1} sit in U[cur], U[prev], U[next] now
      launch_k(k_activation, vg, kVecThreads, 0, s, n, st->U[st->cur], st->U[st->prev], st->U[st->next],
                                              first, dt, (double)st->n * dt, st->act_dmax, st->act_tau);
      SEM_CK(cudaGetLastError());
      ctx->launches += 1;
    }
    if (stats) stats->steps += 1;
  }
  return SEM_OK;
}

}  // namespace sem
