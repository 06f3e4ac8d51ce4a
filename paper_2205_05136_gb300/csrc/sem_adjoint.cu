// Discrete adjoint of the partitioned time stepping and the gradient with
// respect to the per-element conductivities and fibre angle.
//
// Forward (sem_forward_record): the time steps of sem_step, plus the traces
// T[n][s] = u^{n+1}[sensor_s] and a checkpoint of the full BDF2 state
// (u^n, u^{n-1}, h^n, h^{n-1}) every `every` steps.
//
// Reverse (sem_adjoint_grad), for a loss with dL/dT given: segments are
// processed last to first; each is recomputed forward from its checkpoint
// (states kept in memory), then reversed step by step (A_n = alpha_n M + K):
//   ubar^{n+1} += sensor sources dL/dT[n]
//   w = A_n^{-1} ubar^{n+1}                      (A symmetric: same CG solver)
//   grad_e -= w_e^T K_e[dD/dparam] u_e^{n+1}     (sigma_l, sigma_t, theta)
//   gbar = M w;  history, ionic-current and gate terms of the step reversed
//   per node into ubar^n, ubar^{n-1}, hbar^n, hbar^{n-1}.
// dD/dsigma_l = f f^T, dD/dsigma_t = I - f f^T,
// dD/dtheta = (sigma_l - sigma_t)(f' f^T + f f'^T), f = (cos, sin, 0), f' = (-sin, cos, 0).
#include <algorithm>
#include <cmath>
#include <string>
#include <vector>

#include "sem_apply_kernel.cuh"
#include "sem_context.cuh"

namespace sem {

struct Tape {
  int64_t ndofs = 0;
  int nsteps = 0, every = 0, nsens = 0;
  double dt = 0.0;
  int* sensors = nullptr;              // device copy of the sensor indices
  std::vector<double*> ck;             // checkpoints: [u, u_prev, h, h_prev] x ndofs
  std::vector<int64_t> ck_n;           // step count of each checkpoint
  int64_t n0 = 0;                      // step count when recording started
  double *seg_u = nullptr, *seg_h = nullptr;  // (every + 2) x ndofs each
  double *ub = nullptr, *hb = nullptr;        // 3 rolling adjoint accumulators each
  double *w = nullptr, *gbar = nullptr;
  sem_state* st = nullptr;             // private state for the recomputation
  bool recorded = false;
};

namespace {

constexpr int kThreads = 256;

int grid1d(int64_t n) {
  const int64_t g = (n + kThreads - 1) / kThreads;
  return (int)std::max<int64_t>(1, std::min<int64_t>(g, 152 * 8));
}

#define GRID_LOOP(i, n)                                                          \
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < (n); \
       i += (int64_t)gridDim.x * blockDim.x)

#define ADJ_CK(call)                                          \
  do {                                                        \
    cudaError_t e_ = (call);                                  \
    if (e_ != cudaSuccess) return cuda_fail(ctx, e_, #call);  \
  } while (0)

__global__ void k_gather(int nsens, const int* __restrict__ sensors, const double* __restrict__ u,
                         double* __restrict__ out) {
  for (int s = blockIdx.x * blockDim.x + threadIdx.x; s < nsens; s += gridDim.x * blockDim.x)
    out[s] = u[sensors[s]];
}

__global__ void k_sources(int nsens, const int* __restrict__ sensors, const double* __restrict__ tb,
                          double* __restrict__ ubar) {
  for (int s = blockIdx.x * blockDim.x + threadIdx.x; s < nsens; s += gridDim.x * blockDim.x)
    atomicAdd(ubar + sensors[s], tb[s]);
}

__global__ void k_scale_mul(int64_t n, const double* __restrict__ d, const double* __restrict__ x,
                            double* __restrict__ y) {
  GRID_LOOP(i, n) y[i] = d[i] * x[i];
}

struct IonicAdj {
  double u_rest, u_amp, tau_in, tau_out, tau_open, tau_close, v_gate, kappa;
};

// Reverse of the rhs assembly, ionic current and gate update of one step (per node).
__global__ void k_adj_pointwise(int64_t n, const double* __restrict__ gbar,
                                const double* __restrict__ un, const double* __restrict__ unm1,
                                const double* __restrict__ hnp1, double* __restrict__ ub_n,
                                double* __restrict__ ub_nm1, const double* __restrict__ hb_np1,
                                double* __restrict__ hb_n, double* __restrict__ hb_nm1,
                                const IonicAdj prm, double dt, int first) {
  GRID_LOOP(i, n) {
    const double gb = gbar[i];
    double us;
    if (first) {
      ub_n[i] += gb / dt;
      us = un[i];
    } else {
      ub_n[i] += (2.0 / dt) * gb;
      ub_nm1[i] -= gb / (2.0 * dt);
      us = 2.0 * un[i] - unm1[i];
    }
    const double Ibar = -gb;
    const double h1 = hnp1[i];
    const double v = (us - prm.u_rest) / prm.u_amp;
    const double dI_du = -(h1 * (2.0 * v - 3.0 * v * v) / prm.tau_in - 1.0 / prm.tau_out);
    const double dI_dh = -prm.u_amp * v * v * (1.0 - v) / prm.tau_in;
    double ustar_bar = Ibar * dI_du;
    const double hb = hb_np1[i] + Ibar * dI_dh;
    const double s = 1.0 / (1.0 + exp(-(v - prm.v_gate) / prm.kappa));
    const double ds = s * (1.0 - s) / prm.kappa / prm.u_amp;
    const double a = (1.0 - s) / prm.tau_open, b = s / prm.tau_close;
    const double da = -ds / prm.tau_open, db = ds / prm.tau_close;
    if (first) {
      const double D1 = 1.0 + dt * (a + b);
      ustar_bar += hb * dt * (da - h1 * (da + db)) / D1;
      hb_n[i] += hb / D1;
      ub_n[i] += ustar_bar;
    } else {
      const double D2 = 3.0 + 2.0 * dt * (a + b);
      ustar_bar += hb * 2.0 * dt * (da - h1 * (da + db)) / D2;
      hb_n[i] += 4.0 * hb / D2;
      hb_nm1[i] -= hb / D2;
      ub_n[i] += 2.0 * ustar_bar;
      ub_nm1[i] -= ustar_bar;
    }
  }
}

struct GradTab {
  int n, lg;
  double xq[kMaxN], wq[kMaxN];
  double Bi[kMaxN][kMaxN];  // GLL basis at the quadrature points
  double Dc[kMaxN][kMaxN];  // collocation derivative on the quadrature points
};

// One CTA per element: g_k[e] -= sum_q W_q grad w . dD_k grad u at the quadrature points.
__global__ void k_param_grad(int nelem, const int* __restrict__ map, const double* __restrict__ evert,
                             const double* __restrict__ sigma_l, const double* __restrict__ sigma_t,
                             const double* __restrict__ theta, const __grid_constant__ GradTab tab,
                             const double* __restrict__ w, const double* __restrict__ u,
                             double* __restrict__ g_sl, double* __restrict__ g_st,
                             double* __restrict__ g_th) {
  const int e = blockIdx.x;
  if (e >= nelem) return;
  const int n = tab.n, n2 = n * n, n3 = n2 * n;
  __shared__ double V[8][3];
  __shared__ double F[2][kMaxN * kMaxN * kMaxN];
  __shared__ double G[2][kMaxN * kMaxN * kMaxN];
  __shared__ double red[3][32];
  if (threadIdx.x < 24) V[threadIdx.x / 3][threadIdx.x % 3] = evert[(size_t)e * 24 + threadIdx.x];
  for (int a = threadIdx.x; a < n3; a += blockDim.x) {
    const int gidx = map[(size_t)e * n3 + a];
    F[0][a] = w[gidx];
    F[1][a] = u[gidx];
  }
  __syncthreads();
  if (tab.lg) {  // values at the Gauss points: F -> G (x), G -> F (y), F -> G (z), G -> F copy
    for (int a = threadIdx.x; a < 2 * n3; a += blockDim.x) {
      const int c = a / n3, r = a % n3, q = r % n, j = (r / n) % n, k = r / n2;
      double s = 0.0;
      for (int l = 0; l < n; ++l) s += tab.Bi[q][l] * F[c][k * n2 + j * n + l];
      G[c][r] = s;
    }
    __syncthreads();
    for (int a = threadIdx.x; a < 2 * n3; a += blockDim.x) {
      const int c = a / n3, r = a % n3, i = r % n, q = (r / n) % n, k = r / n2;
      double s = 0.0;
      for (int l = 0; l < n; ++l) s += tab.Bi[q][l] * G[c][k * n2 + l * n + i];
      F[c][r] = s;
    }
    __syncthreads();
    for (int a = threadIdx.x; a < 2 * n3; a += blockDim.x) {
      const int c = a / n3, r = a % n3, i = r % n, j = (r / n) % n, q = r / n2;
      double s = 0.0;
      for (int l = 0; l < n; ++l) s += tab.Bi[q][l] * F[c][l * n2 + j * n + i];
      G[c][r] = s;
    }
    __syncthreads();
    for (int a = threadIdx.x; a < 2 * n3; a += blockDim.x) F[a / n3][a % n3] = G[a / n3][a % n3];
    __syncthreads();
  }
  const double sl = sigma_l[e], st = sigma_t[e], th = theta[e];
  const double f[3] = {cos(th), sin(th), 0.0};
  const double fp[3] = {-sin(th), cos(th), 0.0};
  double acc[3] = {0.0, 0.0, 0.0};
  for (int a = threadIdx.x; a < n3; a += blockDim.x) {
    const int qx = a % n, qy = (a / n) % n, qz = a / n2;
    const double xi[3] = {tab.xq[qx], tab.xq[qy], tab.xq[qz]};
    // Jacobian of the trilinear map at xi
    double J[3][3] = {{0, 0, 0}, {0, 0, 0}, {0, 0, 0}};
    for (int v = 0; v < 8; ++v) {
      const double sg[3] = {(v & 1) ? 1.0 : -1.0, (v & 2) ? 1.0 : -1.0, (v & 4) ? 1.0 : -1.0};
      const double fa[3] = {0.5 * (1.0 + sg[0] * xi[0]), 0.5 * (1.0 + sg[1] * xi[1]), 0.5 * (1.0 + sg[2] * xi[2])};
      const double dN[3] = {0.5 * sg[0] * fa[1] * fa[2], fa[0] * 0.5 * sg[1] * fa[2], fa[0] * fa[1] * 0.5 * sg[2]};
      for (int d = 0; d < 3; ++d)
        for (int c = 0; c < 3; ++c) J[d][c] += V[v][d] * dN[c];
    }
    const double det = J[0][0] * (J[1][1] * J[2][2] - J[1][2] * J[2][1]) -
                       J[0][1] * (J[1][0] * J[2][2] - J[1][2] * J[2][0]) +
                       J[0][2] * (J[1][0] * J[2][1] - J[1][1] * J[2][0]);
    double inv[3][3];
    inv[0][0] = (J[1][1] * J[2][2] - J[1][2] * J[2][1]) / det;
    inv[0][1] = (J[0][2] * J[2][1] - J[0][1] * J[2][2]) / det;
    inv[0][2] = (J[0][1] * J[1][2] - J[0][2] * J[1][1]) / det;
    inv[1][0] = (J[1][2] * J[2][0] - J[1][0] * J[2][2]) / det;
    inv[1][1] = (J[0][0] * J[2][2] - J[0][2] * J[2][0]) / det;
    inv[1][2] = (J[0][2] * J[1][0] - J[0][0] * J[1][2]) / det;
    inv[2][0] = (J[1][0] * J[2][1] - J[1][1] * J[2][0]) / det;
    inv[2][1] = (J[0][1] * J[2][0] - J[0][0] * J[2][1]) / det;
    inv[2][2] = (J[0][0] * J[1][1] - J[0][1] * J[1][0]) / det;
    const double W = tab.wq[qx] * tab.wq[qy] * tab.wq[qz] * det;
    double gw[3], gu[3];
    for (int c = 0; c < 2; ++c) {
      double ref[3] = {0.0, 0.0, 0.0};
      for (int l = 0; l < n; ++l) {
        ref[0] += tab.Dc[qx][l] * F[c][qz * n2 + qy * n + l];
        ref[1] += tab.Dc[qy][l] * F[c][qz * n2 + l * n + qx];
        ref[2] += tab.Dc[qz][l] * F[c][l * n2 + qy * n + qx];
      }
      double* out = c == 0 ? gw : gu;
      for (int d = 0; d < 3; ++d) out[d] = inv[0][d] * ref[0] + inv[1][d] * ref[1] + inv[2][d] * ref[2];
    }
    const double wf = gw[0] * f[0] + gw[1] * f[1];
    const double uf = gu[0] * f[0] + gu[1] * f[1];
    const double wfp = gw[0] * fp[0] + gw[1] * fp[1];
    const double ufp = gu[0] * fp[0] + gu[1] * fp[1];
    const double wu = gw[0] * gu[0] + gw[1] * gu[1] + gw[2] * gu[2];
    acc[0] += W * wf * uf;
    acc[1] += W * (wu - wf * uf);
    acc[2] += W * (sl - st) * (wfp * uf + wf * ufp);
  }
  for (int k = 0; k < 3; ++k) {
    const double s = block_sum(acc[k], red[k]);
    __syncthreads();
    if (threadIdx.x == 0) {
      if (k == 0) g_sl[e] -= s;
      if (k == 1) g_st[e] -= s;
      if (k == 2) g_th[e] -= s;
    }
  }
}

GradTab make_grad_tab(const Tables1D& t) {
  GradTab g{};
  g.n = t.n;
  g.lg = t.quad == SEM_QUAD_LG;
  for (int i = 0; i < t.n; ++i) { g.xq[i] = t.xq[i]; g.wq[i] = t.wq[i]; }
  for (int q = 0; q < t.n; ++q)
    for (int l = 0; l < t.n; ++l) {
      g.Bi[q][l] = t.Bi[q][l];
      g.Dc[q][l] = t.Dg[q][l];
    }
  return g;
}

void free_tape(Tape* t) {
  if (!t) return;
  cudaFree(t->sensors);
  for (double* p : t->ck) cudaFree(p);
  cudaFree(t->seg_u); cudaFree(t->seg_h);
  cudaFree(t->ub); cudaFree(t->hb);
  cudaFree(t->w); cudaFree(t->gbar);
  if (t->st) sem_state_destroy(t->st);
  delete t;
}

int save_checkpoint(sem_ctx* ctx, Tape& tp, sem_state* st, cudaStream_t s) {
  const size_t bytes = sizeof(double) * tp.ndofs;
  double* buf = nullptr;
  ADJ_CK(cudaMalloc(&buf, 4 * bytes));
  tp.ck.push_back(buf);
  tp.ck_n.push_back(st->n);
  ADJ_CK(cudaMemcpyAsync(buf, st->U[st->cur], bytes, cudaMemcpyDeviceToDevice, s));
  ADJ_CK(cudaMemcpyAsync(buf + tp.ndofs, st->U[st->prev], bytes, cudaMemcpyDeviceToDevice, s));
  ADJ_CK(cudaMemcpyAsync(buf + 2 * tp.ndofs, st->H[st->cur], bytes, cudaMemcpyDeviceToDevice, s));
  ADJ_CK(cudaMemcpyAsync(buf + 3 * tp.ndofs, st->H[st->prev], bytes, cudaMemcpyDeviceToDevice, s));
  return SEM_OK;
}

}  // namespace

void tape_free(sem_ctx* ctx) {
  free_tape(ctx->tape);
  ctx->tape = nullptr;
}

int forward_record(sem_ctx* ctx, sem_state* st, double dt, int nsteps, int every,
                   const int* sensors, int nsens, double* traces, double rtol, double atol,
                   int maxit, int precond, sem_stats* stats, cudaStream_t s) {
  tape_free(ctx);
  Tape* tp = new Tape();
  ctx->tape = tp;
  tp->ndofs = ctx->L.ndofs;
  tp->nsteps = nsteps;
  tp->every = every;
  tp->nsens = nsens;
  tp->dt = dt;
  tp->n0 = st->n;
  ADJ_CK(cudaMalloc(&tp->sensors, sizeof(int) * std::max(1, nsens)));
  ADJ_CK(cudaMemcpyAsync(tp->sensors, sensors, sizeof(int) * nsens, cudaMemcpyDeviceToDevice, s));
  for (int k = 0; k < nsteps; ++k) {
    if (k % every == 0) {
      int rc = save_checkpoint(ctx, *tp, st, s);
      if (rc != SEM_OK) return rc;
    }
    int rc = time_steps(ctx, st, dt, 1, rtol, atol, maxit, precond, stats, s);
    if (rc != SEM_OK) return rc;
    k_gather<<<1, 128, 0, s>>>(nsens, tp->sensors, st->U[st->cur], traces + (size_t)k * nsens);
    ADJ_CK(cudaGetLastError());
    ctx->launches += 1;
  }
  tp->recorded = true;
  return SEM_OK;
}

int adjoint_grad(sem_ctx* ctx, const double* trace_bar, double* g_sl, double* g_st, double* g_th,
                 double rtol, double atol, int maxit, int precond, sem_stats* stats,
                 cudaStream_t s) {
  Tape* tp = ctx->tape;
  if (tp == nullptr || !tp->recorded)
    return fail(ctx, SEM_ERR_ARG, "no recorded forward run: call sem_forward_record first");
  Level& L = ctx->L;
  const int64_t n = L.ndofs;
  const size_t bytes = sizeof(double) * n;
  const int gr = grid1d(n);
  if (!tp->seg_u) {
    ADJ_CK(cudaMalloc(&tp->seg_u, bytes * (tp->every + 2)));
    ADJ_CK(cudaMalloc(&tp->seg_h, bytes * (tp->every + 2)));
    ADJ_CK(cudaMalloc(&tp->ub, bytes * 3));
    ADJ_CK(cudaMalloc(&tp->hb, bytes * 3));
    ADJ_CK(cudaMalloc(&tp->w, bytes));
    ADJ_CK(cudaMalloc(&tp->gbar, bytes));
    int rc = sem_state_create(ctx, &tp->st);
    if (rc != SEM_OK) return rc;
  }
  ADJ_CK(cudaMemsetAsync(tp->ub, 0, bytes * 3, s));
  ADJ_CK(cudaMemsetAsync(tp->hb, 0, bytes * 3, s));
  ADJ_CK(cudaMemsetAsync(g_sl, 0, sizeof(double) * L.nelem, s));
  ADJ_CK(cudaMemsetAsync(g_st, 0, sizeof(double) * L.nelem, s));
  ADJ_CK(cudaMemsetAsync(g_th, 0, sizeof(double) * L.nelem, s));
  const sem_ionic_params& ip = ctx->ionic;
  const IonicAdj prm{ip.u_rest, ip.u_amp, ip.tau_in, ip.tau_out, ip.tau_open, ip.tau_close, ip.v_gate, ip.kappa};
  const GradTab gtab = make_grad_tab(L.tab);
  const double dt = tp->dt;
  auto UB = [&](int64_t k) { return tp->ub + ((k % 3 + 3) % 3) * n; };
  auto HB = [&](int64_t k) { return tp->hb + ((k % 3 + 3) % 3) * n; };
  sem_state* st = tp->st;
  for (int seg = (int)tp->ck.size() - 1; seg >= 0; --seg) {
    const int64_t start = tp->ck_n[seg];
    const int64_t stop = std::min<int64_t>(start + tp->every, tp->n0 + tp->nsteps);
    const double* ck = tp->ck[seg];
    // restore the checkpoint and recompute the segment's states
    st->cur = 0; st->prev = 1; st->next = 2; st->n = start;
    ADJ_CK(cudaMemcpyAsync(st->U[0], ck, bytes, cudaMemcpyDeviceToDevice, s));
    ADJ_CK(cudaMemcpyAsync(st->U[1], ck + n, bytes, cudaMemcpyDeviceToDevice, s));
    ADJ_CK(cudaMemcpyAsync(st->H[0], ck + 2 * n, bytes, cudaMemcpyDeviceToDevice, s));
    ADJ_CK(cudaMemcpyAsync(st->H[1], ck + 3 * n, bytes, cudaMemcpyDeviceToDevice, s));
    ADJ_CK(cudaMemcpyAsync(tp->seg_u, ck + n, bytes, cudaMemcpyDeviceToDevice, s));        // u^{start-1}
    ADJ_CK(cudaMemcpyAsync(tp->seg_u + n, ck, bytes, cudaMemcpyDeviceToDevice, s));        // u^start
    ADJ_CK(cudaMemcpyAsync(tp->seg_h, ck + 3 * n, bytes, cudaMemcpyDeviceToDevice, s));
    ADJ_CK(cudaMemcpyAsync(tp->seg_h + n, ck + 2 * n, bytes, cudaMemcpyDeviceToDevice, s));
    ctx->carry.valid = false;  // the state was restored from a checkpoint
    for (int64_t k = start; k < stop; ++k) {
      int rc = time_steps(ctx, st, dt, 1, rtol, atol, maxit, precond, nullptr, s);
      if (rc != SEM_OK) return rc;
      const int64_t j = k - start + 2;
      ADJ_CK(cudaMemcpyAsync(tp->seg_u + j * n, st->U[st->cur], bytes, cudaMemcpyDeviceToDevice, s));
      ADJ_CK(cudaMemcpyAsync(tp->seg_h + j * n, st->H[st->cur], bytes, cudaMemcpyDeviceToDevice, s));
    }
    // reverse the segment's steps
    for (int64_t k = stop - 1; k >= start; --k) {
      const int64_t j = k - start;
      const int64_t m = k - tp->n0;  // trace row
      k_sources<<<1, 128, 0, s>>>(tp->nsens, tp->sensors, trace_bar + (size_t)m * tp->nsens, UB(k + 1));
      ADJ_CK(cudaMemsetAsync(tp->w, 0, bytes, s));
      const int first = k == 0 ? 1 : 0;
      const double alpha = first ? 1.0 / dt : 1.5 / dt;
      int rc = cg_solve(ctx, alpha, UB(k + 1), tp->w, rtol, atol, maxit, precond, nullptr, nullptr,
                        stats, s);
      if (rc != SEM_OK) return rc;
      k_param_grad<<<L.nelem, 128, 0, s>>>(L.nelem, L.map, L.evert, ctx->sigma_l, ctx->sigma_t,
                                           ctx->theta, gtab, tp->w, tp->seg_u + (j + 2) * n, g_sl,
                                           g_st, g_th);
      ADJ_CK(cudaGetLastError());
      if (L.quad == SEM_QUAD_LGL) {
        k_scale_mul<<<gr, kThreads, 0, s>>>(n, L.mdiag, tp->w, tp->gbar);
        ADJ_CK(cudaGetLastError());
        ctx->launches += 1;
      } else {
        rc = apply_fp64(ctx, 1.0, 0.0, tp->w, tp->gbar, s);
        if (rc != SEM_OK) return rc;
      }
      k_adj_pointwise<<<gr, kThreads, 0, s>>>(n, tp->gbar, tp->seg_u + (j + 1) * n, tp->seg_u + j * n,
                                              tp->seg_h + (j + 2) * n, UB(k), UB(k - 1), HB(k + 1),
                                              HB(k), HB(k - 1), prm, dt, first);
      ADJ_CK(cudaGetLastError());
      ctx->launches += 3;
      // slot k+1 becomes slot k-2 of the next step: clear it
      ADJ_CK(cudaMemsetAsync(UB(k + 1), 0, bytes, s));
      ADJ_CK(cudaMemsetAsync(HB(k + 1), 0, bytes, s));
    }
  }
  return SEM_OK;
}

}  // namespace sem
