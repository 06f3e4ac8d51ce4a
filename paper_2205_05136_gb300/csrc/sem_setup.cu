// Setup kernels: node coordinates, quadrature-point metric terms with the
// fibre conductivity tensor, assembled diagonals, stimulus masks and the
// low-precision metric copies.
//
// Metric (Section 4: "the Jacobian of the transformation ... is cached";
// Section 4.2: D evaluated at every quadrature point, Eq. diffusiontensor):
//   J[d][c] = dx_d / dxi_c at each quadrature point, obtained by
//   differentiating the element's nodal coordinate field (SEM-NI: D on the
//   GLL nodes; SEM: interpolate to the Gauss points, then the Gauss
//   collocation derivative),
//   D_e = sigma_t I + (sigma_l - sigma_t) f f^T,  f = (cos theta, sin theta, 0),
//   G   = w |det J| J^{-1} D_e J^{-T}  (6 entries),  W = w |det J|.
#include <algorithm>
#include <cmath>
#include <vector>

#include "sem_internal.cuh"

namespace sem {
namespace {

struct SetupTab {
  int n;
  double xg[kMaxN];          // LGL nodes
  double wq[kMaxN];          // quadrature weights
  double Bq[kMaxN][kMaxN];   // GLL basis at the quadrature points (identity for SEM-NI)
  double Dq[kMaxN][kMaxN];   // derivative of the GLL basis at the quadrature points
  double Dc[kMaxN][kMaxN];   // collocation derivative on the quadrature points
};

SetupTab make_setup_tab(const Tables1D& t) {
  SetupTab s{};
  s.n = t.n;
  for (int i = 0; i < t.n; ++i) { s.xg[i] = t.xg[i]; s.wq[i] = t.wq[i]; }
  for (int q = 0; q < t.n; ++q)
    for (int l = 0; l < t.n; ++l) {
      s.Bq[q][l] = t.Bi[q][l];
      s.Dc[q][l] = t.Dg[q][l];
      double d = 0.0;
      if (t.quad == SEM_QUAD_LGL) {
        d = t.D[q][l];
      } else {
        for (int m = 0; m < t.n; ++m) d += t.Dg[q][m] * t.Bi[m][l];
      }
      s.Dq[q][l] = d;
    }
  return s;
}

__device__ __forceinline__ double trilinear(const double (*V)[3], int d, double x, double y,
                                            double z) {
  double acc = 0.0;
#pragma unroll
  for (int v = 0; v < 8; ++v) {
    const double sx = (v & 1) ? 1.0 : -1.0, sy = (v & 2) ? 1.0 : -1.0, sz = (v & 4) ? 1.0 : -1.0;
    const double N = 0.125 * (1.0 + sx * x) * (1.0 + sy * y) * (1.0 + sz * z);
    acc += N * V[v][d];
  }
  return acc;
}

// One CTA per element.
__global__ void k_metric(int nelem, const double* __restrict__ evert,
                         const double* __restrict__ sigma_l, const double* __restrict__ sigma_t,
                         const double* __restrict__ theta, const __grid_constant__ SetupTab tab,
                         int lg, double* __restrict__ metric, int* bad) {
  const int e = blockIdx.x;
  if (e >= nelem) return;
  const int n = tab.n, n2 = n * n, n3 = n2 * n;
  __shared__ double V[8][3];
  __shared__ double X[3][kMaxN * kMaxN * kMaxN];
  __shared__ double Y[3][kMaxN * kMaxN * kMaxN];
  if (threadIdx.x < 24) V[threadIdx.x / 3][threadIdx.x % 3] = evert[(size_t)e * 24 + threadIdx.x];
  __syncthreads();
  for (int a = threadIdx.x; a < n3; a += blockDim.x) {
    const int i = a % n, j = (a / n) % n, k = a / n2;
    for (int d = 0; d < 3; ++d) X[d][a] = trilinear(V, d, tab.xg[i], tab.xg[j], tab.xg[k]);
  }
  __syncthreads();
  if (lg) {  // coordinates at the Gauss points: X -> Y (x), Y -> X (y), X -> Y (z)
    for (int a = threadIdx.x; a < n3; a += blockDim.x) {
      const int q = a % n, j = (a / n) % n, k = a / n2;
      for (int d = 0; d < 3; ++d) {
        double s = 0.0;
        for (int l = 0; l < n; ++l) s += tab.Bq[q][l] * X[d][k * n2 + j * n + l];
        Y[d][a] = s;
      }
    }
    __syncthreads();
    for (int a = threadIdx.x; a < n3; a += blockDim.x) {
      const int i = a % n, q = (a / n) % n, k = a / n2;
      for (int d = 0; d < 3; ++d) {
        double s = 0.0;
        for (int l = 0; l < n; ++l) s += tab.Bq[q][l] * Y[d][k * n2 + l * n + i];
        X[d][a] = s;
      }
    }
    __syncthreads();
    for (int a = threadIdx.x; a < n3; a += blockDim.x) {
      const int i = a % n, j = (a / n) % n, q = a / n2;
      for (int d = 0; d < 3; ++d) {
        double s = 0.0;
        for (int l = 0; l < n; ++l) s += tab.Bq[q][l] * X[d][l * n2 + j * n + i];
        Y[d][a] = s;
      }
    }
    __syncthreads();
  }
  const double(*Xq)[kMaxN * kMaxN * kMaxN] = lg ? Y : X;
  const double sl = sigma_l[e], st = sigma_t[e], th = theta[e];
  const double f0 = cos(th), f1 = sin(th);
  double Dm[3][3];
  const double fv[3] = {f0, f1, 0.0};
  for (int r = 0; r < 3; ++r)
    for (int c = 0; c < 3; ++c) Dm[r][c] = (r == c ? st : 0.0) + (sl - st) * fv[r] * fv[c];
  for (int a = threadIdx.x; a < n3; a += blockDim.x) {
    const int qx = a % n, qy = (a / n) % n, qz = a / n2;
    double J[3][3];
    for (int d = 0; d < 3; ++d) {
      double s0 = 0.0, s1 = 0.0, s2 = 0.0;
      for (int l = 0; l < n; ++l) {
        s0 += tab.Dc[qx][l] * Xq[d][qz * n2 + qy * n + l];
        s1 += tab.Dc[qy][l] * Xq[d][qz * n2 + l * n + qx];
        s2 += tab.Dc[qz][l] * Xq[d][l * n2 + qy * n + qx];
      }
      J[d][0] = s0; J[d][1] = s1; J[d][2] = s2;
    }
    const double det = J[0][0] * (J[1][1] * J[2][2] - J[1][2] * J[2][1]) -
                       J[0][1] * (J[1][0] * J[2][2] - J[1][2] * J[2][0]) +
                       J[0][2] * (J[1][0] * J[2][1] - J[1][1] * J[2][0]);
    if (!(det > 0.0)) atomicExch(bad, 1);
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
    double T[3][3];  // inv * Dm
    for (int r = 0; r < 3; ++r)
      for (int c = 0; c < 3; ++c)
        T[r][c] = inv[r][0] * Dm[0][c] + inv[r][1] * Dm[1][c] + inv[r][2] * Dm[2][c];
    double G[3][3];  // W * T * inv^T
    for (int r = 0; r < 3; ++r)
      for (int c = 0; c < 3; ++c)
        G[r][c] = W * (T[r][0] * inv[c][0] + T[r][1] * inv[c][1] + T[r][2] * inv[c][2]);
    const int n3p = padded_n3(n);
    double* out = metric + (size_t)e * kMetricComps * n3p + a;
    out[0 * n3p] = G[0][0];
    out[1 * n3p] = 0.5 * (G[0][1] + G[1][0]);
    out[2 * n3p] = 0.5 * (G[0][2] + G[2][0]);
    out[3 * n3p] = G[1][1];
    out[4 * n3p] = 0.5 * (G[1][2] + G[2][1]);
    out[5 * n3p] = G[2][2];
    out[6 * n3p] = W;
  }
}

// Node coordinates; each global node is written by exactly one element (the
// highest-index element that holds it).
__global__ void k_nodes(int nelem, int nx, int ny, int nz, const double* __restrict__ evert,
                        const int* __restrict__ map, const __grid_constant__ SetupTab tab,
                        int64_t ndofs, double* __restrict__ xyz) {
  const int e = blockIdx.x;
  if (e >= nelem) return;
  const int n = tab.n, p = n - 1, n3 = n * n * n;
  const int ex = e % nx, ey = (e / nx) % ny, ez = e / (nx * ny);
  __shared__ double V[8][3];
  if (threadIdx.x < 24) V[threadIdx.x / 3][threadIdx.x % 3] = evert[(size_t)e * 24 + threadIdx.x];
  __syncthreads();
  for (int a = threadIdx.x; a < n3; a += blockDim.x) {
    const int i = a % n, j = (a / n) % n, k = a / (n * n);
    const bool own = (i < p || ex == nx - 1) && (j < p || ey == ny - 1) && (k < p || ez == nz - 1);
    if (!own) continue;
    const int g = map[(size_t)e * n3 + a];
    for (int d = 0; d < 3; ++d) xyz[d * ndofs + g] = trilinear(V, d, tab.xg[i], tab.xg[j], tab.xg[k]);
  }
}

// Assembled diagonals of M and K: per element and local node a,
//   M_aa = sum_q W_q phi_a(q)^2,  K_aa = sum_q grad phi_a(q) . G_q grad phi_a(q)
// (reference gradients; G already holds J^{-1} D J^{-T} w |det J|).
__global__ void k_diagonals(int nelem, const int* __restrict__ map,
                            const double* __restrict__ metric, const __grid_constant__ SetupTab tab,
                            double* __restrict__ mdiag, double* __restrict__ kdiag) {
  const int e = blockIdx.x;
  if (e >= nelem) return;
  const int n = tab.n, n2 = n * n, n3 = n2 * n;
  const int n3p = padded_n3(n);
  const double* me = metric + (size_t)e * kMetricComps * n3p;
  for (int a = threadIdx.x; a < n3; a += blockDim.x) {
    const int i = a % n, j = (a / n) % n, k = a / n2;
    double Msum = 0.0, Ksum = 0.0;
    for (int qz = 0; qz < n; ++qz)
      for (int qy = 0; qy < n; ++qy)
        for (int qx = 0; qx < n; ++qx) {
          const int q = qx + n * qy + n2 * qz;
          const double b0 = tab.Bq[qx][i], b1 = tab.Bq[qy][j], b2 = tab.Bq[qz][k];
          const double d0 = tab.Dq[qx][i], d1 = tab.Dq[qy][j], d2 = tab.Dq[qz][k];
          const double gx = d0 * b1 * b2, gy = b0 * d1 * b2, gz = b0 * b1 * d2, ph = b0 * b1 * b2;
          const double G00 = me[0 * n3p + q], G01 = me[1 * n3p + q], G02 = me[2 * n3p + q];
          const double G11 = me[3 * n3p + q], G12 = me[4 * n3p + q], G22 = me[5 * n3p + q];
          const double W = me[6 * n3p + q];
          Ksum += G00 * gx * gx + G11 * gy * gy + G22 * gz * gz +
                  2.0 * (G01 * gx * gy + G02 * gx * gz + G12 * gy * gz);
          Msum += W * ph * ph;
        }
    const int g = map[(size_t)e * n3 + a];
    atomicAdd(mdiag + g, Msum);
    atomicAdd(kdiag + g, Ksum);
  }
}

__global__ void k_region_mask(int64_t ndofs, const double* __restrict__ xyz, int region,
                              double a0, double a1, double a2, double a3, double a4, double a5,
                              double* __restrict__ mask) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < ndofs;
       i += (int64_t)gridDim.x * blockDim.x) {
    const double x = xyz[i], y = xyz[ndofs + i], z = xyz[2 * ndofs + i];
    bool in;
    if (region == SEM_REGION_BOX) {
      in = x >= a0 && y >= a1 && z >= a2 && x <= a3 && y <= a4 && z <= a5;
    } else {
      const double dx = x - a0, dy = y - a1, dz = z - a2;
      in = dx * dx + dy * dy + dz * dz <= a3 * a3;
    }
    mask[i] = in ? 1.0 : 0.0;
  }
}

template <typename OT>
__global__ void k_convert(int64_t n, const double* __restrict__ in, OT* __restrict__ out);

template <>
__global__ void k_convert<float>(int64_t n, const double* __restrict__ in, float* __restrict__ out) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    out[i] = __double2float_rn(in[i]);
}

// FP64 component-major metric -> the column-major bf16 layout (MetricLayout).
__global__ void k_convert_columns_bf16(int64_t n, int np, const double* __restrict__ in,
                                       __nv_bfloat16* __restrict__ out) {
  using ML = MetricLayout<__nv_bfloat16>;
  const int n2 = np * np, cw = ML::col_width(np), blk = ML::block(np), n3p = padded_n3(np);
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t e = i / blk;
    const int r = (int)(i - e * blk), c = r / cw, s = r - c * cw, k = s / kMetricComps,
              comp = s - k * kMetricComps;
    const double v = (c < n2 && k < np) ? in[(e * kMetricComps + comp) * n3p + c + (int64_t)n2 * k] : 0.0;
    out[i] = __float2bfloat16_rn(__double2float_rn(v));
  }
}

__global__ void k_split_pairs(int64_t n, const double* __restrict__ in, df_pair* __restrict__ out) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const double x = in[i];
    const float h = __double2float_rn(x);
    out[i].h = h;
    out[i].l = __double2float_rn(x - (double)h);
  }
}

int setup_threads(int n3) { return n3 <= 64 ? 64 : (n3 <= 128 ? 128 : 256); }

}  // namespace

cudaError_t level_create(Level& L, int nx, int ny, int nz, const double* vertices, int p, int quad,
                         bool coords, cudaStream_t s) {
  L.p = p; L.quad = quad; L.n = p + 1;
  L.nx = nx; L.ny = ny; L.nz = nz;
  L.nelem = nx * ny * nz;
  const int64_t NX = (int64_t)p * nx + 1, NY = (int64_t)p * ny + 1, NZ = (int64_t)p * nz + 1;
  L.ndofs = NX * NY * NZ;
  build_tables(p, quad, &L.tab);
  const int n = L.n, n3 = n * n * n;
  std::vector<int> map((size_t)L.nelem * n3);
  std::vector<double> ev((size_t)L.nelem * 24);
  for (int ez = 0; ez < nz; ++ez)
    for (int ey = 0; ey < ny; ++ey)
      for (int ex = 0; ex < nx; ++ex) {
        const size_t e = (size_t)ex + (size_t)nx * (ey + (size_t)ny * ez);
        for (int k = 0; k < n; ++k)
          for (int j = 0; j < n; ++j)
            for (int i = 0; i < n; ++i) {
              const int64_t g = (ex * (int64_t)p + i) + NX * ((ey * (int64_t)p + j) + NY * (ez * (int64_t)p + k));
              map[e * n3 + i + n * (j + n * k)] = (int)g;
            }
        for (int c = 0; c < 2; ++c)
          for (int b = 0; b < 2; ++b)
            for (int a = 0; a < 2; ++a) {
              const size_t v = (size_t)(ex + a) + (size_t)(nx + 1) * ((ey + b) + (size_t)(ny + 1) * (ez + c));
              for (int d = 0; d < 3; ++d) ev[e * 24 + (a + 2 * b + 4 * c) * 3 + d] = vertices[v * 3 + d];
            }
      }
  const size_t nm = metric_count(L);
  cudaError_t e;
  if ((e = cudaMalloc(&L.map, sizeof(int) * map.size())) != cudaSuccess) return e;
  if ((e = cudaMalloc(&L.evert, sizeof(double) * ev.size())) != cudaSuccess) return e;
  if ((e = cudaMalloc(&L.metric, sizeof(double) * nm)) != cudaSuccess) return e;
  if ((e = cudaMemsetAsync(L.metric, 0, sizeof(double) * nm, s)) != cudaSuccess) return e;  // padding
  if ((e = cudaMalloc(&L.mdiag, sizeof(double) * L.ndofs)) != cudaSuccess) return e;
  if ((e = cudaMalloc(&L.kdiag, sizeof(double) * L.ndofs)) != cudaSuccess) return e;
  if (coords && (e = cudaMalloc(&L.xyz, sizeof(double) * 3 * L.ndofs)) != cudaSuccess) return e;
  if ((e = cudaMemcpyAsync(L.map, map.data(), sizeof(int) * map.size(), cudaMemcpyHostToDevice, s)) != cudaSuccess) return e;
  if ((e = cudaMemcpyAsync(L.evert, ev.data(), sizeof(double) * ev.size(), cudaMemcpyHostToDevice, s)) != cudaSuccess) return e;
  // the host vectors must outlive the copies
  return cudaStreamSynchronize(s);
}

void level_free(Level& L) {
  cudaFree(L.map);
  cudaFree(L.evert);
  cudaFree(L.metric);
  cudaFree(L.metric32);
  cudaFree(L.metric16);
  cudaFree(L.metric2);
  cudaFree(L.metric_tc);
  cudaFree(L.tc_frag);
  cudaFree(L.mdiag);
  cudaFree(L.kdiag);
  cudaFree(L.xyz);
  L = Level();
}

cudaError_t setup_geometry(Level& L, const double* sigma_l, const double* sigma_t,
                           const double* theta, int* d_bad, cudaStream_t s) {
  const SetupTab tab = make_setup_tab(L.tab);
  const int n3 = L.n * L.n * L.n;
  k_metric<<<L.nelem, setup_threads(n3), 0, s>>>(L.nelem, L.evert, sigma_l, sigma_t, theta, tab,
                                                 L.quad == SEM_QUAD_LG, L.metric, d_bad);
  L.metric32_valid = false;
  L.metric16_valid = false;
  L.metric2_valid = false;
  L.metric_tc_valid = false;
  return cudaGetLastError();
}

cudaError_t setup_node_coords(Level& L, cudaStream_t s) {
  const SetupTab tab = make_setup_tab(L.tab);
  const int n3 = L.n * L.n * L.n;
  k_nodes<<<L.nelem, setup_threads(n3), 0, s>>>(L.nelem, L.nx, L.ny, L.nz, L.evert, L.map, tab,
                                                L.ndofs, L.xyz);
  return cudaGetLastError();
}

cudaError_t setup_diagonals(Level& L, cudaStream_t s) {
  const SetupTab tab = make_setup_tab(L.tab);
  const int n3 = L.n * L.n * L.n;
  cudaError_t err = cudaMemsetAsync(L.mdiag, 0, sizeof(double) * L.ndofs, s);
  if (err != cudaSuccess) return err;
  err = cudaMemsetAsync(L.kdiag, 0, sizeof(double) * L.ndofs, s);
  if (err != cudaSuccess) return err;
  k_diagonals<<<L.nelem, setup_threads(n3), 0, s>>>(L.nelem, L.map, L.metric, tab, L.mdiag,
                                                    L.kdiag);
  return cudaGetLastError();
}

cudaError_t setup_metric_lowp(Level& L, bool bf16, cudaStream_t s) {
  const int64_t count = (int64_t)metric_count(L);
  const int threads = 256;
  const int blocks = (int)std::min<int64_t>((count + threads - 1) / threads, 152 * 16);
  if (bf16) {
    const int64_t count16 = (int64_t)metric16_count(L);
    const int blocks16 = (int)std::min<int64_t>((count16 + threads - 1) / threads, 152 * 16);
    k_convert_columns_bf16<<<blocks16, threads, 0, s>>>(count16, L.n, L.metric, L.metric16);
    L.metric16_valid = true;
  } else {
    k_convert<float><<<blocks, threads, 0, s>>>(count, L.metric, L.metric32);
    L.metric32_valid = true;
  }
  return cudaGetLastError();
}

cudaError_t setup_metric_df(Level& L, cudaStream_t s) {
  const int64_t count = (int64_t)metric_count(L);
  const int threads = 256;
  const int blocks = (int)std::min<int64_t>((count + threads - 1) / threads, 152 * 16);
  k_split_pairs<<<blocks, threads, 0, s>>>(count, L.metric, L.metric2);
  L.metric2_valid = true;
  return cudaGetLastError();
}

cudaError_t setup_region_mask(const Level& L, int region, const double* prm, double* mask,
                              cudaStream_t s) {
  double a[6] = {0, 0, 0, 0, 0, 0};
  const int cnt = region == SEM_REGION_BOX ? 6 : 4;
  for (int i = 0; i < cnt; ++i) a[i] = prm[i];
  const int threads = 256;
  const int blocks = (int)std::min<int64_t>((L.ndofs + threads - 1) / threads, 152 * 8);
  k_region_mask<<<blocks, threads, 0, s>>>(L.ndofs, L.xyz, region, a[0], a[1], a[2], a[3], a[4],
                                           a[5], mask);
  return cudaGetLastError();
}

}  // namespace sem
