// 1-D tables of the Q_p spectral element (Section 3): LGL nodes and weights
// (the nodal basis and the SEM-NI rule), LG nodes and weights (the SEM rule),
// and the interpolation / collocation-derivative matrices of the Lagrange
// basis.
//
// Nodes are the eigenvalues of symmetric tridiagonal Jacobi matrices
// (Golub-Welsch), found by Sturm-sequence bisection:
//   LG nodes      = zeros of P_n:            Jacobi matrix of the Legendre
//                   polynomials, off-diagonal k / sqrt(4k^2 - 1);
//   interior LGL  = zeros of P_p' = Jacobi P^(1,1)_{p-1}: Gegenbauer(3/2)
//                   recurrence, off-diagonal sqrt(k (k+2) / ((2k+1)(2k+3))).
// Weights: LG  w = 2 / ((1 - x^2) P_n'(x)^2),  LGL  w = 2 / (p (p+1) P_p(x)^2).
// Matrices use the barycentric form of Lagrange interpolation.
#include <cmath>
#include <vector>

#include "sem_internal.cuh"

namespace sem {
namespace {

// Number of eigenvalues of the zero-diagonal symmetric tridiagonal matrix with
// squared off-diagonals b2[0..m-2] that are smaller than x.
int sturm_count(const std::vector<double>& b2, int m, double x) {
  int count = 0;
  double d = -x;
  for (int i = 0; i < m; ++i) {
    if (i > 0) d = -x - b2[i - 1] / d;
    if (d == 0.0) d = -1e-300;
    if (d < 0.0) ++count;
  }
  return count;
}

std::vector<double> tridiag_eigs(const std::vector<double>& b2, int m) {
  std::vector<double> ev(m);
  for (int k = 0; k < m; ++k) {
    double lo = -1.0, hi = 1.0;  // all zeros of these families lie in (-1, 1)
    for (int it = 0; it < 200 && hi - lo > 0.0; ++it) {
      double mid = 0.5 * (lo + hi);
      if (mid <= lo || mid >= hi) break;
      if (sturm_count(b2, m, mid) > k) hi = mid; else lo = mid;
    }
    ev[k] = 0.5 * (lo + hi);
  }
  return ev;
}

// Legendre P_n(x) and P_n'(x).
void legendre_eval(int n, double x, double* P, double* dP) {
  double p0 = 1.0, p1 = x, d0 = 0.0, d1 = 1.0;
  if (n == 0) { *P = 1.0; *dP = 0.0; return; }
  for (int k = 2; k <= n; ++k) {
    double p2 = ((2.0 * k - 1.0) * x * p1 - (k - 1.0) * p0) / k;
    double d2 = d0 + (2.0 * k - 1.0) * p1;  // P_k' = P_{k-2}' + (2k-1) P_{k-1}
    p0 = p1; p1 = p2; d0 = d1; d1 = d2;
  }
  *P = p1; *dP = d1;
}

void barycentric_weights(const double* x, int n, double* lam) {
  for (int j = 0; j < n; ++j) {
    double prod = 1.0;
    for (int k = 0; k < n; ++k) if (k != j) prod *= (x[j] - x[k]);
    lam[j] = 1.0 / prod;
  }
}

// M[q][l] = d/dx l_l at x_q, for the Lagrange basis on nodes x (collocation derivative).
void collocation_derivative(const double* x, int n, double (*M)[kMaxN]) {
  double lam[kMaxN];
  barycentric_weights(x, n, lam);
  for (int q = 0; q < n; ++q) {
    double diag = 0.0;
    for (int l = 0; l < n; ++l) {
      if (l == q) continue;
      M[q][l] = (lam[l] / lam[q]) / (x[q] - x[l]);
      diag -= M[q][l];
    }
    M[q][q] = diag;
  }
}

// M[q][l] = l_l(t_q) for the Lagrange basis on nodes x, evaluated at points t.
void interpolation_matrix(const double* x, int n, const double* t, int m, double (*M)[kMaxN]) {
  double lam[kMaxN];
  barycentric_weights(x, n, lam);
  for (int q = 0; q < m; ++q) {
    int hit = -1;
    for (int l = 0; l < n; ++l)
      if (std::fabs(t[q] - x[l]) < 1e-15) hit = l;
    if (hit >= 0) {
      for (int l = 0; l < n; ++l) M[q][l] = (l == hit) ? 1.0 : 0.0;
      continue;
    }
    double den = 0.0;
    for (int l = 0; l < n; ++l) den += lam[l] / (t[q] - x[l]);
    for (int l = 0; l < n; ++l) M[q][l] = (lam[l] / (t[q] - x[l])) / den;
  }
}

}  // namespace

void build_tables(int p, int quad, Tables1D* t) {
  *t = Tables1D();
  const int n = p + 1;
  t->p = p; t->n = n; t->quad = quad;
  // LGL nodes: -1, zeros of P_p', +1
  t->xg[0] = -1.0; t->xg[p] = 1.0;
  if (p >= 2) {
    std::vector<double> b2(p - 2);
    for (int k = 1; k <= p - 2; ++k) b2[k - 1] = double(k) * (k + 2) / ((2.0 * k + 1.0) * (2.0 * k + 3.0));
    std::vector<double> ev = tridiag_eigs(b2, p - 1);
    for (int i = 0; i < p - 1; ++i) t->xg[i + 1] = ev[i];
  }
  for (int i = 0; i < n; ++i) {
    double P, dP;
    legendre_eval(p, t->xg[i], &P, &dP);
    t->wg[i] = 2.0 / (p * (p + 1.0) * P * P);
  }
  collocation_derivative(t->xg, n, t->D);
  if (quad == SEM_QUAD_LGL) {
    for (int i = 0; i < n; ++i) { t->xq[i] = t->xg[i]; t->wq[i] = t->wg[i]; }
    for (int q = 0; q < n; ++q)
      for (int l = 0; l < n; ++l) { t->Bi[q][l] = (q == l) ? 1.0 : 0.0; t->Dg[q][l] = t->D[q][l]; }
  } else {
    std::vector<double> b2(n - 1);
    for (int k = 1; k <= n - 1; ++k) b2[k - 1] = double(k) * k / (4.0 * k * k - 1.0);
    std::vector<double> ev = tridiag_eigs(b2, n);
    for (int i = 0; i < n; ++i) {
      t->xq[i] = ev[i];
      double P, dP;
      legendre_eval(n, ev[i], &P, &dP);
      t->wq[i] = 2.0 / ((1.0 - ev[i] * ev[i]) * dP * dP);
    }
    interpolation_matrix(t->xg, n, t->xq, n, t->Bi);
    collocation_derivative(t->xq, n, t->Dg);
  }
}

}  // namespace sem
