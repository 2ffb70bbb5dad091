// 1D quadrature and Lagrange operators of the tensor-product DG basis (host code).
//
// Sec. 3.1: the element spaces hold polynomials of degree k = n - 1. The library represents them by
// the Lagrange basis on n Gauss-Lobatto-Legendre (GLL) nodes (the nodal layout of the ABI) and
// integrates with the n-point Gauss-Legendre rule. Internally the kernels work with values at the
// Gauss points (the map between the two is the invertible tensor matrix B x B x B).
#include <cmath>
#include <cstring>

#include "dg_internal.cuh"

namespace dg {

namespace {

// Legendre P_n(x) and its derivative by the three-term recurrence
void legendre(int n, double x, double* p, double* dp) {
  double p0 = 1.0, p1 = x;
  if (n == 0) { *p = 1.0; *dp = 0.0; return; }
  for (int k = 2; k <= n; ++k) {
    double p2 = ((2.0 * k - 1.0) * x * p1 - (k - 1.0) * p0) / k;
    p0 = p1;
    p1 = p2;
  }
  *p = p1;
  *dp = (std::fabs(x) < 1.0) ? n * (p0 - x * p1) / (1.0 - x * x) : 0.5 * n * (n + 1) * std::pow(x, n + 1);
}

// Gauss-Legendre: roots of P_n by Newton from Chebyshev-like guesses, weights 2/((1-x^2) P_n'^2)
void gauss_rule(int n, double* x, double* w) {
  for (int i = 0; i < n; ++i) {
    double z = -std::cos(M_PI * (i + 0.75) / (n + 0.5));
    for (int it = 0; it < 100; ++it) {
      double p, dp;
      legendre(n, z, &p, &dp);
      double dz = p / dp;
      z -= dz;
      if (std::fabs(dz) < 1e-16) break;
    }
    double p, dp;
    legendre(n, z, &p, &dp);
    x[i] = z;
    w[i] = 2.0 / ((1.0 - z * z) * dp * dp);
  }
}

// GLL nodes: -1, roots of P'_{n-1}, +1. Newton on q(x) = (1 - x^2) P'_{n-1}(x), whose
// derivative is -(n-1) n P_{n-1}(x) (Legendre's equation).
void gll_nodes(int n, double* x) {
  int N = n - 1;
  x[0] = -1.0;
  x[N] = 1.0;
  for (int i = 1; i < N; ++i) {
    double z = -std::cos(M_PI * i / N);
    for (int it = 0; it < 100; ++it) {
      double p, dp;
      legendre(N, z, &p, &dp);
      double qv = (1.0 - z * z) * dp;
      double dq = -double(N) * (N + 1) * p;
      double dz = qv / dq;
      z -= dz;
      if (std::fabs(dz) < 1e-16) break;
    }
    x[i] = z;
  }
}

// barycentric weights of a node set
void bary(int n, const double* x, double* lam) {
  for (int k = 0; k < n; ++k) {
    double prod = 1.0;
    for (int m = 0; m < n; ++m)
      if (m != k) prod *= (x[k] - x[m]);
    lam[k] = 1.0 / prod;
  }
}

// Lagrange basis of node set x evaluated at point t: out[k] = l_k(t) (product form)
void lagrange_at(int n, const double* x, double t, double* out) {
  for (int k = 0; k < n; ++k) {
    double v = 1.0;
    for (int m = 0; m < n; ++m)
      if (m != k) v *= (t - x[m]) / (x[k] - x[m]);
    out[k] = v;
  }
}

}  // namespace

void build_ops(int n, Ops* o) {
  std::memset(o, 0, sizeof(Ops));
  gauss_rule(n, o->eta, o->w);
  gll_nodes(n, o->xi);
  double row[MAXN];
  for (int q = 0; q < n; ++q) {
    lagrange_at(n, o->xi, o->eta[q], row);
    for (int a = 0; a < n; ++a) o->B[q * n + a] = row[a];
  }
  for (int a = 0; a < n; ++a) {
    lagrange_at(n, o->eta, o->xi[a], row);
    for (int q = 0; q < n; ++q) o->Binv[a * n + q] = row[q];
  }
  lagrange_at(n, o->eta, -1.0, o->eL);
  lagrange_at(n, o->eta, 1.0, o->eR);
  // derivative matrix on the Gauss points: D[q][k] = lam_k / lam_q / (eta_q - eta_k), q != k;
  // the diagonal makes every row sum to zero (derivative of a constant)
  double lam[MAXN];
  bary(n, o->eta, lam);
  for (int q = 0; q < n; ++q) {
    double diag = 0.0;
    for (int k = 0; k < n; ++k) {
      if (k == q) continue;
      double v = lam[k] / lam[q] / (o->eta[q] - o->eta[k]);
      o->D[q * n + k] = v;
      diag -= v;
    }
    o->D[q * n + q] = diag;
  }
}

}  // namespace dg
