// fe_tables.cpp -- 1D rules of libfe, computed once per degree on the host in double precision.
//
// The paper names only the 1D matrices of sum factorization (Sec. 2.3: V evaluates nodal values
// at quadrature points, D differentiates); the node and quadrature families used here are
// Gauss-Lobatto-Legendre nodes and an n = p+1 point Gauss-Legendre rule, both mapped to [0,1].
//  - Gauss points: Newton on P_n, derivative from the recurrence P'_{k+1} = P'_{k-1} + (2k+1) P_k.
//  - GLL interior nodes: Newton on f = P_{p-1} - x P_p (which is (1-x^2) P_p'/p), using the
//    Legendre equation f' = -(p+1) P_p.
//  - Lagrange interpolation and differentiation matrices in barycentric form.
#include <cmath>
#include <cstring>

#include "fe_internal.h"

namespace {

// P_k(x) and P_k'(x) for k = 0..n by recurrence
void legendre_all(int n, double x, double* P, double* dP) {
  P[0] = 1.0;
  dP[0] = 0.0;
  if (n == 0) return;
  P[1] = x;
  dP[1] = 1.0;
  for (int k = 1; k < n; ++k) {
    P[k + 1] = ((2 * k + 1) * x * P[k] - k * P[k - 1]) / (k + 1);
    dP[k + 1] = dP[k - 1] + (2 * k + 1) * P[k];
  }
}

void gauss_pm1(int n, double* x, double* w) {
  const double pi = 3.14159265358979323846;
  double P[FE_MAXN + 2], dP[FE_MAXN + 2];
  for (int i = 0; i < n; ++i) {
    // Tricomi-type first guess for the i-th root, ascending order
    double r = -std::cos(pi * (4.0 * i + 3.0) / (4.0 * n + 2.0));
    for (int it = 0; it < 60; ++it) {
      legendre_all(n, r, P, dP);
      double dr = P[n] / dP[n];
      r -= dr;
      if (std::fabs(dr) <= 1e-17) break;
    }
    legendre_all(n, r, P, dP);
    x[i] = r;
    w[i] = 2.0 / ((1.0 - r * r) * dP[n] * dP[n]);
  }
}

void gll_pm1(int p, double* x) {
  const double pi = 3.14159265358979323846;
  double P[FE_MAXN + 2], dP[FE_MAXN + 2];
  x[0] = -1.0;
  x[p] = 1.0;
  for (int i = 1; i < p; ++i) {
    double r = -std::cos(pi * i / p);
    for (int it = 0; it < 60; ++it) {
      legendre_all(p, r, P, dP);
      double f = P[p - 1] - r * P[p];
      double df = -(p + 1) * P[p];
      double dr = f / df;
      r -= dr;
      if (std::fabs(dr) <= 1e-17) break;
    }
    x[i] = r;
  }
}

// barycentric weights lambda_j = 1 / prod_{k != j} (x_j - x_k)
void bary_weights(int n, const double* x, double* lam) {
  for (int j = 0; j < n; ++j) {
    double prod = 1.0;
    for (int k = 0; k < n; ++k)
      if (k != j) prod *= (x[j] - x[k]);
    lam[j] = 1.0 / prod;
  }
}

// values of all Lagrange polynomials through nodes x at the point s (barycentric, second form)
void lagrange_values(int n, const double* x, const double* lam, double s, double* out) {
  for (int j = 0; j < n; ++j)
    if (s == x[j]) {
      for (int k = 0; k < n; ++k) out[k] = (k == j) ? 1.0 : 0.0;
      return;
    }
  double den = 0.0;
  for (int j = 0; j < n; ++j) den += lam[j] / (s - x[j]);
  for (int j = 0; j < n; ++j) out[j] = lam[j] / (s - x[j]) / den;
}

}  // namespace

void fe_host_tables(int p, HostTab* h) {
  std::memset(h, 0, sizeof(*h));
  int n = p + 1;
  h->p = p;
  h->n = n;
  double g[FE_MAXN], gw[FE_MAXN], l[FE_MAXN];
  gauss_pm1(n, g, gw);
  gll_pm1(p, l);
  for (int i = 0; i < n; ++i) {
    h->t[i] = 0.5 * (l[i] + 1.0);
    h->s[i] = 0.5 * (g[i] + 1.0);
    h->w[i] = 0.5 * gw[i];
  }
  double lt[FE_MAXN], ls[FE_MAXN];
  bary_weights(n, h->t, lt);
  bary_weights(n, h->s, ls);
  for (int q = 0; q < n; ++q) lagrange_values(n, h->t, lt, h->s[q], h->V[q]);
  // collocation derivative at the Gauss points: D[q][r] = (ls_r/ls_q)/(s_q - s_r), rows sum to 0
  for (int q = 0; q < n; ++q) {
    double diag = 0.0;
    for (int r = 0; r < n; ++r) {
      if (r == q) continue;
      h->D[q][r] = (ls[r] / ls[q]) / (h->s[q] - h->s[r]);
      diag -= h->D[q][r];
    }
    h->D[q][q] = diag;
  }
  for (int q = 0; q < n; ++q)
    for (int i = 0; i < n; ++i) {
      double acc = 0.0;
      for (int r = 0; r < n; ++r) acc += h->D[q][r] * h->V[r][i];
      h->Dh[q][i] = acc;
    }
}
