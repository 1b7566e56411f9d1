/*
 * oracle.c -- plain, slow FP64 CPU oracle (TEST INFRASTRUCTURE ONLY; see oracle.h).
 *
 * Every routine follows a definition of the method directly: no sum factorization, no
 * blocking, no fusion.  Element matrices are formed entry by entry from the tensor-product
 * Lagrange basis evaluated at every quadrature point, then assembled or applied cell by cell.
 * Compile with -ffp-contract=off so that every product and sum is rounded as written.
 */
#include "oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define OR_MAXN 8
#define OR_PI 3.14159265358979323846

static void set_threads(int nthreads) {
#ifdef _OPENMP
  if (nthreads > 0) omp_set_num_threads(nthreads);
#else
  (void)nthreads;
#endif
}

/* ------------------------------------------------------------------------------------------
 * 1D rules.  The paper leaves the node and quadrature families open (Sec. 2.3 names only the
 * 1D matrices V, D, M); the reading used here is Gauss-Lobatto-Legendre nodes and an
 * n = p+1 point Gauss-Legendre rule per direction.
 * ---------------------------------------------------------------------------------------- */

/* Legendre P_k(x) for k = n and n-1 by the three-term recurrence
 * (k+1) P_{k+1} = (2k+1) x P_k - k P_{k-1}. */
static void legendre_pair(int n, double x, double* pn, double* pnm1) {
  double p0 = 1.0, p1 = x;
  if (n == 0) {
    *pn = 1.0;
    *pnm1 = 0.0;
    return;
  }
  for (int k = 1; k < n; ++k) {
    double p2 = ((2.0 * k + 1.0) * x * p1 - k * p0) / (k + 1.0);
    p0 = p1;
    p1 = p2;
  }
  *pn = p1;
  *pnm1 = p0;
}

/* P_n'(x) for |x| < 1 from (x^2-1) P_n' = n (x P_n - P_{n-1}). */
static double legendre_deriv(int n, double x) {
  double pn, pnm1;
  legendre_pair(n, x, &pn, &pnm1);
  return n * (x * pn - pnm1) / (x * x - 1.0);
}

int or_gauss(int n, double* x, double* w) {
  if (n < 1 || n > 64) return 1;
  for (int i = 0; i < n; ++i) {
    double r = -cos(OR_PI * (i + 0.75) / (n + 0.5));
    for (int it = 0; it < 100; ++it) {
      double pn, pnm1;
      legendre_pair(n, r, &pn, &pnm1);
      double dp = n * (r * pn - pnm1) / (r * r - 1.0);
      double dr = pn / dp;
      r -= dr;
      if (fabs(dr) < 1e-16) break;
    }
    double dp = legendre_deriv(n, r);
    x[i] = r;
    w[i] = 2.0 / ((1.0 - r * r) * dp * dp);
  }
  return 0;
}

int or_gll(int p, double* x) {
  if (p < 1 || p > 63) return 1;
  x[0] = -1.0;
  x[p] = 1.0;
  for (int i = 1; i < p; ++i) {
    /* interior nodes: roots of P_p'; Newton with P_p'' = (2x P_p' - p(p+1) P_p)/(1-x^2) */
    double r = -cos(OR_PI * i / p);
    for (int it = 0; it < 100; ++it) {
      double pn, pnm1;
      legendre_pair(p, r, &pn, &pnm1);
      double d1 = p * (r * pn - pnm1) / (r * r - 1.0);
      double d2 = (2.0 * r * d1 - p * (p + 1.0) * pn) / (1.0 - r * r);
      double dr = d1 / d2;
      r -= dr;
      if (fabs(dr) < 1e-16) break;
    }
    x[i] = r;
  }
  return 0;
}

/* Lagrange polynomial through nodes t[0..n-1]: l_i(s) = prod_{j != i} (s - t_j)/(t_i - t_j). */
double or_lagrange(const double* t, int n, int i, double s) {
  double v = 1.0;
  for (int j = 0; j < n; ++j)
    if (j != i) v *= (s - t[j]) / (t[i] - t[j]);
  return v;
}

/* l_i'(s) = sum_{m != i} 1/(t_i - t_m) prod_{j != i, m} (s - t_j)/(t_i - t_j). */
double or_lagrange_deriv(const double* t, int n, int i, double s) {
  double d = 0.0;
  for (int m = 0; m < n; ++m) {
    if (m == i) continue;
    double v = 1.0 / (t[i] - t[m]);
    for (int j = 0; j < n; ++j)
      if (j != i && j != m) v *= (s - t[j]) / (t[i] - t[j]);
    d += v;
  }
  return d;
}

/* ------------------------------------------------------------------------------------------
 * Counts (Sec. 6: unique count (n p + 1)^d on structured grids; cell-wise (p+1)^d per cell).
 * ---------------------------------------------------------------------------------------- */
long long or_n_cells(const or_mesh* m) { return (long long)m->mx * m->my * m->mz; }
long long or_n_cellwise(const or_mesh* m) {
  long long n = m->p + 1;
  return or_n_cells(m) * n * n * n;
}
long long or_n_unique(const or_mesh* m) {
  return (long long)(m->mx * m->p + 1) * (m->my * m->p + 1) * (m->mz * m->p + 1);
}

/* ------------------------------------------------------------------------------------------
 * Geometry.  The map Phi(X) = X + amp * sin(pi X) sin(pi Y) sin(pi Z) * (1,1,1) is sampled at
 * the GLL nodes of every cell and interpolated isoparametrically with the Q_p basis.  Reference
 * coordinates xi are in [0,1]^3.
 * ---------------------------------------------------------------------------------------- */
void or_map(double amp, const double X[3], double x[3]) {
  double s = sin(OR_PI * X[0]) * sin(OR_PI * X[1]) * sin(OR_PI * X[2]);
  x[0] = X[0] + amp * s;
  x[1] = X[1] + amp * s;
  x[2] = X[2] + amp * s;
}

static void ref_nodes01(int p, double* t) {
  double g[OR_MAXN];
  or_gll(p, g);
  for (int i = 0; i <= p; ++i) t[i] = 0.5 * (1.0 + g[i]);
}

static void gauss01(int n, double* s, double* w) {
  double g[64], gw[64];
  or_gauss(n, g, gw);
  for (int i = 0; i < n; ++i) {
    s[i] = 0.5 * (1.0 + g[i]);
    w[i] = 0.5 * gw[i];
  }
}

void or_cell_nodes(const or_mesh* m, int cx, int cy, int cz, double* xn) {
  int n = m->p + 1;
  double t[OR_MAXN];
  ref_nodes01(m->p, t);
  for (int k = 0; k < n; ++k)
    for (int j = 0; j < n; ++j)
      for (int i = 0; i < n; ++i) {
        double X[3] = {(cx + t[i]) / m->mx, (cy + t[j]) / m->my, (cz + t[k]) / m->mz};
        or_map(m->amp, X, xn + 3 * ((k * n + j) * n + i));
      }
}

/* value and reference gradient of the tensor-product basis function (i,j,k) at xi */
static void basis_eval(const double* t, int n, int i, int j, int k, const double xi[3], double* v,
                       double g[3]) {
  double li = or_lagrange(t, n, i, xi[0]), lj = or_lagrange(t, n, j, xi[1]),
         lk = or_lagrange(t, n, k, xi[2]);
  double di = or_lagrange_deriv(t, n, i, xi[0]), dj = or_lagrange_deriv(t, n, j, xi[1]),
         dk = or_lagrange_deriv(t, n, k, xi[2]);
  *v = li * lj * lk;
  g[0] = di * lj * lk;
  g[1] = li * dj * lk;
  g[2] = li * lj * dk;
}

/* J[a*3+b] = d x_a / d xi_b of the isoparametric map at xi */
void or_jacobian(const or_mesh* m, const double* xn, const double xi[3], double J[9]) {
  int n = m->p + 1;
  double t[OR_MAXN];
  ref_nodes01(m->p, t);
  for (int e = 0; e < 9; ++e) J[e] = 0.0;
  for (int k = 0; k < n; ++k)
    for (int j = 0; j < n; ++j)
      for (int i = 0; i < n; ++i) {
        double v, g[3];
        basis_eval(t, n, i, j, k, xi, &v, g);
        const double* X = xn + 3 * ((k * n + j) * n + i);
        for (int a = 0; a < 3; ++a)
          for (int b = 0; b < 3; ++b) J[a * 3 + b] += X[a] * g[b];
      }
}

static double det3(const double J[9]) {
  return J[0] * (J[4] * J[8] - J[5] * J[7]) - J[1] * (J[3] * J[8] - J[5] * J[6]) +
         J[2] * (J[3] * J[7] - J[4] * J[6]);
}

static void inv3(const double J[9], double det, double Ji[9]) {
  Ji[0] = (J[4] * J[8] - J[5] * J[7]) / det;
  Ji[1] = (J[2] * J[7] - J[1] * J[8]) / det;
  Ji[2] = (J[1] * J[5] - J[2] * J[4]) / det;
  Ji[3] = (J[5] * J[6] - J[3] * J[8]) / det;
  Ji[4] = (J[0] * J[8] - J[2] * J[6]) / det;
  Ji[5] = (J[2] * J[3] - J[0] * J[5]) / det;
  Ji[6] = (J[3] * J[7] - J[4] * J[6]) / det;
  Ji[7] = (J[1] * J[6] - J[0] * J[7]) / det;
  Ji[8] = (J[0] * J[4] - J[1] * J[3]) / det;
}

static void cell_coords(const or_mesh* m, long long cell, int* cx, int* cy, int* cz) {
  *cx = (int)(cell % m->mx);
  *cy = (int)((cell / m->mx) % m->my);
  *cz = (int)(cell / ((long long)m->mx * m->my));
}

/* Per-quadrature-point data of one cell: weight*detJ, basis values and physical gradients.
 * phi[q*nn+i], grad[(q*nn+i)*3+a], wdet[q]. */
typedef struct {
  int n, nn, nq;
  double* wdet;
  double* phi;
  double* grad;
} qdata;

/* quadrature data of a cell of degree p from its nodal coordinates xn (n^3 x 3) */
static int qdata_build_nodes(int p, const double* xn, qdata* d) {
  int n = p + 1, nn = n * n * n, nq = nn;
  or_mesh m1;
  memset(&m1, 0, sizeof(m1));
  m1.p = p;
  const or_mesh* m = &m1;
  double t[OR_MAXN], s[OR_MAXN], w[OR_MAXN];
  ref_nodes01(p, t);
  gauss01(n, s, w);
  d->n = n;
  d->nn = nn;
  d->nq = nq;
  d->wdet = (double*)malloc(sizeof(double) * nq);
  d->phi = (double*)malloc(sizeof(double) * (size_t)nq * nn);
  d->grad = (double*)malloc(sizeof(double) * (size_t)nq * nn * 3);
  if (!d->wdet || !d->phi || !d->grad) return 2;
  int status = 0;
  for (int q3 = 0; q3 < n; ++q3)
    for (int q2 = 0; q2 < n; ++q2)
      for (int q1 = 0; q1 < n; ++q1) {
        int q = (q3 * n + q2) * n + q1;
        double xi[3] = {s[q1], s[q2], s[q3]};
        double J[9], Ji[9];
        or_jacobian(m, xn, xi, J);
        double det = det3(J);
        if (!(det > 0.0)) status = 3;
        inv3(J, det, Ji);
        d->wdet[q] = w[q1] * w[q2] * w[q3] * det;
        for (int k = 0; k < n; ++k)
          for (int j = 0; j < n; ++j)
            for (int i = 0; i < n; ++i) {
              int a = (k * n + j) * n + i;
              double v, g[3];
              basis_eval(t, n, i, j, k, xi, &v, g);
              d->phi[(size_t)q * nn + a] = v;
              /* physical gradient: (grad phi)_c = sum_b g_b (J^{-1})_{b c} */
              for (int c = 0; c < 3; ++c)
                d->grad[((size_t)q * nn + a) * 3 + c] =
                    g[0] * Ji[0 * 3 + c] + g[1] * Ji[1 * 3 + c] + g[2] * Ji[2 * 3 + c];
            }
      }
  return status;
}

static int qdata_build(const or_mesh* m, long long cell, qdata* d) {
  int n = m->p + 1, nn = n * n * n;
  int cx, cy, cz;
  cell_coords(m, cell, &cx, &cy, &cz);
  double* xn = (double*)malloc(sizeof(double) * 3 * nn);
  if (!xn) return 2;
  or_cell_nodes(m, cx, cy, cz, xn);
  int st = qdata_build_nodes(m->p, xn, d);
  free(xn);
  return st;
}

static void qdata_free(qdata* d) {
  free(d->wdet);
  free(d->phi);
  free(d->grad);
}

/* Element matrix, formed entry by entry:
 *   Laplace  K_ij = sum_q w_q detJ_q (J^{-T} grad phi_i).(J^{-T} grad phi_j)
 *   mass     M_ij = sum_q w_q detJ_q phi_i phi_j
 * (Eq. (laplace_operator) and Eq. (mass_operator) with general per-quadrature-point geometry). */
static void element_matrix_from_qdata(const qdata* dp, int op, double* A);

int or_element_matrix(const or_mesh* m, int op, long long cell, double* A) {
  qdata d;
  int st = qdata_build(m, cell, &d);
  if (st == 2) return 2;
  element_matrix_from_qdata(&d, op, A);
  qdata_free(&d);
  return st;
}

static void element_matrix_from_qdata(const qdata* dp, int op, double* A) {
  const qdata d = *dp;
  int nn = d.nn;
  for (long long e = 0; e < (long long)nn * nn; ++e) A[e] = 0.0;
  for (int q = 0; q < d.nq; ++q) {
    double wd = d.wdet[q];
    for (int i = 0; i < nn; ++i)
      for (int j = 0; j < nn; ++j) {
        double v;
        if (op == OR_LAPLACE) {
          const double* gi = d.grad + ((size_t)q * nn + i) * 3;
          const double* gj = d.grad + ((size_t)q * nn + j) * 3;
          v = gi[0] * gj[0] + gi[1] * gj[1] + gi[2] * gj[2];
        } else {
          v = d.phi[(size_t)q * nn + i] * d.phi[(size_t)q * nn + j];
        }
        A[(size_t)i * nn + j] += wd * v;
      }
  }
}

int or_element_row(const or_mesh* m, int op, long long cell, int row, double* out) {
  qdata d;
  int st = qdata_build(m, cell, &d);
  if (st == 2) return 2;
  int nn = d.nn;
  for (int j = 0; j < nn; ++j) out[j] = 0.0;
  for (int q = 0; q < d.nq; ++q) {
    double wd = d.wdet[q];
    for (int j = 0; j < nn; ++j) {
      double v;
      if (op == OR_LAPLACE) {
        const double* gi = d.grad + ((size_t)q * nn + row) * 3;
        const double* gj = d.grad + ((size_t)q * nn + j) * 3;
        v = gi[0] * gj[0] + gi[1] * gj[1] + gi[2] * gj[2];
      } else {
        v = d.phi[(size_t)q * nn + row] * d.phi[(size_t)q * nn + j];
      }
      out[j] += wd * v;
    }
  }
  qdata_free(&d);
  return st;
}

/* ------------------------------------------------------------------------------------------
 * Gather G, scatter G^T (Sec. 2.1), boundary mask and multiplicity.
 * ---------------------------------------------------------------------------------------- */
static long long global_index(const or_mesh* m, long long cell, int i, int j, int k) {
  int cx, cy, cz;
  cell_coords(m, cell, &cx, &cy, &cz);
  long long Nx = (long long)m->mx * m->p + 1, Ny = (long long)m->my * m->p + 1;
  long long gx = (long long)cx * m->p + i, gy = (long long)cy * m->p + j,
            gz = (long long)cz * m->p + k;
  return (gz * Ny + gy) * Nx + gx;
}

void or_gather(const or_mesh* m, const double* xg, double* xc) {
  int n = m->p + 1, nn = n * n * n;
  long long nc = or_n_cells(m);
  for (long long c = 0; c < nc; ++c)
    for (int k = 0; k < n; ++k)
      for (int j = 0; j < n; ++j)
        for (int i = 0; i < n; ++i)
          xc[c * nn + (k * n + j) * n + i] = xg[global_index(m, c, i, j, k)];
}

void or_scatter(const or_mesh* m, const double* yc, double* yg) {
  int n = m->p + 1, nn = n * n * n;
  long long nc = or_n_cells(m), nu = or_n_unique(m);
  for (long long g = 0; g < nu; ++g) yg[g] = 0.0;
  for (long long c = 0; c < nc; ++c)
    for (int k = 0; k < n; ++k)
      for (int j = 0; j < n; ++j)
        for (int i = 0; i < n; ++i)
          yg[global_index(m, c, i, j, k)] += yc[c * nn + (k * n + j) * n + i];
}

void or_boundary_global(const or_mesh* m, unsigned char* is_bnd) {
  long long Nx = (long long)m->mx * m->p + 1, Ny = (long long)m->my * m->p + 1,
            Nz = (long long)m->mz * m->p + 1;
  for (long long gz = 0; gz < Nz; ++gz)
    for (long long gy = 0; gy < Ny; ++gy)
      for (long long gx = 0; gx < Nx; ++gx)
        is_bnd[(gz * Ny + gy) * Nx + gx] = (gx == 0 || gx == Nx - 1 || gy == 0 ||
                                            gy == Ny - 1 || gz == 0 || gz == Nz - 1);
}

/* multiplicity of every cell-wise entry = number of copies of its global node, G^T 1 gathered */
void or_multiplicity(const or_mesh* m, double* mult) {
  long long nc = or_n_cellwise(m), nu = or_n_unique(m);
  double* ones = (double*)malloc(sizeof(double) * nc);
  double* cnt = (double*)malloc(sizeof(double) * nu);
  for (long long e = 0; e < nc; ++e) ones[e] = 1.0;
  or_scatter(m, ones, cnt);
  or_gather(m, cnt, mult);
  free(ones);
  free(cnt);
}

/* ------------------------------------------------------------------------------------------
 * Operators.  Dirichlet (the paper has no boundary conditions; reading: homogeneous Dirichlet
 * by masking rows and columns of boundary nodes, A_D = R^T R A_CG R^T R).
 * ---------------------------------------------------------------------------------------- */
static int local_is_bnd(const or_mesh* m, long long cell, int i, int j, int k) {
  int cx, cy, cz;
  cell_coords(m, cell, &cx, &cy, &cz);
  int p = m->p;
  return (cx * p + i == 0) || (cx * p + i == m->mx * p) || (cy * p + j == 0) ||
         (cy * p + j == m->my * p) || (cz * p + k == 0) || (cz * p + k == m->mz * p);
}

/* y_K = A_K x_K for every cell K (unassembled dual output, Sec. 3.1 "local operator") */
int or_apply_local(const or_mesh* m, int op, const double* xc, double* yc, int nthreads) {
  int n = m->p + 1, nn = n * n * n;
  long long nc = or_n_cells(m);
  int status = 0;
  set_threads(nthreads);
#pragma omp parallel for schedule(dynamic, 1)
  for (long long c = 0; c < nc; ++c) {
    double* A = (double*)malloc(sizeof(double) * (size_t)nn * nn);
    double* xl = (double*)malloc(sizeof(double) * nn);
    int st = or_element_matrix(m, op, c, A);
    if (st) status = st;
    for (int a = 0; a < nn; ++a) {
      int i = a % n, j = (a / n) % n, k = a / (n * n);
      xl[a] = (m->dirichlet && local_is_bnd(m, c, i, j, k)) ? 0.0 : xc[c * nn + a];
    }
    for (int a = 0; a < nn; ++a) {
      int i = a % n, j = (a / n) % n, k = a / (n * n);
      double s = 0.0;
      for (int b = 0; b < nn; ++b) s += A[(size_t)a * nn + b] * xl[b];
      yc[c * nn + a] = (m->dirichlet && local_is_bnd(m, c, i, j, k)) ? 0.0 : s;
    }
    free(A);
    free(xl);
  }
  return status;
}

/* y_glob = A_D x_glob = R ( sum_K G_K^T A_K G_K (R x) )  (Eq. (constrained_system)) */
int or_apply_assembled(const or_mesh* m, int op, const double* xg, double* yg, int nthreads) {
  long long nc = or_n_cellwise(m);
  double* xc = (double*)malloc(sizeof(double) * nc);
  double* yc = (double*)malloc(sizeof(double) * nc);
  if (!xc || !yc) return 2;
  or_gather(m, xg, xc);
  int st = or_apply_local(m, op, xc, yc, nthreads);
  or_scatter(m, yc, yg);
  free(xc);
  free(yc);
  return st;
}

/* DSS, S = G I_Riesz G^T (Eq. (dss_operator)): assemble, read the sums as nodal values, gather */
int or_dss(const or_mesh* m, const double* yc, double* zc) {
  long long nu = or_n_unique(m);
  double* g = (double*)malloc(sizeof(double) * nu);
  if (!g) return 2;
  or_scatter(m, yc, g);
  or_gather(m, g, zc);
  free(g);
  return 0;
}

/* diagonal of A_D, with 1 on Dirichlet nodes (the Jacobi diagonal D_CG, Sec. 3.3) */
int or_diag_global(const or_mesh* m, int op, double* dg, int nthreads) {
  int n = m->p + 1, nn = n * n * n;
  long long nc = or_n_cells(m), nu = or_n_unique(m);
  double* dc = (double*)malloc(sizeof(double) * nc * nn);
  if (!dc) return 2;
  int status = 0;
  set_threads(nthreads);
#pragma omp parallel for schedule(dynamic, 1)
  for (long long c = 0; c < nc; ++c) {
    double* A = (double*)malloc(sizeof(double) * (size_t)nn * nn);
    int st = or_element_matrix(m, op, c, A);
    if (st) status = st;
    for (int a = 0; a < nn; ++a) dc[c * nn + a] = A[(size_t)a * nn + a];
    free(A);
  }
  or_scatter(m, dc, dg);
  if (m->dirichlet) {
    unsigned char* b = (unsigned char*)malloc(nu);
    or_boundary_global(m, b);
    for (long long g = 0; g < nu; ++g)
      if (b[g]) dg[g] = 1.0;
    free(b);
  }
  free(dc);
  return status;
}

int or_element_matrices(const or_mesh* m, int op, long long cell0, long long ncell, double* mats,
                        int nthreads) {
  int n = m->p + 1, nn = n * n * n;
  int status = 0;
  set_threads(nthreads);
#pragma omp parallel for schedule(dynamic, 1)
  for (long long c = 0; c < ncell; ++c) {
    int st = or_element_matrix(m, op, cell0 + c, mats + (size_t)c * nn * nn);
    if (st) status = st;
  }
  return status;
}

/* y_K = A_K x_K with precomputed element matrices for cells cell0 .. cell0+ncell-1;
 * xc and yc hold only those cells (ncell * n^3 entries). */
int or_apply_local_mats(const or_mesh* m, long long cell0, long long ncell, const double* mats,
                        const double* xc, double* yc, int nthreads) {
  int n = m->p + 1, nn = n * n * n;
  set_threads(nthreads);
#pragma omp parallel for schedule(static)
  for (long long c = 0; c < ncell; ++c) {
    const double* A = mats + (size_t)c * nn * nn;
    double xl[OR_MAXN * OR_MAXN * OR_MAXN];
    for (int a = 0; a < nn; ++a) {
      int i = a % n, j = (a / n) % n, k = a / (n * n);
      xl[a] = (m->dirichlet && local_is_bnd(m, cell0 + c, i, j, k)) ? 0.0 : xc[c * nn + a];
    }
    for (int a = 0; a < nn; ++a) {
      int i = a % n, j = (a / n) % n, k = a / (n * n);
      double s = 0.0;
      for (int b = 0; b < nn; ++b) s += A[(size_t)a * nn + b] * xl[b];
      yc[c * nn + a] = (m->dirichlet && local_is_bnd(m, cell0 + c, i, j, k)) ? 0.0 : s;
    }
  }
  return 0;
}

/* ------------------------------------------------------------------------------------------
 * CSR assembly of A_CG = G^T blockdiag(A_K) G (unconstrained).  Row g couples to every node of
 * every cell containing g; per axis that is a contiguous index range, so the columns of a row
 * are the Cartesian product of three ranges (stored in ascending order).
 * ---------------------------------------------------------------------------------------- */
static void axis_range(long long g, int p, int mcells, long long* lo, long long* hi) {
  long long c0, c1; /* first and last cell along the axis containing node g */
  if (g % p == 0) {
    c0 = g / p - 1;
    c1 = g / p;
  } else {
    c0 = g / p;
    c1 = g / p;
  }
  if (c0 < 0) c0 = 0;
  if (c1 > mcells - 1) c1 = mcells - 1;
  *lo = c0 * p;
  *hi = c1 * p + p;
}

long long or_csr_nnz(const or_mesh* m) {
  long long Nx = (long long)m->mx * m->p + 1, Ny = (long long)m->my * m->p + 1,
            Nz = (long long)m->mz * m->p + 1;
  long long sx = 0, sy = 0, sz = 0, lo, hi;
  for (long long g = 0; g < Nx; ++g) {
    axis_range(g, m->p, m->mx, &lo, &hi);
    sx += hi - lo + 1;
  }
  for (long long g = 0; g < Ny; ++g) {
    axis_range(g, m->p, m->my, &lo, &hi);
    sy += hi - lo + 1;
  }
  for (long long g = 0; g < Nz; ++g) {
    axis_range(g, m->p, m->mz, &lo, &hi);
    sz += hi - lo + 1;
  }
  return sx * sy * sz;
}

int or_assemble_csr(const or_mesh* m, int op, long long* rowptr, int* colidx, double* vals,
                    int nthreads) {
  int p = m->p, n = p + 1, nn = n * n * n;
  long long Nx = (long long)m->mx * p + 1, Ny = (long long)m->my * p + 1,
            Nz = (long long)m->mz * p + 1;
  long long nu = Nx * Ny * Nz, nc = or_n_cells(m);
  double* mats = (double*)malloc(sizeof(double) * (size_t)nc * nn * nn);
  if (!mats) return 2;
  int st = or_element_matrices(m, op, 0, nc, mats, nthreads);
  /* row pointers */
  rowptr[0] = 0;
  for (long long g = 0; g < nu; ++g) {
    long long gx = g % Nx, gy = (g / Nx) % Ny, gz = g / (Nx * Ny), lx, hx, ly, hy, lz, hz;
    axis_range(gx, p, m->mx, &lx, &hx);
    axis_range(gy, p, m->my, &ly, &hy);
    axis_range(gz, p, m->mz, &lz, &hz);
    rowptr[g + 1] = rowptr[g] + (hx - lx + 1) * (hy - ly + 1) * (hz - lz + 1);
  }
  set_threads(nthreads);
#pragma omp parallel for schedule(dynamic, 64)
  for (long long g = 0; g < nu; ++g) {
    long long gx = g % Nx, gy = (g / Nx) % Ny, gz = g / (Nx * Ny), lx, hx, ly, hy, lz, hz;
    axis_range(gx, p, m->mx, &lx, &hx);
    axis_range(gy, p, m->my, &ly, &hy);
    axis_range(gz, p, m->mz, &lz, &hz);
    long long wx = hx - lx + 1, wy = hy - ly + 1;
    long long base = rowptr[g];
    for (long long z = lz; z <= hz; ++z)
      for (long long y = ly; y <= hy; ++y)
        for (long long x = lx; x <= hx; ++x) {
          long long pos = base + ((z - lz) * wy + (y - ly)) * wx + (x - lx);
          colidx[pos] = (int)((z * Ny + y) * Nx + x);
          vals[pos] = 0.0;
        }
    /* every cell containing g contributes its element-matrix row */
    for (long long cz = lz / p; cz < hz / p; ++cz)
      for (long long cy = ly / p; cy < hy / p; ++cy)
        for (long long cx = lx / p; cx < hx / p; ++cx) {
          long long cell = (cz * m->my + cy) * m->mx + cx;
          int i = (int)(gx - cx * p), j = (int)(gy - cy * p), k = (int)(gz - cz * p);
          const double* A = mats + (size_t)cell * nn * nn + (size_t)((k * n + j) * n + i) * nn;
          for (int kk = 0; kk < n; ++kk)
            for (int jj = 0; jj < n; ++jj)
              for (int ii = 0; ii < n; ++ii) {
                long long x = cx * p + ii, y = cy * p + jj, z = cz * p + kk;
                long long pos = base + ((z - lz) * wy + (y - ly)) * wx + (x - lx);
                vals[pos] += A[(kk * n + jj) * n + ii];
              }
        }
  }
  free(mats);
  return st;
}

void or_csr_spmv(long long nrows, const long long* rowptr, const int* colidx, const double* vals,
                 const double* x, double* y) {
#pragma omp parallel for schedule(static)
  for (long long r = 0; r < nrows; ++r) {
    double s = 0.0;
    for (long long e = rowptr[r]; e < rowptr[r + 1]; ++e) s += vals[e] * x[colidx[e]];
    y[r] = s;
  }
}

/* ------------------------------------------------------------------------------------------
 * Right-hand side and error.  Manufactured problems for -Laplace(u) = f on the unit cube with
 * u = 0 on the boundary:
 *   sine:      u = sin(pi x) sin(pi y) sin(pi z),  f = 3 pi^2 u
 *   quadratic: u = x(1-x) y(1-y) z(1-z),           f = 2 [y(1-y)z(1-z) + x(1-x)z(1-z) + x(1-x)y(1-y)]
 * ---------------------------------------------------------------------------------------- */
static double exact_u(int kind, const double x[3]) {
  if (kind == OR_RHS_SINE) return sin(OR_PI * x[0]) * sin(OR_PI * x[1]) * sin(OR_PI * x[2]);
  return x[0] * (1.0 - x[0]) * x[1] * (1.0 - x[1]) * x[2] * (1.0 - x[2]);
}

static double exact_f(int kind, const double x[3]) {
  if (kind == OR_RHS_SINE) return 3.0 * OR_PI * OR_PI * exact_u(kind, x);
  double a = x[0] * (1.0 - x[0]), b = x[1] * (1.0 - x[1]), c = x[2] * (1.0 - x[2]);
  return 2.0 * (b * c + a * c + a * b);
}

/* unassembled dual load b_K,i = sum_q w_q detJ_q f(x(xi_q)) phi_i(xi_q) */
int or_rhs(const or_mesh* m, int kind, double* bc) {
  int n = m->p + 1, nn = n * n * n;
  long long nc = or_n_cells(m);
  int status = 0;
#pragma omp parallel for schedule(dynamic, 1)
  for (long long c = 0; c < nc; ++c) {
    int cx, cy, cz;
    cell_coords(m, c, &cx, &cy, &cz);
    qdata d;
    int st = qdata_build(m, c, &d);
    if (st) status = st;
    double* xn = (double*)malloc(sizeof(double) * 3 * nn);
    or_cell_nodes(m, cx, cy, cz, xn);
    for (int a = 0; a < nn; ++a) bc[c * nn + a] = 0.0;
    for (int q = 0; q < nn; ++q) {
      double x[3] = {0.0, 0.0, 0.0};
      for (int a = 0; a < nn; ++a)
        for (int e = 0; e < 3; ++e) x[e] += xn[3 * a + e] * d.phi[(size_t)q * nn + a];
      double fw = d.wdet[q] * exact_f(kind, x);
      for (int a = 0; a < nn; ++a) bc[c * nn + a] += fw * d.phi[(size_t)q * nn + a];
    }
    free(xn);
    qdata_free(&d);
  }
  return status;
}

/* exact solution sampled at the (physical) global nodes */
void or_exact_nodal(const or_mesh* m, int kind, double* ug) {
  int p = m->p;
  double t[OR_MAXN];
  ref_nodes01(p, t);
  long long Nx = (long long)m->mx * p + 1, Ny = (long long)m->my * p + 1,
            Nz = (long long)m->mz * p + 1;
  for (long long gz = 0; gz < Nz; ++gz)
    for (long long gy = 0; gy < Ny; ++gy)
      for (long long gx = 0; gx < Nx; ++gx) {
        long long c[3], l[3], g[3] = {gx, gy, gz};
        int mm[3] = {m->mx, m->my, m->mz};
        double X[3], x[3];
        for (int e = 0; e < 3; ++e) {
          c[e] = g[e] / p;
          if (c[e] > mm[e] - 1) c[e] = mm[e] - 1;
          l[e] = g[e] - c[e] * p;
          X[e] = (c[e] + t[l[e]]) / mm[e];
        }
        or_map(m->amp, X, x);
        ug[(gz * Ny + gy) * Nx + gx] = exact_u(kind, x);
      }
}

/* L2 error sum_K sum_q w_q detJ (u_h - u)^2 with an (n+2)-point Gauss rule per direction */
int or_l2_error(const or_mesh* m, int kind, const double* uc, double* err) {
  int n = m->p + 1, nn = n * n * n, nq1 = n + 2;
  long long nc = or_n_cells(m);
  double t[OR_MAXN], s[64], w[64];
  ref_nodes01(m->p, t);
  gauss01(nq1, s, w);
  double total = 0.0;
  for (long long c = 0; c < nc; ++c) {
    int cx, cy, cz;
    cell_coords(m, c, &cx, &cy, &cz);
    double* xn = (double*)malloc(sizeof(double) * 3 * nn);
    or_cell_nodes(m, cx, cy, cz, xn);
    for (int q3 = 0; q3 < nq1; ++q3)
      for (int q2 = 0; q2 < nq1; ++q2)
        for (int q1 = 0; q1 < nq1; ++q1) {
          double xi[3] = {s[q1], s[q2], s[q3]};
          double J[9], x[3] = {0, 0, 0}, uh = 0.0;
          or_jacobian(m, xn, xi, J);
          for (int k = 0; k < n; ++k)
            for (int j = 0; j < n; ++j)
              for (int i = 0; i < n; ++i) {
                int a = (k * n + j) * n + i;
                double v, g[3];
                basis_eval(t, n, i, j, k, xi, &v, g);
                uh += uc[c * nn + a] * v;
                for (int e = 0; e < 3; ++e) x[e] += xn[3 * a + e] * v;
              }
          double diff = uh - exact_u(kind, x);
          total += w[q1] * w[q2] * w[q3] * det3(J) * diff * diff;
        }
    free(xn);
  }
  *err = sqrt(total);
  return 0;
}

/* ------------------------------------------------------------------------------------------
 * Assembled Jacobi-PCG / FCG on A_D u = b (the "standard FCG applied to the explicitly assembled
 * minimal global system" of Theorem "Equivalence of Communication-Free FCG"), following the
 * steps of Algorithm "Communication-Free (Flexible) PCG" on global vectors.  Convergence
 * (unspecified in the paper): ||r||_2 / ||b||_2 <= rtol.  alpha[k], beta[k] for k < iters;
 * relres[k] for k <= iters (relres[0] is the initial residual).
 * Returns 0 converged, 4 not converged at maxit, 5 breakdown (<q,p> <= 0 or not finite).
 * ---------------------------------------------------------------------------------------- */
static double dot(long long n, const double* a, const double* b) {
  double s = 0.0;
  for (long long i = 0; i < n; ++i) s += a[i] * b[i];
  return s;
}

int or_cg(const or_mesh* m, int op, const double* bg, double* xg, const or_cg_opts* o, int* iters,
          double* alpha, double* beta, double* relres, int nthreads) {
  long long nu = or_n_unique(m);
  long long nnz = or_csr_nnz(m);
  long long* rowptr = (long long*)malloc(sizeof(long long) * (nu + 1));
  int* col = (int*)malloc(sizeof(int) * nnz);
  double* val = (double*)malloc(sizeof(double) * nnz);
  double *d = (double*)malloc(sizeof(double) * nu), *r = (double*)malloc(sizeof(double) * nu),
         *z = (double*)malloc(sizeof(double) * nu), *pv = (double*)malloc(sizeof(double) * nu),
         *q = (double*)malloc(sizeof(double) * nu), *b = (double*)malloc(sizeof(double) * nu),
         *t = (double*)malloc(sizeof(double) * nu);
  unsigned char* bnd = (unsigned char*)malloc(nu);
  if (!rowptr || !col || !val || !d || !r || !z || !pv || !q || !b || !t || !bnd) return 2;
  or_assemble_csr(m, op, rowptr, col, val, nthreads);
  or_diag_global(m, op, d, nthreads);
  or_boundary_global(m, bnd);
  int dir = m->dirichlet;
  /* A_D v = R A_CG R v */
#define APPLY_AD(src, dst)                                                   \
  do {                                                                       \
    for (long long g = 0; g < nu; ++g) t[g] = (dir && bnd[g]) ? 0.0 : src[g]; \
    or_csr_spmv(nu, rowptr, col, val, t, dst);                               \
    if (dir)                                                                 \
      for (long long g = 0; g < nu; ++g)                                     \
        if (bnd[g]) dst[g] = 0.0;                                            \
  } while (0)
  for (long long g = 0; g < nu; ++g) {
    b[g] = (dir && bnd[g]) ? 0.0 : bg[g];
    if (dir && bnd[g]) xg[g] = 0.0;
  }
  double bnorm = sqrt(dot(nu, b, b));
  APPLY_AD(xg, q);
  for (long long g = 0; g < nu; ++g) r[g] = b[g] - q[g];
  double rn = sqrt(dot(nu, r, r));
  relres[0] = bnorm > 0.0 ? rn / bnorm : 0.0;
  int status = 4, k = 0;
  if (bnorm == 0.0 || relres[0] <= o->rtol) {
    status = 0;
  } else {
    for (long long g = 0; g < nu; ++g) z[g] = r[g] / d[g];
    for (long long g = 0; g < nu; ++g) pv[g] = z[g];
    double rz = dot(nu, r, z);
    for (k = 0; k < o->maxit; ++k) {
      APPLY_AD(pv, q);
      double qp = dot(nu, q, pv);
      if (!(qp > 0.0) || !isfinite(qp)) {
        status = 5;
        break;
      }
      double a = rz / qp;
      alpha[k] = a;
      for (long long g = 0; g < nu; ++g) xg[g] += a * pv[g];
      for (long long g = 0; g < nu; ++g) r[g] -= a * q[g];
      rn = sqrt(dot(nu, r, r));
      relres[k + 1] = rn / bnorm;
      if (relres[k + 1] <= o->rtol) {
        status = 0;
        ++k;
        break;
      }
      for (long long g = 0; g < nu; ++g) z[g] = r[g] / d[g];
      double rz_new = dot(nu, r, z), bt;
      if (o->flexible)
        bt = -dot(nu, q, z) / qp;
      else
        bt = rz_new / rz;
      beta[k] = bt;
      rz = rz_new;
      for (long long g = 0; g < nu; ++g) pv[g] = z[g] + bt * pv[g];
    }
  }
#undef APPLY_AD
  *iters = k;
  free(rowptr);
  free(col);
  free(val);
  free(d);
  free(r);
  free(z);
  free(pv);
  free(q);
  free(b);
  free(t);
  free(bnd);
  return status;
}

/* ------------------------------------------------------------------------------------------
 * Block-structured meshes (Sec. 4.2 "Generalization to Block-Structured Grids"): macro-blocks,
 * each a structured grid of cells whose geometry is the trilinear map of its eight corner
 * vertices.  The global (unique) numbering is found from the nodes' physical coordinates --
 * conforming blocks place shared nodes at the same points -- so it knows nothing of faces,
 * orientations or sharing lists.
 * ---------------------------------------------------------------------------------------- */
long long or_mb_n_cellwise(const or_mb* mb) {
  long long n3 = (long long)(mb->p + 1) * (mb->p + 1) * (mb->p + 1), c = 0;
  for (int b = 0; b < mb->nblocks; ++b)
    c += (long long)mb->dims[3 * b] * mb->dims[3 * b + 1] * mb->dims[3 * b + 2];
  return c * n3;
}

long long or_mb_cell_offset(const or_mb* mb, int block) {
  long long c = 0;
  for (int b = 0; b < block; ++b)
    c += (long long)mb->dims[3 * b] * mb->dims[3 * b + 1] * mb->dims[3 * b + 2];
  return c;
}

/* x(xi) = sum_c N_c(xi) X_c over the corners c = i + 2j + 4k at xi = (i, j, k) */
static void trilinear(const or_mb* mb, int block, const double xi[3], double x[3]) {
  for (int a = 0; a < 3; ++a) x[a] = 0.0;
  for (int c = 0; c < 8; ++c) {
    double w = ((c & 1) ? xi[0] : 1.0 - xi[0]) * ((c & 2) ? xi[1] : 1.0 - xi[1]) *
               ((c & 4) ? xi[2] : 1.0 - xi[2]);
    const double* X = mb->vxyz + 3 * mb->block_verts[8 * block + c];
    for (int a = 0; a < 3; ++a) x[a] += w * X[a];
  }
}

void or_mb_cell_nodes(const or_mb* mb, int block, int cx, int cy, int cz, double* xn) {
  int n = mb->p + 1;
  const int* d = mb->dims + 3 * block;
  double t[OR_MAXN];
  ref_nodes01(mb->p, t);
  for (int k = 0; k < n; ++k)
    for (int j = 0; j < n; ++j)
      for (int i = 0; i < n; ++i) {
        double xi[3] = {(cx + t[i]) / d[0], (cy + t[j]) / d[1], (cz + t[k]) / d[2]};
        trilinear(mb, block, xi, xn + 3 * ((k * n + j) * n + i));
      }
}

/* block and cell coordinates of a cell numbered over all blocks */
static void mb_cell(const or_mb* mb, long long cell, int* block, int* cx, int* cy, int* cz) {
  int b = 0;
  long long c = cell;
  for (;;) {
    long long nb = (long long)mb->dims[3 * b] * mb->dims[3 * b + 1] * mb->dims[3 * b + 2];
    if (c < nb || b == mb->nblocks - 1) break;
    c -= nb;
    ++b;
  }
  const int* d = mb->dims + 3 * b;
  *block = b;
  *cx = (int)(c % d[0]);
  *cy = (int)((c / d[0]) % d[1]);
  *cz = (int)(c / ((long long)d[0] * d[1]));
}

int or_mb_element_matrix(const or_mb* mb, int op, long long cell, double* A) {
  int n = mb->p + 1, nn = n * n * n, b, cx, cy, cz;
  mb_cell(mb, cell, &b, &cx, &cy, &cz);
  double* xn = (double*)malloc(sizeof(double) * 3 * nn);
  if (!xn) return 2;
  or_mb_cell_nodes(mb, b, cx, cy, cz, xn);
  qdata d;
  int st = qdata_build_nodes(mb->p, xn, &d);
  free(xn);
  if (st == 2) return 2;
  element_matrix_from_qdata(&d, op, A);
  qdata_free(&d);
  return st;
}

int or_mb_apply_local(const or_mb* mb, int op, const double* xc, double* yc, int nthreads) {
  int n = mb->p + 1, nn = n * n * n;
  long long nc = or_mb_n_cellwise(mb) / nn;
  int status = 0;
  set_threads(nthreads);
#pragma omp parallel for schedule(dynamic, 1)
  for (long long c = 0; c < nc; ++c) {
    double* A = (double*)malloc(sizeof(double) * (size_t)nn * nn);
    int st = or_mb_element_matrix(mb, op, c, A);
    if (st) status = st;
    for (int a = 0; a < nn; ++a) {
      double s = 0.0;
      for (int b = 0; b < nn; ++b) s += A[(size_t)a * nn + b] * xc[c * nn + b];
      yc[c * nn + a] = s;
    }
    free(A);
  }
  return status;
}

typedef struct {
  double x[3];
  long long idx;
} mb_pt;

static int cmp_pt(const void* a, const void* b) {
  const mb_pt* p = (const mb_pt*)a;
  const mb_pt* q = (const mb_pt*)b;
  for (int d = 0; d < 3; ++d) {
    if (p->x[d] < q->x[d]) return -1;
    if (p->x[d] > q->x[d]) return 1;
  }
  return (p->idx > q->idx) - (p->idx < q->idx);
}

static long long uf_find(long long* par, long long i) {
  while (par[i] != i) {
    par[i] = par[par[i]];
    i = par[i];
  }
  return i;
}

/* gid[e] for every cell-wise entry e: nodes closer than tol get the same number; numbers follow
 * the ascending (x, y, z) order of the nodes.  Returns the unique count (< 0 on failure). */
long long or_mb_numbering(const or_mb* mb, double tol, long long* gid) {
  int n = mb->p + 1, nn = n * n * n;
  long long ncw = or_mb_n_cellwise(mb), nc = ncw / nn;
  mb_pt* pts = (mb_pt*)malloc(sizeof(mb_pt) * ncw);
  long long* par = (long long*)malloc(sizeof(long long) * ncw);
  double* xn = (double*)malloc(sizeof(double) * 3 * nn);
  if (!pts || !par || !xn) return -1;
  for (long long c = 0; c < nc; ++c) {
    int b, cx, cy, cz;
    mb_cell(mb, c, &b, &cx, &cy, &cz);
    or_mb_cell_nodes(mb, b, cx, cy, cz, xn);
    for (int a = 0; a < nn; ++a) {
      long long e = c * nn + a;
      for (int d = 0; d < 3; ++d) pts[e].x[d] = xn[3 * a + d];
      pts[e].idx = e;
    }
  }
  qsort(pts, (size_t)ncw, sizeof(mb_pt), cmp_pt);
  for (long long e = 0; e < ncw; ++e) par[e] = e;
  /* nodes within tol of each other are neighbours in the x-sorted order up to an x-window */
  for (long long i = 0; i < ncw; ++i)
    for (long long j = i + 1; j < ncw && pts[j].x[0] - pts[i].x[0] <= tol; ++j)
      if (fabs(pts[j].x[1] - pts[i].x[1]) <= tol && fabs(pts[j].x[2] - pts[i].x[2]) <= tol) {
        long long ri = uf_find(par, i), rj = uf_find(par, j);
        if (ri != rj) par[rj < ri ? ri : rj] = rj < ri ? rj : ri;
      }
  long long nu = 0;
  long long* rootid = (long long*)malloc(sizeof(long long) * ncw);
  if (!rootid) return -1;
  for (long long i = 0; i < ncw; ++i) rootid[i] = -1;
  for (long long i = 0; i < ncw; ++i) {
    long long r = uf_find(par, i);
    if (rootid[r] < 0) rootid[r] = nu++;
    gid[pts[i].idx] = rootid[r];
  }
  free(rootid);
  free(pts);
  free(par);
  free(xn);
  return nu;
}
