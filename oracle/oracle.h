/*
 * oracle.h -- plain, slow FP64 CPU oracle for the cell-wise matrix-free finite-element path.
 *
 * TEST INFRASTRUCTURE ONLY.  Only the tests, the smoke check and the CPU-baseline leg of the
 * benchmark may load this library.  It shares no code, header, table or constant generator
 * with the CUDA library: it is written from the definitions of the method
 * ("Coalesced Matrix-Free Finite Elements in Cell-Wise Storage"):
 *   - discrete problem A u = f, gather G, scatter G^T           (Sec. 2, Sec. 2.1)
 *   - element operators, mass and Laplace                       (Sec. 2.3, Eq. (mass_operator),
 *                                                                Eq. (laplace_operator))
 *   - constrained system C^T A C u = C^T b, A_CG = G^T A G      (Sec. 3.1, Eq. (constrained_system))
 *   - DSS S = G I_Riesz G^T and Jacobi P = D_cell^{-1} S         (Sec. 3.3, Eq. (dss_operator))
 *   - (flexible) PCG                                             (Algorithm "Communication-Free
 *                                                                (Flexible) PCG", Sec. 3.2)
 *
 * Conventions (shared with the test harness, not with the CUDA path):
 *   degree p in [1,7], n = p+1 nodes (GLL) and n Gauss points per direction;
 *   mesh: mx*my*mz hexahedral cells of the unit cube, cell (cx,cy,cz) covers
 *   [cx/mx,(cx+1)/mx] x ... before the map Phi(X) = X + amp*sin(pi X)sin(pi Y)sin(pi Z)*(1,1,1);
 *   canonical cell-wise index   ((cz*my+cy)*mx+cx)*n^3 + (k*n+j)*n+i   (local node (i,j,k), i fastest);
 *   global (unique) index       (gz*Ny+gy)*Nx+gx with Nx = mx*p+1 etc., gx = cx*p+i.
 * Every floating-point routine works in double precision; sums run sequentially.
 */
#ifndef FE_ORACLE_H
#define FE_ORACLE_H
#ifdef __cplusplus
extern "C" {
#endif

#define OR_LAPLACE 0
#define OR_MASS 1

#define OR_RHS_SINE 0      /* f = 3 pi^2 sin(pi x) sin(pi y) sin(pi z), u = sin sin sin       */
#define OR_RHS_QUADRATIC 1 /* u = prod x_a (1-x_a),  f = -Laplace(u)                          */

typedef struct {
  int mx, my, mz; /* cells per direction */
  int p;          /* polynomial degree, 1..7 */
  double amp;     /* deformation amplitude (0 = affine) */
  int dirichlet;  /* 1 = homogeneous Dirichlet on the whole boundary */
} or_mesh;

/* ---- 1D rules ---- */
int or_gauss(int n, double* x, double* w); /* Gauss-Legendre on [-1,1], ascending */
int or_gll(int p, double* x);              /* p+1 Gauss-Lobatto-Legendre nodes on [-1,1] */
double or_lagrange(const double* t, int n, int i, double s);
double or_lagrange_deriv(const double* t, int n, int i, double s);

/* ---- counts ---- */
long long or_n_cells(const or_mesh* m);
long long or_n_cellwise(const or_mesh* m);
long long or_n_unique(const or_mesh* m);

/* ---- geometry ---- */
void or_map(double amp, const double X[3], double x[3]);
void or_cell_nodes(const or_mesh* m, int cx, int cy, int cz, double* xn /* n^3 x 3 */);
void or_jacobian(const or_mesh* m, const double* xn, const double xi[3], double J[9]);

/* ---- element level ---- */
int or_element_matrix(const or_mesh* m, int op, long long cell, double* A /* n^3 x n^3 */);
int or_element_row(const or_mesh* m, int op, long long cell, int row, double* out /* n^3 */);

/* ---- gather / scatter / masks ---- */
void or_gather(const or_mesh* m, const double* xg, double* xc);
void or_scatter(const or_mesh* m, const double* yc, double* yg);
void or_boundary_global(const or_mesh* m, unsigned char* is_bnd);
void or_multiplicity(const or_mesh* m, double* mult_cellwise);

/* ---- operators ---- */
int or_apply_local(const or_mesh* m, int op, const double* xc, double* yc, int nthreads);
int or_apply_assembled(const or_mesh* m, int op, const double* xg, double* yg, int nthreads);
int or_dss(const or_mesh* m, const double* yc, double* zc);
int or_diag_global(const or_mesh* m, int op, double* dg, int nthreads);

/* precomputed element matrices for a contiguous range of cells (CPU-baseline timing) */
int or_element_matrices(const or_mesh* m, int op, long long cell0, long long ncell, double* mats,
                        int nthreads);
int or_apply_local_mats(const or_mesh* m, long long cell0, long long ncell, const double* mats,
                        const double* xc, double* yc, int nthreads);

/* ---- CSR assembly of A_CG (unconstrained) ---- */
long long or_csr_nnz(const or_mesh* m);
int or_assemble_csr(const or_mesh* m, int op, long long* rowptr, int* colidx, double* vals,
                    int nthreads);
void or_csr_spmv(long long nrows, const long long* rowptr, const int* colidx, const double* vals,
                 const double* x, double* y);

/* ---- right-hand side, exact solution, error ---- */
int or_rhs(const or_mesh* m, int kind, double* bc);
void or_exact_nodal(const or_mesh* m, int kind, double* ug);
int or_l2_error(const or_mesh* m, int kind, const double* uc, double* err);

/* ---- assembled Jacobi-PCG / FCG on the global (unique) system ---- */
typedef struct {
  double rtol;
  int maxit;
  int flexible;
} or_cg_opts;
int or_cg(const or_mesh* m, int op, const double* bg, double* xg, const or_cg_opts* o, int* iters,
          double* alpha, double* beta, double* relres, int nthreads);

/* ---- block-structured meshes (Sec. 4.2): trilinear macro-blocks, numbering by coordinates ---- */
typedef struct {
  int nblocks, p;
  const int* dims;        /* 3 per block: cells along the block's local x, y, z */
  const int* block_verts; /* 8 per block: macro-vertex of local corner c = i + 2j + 4k */
  const double* vxyz;     /* 3 per macro-vertex */
} or_mb;
long long or_mb_n_cellwise(const or_mb* mb);
long long or_mb_cell_offset(const or_mb* mb, int block);
void or_mb_cell_nodes(const or_mb* mb, int block, int cx, int cy, int cz, double* xn);
int or_mb_element_matrix(const or_mb* mb, int op, long long cell, double* A);
int or_mb_apply_local(const or_mb* mb, int op, const double* xc, double* yc, int nthreads);
long long or_mb_numbering(const or_mb* mb, double tol, long long* gid);

#ifdef __cplusplus
}
#endif
#endif
