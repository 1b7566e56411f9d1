/*
 * fe.h -- C ABI of libfe: matrix-free high-order finite elements in persistent cell-wise storage
 * on one GB300 GPU (hand-written CUDA for sm_103a).
 *
 * Method: "Coalesced Matrix-Free Finite Elements in Cell-Wise Storage".  Every field lives
 * persistently in the redundant cell-wise representation V_cell (primal) / V_cell* (dual)
 * (Sec. 2.2); the local operator A : V_cell -> V_cell* is applied cell by cell with sum
 * factorization (Sec. 2.3, Eq. (mass_operator), Eq. (laplace_operator)); continuity is restored
 * only by the direct stiffness summation S = G I_Riesz G^T (Sec. 3.3, Eq. (dss_operator)),
 * realised as dimension-split one-to-one face exchanges without atomics (Sec. 4.1, Algorithm
 * "Dimensionally-Split Structured Summation"); Krylov solves run on cell-wise data (Sec. 3.2,
 * Algorithm "Communication-Free (Flexible) PCG").
 *
 * Conventions
 *  - Mesh: mx*my*mz hexahedra of the unit cube, deformed by
 *    Phi(X) = X + deform_amp * sin(pi X) sin(pi Y) sin(pi Z) * (1,1,1), sampled at the
 *    Gauss-Lobatto-Legendre (GLL) nodes of every cell and interpolated isoparametrically with
 *    Q_p; n = p+1 GLL nodes and n Gauss points per direction.
 *  - Cell-wise layout (layout_id 0): cell-major, cells in lexicographic order
 *    (cell = (cz*my + cy)*mx + cx), each cell's n^3 values contiguous with local node
 *    (i,j,k) at (k*n + j)*n + i.  Element e of a cell-wise vector is cell e / n^3, node e % n^3.
 *  - Vectors are caller-owned DEVICE memory of `cellwise_len` elements: double for FE_F64,
 *    float for the other precisions.  Pointers must be 16-byte aligned.  HOST arrays appear only
 *    where a declaration says so (fe_gather, fe_apply_host, the server, CG histories).
 *    Library-owned state (geometry, tables, solver workspaces, staging buffers) lives inside the
 *    opaque fe_mesh / fe_mbmesh / fe_amr / fe_server objects.
 *  - `stream` is a cudaStream_t (NULL = legacy default stream).  Calls are asynchronous on it
 *    unless stated otherwise.
 *  - Errors: every call returns an fe_status; fe_last_error() gives a thread-local message.
 *    No exception crosses the ABI.  A CUDA error from a launch is reported as FE_ERR_CUDA.
 *  - Dirichlet (the paper has no boundary conditions; reading used here): when the mesh is
 *    created with dirichlet = 1, rows and columns of boundary nodes are masked, i.e. the
 *    operator is A_D = R^T R A_CG R^T R; every copy of a boundary node is zero in the output of
 *    fe_apply, and the Jacobi diagonal is 1 there.
 */
#ifndef LIBFE_FE_H
#define LIBFE_FE_H
#include <stddef.h>
#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  FE_OK = 0,
  FE_ERR_INVALID = 1,       /* bad argument: null/misaligned pointer, degree outside [1,7], ... */
  FE_ERR_OOM = 2,           /* device allocation failed, or request over the memory budget */
  FE_ERR_CUDA = 3,          /* CUDA runtime or launch error */
  FE_ERR_NOT_CONVERGED = 4, /* CG reached maxit */
  FE_ERR_BREAKDOWN = 5,     /* CG breakdown: <q,p> <= 0 or a non-finite scalar */
  FE_ERR_TIMEOUT = 6,       /* a bounded device-side wait ran out */
  FE_ERR_BUSY = 7,          /* fe_serve_poll: the request is still pending */
  FE_ERR_COMM = 8           /* a communication callback of an fe_comm returned non-zero */
} fe_status;

typedef enum { FE_LAPLACE = 0, FE_MASS = 1 } fe_op;

/* Arithmetic of a call.  FE_F64: double storage, FP64-accurate arithmetic (see FE_NATIVE_F64).
 * FE_F32: float storage and float arithmetic.  FE_BF16_F32ACC / FE_F16_F32ACC: float vectors, but
 * every operand of a product in the contractions is rounded to bf16 / fp16 and the products
 * accumulate in FP32 (Sec. 3.2's reduced-precision preconditioner; stored geometry only; the
 * stored metric is kept in the 16-bit format scaled by a power of two).  For n = p+1 = 2..4 on
 * FE_LAYOUT_CELLS meshes the contractions run on the tensor cores as two dense products per cell
 * (the 3n^3 x n^3 Kronecker gradient matrix, or the n^3 x n^3 interpolation matrix for mass,
 * entries rounded once; the metric product in FP32); otherwise, or with FE_LOWP_FMA=1 in the
 * environment, as sum-factorized sweeps on the FMA pipe with every sweep value rounded. */
typedef enum { FE_F64 = 0, FE_F32 = 1, FE_BF16_F32ACC = 2, FE_F16_F32ACC = 3 } fe_prec;

/* Geometry representation (Sec. 2.3 and Sec. 6.2: "per-quadrature-point Jacobians"):
 *  STORED    -- w_q detJ J^{-1}J^{-T} (6 symmetric entries, Laplace) and w_q detJ (mass) per
 *               quadrature point, precomputed by fe_mesh_create;
 *  RECOMPUTE -- only the cell-wise nodal coordinates are stored (3 values per cell node, as
 *               offsets from the cell's first node); each apply forms J and the metric from them,
 *               chunk by chunk into an L2-sized library scratch of the mesh, so applies on one
 *               RECOMPUTE mesh must not run concurrently on different streams.  Not accepted by
 *               fe_cg_solve_batched and the request server;
 *  AFFINE    -- undeformed Cartesian mesh (deform_amp must be 0): one diagonal J for all cells,
 *               the paper's "scalar h" setting. */
enum { FE_GEOM_STORED = 0, FE_GEOM_RECOMPUTE = 1, FE_GEOM_AFFINE = 2 };

/* fe_apply flags */
#define FE_ASSEMBLE 1u   /* y = S(A x): continuous output equal to G A_D x_glob when x = G x_glob */
#define FE_NATIVE_F64 2u /* FE_F64 only: use the FP64 pipe instead of double-float arithmetic on
                            the FP32 pipe (reference variant; slow on GB300) */

typedef struct {
  int mx, my, mz;    /* cells per direction, each >= 1 */
  int degree;        /* p in [1, 7] */
  double deform_amp; /* amplitude of the sine deformation (0 = affine) */
  int geom_mode;     /* FE_GEOM_* */
  int dirichlet;     /* 1 = homogeneous Dirichlet on the whole boundary */
  int device;        /* CUDA device ordinal */
  int layout;        /* storage of cell-wise vectors: FE_LAYOUT_CELLS or FE_LAYOUT_PACKED2 */
} fe_mesh_desc;

/* Storage layouts (Sec. 2.2 "Persistent cell-wise storage", Table "tab:memory_overhead").
 *  FE_LAYOUT_CELLS   (0) -- one cell per storage unit: cell-major, cells lexicographic, n^3 values
 *                          per cell, local node (i,j,k) at (k n + j) n + i.
 *  FE_LAYOUT_PACKED2 (1) -- a 2x2x2 cluster of cells per storage unit with its interior interface
 *                          nodes stored once: units lexicographic over (mx/2, my/2, mz/2),
 *                          (2p+1)^3 values per unit, local node (i,j,k) at (k N + j) N + i with
 *                          N = 2p+1.  Even cell counts, degree 1 to 3, FE_GEOM_STORED or
 *                          FE_GEOM_AFFINE.  fe_apply (its unassembled output is assembled inside
 *                          each unit), fe_dss and fe_pairing accept it; the solvers, fe_diag,
 *                          fe_gather, fe_rhs and fe_l2_error take FE_LAYOUT_CELLS meshes only. */
enum { FE_LAYOUT_CELLS = 0, FE_LAYOUT_PACKED2 = 1 };

typedef struct {
  long long n_cells;        /* storage units: mx*my*mz cells (layout 0), mx*my*mz/8 units (1) */
  long long nodes_per_cell; /* values per storage unit: (p+1)^3, or (2p+1)^3 packed */
  long long cellwise_len;   /* n_cells * nodes_per_cell: the length of every mesh vector */
  long long unique_dofs;    /* (mx p + 1)(my p + 1)(mz p + 1), Sec. 6 closed form */
  int layout_id;            /* FE_LAYOUT_CELLS or FE_LAYOUT_PACKED2 */
} fe_layout;

typedef struct fe_mesh fe_mesh;
typedef struct fe_server fe_server;

/* Build a mesh: 1D tables, geometry kernel on `stream` (Sec. 2.3 geometry, Sec. 6.2).  The call
 * returns once the geometry is built (it synchronizes `stream`).  *out is library-owned; free it
 * with fe_mesh_destroy.  FE_ERR_INVALID for degree outside [1,7], non-positive cell counts,
 * geom_mode AFFINE with deform_amp != 0; FE_ERR_OOM if device memory runs out. */
fe_status fe_mesh_create(const fe_mesh_desc* desc, void* stream, fe_mesh** out);
fe_status fe_mesh_destroy(fe_mesh* mesh);
fe_status fe_mesh_layout(const fe_mesh* mesh, fe_layout* out);

/* Gather G (Sec. 2.1): x_cell = G x_unique.  Test and input helper: x_unique_host is a HOST
 * array of unique_dofs doubles in lexicographic global order (gz*Ny + gy)*Nx + gx,
 * Nx = mx p + 1; x_cell_dev is a device array of cellwise_len doubles.  Synchronous. */
fe_status fe_gather(const fe_mesh* mesh, const double* x_unique_host, double* x_cell_dev,
                    void* stream);

/* Operator apply on HOST vectors in unique-node form: for each of the nop (1 or 2) operators
 * ops[k], y_unique_host[k] = G^T A_D G x_unique_host, the assembled operator on the global node
 * vector (Sec. 2.1: G the gather, A_D the operator of fe_apply).  x_unique_host and each
 * y_unique_host[k] hold unique_dofs doubles in fe_gather's lexicographic order.  Only these
 * unique-node vectors cross the host link (cell-wise storage, 2.4x larger at Q3, stays on the
 * device): the call copies x in once, expands it to cell-wise form with a kernel, runs the
 * assembled apply per operator, and copies one copy of every node back.  Large meshes are
 * pipelined in chunks of z-layers (uploads, applies and read-backs of different chunks overlap);
 * the result is bitwise that of fe_apply with FE_ASSEMBLE.  The environment variable
 * FE_HOST_CHUNKS sets the chunk count.  Stream-ordered: it returns once the work is enqueued;
 * with page-locked host buffers (cudaHostAlloc) the copies are asynchronous and the buffers must
 * stay untouched until `stream` has passed the call (synchronize it or wait on an event).  The
 * device staging (one unique and two cell-wise vectors, plus one unique vector per output) belongs
 * to the mesh and is allocated on first use, so calls on one mesh must be ordered on one stream.
 * FE_F64 arithmetic; flags 0 or FE_NATIVE_F64; FE_LAYOUT_CELLS meshes (slabs included). */
fe_status fe_apply_host(const fe_mesh* mesh, int nop, const fe_op* ops, const double* x_unique_host,
                        double* const* y_unique_host, unsigned flags, void* stream);

/* Local operator apply (Sec. 3.1 "local operator"; Eq. (mass_operator) / (laplace_operator)
 * with per-quadrature-point geometry): y_K = A_K x_K for every cell K (dual, unassembled).
 * With FE_ASSEMBLE the structured DSS follows (Sec. 4.1): y = S(A x), continuous.  x and y must
 * not overlap.  x and y are float arrays for every prec but FE_F64.  FE_BF16_F32ACC /
 * FE_F16_F32ACC need FE_GEOM_STORED (else FE_ERR_INVALID); their first call on a mesh builds the
 * 16-bit metric from the FP64 one (and, for n <= 4, the operand tables of the tensor-core
 * kernels).  Assembled applies at degree <= 3 (but the tensor-core ones) sum the x/y interfaces
 * inside bricks of cells in the kernel, and on large meshes also the z-interfaces inside chunks
 * of z-layers (the environment variable FE_ZCARRY_CHUNK=k forces k layers per chunk, 0 or 1
 * none); the result is bitwise the same either way. */
fe_status fe_apply(const fe_mesh* mesh, fe_op op, fe_prec prec, const void* x, void* y,
                   unsigned flags, void* stream);

/* Direct stiffness summation S = G I_Riesz G^T (Eq. (dss_operator)), structured
 * dimension-split passes (Algorithm "Dimensionally-Split Structured Summation"):
 * z = S r.  In place (z == r) is allowed.  prec FE_F64 (double) or FE_F32 (float). */
fe_status fe_dss(const fe_mesh* mesh, fe_prec prec, const void* r, void* z, void* stream);

/* Jacobi diagonal D_cell = diag(G d), d = diag(A_D) (Sec. 3.3): d_cell is a device array of
 * cellwise_len doubles; every copy of a node holds the assembled diagonal; 1 on Dirichlet nodes. */
fe_status fe_diag(const fe_mesh* mesh, fe_op op, double* d_cell, void* stream);

/* Duality pairing <a, b> = sum_e a_e b_e over all cell-wise entries (Lemma "Duality Pairing
 * Identity": pairing a dual with a continuous primal vector gives the assembled inner
 * product).  Products and sums in binary64 (the FP64 pipe; the whole binary64 range, rounding
 * error below (n / 155,648 + 20) units of 2^-53 of sum |a_e b_e|), fixed reduction order
 * (bitwise reproducible).  result_dev is a device pointer to one double.  prec FE_F64 (double
 * inputs) or FE_F32 (float inputs). */
fe_status fe_pairing(const fe_mesh* mesh, fe_prec prec, const void* a, const void* b,
                     double* result_dev, void* stream);

/* Duality pairing <a, b> as fe_pairing, but allocating nothing on any call.  The paper has no
 * counterpart: this entry point serves callers that cannot let the library call cudaMalloc, such
 * as a process whose device memory is all handed to its own pool (a caching allocator, or a
 * serving loop that admits work against a fixed memory budget) or a latency-critical loop where
 * an allocation, which may synchronize the device, is not acceptable.  Its scratch is a static
 * device array of 8192 doubles (64 KiB, held on every device that loads the library until the
 * process exits); one CTA reduces 8192 consecutive entries per scratch slot, so meshes with more
 * than 67,108,864 cell-wise entries are rejected with FE_ERR_INVALID.  The first call on a device
 * looks up the array's device address (cudaGetSymbolAddress) and should come before any stream
 * capture; the address is kept for the life of the process, so the entry point must not be
 * called after a reset of that device (cudaDeviceReset).  All calls share the array: calls that
 * overlap on the GPU race.  Each call rewrites every slot it reads, so no clearing is needed.
 * Same arguments, arithmetic and errors as fe_pairing. */
fe_status fe_pairing_noalloc(const fe_mesh* mesh, fe_prec prec, const void* a, const void* b,
                             double* result_dev, void* stream);

/* Manufactured Poisson problems -Laplace(u) = f, u = 0 on the boundary of the unit cube:
 * FE_RHS_SINE (u = sin(pi x) sin(pi y) sin(pi z), f = 3 pi^2 u) and FE_RHS_QUADRATIC
 * (u = prod x_a (1 - x_a)).  fe_rhs writes the unassembled load vector b~ (dual, cell-wise:
 * b_K,i = sum_q w_q detJ f(x(xi_q)) phi_i(xi_q)), the right-hand side of Eq. (constrained_system),
 * into the device array b (cellwise_len doubles).  fe_l2_error computes the L2 norm of u_h - u for
 * a cell-wise FP64 solution u (device) with an (n+2)-point Gauss rule per direction and writes it
 * to the HOST double *err (synchronous).  FP64 arithmetic. */
#define FE_RHS_SINE 0
#define FE_RHS_QUADRATIC 1
fe_status fe_rhs(const fe_mesh* mesh, int kind, double* b, void* stream);
fe_status fe_l2_error(const fe_mesh* mesh, int kind, const double* u, double* err, void* stream);

/* Conjugate gradients on cell-wise data (Algorithm "Communication-Free (Flexible) PCG") with the
 * Jacobi preconditioner P = D_cell^{-1} S.  Convergence (unspecified in the paper; reading):
 * ||G^T r||_2 / ||G^T b||_2 <= rtol over free nodes, evaluated on the device as
 * sum_e (S r)_e^2 / mult_e.  mixed = 0: FP64 throughout; flexible = 1 uses the FCG beta.
 * mixed = FE_F32, flexible = 0: FP32 PCG (FP32 vectors and operator, pairings accumulated in
 * double-word arithmetic) with FP64 reliable updates: whenever the recursive residual has dropped
 * by inner_rtol since the last update, the FP32 correction is added to the FP64 solution x, the
 * true residual b - A x is formed with the FP64 operator and replaces the recursive one, and the
 * search direction is kept (iterative refinement that keeps the Krylov space).
 * mixed = FE_F32, flexible = 1: FP64 FCG whose (variable) preconditioner is an FP32 PCG solve to
 * inner_rtol, the reduced-precision preconditioner that motivates FCG in Sec. 3.2.
 * mixed = FE_BF16_F32ACC or FE_F16_F32ACC: the FCG scheme (whatever `flexible` says) with the
 * inner operator in 16-bit operands and FP32 accumulation (stored geometry only; inner vectors
 * stay FP32).  The FP32 iteration receives the residual assembled in FP64 and split evenly over
 * the copies of each node.  The FP64 residual of the returned x decides convergence.  b (dual)
 * and x (primal, in/out) are device arrays of cellwise_len doubles.  Every solve (this one, the
 * batched and served ones, fe_slab_cg_solve) runs on the system scaled by an exact power of two
 * that brings max|b| into [1, 2), and scales x back, so any finite scale of b behaves like unit
 * size; a non-finite entry of b returns FE_ERR_INVALID.  Synchronous: returns after the solve. */
typedef struct {
  double rtol;       /* relative residual target */
  int maxit;         /* iteration cap (inner iterations in total for mixed) */
  int mixed;         /* 0 = FP64; FE_F32, FE_BF16_F32ACC, FE_F16_F32ACC = inner solve in that
                        arithmetic under FP64 refinement */
  int flexible;      /* 1 = FCG beta */
  double inner_rtol; /* mixed only: residual reduction between two reliable updates (<= 0: 0.1),
                        or per inner FCG solve (<= 0: 1e-2; an inner FCG solve also stops after
                        20 iterations without a 10% residual drop) */
  double* history;   /* nullable HOST array of 3*maxit doubles; FP64 solves write, for iteration
                        k, alpha_k, beta_k and the relative residual after the update */
} fe_cg_opts;
typedef struct {
  int iters;        /* total CG iterations (inner iterations for mixed) */
  int outer_iters;  /* refinement steps (mixed), 1 otherwise */
  double rel_res;   /* final ||G^T r|| / ||G^T b|| in FP64 */
  fe_status status; /* FE_OK, FE_ERR_NOT_CONVERGED, FE_ERR_BREAKDOWN */
} fe_cg_result;
fe_status fe_cg_solve(const fe_mesh* mesh, const double* b, double* x, const fe_cg_opts* opts,
                      fe_cg_result* res, void* stream);

/* Batched solve of nprob independent problems (each its own mesh, degree and right-hand side)
 * with the options of fe_cg_solve (mixed = 0: FP64 PCG; mixed = FE_F32: FP32 PCG with FP64 reliable
 * updates, whatever `flexible` says).  Every CG iteration applies the operators of all
 * unconverged problems in one persistent launch over (problem, cell-tile) work items; vector
 * kernels run over (problem, chunk) items and every problem's scalars are reduced in a fixed
 * order, so each result is bitwise the same alone and in any mix.  meshes must be distinct and on
 * one device; b[i] (dual) and x[i] (primal, in/out) are device arrays of each mesh's
 * cellwise_len doubles; res[i] receives each result.  Synchronous.  Returns FE_OK when every
 * problem converged, else the first failing status (all results are still filled in). */
fe_status fe_cg_solve_batched(int nprob, const fe_mesh* const* meshes, const double* const* b,
                              double* const* x, const fe_cg_opts* opts, fe_cg_result* res,
                              void* stream);

/* Request server with continuous batching (the paper has no serving; this follows the same
 * batched engine as fe_cg_solve_batched).  A worker thread admits submitted solves in arrival
 * order while one of max_slots slots is free and the request's device-memory estimate fits
 * mem_budget bytes, builds its mesh and workspace, and joins it to the running batch: FP64
 * requests at once, mixed-precision requests at the next outer-iteration boundary.  One
 * persistent launch per iteration applies the operators of every solve in the batch; converged
 * solves retire, copy their solution to host memory and free their device memory (a library-owned
 * stream-ordered pool).  Each result is bitwise the same as when the request is served alone.
 *  fe_serve_create: device is the CUDA device the server uses.
 *  fe_serve_submit: desc describes the mesh (geom_mode STORED or AFFINE, device = the server's);
 *    b_host is a HOST cell-wise dual right-hand side of the mesh's cellwise_len doubles, copied at
 *    submission, or NULL for the manufactured sine load (FE_RHS_SINE); opts as in fe_cg_solve
 *    (mixed = FE_F32 runs FP32 PCG with FP64 reliable updates).  *ticket identifies the
 *    request.  FE_ERR_OOM if the request alone exceeds the budget.
 *  fe_serve_poll: FE_ERR_BUSY while pending; FE_OK fills *res and, if x_host is not NULL, copies
 *    the solution (cellwise_len doubles) and forgets the ticket.  Non-blocking.
 *  fe_serve_stats: p50 and p99 of (completion - submission) over completed requests, in seconds,
 *    and completed solves per second since the first submission.
 *  fe_serve_destroy: drops requests still waiting for admission, finishes the admitted ones,
 *    then frees the server. */
fe_status fe_serve_create(size_t mem_budget, int max_slots, int device, fe_server** out);
fe_status fe_serve_submit(fe_server* server, const fe_mesh_desc* desc, const double* b_host,
                          const fe_cg_opts* opts, long long* ticket);
fe_status fe_serve_poll(fe_server* server, long long ticket, fe_cg_result* res, double* x_host);
fe_status fe_serve_stats(fe_server* server, double* p50_s, double* p99_s, double* solves_per_s);
fe_status fe_serve_destroy(fe_server* server);

/* Block-structured meshes (Sec. 4.2 "Generalization to Block-Structured Grids").  A macro-mesh
 * of nblocks hexahedral blocks: block b has the macro-vertices block_verts[8b + c] at its local
 * corners c = i + 2j + 4k (i, j, k in {0,1} along its local x, y, z), trilinear geometry from the
 * vertex coordinates vxyz (3 per vertex; every block must be right-handed) and a structured grid
 * of dims[3b..3b+2] cells of the given degree.  Blocks that share a face must agree on its cell
 * counts (conforming); shared faces may meet with any relative rotation or reflection.
 * Cell-wise layout: the blocks one after the other, each block in layout 0.  No Dirichlet
 * masking.  fe_mb_create derives the interface structure on the host from the vertex numbers:
 * face pairs with a 3-bit relative orientation (swap, flip s, flip t), and sharing lists of the
 * macro-edge and macro-vertex nodes with one representative copy per block.  Synchronous.
 * FE_ERR_INVALID for non-conforming faces, left-handed blocks, or bad sizes. */
typedef struct {
  int nblocks, nverts, degree;
  const int* dims;        /* 3 per block (host) */
  const int* block_verts; /* 8 per block (host) */
  const double* vxyz;     /* 3 per vertex (host) */
  int device;
} fe_mb_desc;
typedef struct fe_mbmesh fe_mbmesh;
fe_status fe_mb_create(const fe_mb_desc* desc, void* stream, fe_mbmesh** out);
fe_status fe_mb_destroy(fe_mbmesh* mesh);
/* n_cells and cellwise_len over all blocks; unique_dofs counted from the macro-topology */
fe_status fe_mb_layout(const fe_mbmesh* mesh, fe_layout* out);
/* counts of the inter-block structure: face pairs, macro-edge node entities, macro-vertex
 * entities, and the largest number of blocks sharing an entity (any pointer may be NULL) */
fe_status fe_mb_info(const fe_mbmesh* mesh, int* face_pairs, long long* edge_entities,
                     int* vertex_entities, int* max_valence);
/* Local apply of every block (fe_apply per block; prec FE_F64 / FE_F32, flag FE_NATIVE_F64).
 * With FE_ASSEMBLE: the structured DSS inside every block, then the inter-block summation of
 * Algorithm "Unstructured Inter-Block Summation" (faces, lines, vertices). */
fe_status fe_mb_apply(const fe_mbmesh* mesh, fe_op op, fe_prec prec, const void* x, void* y,
                      unsigned flags, void* stream);
/* DSS of the block-structured mesh: structured passes inside every block (Algorithm
 * "Dimensionally-Split Structured Summation"), then the inter-block summation.  r == z allowed. */
fe_status fe_mb_dss(const fe_mbmesh* mesh, fe_prec prec, const void* r, void* z, void* stream);

/* Hanging nodes (Appendix "Extension of DSS algorithms onto Non-Conforming Interfaces",
 * Algorithm "Full DSS Operator with Hanging Node Resolution") on a two-level Cartesian
 * refinement of the unit cube: a coarse grid of mc^3 cells whose cells inside the box
 * [lo, hi) (coarse cell coordinates, strictly inside: 1 <= lo < hi <= mc-1) are each refined
 * into 2x2x2 fine cells.  The conforming space constrains every fine node on the box boundary to
 * the trace of its parent's coarse polynomial.  Vectors (cellwise_len entries, layout 0 per
 * level): the full coarse grid -- its cells inside the box are dormant, zero on output, and act
 * as the shadow cells of the exchange -- then the fine grid of the box (2(hi-lo) cells per
 * direction).  unique_dofs counts the conforming space.  Stored trilinear geometry, no Dirichlet
 * masking.  fe_amr_dss: shadow restriction, structured DSS on both levels, prolongation (an
 * assignment, which makes the paper's vertex save-and-restore unnecessary), result G_c G_c^T r on
 * the active copies.  fe_amr_apply: the local operator of every active cell, with FE_ASSEMBLE
 * followed by fe_amr_dss.  FE_F64 / FE_F32; FE_NATIVE_F64 accepted. */
typedef struct {
  int mc;         /* coarse cells per direction, >= 3 */
  int lo[3], hi[3];
  int degree;     /* p in [1, 7] */
  int device;
} fe_amr_desc;
typedef struct fe_amr fe_amr;
fe_status fe_amr_create(const fe_amr_desc* desc, void* stream, fe_amr** out);
fe_status fe_amr_destroy(fe_amr* mesh);
fe_status fe_amr_layout(const fe_amr* mesh, fe_layout* out);
fe_status fe_amr_apply(const fe_amr* mesh, fe_op op, fe_prec prec, const void* x, void* y,
                       unsigned flags, void* stream);
fe_status fe_amr_dss(const fe_amr* mesh, fe_prec prec, const void* r, void* z, void* stream);

/* ---- Slab decomposition of a structured mesh over several processes or devices ----------------
 * The cells of a structured mesh (fe_mesh_desc, FE_LAYOUT_CELLS) split into slabs of whole
 * z-layers; slab s holds the layers z0 <= cz < z1.  Cells are lexicographic with z slowest, so a
 * slab's cell-wise vectors are the contiguous range of cells [z0 mx my, z1 mx my) of the whole
 * mesh's vectors.  The volumetric apply is independent per cell; the structured DSS (Sec. 4.1)
 * needs one exchange per call.  Its passes run in the order z, y, x; a node's copies on the two
 * sides of a slab interface form one pair of the z-pass, so after the z-pass inside the slab each
 * slab adds the neighbour's copy of the interface plane to its own, and the y- and x-passes
 * follow.  The result is bitwise the whole mesh's.  A slab sends and receives mx * my * n^2
 * values per neighbour and DSS.
 *
 * fe_slab_create: an fe_mesh of mx x my x (z1 - z0) cells whose geometry, affine scaling,
 *   Dirichlet boundary and manufactured data (fe_rhs, fe_l2_error) are those of the whole mesh
 *   desc->global describes; the interface planes to neighbouring slabs are not Dirichlet
 *   boundary.  Every fe_* call on a single mesh accepts it and works on the slab alone (fe_dss,
 *   fe_diag and FE_ASSEMBLE sum inside the slab; fe_layout.unique_dofs counts the slab's nodes,
 *   interface planes included; fe_pairing of a dual and a primal vector is this slab's part of the
 *   whole pairing), except fe_cg_solve and fe_cg_solve_batched (use fe_slab_cg_solve).
 *   FE_ERR_INVALID unless 0 <= z0 < z1 <= global.mz and layout is FE_LAYOUT_CELLS.
 * Interface planes: side 0 is the slab's bottom (local node k = 0 of layer 0), side 1 its top
 *   (k = p of the last layer).  A plane holds mx my n^2 values, entry ((cy mx + cx) n + j) n + i
 *   for node (i, j) of cell (cx, cy); two slabs that share an interface see it in the same order.
 * fe_slab_face_pack: plane[e] = v[node e of `side`].  fe_slab_face_add: v[node e] += plane[e].
 *   v and plane are device arrays of double (FE_F64) or float (FE_F32).  Building blocks for
 *   callers that run their own exchange; fe_slab_dss uses them between its z- and y-passes.
 * fe_slab_plane_len: mx my n^2. */
typedef struct {
  fe_mesh_desc global; /* the whole mesh */
  int z0, z1;          /* this slab's layers: z0 <= cz < z1 */
} fe_slab_desc;
fe_status fe_slab_create(const fe_slab_desc* desc, void* stream, fe_mesh** out);
fe_status fe_slab_plane_len(const fe_mesh* slab, long long* count);
fe_status fe_slab_face_pack(const fe_mesh* slab, fe_prec prec, const void* v, int side, void* plane,
                            void* stream);
fe_status fe_slab_face_add(const fe_mesh* slab, fe_prec prec, void* v, int side, const void* plane,
                           void* stream);

/* Communication between the slabs, supplied by the caller (NCCL, MPI, host threads ...).  All
 * slabs call the same fe_slab_* functions in the same order; each call invokes the callbacks the
 * same number of times on every slab.  Buffers are caller-owned device memory on the slab's
 * device: send[s] / recv[s] hold plane_len doubles for the neighbour on side s (NULL where the slab
 * has no neighbour), red_send 4 doubles and red_all 4 * size doubles.
 *  exchange(ctx, sides, elem_bytes, count, stream): for every side s in the bitmask `sides`
 *    (1: below, 2: above) send the first count elements of elem_bytes bytes of send[s] to the
 *    neighbour there and receive its plane into recv[s].
 *  allgather(ctx, n, stream): every slab's red_send[0..n) into red_all[r * n + i], r the slab's
 *    rank (slab r - 1 lies below slab r).
 * The library enqueues the work that fills the send buffers on `stream` before a call; the callback
 * must order its transfers after that work (issue them on `stream`, or synchronize it) and leave
 * the received data ready for work enqueued on `stream` after it returns.  A non-zero return
 * makes the calling fe_slab_* function return FE_ERR_COMM. */
typedef struct {
  int rank, size;      /* this slab's rank and the number of slabs (rank 0 holds z0 = 0) */
  void* send[2];
  void* recv[2];
  double* red_send;
  double* red_all;
  int (*exchange)(void* ctx, int sides, int elem_bytes, long long count, void* stream);
  int (*allgather)(void* ctx, int n, void* stream);
  void* ctx;
} fe_comm;

/* fe_slab_dss: z = S r on the whole mesh, restricted to this slab: the z-pass, one exchange of both
 *   interface planes, the y- and x-passes.  Bitwise fe_dss of the whole mesh.  FE_F64 / FE_F32.
 * fe_slab_apply: fe_apply on the slab; with FE_ASSEMBLE the DSS passes run as in fe_slab_dss, so y
 *   is this slab's part of the whole mesh's assembled output, bit for bit.  comm may be NULL
 *   without FE_ASSEMBLE.
 * fe_slab_cg_solve: Jacobi PCG on the whole mesh (Sec. 3.2 with P = D^{-1} S, Sec. 3.3), this
 *   slab's part of b (dual) and x (primal, in/out) in its cell-wise vectors.  The iteration is the
 *   single-reduction recurrence of Chronopoulos and Gear (1989): per iteration one apply
 *   s = A z, one DSS with its plane exchange, and one allgather of three scalars (<r,z>, <s,z> and
 *   sum w^2/mult for the residual) summed over the slabs in rank order, so every slab takes the
 *   same decisions.  The Jacobi diagonal is assembled across the interfaces once per call.  Same
 *   stopping rule, result and history semantics as fe_cg_solve; opts->mixed and opts->flexible
 *   must be 0 (FE_ERR_INVALID).  Synchronous. */
fe_status fe_slab_dss(const fe_mesh* slab, fe_prec prec, const void* r, void* z, const fe_comm* comm,
                      void* stream);
fe_status fe_slab_apply(const fe_mesh* slab, fe_op op, fe_prec prec, const void* x, void* y,
                        unsigned flags, const fe_comm* comm, void* stream);
fe_status fe_slab_cg_solve(const fe_mesh* slab, const double* b, double* x, const fe_cg_opts* opts,
                           const fe_comm* comm, fe_cg_result* res, void* stream);

/* Thread-local message describing the last error of this thread ("" if none). */
const char* fe_last_error(void);

#ifdef __cplusplus
}
#endif
#endif
