// fe_cgcore.h -- pieces shared by the single-problem CG (fe_cg.cu) and the batched engine
// (fe_batch.cu): device-resident scalars, their finishing logic, and the per-mesh workspace.
#pragma once
#include <cmath>

#include "fe_internal.h"

struct CgScal {
  double rz, rz_new, qp, qz, alpha, beta, rnorm2, bnorm2, relres;
  double best;      // smallest relative residual so far
  int done, status, iter, maxit;
  int stall;        // iterations since `best` last dropped by 10%
  int stall_limit;  // stop after this many iterations without progress (0 = never)
  int stall_total;  // batched mixed solves: inner iterations accumulated over outer steps
  int pad;
  double rtol;      // stopping tolerance of graph-replayed iterations (set by the host per run)
};

// FIN_INIT_B: ||G^T b||^2.  FIN_INIT_R: initial residual, <r,z>.  FIN_ITER: residual, convergence,
// beta.  FIN_NORM: residual only.  FIN_OUTER: residual, outer count, convergence.
enum { FIN_INIT_B = 0, FIN_INIT_R = 1, FIN_ITER = 2, FIN_NORM = 3, FIN_OUTER = 4 };

__device__ __forceinline__ void fin_scalars(CgScal* sc, double rn2, double rz, double qz, double rtol,
                                            int mode, int flexible) {
  if (mode == FIN_INIT_B) {
    sc->bnorm2 = rn2;
    return;
  }
  sc->rnorm2 = rn2;
  const double rel = sc->bnorm2 > 0.0 ? sqrt(rn2 / sc->bnorm2) : 0.0;
  sc->relres = rel;
  if (mode == FIN_NORM) return;
  if (mode == FIN_OUTER) {
    sc->iter += 1;
    if (!isfinite(rel)) {
      sc->status = FE_ERR_BREAKDOWN;
      sc->done = 1;
    } else if (rel <= rtol) {
      sc->status = FE_OK;
      sc->done = 1;
    }
    return;
  }
  if (mode == FIN_INIT_R) {
    sc->rz = rz;
    sc->best = rel;
    sc->stall = 0;
    sc->iter = 0;
    sc->status = FE_OK;
    sc->done = (rel <= rtol) ? 1 : 0;
    return;
  }
  const int k = sc->iter;
  sc->iter = k + 1;
  if (!isfinite(rel)) {
    sc->status = FE_ERR_BREAKDOWN;
    sc->done = 1;
    return;
  }
  if (rel <= rtol) {
    sc->status = FE_OK;
    sc->done = 1;
    return;
  }
  // Stagnation guard of FP32 inner solves: FP32 rounding makes the operator slightly
  // non-symmetric and CG then levels off near eps_32 * cond(A); the FP64 outer loop takes over.
  if (rel < 0.9 * sc->best) {
    sc->best = rel;
    sc->stall = 0;
  } else if (sc->stall_limit > 0 && ++sc->stall >= sc->stall_limit) {
    sc->status = FE_OK;
    sc->done = 1;
    return;
  }
  if (k + 1 >= sc->maxit) {
    sc->status = FE_ERR_NOT_CONVERGED;
    sc->done = 1;
    return;
  }
  sc->beta = flexible ? -qz / sc->qp : rz / sc->rz;
  sc->rz = rz;
}

// per-mesh CG workspace (allocated on first use, owned by the mesh)
struct CgWork {
  long long n = 0;
  double *x = nullptr, *r = nullptr, *z = nullptr, *p = nullptr, *q = nullptr, *w = nullptr;
  double* bs = nullptr;  // the right-hand side scaled by the solve's power of two
  float *r32 = nullptr, *z32 = nullptr, *p32 = nullptr, *q32 = nullptr, *w32 = nullptr,
        *d32 = nullptr;
  double* invdiag64 = nullptr;
  float* invdiag32 = nullptr;
  float* invmult = nullptr;
  double* partials = nullptr;
  CgScal* sc = nullptr;   // [0] outer / FP64 solve, [1] inner FP32 solve
  CgScal* hsc = nullptr;  // pinned host mirror
  double* hist = nullptr;
  int hist_cap = 0;
  int diag_op = -1;
  cudaStream_t st = nullptr;
  cudaGraphExec_t g64[2] = {nullptr, nullptr};  // [flexible]
  cudaGraphExec_t g32[2] = {nullptr, nullptr};
  int inner_prec = FE_F32;  // arithmetic of the inner solve's operator (FP32 or 16-bit operands)
  int g32_prec = FE_F32;    // the one the g32 graphs were captured with
  double* g64_hist = nullptr;
};

fe_status fe_cg_get_work(const fe_mesh* m, bool mixed, CgWork** out);  // fe_cg.cu
// The power of two 2^-e with e the binary exponent of max|b| (1 for b = 0): solves run on
// 2^-e b and 2^-e x, exact scalings that keep the pairings' double-word sums (FP32's exponent
// range) away from overflow and underflow whatever the scale of b.  FE_ERR_INVALID when b holds a
// non-finite value.  Synchronizes w->st.
fe_status fe_cg_rhs_scale(CgWork* w, const double* b, long long n, double* s);
// *out = bit pattern of max|v| (a non-negative double), on st
fe_status fe_launch_absmax(const double* v, long long n, unsigned long long* out, cudaStream_t st);
// the power of two 2^-e with e the binary exponent of mx (1 for mx = 0); false if mx is not finite
bool fe_scale_of_max(double mx, double* s);
// dst = s src on st (src may equal dst)
fe_status fe_cg_scale(const double* src, double* dst, double s, long long n, cudaStream_t st);
fe_status fe_cg_ensure_diag(const fe_mesh* m, CgWork* w, int op);       // fe_cg.cu
