// fe_batch.h -- batched engine shared by fe_cg_solve_batched and the request server.
#pragma once
#include <vector>

#include "fe_cgcore.h"

// one problem of a batch (device-visible copy lives in FeBatch::d_probs)
struct BProb {
  int n, affine;
  long long ncells, ncw;
  int mx, my, mz, dirichlet;
  double aff[4];  // affine metric constants detJ/h_x^2, detJ/h_y^2, detJ/h_z^2, detJ
  const float2* geodw;
  const float* geo32;
  double *x64, *r64, *z64, *p64, *q64, *w64;
  const double* b64;
  float *d32, *r32, *z32, *p32, *q32, *w32;
  const double* invdiag64;
  const float* invdiag32;
  const float* invmult;
  CgScal* sc;  // [0] outer / FP64, [1] inner FP32
  int chunk0, chunk1;
  double rtol, irtol;  // outer (or FP64) and inner relative tolerances
  int maxit;           // iteration cap (inner iterations in total for mixed)
  int flexible;        // FP64 solves: FCG beta
};

struct FeBatch {
  std::vector<BProb> hp;
  std::vector<char> active;
  BProb* d_probs = nullptr;
  size_t cap_probs = 0;
  void* d_tiles = nullptr;
  size_t cap_tiles = 0;
  long long ntiles = 0;
  long long tile_lo[FE_MAXN + 1] = {}, tile_hi[FE_MAXN + 1] = {};  // tiles of each degree n
  void* d_vch = nullptr;
  size_t cap_vch = 0;
  int nvch = 0;
  void* d_dch[3] = {nullptr, nullptr, nullptr};
  size_t cap_dch[3] = {0, 0, 0};
  int ndch[3] = {0, 0, 0};
  double* d_partials = nullptr;
  size_t cap_partials = 0;
  unsigned long long* d_counter = nullptr;
  CgScal* d_sc = nullptr;  // gathered scalar records for one readback
  size_t cap_sc = 0;
  cudaStream_t st = nullptr;
  bool own_stream = true;
  CgScal* hsc = nullptr;  // pinned, 2 per problem
  size_t cap_hsc = 0;
  int any_flexible = 0;
  ~FeBatch();
};

fe_status fe_batch_prepare();
fe_status fe_batch_build(FeBatch* B);
fe_status fe_batch_read(FeBatch* B);
fe_status fe_batch_setup(FeBatch* B);  // fresh scalars, ||G^T b||, r = b - A x
bool fe_batch_all_done(FeBatch* B, int slot);
template <class S>
fe_status fe_batch_iteration(FeBatch* B, int slot, int redistribute);
template <class S>
fe_status fe_batch_norm(FeBatch* B, int slot, int src, int mode, int redistribute);
// mixed solves: start of an FP32 run, and its end with the FP64 reliable update
fe_status fe_batch_inner_start(FeBatch* B);
fe_status fe_batch_inner_finish(FeBatch* B);
fe_status fe_batch_fill(FeBatch* B, int i, const fe_mesh* m, CgWork* w, const double* b,
                        const fe_cg_opts* opts);
// first steps of a solve for every problem of B: fresh scalars, ||G^T b||, r = b - A x, and the
// initial preconditioned direction (FP64) or the initial residual check (mixed)
fe_status fe_batch_start(FeBatch* B, bool mixed);
// run a full solve of every active problem (FP64 PCG or the mixed reliable-update scheme)
fe_status fe_batch_solve(FeBatch* B, const fe_cg_opts* opts);
