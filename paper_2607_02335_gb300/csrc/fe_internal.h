// fe_internal.h -- internal types of libfe (not part of the ABI): mesh object, launch descriptors,
// memory pool, error reporting.  The number types of the kernels are in fe_arith.h.
#pragma once
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "fe.h"

#include "fe_arith.h"

struct HostTab {
  int p, n;
  double t[FE_MAXN];      // GLL nodes on [0,1]
  double s[FE_MAXN];      // Gauss points on [0,1]
  double w[FE_MAXN];      // Gauss weights on [0,1]
  double V[FE_MAXN][FE_MAXN];   // V[q][i]  = l_i(s_q)
  double D[FE_MAXN][FE_MAXN];   // D[q][r]  = l~_r'(s_q), Gauss-point collocation derivative
  double Dh[FE_MAXN][FE_MAXN];  // Dh[q][i] = l_i'(s_q) = (D V)[q][i]
};

// host-side 1D rules in double precision for one degree
void fe_host_tables(int p, HostTab* out);  // fe_tables.cu

template <int N, class V>
Tab1D<N, V> make_tab(const HostTab& h);

// ---------------------------------------------------------------------------------------------
// mesh object
// ---------------------------------------------------------------------------------------------
#define FE_GEO_COMPS 7  // xx, yy, zz, xy, xz, yz of w detJ J^{-1}J^{-T}, then w detJ

// Recompute mode: cells per chunk of the metric scratch (about FE_RC_CHUNK_BYTES, a multiple of the
// apply's cells per CTA), for a metric value of gv_bytes bytes.
#ifndef FE_RC_CHUNK_BYTES
#define FE_RC_CHUNK_BYTES (48LL << 20)
#endif
inline long long fe_rc_chunk_cells(int n, long long ncells, size_t gv_bytes) {
  const long long per_cell = (long long)FE_GEO_COMPS * n * n * n * (long long)gv_bytes;
  const long long cpb = 256 / (n * n);
  long long c = FE_RC_CHUNK_BYTES / per_cell;
  c = c >= cpb ? c / cpb * cpb : (c > 0 ? c : 1);
  return c < ncells ? c : (ncells > 0 ? ncells : 1);
}

struct fe_mesh {
  fe_mesh_desc d;
  int p, n, n3;
  long long ncells, ncw, nu;
  HostTab tab;
  // stored geometry [cell][FE_GEO_COMPS][n3] (FP64, double-word, FP32 copies)
  double* geo64 = nullptr;
  float2* geodw = nullptr;
  float* geo32 = nullptr;
  unsigned short* geo16[2] = {nullptr, nullptr};  // bf16 / fp16 metric, scaled by gscale[op]
  float gscale[2] = {1.0f, 1.0f};                 // powers of two: Laplace terms, w detJ
  // fragment tables of the tensor-core 16-bit kernels [bf16, fp16][Laplace, mass] (n = 2..4)
  unsigned* kron_tab[2][2] = {{nullptr, nullptr}, {nullptr, nullptr}};
  bool tri = false;  // a block of a block-structured mesh (trilinear map of its corners)
  // slab of a larger structured mesh (fe_slab_create): d.mz is the slab's own layer count, the
  // slab starts at global layer zoff of mzg, and has neighbouring slabs below / above when
  // nbr_lo / nbr_hi (their interface planes are not Dirichlet boundary)
  int zoff = 0, mzg = 0;
  bool nbr_lo = false, nbr_hi = false;
  // storage grid of the vectors (FE_LAYOUT_PACKED2: units of 2x2x2 cells with sn = 2p+1 nodes per
  // side; otherwise the cells with sn = n) -- what the DSS passes walk
  bool packed = false;
  int sgx = 0, sgy = 0, sgz = 0, sn = 0;
  // recompute mode: nodal coordinates [cell][3][n3], and an L2-sized scratch for the metric of one
  // chunk of cells (per arithmetic: 0 double-word, 1 FP64, 2 FP32)
  double* xyz64 = nullptr;
  float2* xyzdw = nullptr;
  float* xyz32 = nullptr;
  void* rc_scratch[3] = {nullptr, nullptr, nullptr};
  long long rc_cells = 0;  // cells per chunk
  // Jacobi diagonal caches (cell-wise, continuous), per operator
  double* diag64[2] = {nullptr, nullptr};
  float* invdiag32[2] = {nullptr, nullptr};
  double* invdiag64[2] = {nullptr, nullptr};
  // inverse multiplicity (cell-wise), for the residual norm
  double* invmult64 = nullptr;
  // reduction scratch
  double* red = nullptr;
  int red_len = 0;
  // host-vector applies (fe_host.cu): device staging of the unique-node input, its cell-wise
  // expansion, the assembled cell-wise output and up to two unique-node outputs; streams for the
  // uploads and the read-backs, and events ordering them against the caller's stream
  double *hs_xu = nullptr, *hs_xc = nullptr, *hs_yc = nullptr, *hs_yu[2] = {nullptr, nullptr};
  cudaStream_t hs_copy = nullptr, hs_up = nullptr;
  static constexpr int HS_EVENTS = 52;  // start, done, an upload and two read-backs per chunk
  cudaEvent_t hs_ev[HS_EVENTS] = {};
  // conjugate-gradient workspace (fe_cg.cu), released through cg_free
  void* cg_work = nullptr;
  void (*cg_free)(void*, cudaStream_t) = nullptr;
  cudaStream_t st = nullptr;  // stream of the mesh's own set-up work
};

// Dirichlet faces of a mesh as the kernels take them: bit 0 the x and y faces, bit 1 the bottom
// z face, bit 2 the top z face (0: no Dirichlet boundary)
enum { FE_DIR_XY = 1, FE_DIR_ZLO = 2, FE_DIR_ZHI = 4 };
inline int fe_dir_mask(const fe_mesh* m) {
  if (!m->d.dirichlet) return 0;
  return FE_DIR_XY | (m->nbr_lo ? 0 : FE_DIR_ZLO) | (m->nbr_hi ? 0 : FE_DIR_ZHI);
}
// global layer count of the mesh a (slab) mesh belongs to
inline int fe_mz_global(const fe_mesh* m) { return m->mzg > 0 ? m->mzg : m->d.mz; }

// ---------------------------------------------------------------------------------------------
// helpers shared by the translation units of the library
// ---------------------------------------------------------------------------------------------
void fe_set_error(const char* fmt, ...);
fe_status fe_cuda_check(cudaError_t e, const char* what);
#define FE_TRY(expr)                      \
  do {                                    \
    fe_status _s = (expr);                \
    if (_s != FE_OK) return _s;           \
  } while (0)
#define FE_CUDA(expr, what) FE_TRY(fe_cuda_check((expr), (what)))

fe_status fe_ensure_geometry(const fe_mesh* m, int prec, bool native);  // fe_mesh.cu
// fe_mesh_create with an optional trilinear block map (8 corners, 24 doubles; null = unit cube)
// z0 < z1: build only the slab of layers [z0, z1) of the mesh d describes (z1 = 0: all of it)
fe_status fe_mesh_create_impl(const fe_mesh_desc* d, const double* corners, void* stream,
                              fe_mesh** out, int z0 = 0, int z1 = 0);

// Stream-ordered device memory from a library-owned pool of the current device (fe_mesh.cu).
// Frees never synchronize the device; the pool keeps freed memory for reuse until fe_pool_trim.
fe_status fe_dalloc(void** p, size_t bytes, cudaStream_t st, const char* what);
void fe_dfree(void* p, cudaStream_t st);
void fe_pool_trim();
// destroy a mesh without synchronizing the device: frees are ordered on `st`, which must carry
// (or follow) every use of the mesh
void fe_mesh_release_async(fe_mesh* m, cudaStream_t st);
// drop the FP64 copy of the stored geometry once the double-word / FP32 copies and the Jacobi
// diagonal exist (the server keeps only what its solves read)
void fe_mesh_drop_geo64(fe_mesh* m, cudaStream_t st);

// apply (fe_apply.cu / fe_apply_*.cu)
struct ApplyLaunch {
  const fe_mesh* m;
  int op;         // FE_LAPLACE / FE_MASS
  const void* x;
  void* y;
  cudaStream_t st;
  const int* skip = nullptr;  // optional device flag that turns the launch into a no-op
  bool assemble = false;      // FE_ASSEMBLE: the launcher also runs the DSS on y
  int* brick_out = nullptr;   // assembled launches with this set leave the DSS passes to the
                              // caller and report the brick (bx, by) the kernel summed inside
};
// fe_apply with its checks; an assembled call with brick_out set leaves the DSS passes to the
// caller as ApplyLaunch::brick_out does (fe_api.cu)
fe_status fe_apply_impl(const fe_mesh* m, fe_op op, fe_prec prec, const void* x, void* y,
                        unsigned flags, void* stream, int* brick_out);
fe_status fe_launch_apply_f64dw(const ApplyLaunch& a);
fe_status fe_launch_apply_f64native(const ApplyLaunch& a);
fe_status fe_launch_apply_f32(const ApplyLaunch& a);
// FE_BF16_F32ACC / FE_F16_F32ACC: float vectors, 16-bit operands, stored geometry only
fe_status fe_launch_apply_lowp(const ApplyLaunch& a, int prec);
// the same on the tensor cores (mma.sync, fe_apply_kron.cu) for unpacked stored-geometry meshes
// of n = 2..4; FE_LOWP_FMA=1 in the environment selects the FMA-pipe kernels instead
bool fe_kron_eligible(const fe_mesh* m);
bool fe_kron_supported(const fe_mesh* m);
fe_status fe_kron_build_tables(fe_mesh* m, int prec);  // with the 16-bit metric, on m->st
fe_status fe_launch_apply_kron(const ApplyLaunch& a, int prec);

// dss / vectors (fe_dss.cu)
fe_status fe_launch_dss(const fe_mesh* m, int prec, void* v, cudaStream_t st);
// DSS passes of an apply whose kernel already summed the x- and y-interfaces inside bricks of
// bx x by cells: all z-interfaces, then the y- and x-interfaces between bricks
fe_status fe_launch_dss_strided(const fe_mesh* m, int prec, void* v, int bx, int by,
                                cudaStream_t st);
// fe_launch_dss_strided whose z-pass also visits only every bz-th z-interface (the boundaries of
// the z-chunks of a z-carry apply)
fe_status fe_launch_dss_strided3(const fe_mesh* m, int prec, void* v, int bx, int by, int bz,
                                 cudaStream_t st);
// the passes of axes axis_hi down to axis_lo (2 = z, 1 = y, 0 = x) of fe_launch_dss_strided
fe_status fe_launch_dss_axes(const fe_mesh* m, int prec, void* v, int bx, int by, int axis_hi,
                             int axis_lo, cudaStream_t st);
// the structured passes inside every block of a block-structured mesh, one launch per axis
// (sx, sy > 1: only the x/y interfaces between bricks, after a brick-fused apply)
fe_status fe_launch_dss_blocks(const fe_mesh* const* blocks, const long long* off, int nb,
                               int prec, void* v, int sx, int sy, cudaStream_t st);
fe_status fe_launch_diag(const fe_mesh* m, int op, double* d, cudaStream_t st);
// 1 / multiplicity of every cell-wise node (interface copies of neighbouring slabs counted), 0 on
// Dirichlet nodes (fe_cg.cu)
fe_status fe_launch_invmult(const fe_mesh* m, float* out, cudaStream_t st);
fe_status fe_launch_pairing(const fe_mesh* m, int prec, const void* a, const void* b,
                            double* out, cudaStream_t st);

static inline bool fe_aligned(const void* p) { return ((uintptr_t)p & 15u) == 0; }

// Switches the calling thread to a mesh's device for the duration of an entry point and restores
// the caller's current device when the entry point returns.
struct FeDeviceGuard {
  int prev = -1;
  cudaError_t set(int dev) {
    if (prev < 0 && cudaGetDevice(&prev) != cudaSuccess) prev = -1;
    return cudaSetDevice(dev);
  }
  ~FeDeviceGuard() {
    if (prev >= 0) cudaSetDevice(prev);
  }
};
