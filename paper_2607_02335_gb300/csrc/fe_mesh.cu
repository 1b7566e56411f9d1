// fe_mesh.cu -- mesh object, geometry set-up kernel, gather helper, error reporting.
//
// Geometry (Sec. 2.3 and Sec. 6.2 "per-quadrature-point Jacobians"): the map
// Phi(X) = X + amp sin(pi X) sin(pi Y) sin(pi Z) (1,1,1) is sampled at the GLL nodes of every
// cell and interpolated isoparametrically with Q_p.  For every Gauss point q the kernel forms
// J_ab = d x_a / d xi_b (xi in [0,1]^3) by sum factorization, then stores
// G = w_q detJ J^{-1} J^{-T} (6 symmetric entries) and w_q detJ, in FP64, laid out
// [cell][component][q] so that the apply kernels read them with coalesced loads.
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <new>

#include "fe_internal.h"

// ---------------------------------------------------------------------------------------------
// errors
// ---------------------------------------------------------------------------------------------
static thread_local char g_err[512] = "";

void fe_set_error(const char* fmt, ...) {
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(g_err, sizeof(g_err), fmt, ap);
  va_end(ap);
}

fe_status fe_cuda_check(cudaError_t e, const char* what) {
  if (e == cudaSuccess) return FE_OK;
  fe_set_error("%s: %s", what, cudaGetErrorString(e));
  return e == cudaErrorMemoryAllocation ? FE_ERR_OOM : FE_ERR_CUDA;
}

extern "C" const char* fe_last_error(void) { return g_err; }

// ---------------------------------------------------------------------------------------------
// library memory pool (one per device)
// ---------------------------------------------------------------------------------------------
static std::mutex g_pool_mu;
static cudaMemPool_t g_pool[64] = {};

static fe_status pool_of_current(cudaMemPool_t* out) {
  int dev = 0;
  FE_CUDA(cudaGetDevice(&dev), "cudaGetDevice");
  if (dev < 0 || dev >= 64) {
    fe_set_error("device ordinal %d out of range", dev);
    return FE_ERR_INVALID;
  }
  std::lock_guard<std::mutex> lock(g_pool_mu);
  if (!g_pool[dev]) {
    cudaMemPoolProps props;
    std::memset(&props, 0, sizeof(props));
    props.allocType = cudaMemAllocationTypePinned;
    props.location.type = cudaMemLocationTypeDevice;
    props.location.id = dev;
    FE_CUDA(cudaMemPoolCreate(&g_pool[dev], &props), "cudaMemPoolCreate");
    unsigned long long thr = ~0ULL;
    FE_CUDA(cudaMemPoolSetAttribute(g_pool[dev], cudaMemPoolAttrReleaseThreshold, &thr),
            "pool release threshold");
  }
  *out = g_pool[dev];
  return FE_OK;
}

fe_status fe_dalloc(void** p, size_t bytes, cudaStream_t st, const char* what) {
  *p = nullptr;
  cudaMemPool_t pool;
  FE_TRY(pool_of_current(&pool));
  return fe_cuda_check(cudaMallocFromPoolAsync(p, bytes > 0 ? bytes : 16, pool, st), what);
}

void fe_dfree(void* p, cudaStream_t st) {
  if (p) cudaFreeAsync(p, st);
}

void fe_pool_trim() {
  std::lock_guard<std::mutex> lock(g_pool_mu);
  int dev = 0;
  if (cudaGetDevice(&dev) == cudaSuccess && dev >= 0 && dev < 64 && g_pool[dev])
    cudaMemPoolTrimTo(g_pool[dev], 0);
}

// ---------------------------------------------------------------------------------------------
// geometry kernel: one CTA per cell, n^3 threads (one per node, then one per Gauss point)
// ---------------------------------------------------------------------------------------------
struct GeoTab {
  double t[FE_MAXN];
  double w[FE_MAXN];
  double V[FE_MAXN][FE_MAXN];
  double Dh[FE_MAXN][FE_MAXN];
};

struct GeoArgs {
  double* geo;  // [cell][7][n3] or null
  double* xyz;  // [cell][3][n3] or null
  long long ncells;
  int mx, my, mz;  // cells of the whole mesh
  int z0;          // global layer of the first layer of cells built (a slab's offset)
  double amp;
  int tri;              // 1: trilinear block map of `corners` instead of the unit-cube map Phi
  double corners[24];   // block corners c = i + 2j + 4k (x, y, z each)
  GeoTab tab;
};

// physical point of the block-reference point X in [0,1]^3
__device__ __forceinline__ void geo_point(const GeoArgs& a, double X0, double X1, double X2,
                                          double out[3]) {
  if (a.tri) {
    out[0] = out[1] = out[2] = 0.0;
#pragma unroll
    for (int c = 0; c < 8; ++c) {
      const double w = ((c & 1) ? X0 : 1.0 - X0) * ((c & 2) ? X1 : 1.0 - X1) *
                       ((c & 4) ? X2 : 1.0 - X2);
#pragma unroll
      for (int d = 0; d < 3; ++d) out[d] = fma(w, a.corners[3 * c + d], out[d]);
    }
  } else {
    const double s = a.amp * sinpi(X0) * sinpi(X1) * sinpi(X2);
    out[0] = X0 + s;
    out[1] = X1 + s;
    out[2] = X2 + s;
  }
}

template <int N>
__global__ void __launch_bounds__(N* N* N) k_geometry(const __grid_constant__ GeoArgs a) {
  constexpr int N2 = N * N, N3 = N2 * N;
  extern __shared__ double gsm[];
  double* sX = gsm;             // [3][N3] node coordinates
  double* sA = gsm + 3 * N3;    // [3][N3] V along x
  double* sB = gsm + 6 * N3;    // [3][N3] Dh along x
  double* sAA = gsm + 9 * N3;   // [3][N3] V x, V y
  double* sAB = gsm + 12 * N3;  // [3][N3] V x, Dh y
  double* sBA = gsm + 15 * N3;  // [3][N3] Dh x, V y
  const long long cell = blockIdx.x;
  const int t = threadIdx.x;
  const int i = t % N, j = (t / N) % N, k = t / N2;
  const int cx = (int)(cell % a.mx), cy = (int)((cell / a.mx) % a.my),
            cz = a.z0 + (int)(cell / ((long long)a.mx * a.my));
  {
    double x[3];
    geo_point(a, (cx + a.tab.t[i]) / a.mx, (cy + a.tab.t[j]) / a.my, (cz + a.tab.t[k]) / a.mz, x);
    sX[0 * N3 + t] = x[0];
    sX[1 * N3 + t] = x[1];
    sX[2 * N3 + t] = x[2];
    if (a.xyz) {  // offsets from the cell's first node (the corner, GLL node 0 is 0)
      double c0[3];
      geo_point(a, (double)cx / a.mx, (double)cy / a.my, (double)cz / a.mz, c0);
      double* out = a.xyz + (size_t)cell * 3 * N3;
      out[0 * N3 + t] = x[0] - c0[0];
      out[1 * N3 + t] = x[1] - c0[1];
      out[2 * N3 + t] = x[2] - c0[2];
    }
  }
  if (!a.geo) return;
  __syncthreads();
  // x: thread (q1 = i, j, k) contracts over the node index along x
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    double A = 0.0, B = 0.0;
#pragma unroll
    for (int r = 0; r < N; ++r) {
      const double v = sX[c * N3 + (k * N + j) * N + r];
      A = fma(a.tab.V[i][r], v, A);
      B = fma(a.tab.Dh[i][r], v, B);
    }
    sA[c * N3 + t] = A;
    sB[c * N3 + t] = B;
  }
  __syncthreads();
  // y: thread (q1 = i, q2 = j, k)
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    double AA = 0.0, AB = 0.0, BA = 0.0;
#pragma unroll
    for (int r = 0; r < N; ++r) {
      const int e = c * N3 + (k * N + r) * N + i;
      AA = fma(a.tab.V[j][r], sA[e], AA);
      AB = fma(a.tab.Dh[j][r], sA[e], AB);
      BA = fma(a.tab.V[j][r], sB[e], BA);
    }
    sAA[c * N3 + t] = AA;
    sAB[c * N3 + t] = AB;
    sBA[c * N3 + t] = BA;
  }
  __syncthreads();
  // z: thread (q1 = i, q2 = j, q3 = k) finishes J[c][b] = d x_c / d xi_b
  double J[3][3];
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    double j0 = 0.0, j1 = 0.0, j2 = 0.0;
#pragma unroll
    for (int r = 0; r < N; ++r) {
      const int e = c * N3 + (r * N + j) * N + i;
      j0 = fma(a.tab.V[k][r], sBA[e], j0);
      j1 = fma(a.tab.V[k][r], sAB[e], j1);
      j2 = fma(a.tab.Dh[k][r], sAA[e], j2);
    }
    J[c][0] = j0;
    J[c][1] = j1;
    J[c][2] = j2;
  }
  const double det = J[0][0] * (J[1][1] * J[2][2] - J[1][2] * J[2][1]) -
                     J[0][1] * (J[1][0] * J[2][2] - J[1][2] * J[2][0]) +
                     J[0][2] * (J[1][0] * J[2][1] - J[1][1] * J[2][0]);
  const double id = 1.0 / det;
  double Ji[3][3];  // inverse via the adjugate
  Ji[0][0] = (J[1][1] * J[2][2] - J[1][2] * J[2][1]) * id;
  Ji[0][1] = (J[0][2] * J[2][1] - J[0][1] * J[2][2]) * id;
  Ji[0][2] = (J[0][1] * J[1][2] - J[0][2] * J[1][1]) * id;
  Ji[1][0] = (J[1][2] * J[2][0] - J[1][0] * J[2][2]) * id;
  Ji[1][1] = (J[0][0] * J[2][2] - J[0][2] * J[2][0]) * id;
  Ji[1][2] = (J[0][2] * J[1][0] - J[0][0] * J[1][2]) * id;
  Ji[2][0] = (J[1][0] * J[2][1] - J[1][1] * J[2][0]) * id;
  Ji[2][1] = (J[0][1] * J[2][0] - J[0][0] * J[2][1]) * id;
  Ji[2][2] = (J[0][0] * J[1][1] - J[0][1] * J[1][0]) * id;
  const double wd = a.tab.w[i] * a.tab.w[j] * a.tab.w[k] * det;
  // G_ab = wd * sum_c Ji[a][c] Ji[b][c]
  auto G = [&](int p, int q) {
    return wd * (Ji[p][0] * Ji[q][0] + Ji[p][1] * Ji[q][1] + Ji[p][2] * Ji[q][2]);
  };
  double* out = a.geo + (size_t)cell * FE_GEO_COMPS * N3;
  out[0 * N3 + t] = G(0, 0);
  out[1 * N3 + t] = G(1, 1);
  out[2 * N3 + t] = G(2, 2);
  out[3 * N3 + t] = G(0, 1);
  out[4 * N3 + t] = G(0, 2);
  out[5 * N3 + t] = G(1, 2);
  out[6 * N3 + t] = wd;
}

template <int N>
static fe_status launch_geometry(const GeoArgs& a, cudaStream_t st) {
  constexpr int N3 = N * N * N;
  size_t smem = 18 * N3 * sizeof(double);
  FE_CUDA(cudaFuncSetAttribute(k_geometry<N>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem),
          "geometry smem attribute");
  if (a.ncells > 0) k_geometry<N><<<(unsigned)a.ncells, N3, smem, st>>>(a);
  return fe_cuda_check(cudaGetLastError(), "geometry kernel launch");
}

// ---------------------------------------------------------------------------------------------
// precision copies of FP64 arrays (set-up only)
// ---------------------------------------------------------------------------------------------
__global__ void k_split_dw(const double* __restrict__ in, float2* __restrict__ out, long long n) {
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < n;
       e += (long long)gridDim.x * blockDim.x) {
    const double v = in[e];
    const float h = __double2float_rn(v);
    out[e] = make_float2(h, __double2float_rn(v - (double)h));
  }
}
__global__ void k_to_f32(const double* __restrict__ in, float* __restrict__ out, long long n) {
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < n;
       e += (long long)gridDim.x * blockDim.x)
    out[e] = __double2float_rn(in[e]);
}

// 16-bit metric copies: max |value| of the Laplace terms (components 0-5) and of w detJ
// (component 6), as ordered bit patterns of non-negative doubles
__global__ void k_geo_absmax(const double* __restrict__ g, long long n, int n3,
                             unsigned long long* __restrict__ out) {
  unsigned long long m0 = 0, m1 = 0;
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < n;
       e += (long long)gridDim.x * blockDim.x) {
    const unsigned long long b = (unsigned long long)__double_as_longlong(fabs(g[e]));
    if ((e / n3) % FE_GEO_COMPS == 6)
      m1 = b > m1 ? b : m1;
    else
      m0 = b > m0 ? b : m0;
  }
  atomicMax(out + 0, m0);
  atomicMax(out + 1, m1);
}
template <bool BF>
__global__ void k_to_h16(const double* __restrict__ g, unsigned short* __restrict__ out, long long n,
                         int n3, float s0, float s1) {
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < n;
       e += (long long)gridDim.x * blockDim.x) {
    const float v = (float)g[e] * ((e / n3) % FE_GEO_COMPS == 6 ? s1 : s0);
    if constexpr (BF)
      out[e] = __bfloat16_as_ushort(__float2bfloat16_rn(v));
    else
      out[e] = __half_as_ushort(__float2half_rn(v));
  }
}

static unsigned grid_for(long long n, int threads) {
  long long b = (n + threads - 1) / threads;
  if (b > 152LL * 64) b = 152LL * 64;
  if (b < 1) b = 1;
  return (unsigned)b;
}

fe_status fe_ensure_geometry(const fe_mesh* cm, int prec, bool native) {
  fe_mesh* m = const_cast<fe_mesh*>(cm);
  if (m->d.geom_mode == FE_GEOM_RECOMPUTE) {
    // coordinate copy in the arithmetic of the call, and that arithmetic's metric scratch
    const long long n = m->ncells * 3 * m->n3;
    const int idx = prec == FE_F32 ? 2 : (native ? 1 : 0);
    const size_t gv = idx == 2 ? sizeof(float) : (idx == 1 ? sizeof(double) : sizeof(float2));
    if (idx == 0 && !m->xyzdw) {
      FE_TRY(fe_dalloc((void**)&m->xyzdw, n * sizeof(float2), m->st, "coordinates (double-word)"));
      k_split_dw<<<grid_for(n, 256), 256, 0, m->st>>>(m->xyz64, m->xyzdw, n);
      FE_CUDA(cudaStreamSynchronize(m->st), "coordinates double-word split");
    } else if (idx == 2 && !m->xyz32) {
      FE_TRY(fe_dalloc((void**)&m->xyz32, n * sizeof(float), m->st, "coordinates (fp32)"));
      k_to_f32<<<grid_for(n, 256), 256, 0, m->st>>>(m->xyz64, m->xyz32, n);
      FE_CUDA(cudaStreamSynchronize(m->st), "coordinates fp32 copy");
    }
    if (!m->rc_scratch[idx]) {
      const long long cells = fe_rc_chunk_cells(m->n, m->ncells, gv);
      FE_TRY(fe_dalloc(&m->rc_scratch[idx], (size_t)cells * FE_GEO_COMPS * m->n3 * gv, m->st,
                       "recompute metric scratch"));
      FE_CUDA(cudaStreamSynchronize(m->st), "recompute metric scratch");
    }
    return FE_OK;
  }
  if (m->d.geom_mode != FE_GEOM_STORED) return FE_OK;
  const long long n = m->ncells * FE_GEO_COMPS * m->n3;
  if (prec == FE_BF16_F32ACC || prec == FE_F16_F32ACC) {
    const int k = prec == FE_BF16_F32ACC ? 0 : 1;
    if (m->geo16[k]) return fe_kron_build_tables(m, prec);
    if (!m->geo64) {
      fe_set_error("16-bit metric: the FP64 metric of this mesh has been released");
      return FE_ERR_INVALID;
    }
    // scale each metric family by a power of two that brings its largest value into [1/2, 1],
    // which keeps w detJ (about h^3) inside the fp16 range
    unsigned long long* dmax = nullptr;
    FE_TRY(fe_dalloc((void**)&dmax, 2 * sizeof(unsigned long long), m->st, "metric max"));
    FE_CUDA(cudaMemsetAsync(dmax, 0, 2 * sizeof(unsigned long long), m->st), "metric max");
    k_geo_absmax<<<grid_for(n, 256), 256, 0, m->st>>>(m->geo64, n, (int)m->n3, dmax);
    unsigned long long hmax[2] = {0, 0};
    FE_CUDA(cudaMemcpyAsync(hmax, dmax, sizeof(hmax), cudaMemcpyDeviceToHost, m->st), "metric max");
    FE_CUDA(cudaStreamSynchronize(m->st), "metric max");
    fe_dfree(dmax, m->st);
    for (int c = 0; c < 2; ++c) {
      double gm;
      std::memcpy(&gm, &hmax[c], sizeof(gm));
      m->gscale[c] = gm > 0.0 ? (float)std::ldexp(1.0, -std::ilogb(gm) - 1) : 1.0f;
    }
    FE_TRY(fe_dalloc((void**)&m->geo16[k], n * sizeof(unsigned short), m->st, "metric (16-bit)"));
    if (k == 0)
      k_to_h16<true><<<grid_for(n, 256), 256, 0, m->st>>>(m->geo64, m->geo16[k], n, (int)m->n3,
                                                          m->gscale[0], m->gscale[1]);
    else
      k_to_h16<false><<<grid_for(n, 256), 256, 0, m->st>>>(m->geo64, m->geo16[k], n, (int)m->n3,
                                                           m->gscale[0], m->gscale[1]);
    FE_CUDA(cudaStreamSynchronize(m->st), "metric (16-bit) copy");
    return fe_kron_build_tables(m, prec);
  }
  if ((prec == FE_F64 && !native && !m->geodw) || (prec == FE_F32 && !m->geo32) ||
      (prec == FE_F64 && native && !m->geo64)) {
    if (!m->geo64) {
      fe_set_error("geometry: the FP64 copy was released and the requested copy does not exist");
      return FE_ERR_INVALID;
    }
  }
  if (prec == FE_F64 && !native) {
    if (!m->geodw) {
      FE_TRY(fe_dalloc((void**)&m->geodw, n * sizeof(float2), m->st, "geometry (double-word)"));
      k_split_dw<<<grid_for(n, 256), 256, 0, m->st>>>(m->geo64, m->geodw, n);
      FE_CUDA(cudaStreamSynchronize(m->st), "geometry double-word split");
    }
  } else if (prec == FE_F32) {
    if (!m->geo32) {
      FE_TRY(fe_dalloc((void**)&m->geo32, n * sizeof(float), m->st, "geometry (fp32)"));
      k_to_f32<<<grid_for(n, 256), 256, 0, m->st>>>(m->geo64, m->geo32, n);
      FE_CUDA(cudaStreamSynchronize(m->st), "geometry fp32 copy");
    }
  }
  return FE_OK;
}

// ---------------------------------------------------------------------------------------------
// mesh object
// ---------------------------------------------------------------------------------------------
static void free_mesh(fe_mesh* m, cudaStream_t st) {
  if (!m) return;
  if (m->cg_work && m->cg_free) m->cg_free(m->cg_work, st);
  void* bufs[] = {m->geo64, m->geodw, m->geo32, m->geo16[0], m->geo16[1], m->xyz64, m->xyzdw,
                  m->xyz32, m->rc_scratch[0],
                  m->rc_scratch[1], m->rc_scratch[2], m->diag64[0],
                  m->diag64[1], m->invdiag32[0], m->invdiag32[1], m->invdiag64[0],
                  m->invdiag64[1], m->invmult64, m->red, m->hs_xu, m->hs_xc, m->hs_yc,
                  m->hs_yu[0], m->hs_yu[1], m->kron_tab[0][0], m->kron_tab[0][1],
                  m->kron_tab[1][0], m->kron_tab[1][1]};
  for (void* b : bufs) fe_dfree(b, st);
  for (cudaEvent_t e : m->hs_ev)
    if (e) cudaEventDestroy(e);
  if (m->hs_copy) cudaStreamDestroy(m->hs_copy);
  if (m->hs_up) cudaStreamDestroy(m->hs_up);
  if (m->st) cudaStreamDestroy(m->st);
  delete m;
}

void fe_mesh_release_async(fe_mesh* m, cudaStream_t st) { free_mesh(m, st); }

void fe_mesh_drop_geo64(fe_mesh* m, cudaStream_t st) {
  fe_dfree(m->geo64, st);
  m->geo64 = nullptr;
}

extern "C" fe_status fe_mesh_create(const fe_mesh_desc* d, void* stream, fe_mesh** out) {
  return fe_mesh_create_impl(d, nullptr, stream, out);
}

// corners: null for the unit-cube map Phi, else the 8 corners of a trilinear block (24 doubles)
fe_status fe_mesh_create_impl(const fe_mesh_desc* d, const double* corners, void* stream,
                              fe_mesh** out, int z0, int z1) {
  if (!d || !out) {
    fe_set_error("fe_mesh_create: null argument");
    return FE_ERR_INVALID;
  }
  *out = nullptr;
  if (d->degree < 1 || d->degree > 7) {
    fe_set_error("fe_mesh_create: degree %d outside [1,7]", d->degree);
    return FE_ERR_INVALID;
  }
  if (d->mx < 1 || d->my < 1 || d->mz < 1) {
    fe_set_error("fe_mesh_create: cell counts must be positive (%d,%d,%d)", d->mx, d->my, d->mz);
    return FE_ERR_INVALID;
  }
  if (d->geom_mode < FE_GEOM_STORED || d->geom_mode > FE_GEOM_AFFINE) {
    fe_set_error("fe_mesh_create: unknown geom_mode %d", d->geom_mode);
    return FE_ERR_INVALID;
  }
  if (d->geom_mode == FE_GEOM_AFFINE && d->deform_amp != 0.0) {
    fe_set_error("fe_mesh_create: FE_GEOM_AFFINE needs deform_amp == 0");
    return FE_ERR_INVALID;
  }
  if (d->layout != FE_LAYOUT_CELLS && d->layout != FE_LAYOUT_PACKED2) {
    fe_set_error("fe_mesh_create: unknown layout %d", d->layout);
    return FE_ERR_INVALID;
  }
  if (d->layout == FE_LAYOUT_PACKED2 &&
      ((d->mx | d->my | d->mz) & 1 || d->degree > 3 || d->geom_mode == FE_GEOM_RECOMPUTE)) {
    fe_set_error("fe_mesh_create: FE_LAYOUT_PACKED2 needs even cell counts, degree 1 to 3 and "
                 "stored or affine geometry");
    return FE_ERR_INVALID;
  }
  const bool slab = z1 > 0;
  if (slab && (z0 < 0 || z1 <= z0 || z1 > d->mz || d->layout != FE_LAYOUT_CELLS || corners)) {
    fe_set_error("fe_slab_create: need 0 <= z0 < z1 <= mz (%d, %d, %d) and FE_LAYOUT_CELLS", z0, z1,
                 d->mz);
    return FE_ERR_INVALID;
  }
  const int mzl = slab ? z1 - z0 : d->mz;  // layers of cells built here
  if (!(std::fabs(d->deform_amp) <= 0.2)) {
    fe_set_error("fe_mesh_create: |deform_amp| must be <= 0.2 (keeps the map invertible)");
    return FE_ERR_INVALID;
  }
  const long long ncells = (long long)d->mx * d->my * mzl;
  const long long n3 = (long long)(d->degree + 1) * (d->degree + 1) * (d->degree + 1);
  if (ncells * n3 > (1LL << 40)) {
    fe_set_error("fe_mesh_create: mesh too large");
    return FE_ERR_INVALID;
  }
  FeDeviceGuard device_guard;
  FE_CUDA(device_guard.set(d->device), "cudaSetDevice");
  fe_mesh* m = new (std::nothrow) fe_mesh();
  if (!m) {
    fe_set_error("fe_mesh_create: host allocation failed");
    return FE_ERR_OOM;
  }
  m->d = *d;
  m->d.mz = mzl;
  if (slab) {
    m->zoff = z0;
    m->mzg = d->mz;
    m->nbr_lo = z0 > 0;
    m->nbr_hi = z1 < d->mz;
  }
  m->p = d->degree;
  m->n = d->degree + 1;
  m->n3 = (int)n3;
  m->ncells = ncells;
  m->ncw = ncells * n3;
  m->nu = (long long)(d->mx * m->p + 1) * (d->my * m->p + 1) * ((long long)mzl * m->p + 1);
  m->packed = d->layout == FE_LAYOUT_PACKED2;
  m->sgx = m->packed ? d->mx / 2 : d->mx;
  m->sgy = m->packed ? d->my / 2 : d->my;
  m->sgz = m->packed ? d->mz / 2 : mzl;
  m->sn = m->packed ? 2 * m->p + 1 : m->n;
  if (m->packed) m->ncw = (long long)m->sgx * m->sgy * m->sgz * m->sn * m->sn * m->sn;
  fe_host_tables(m->p, &m->tab);
  cudaStream_t st = (cudaStream_t)stream;
  {
    fe_status cs = fe_cuda_check(cudaStreamCreateWithFlags(&m->st, cudaStreamNonBlocking), "mesh stream");
    if (cs != FE_OK) {
      delete m;
      return cs;
    }
  }

  GeoArgs g;
  std::memset(&g, 0, sizeof(g));
  g.ncells = ncells;
  g.mx = d->mx;
  g.my = d->my;
  g.mz = d->mz;
  g.z0 = slab ? z0 : 0;
  g.amp = d->deform_amp;
  if (corners) {
    g.tri = 1;
    for (int c = 0; c < 24; ++c) g.corners[c] = corners[c];
    m->tri = true;
  }
  for (int a = 0; a < m->n; ++a) {
    g.tab.t[a] = m->tab.t[a];
    g.tab.w[a] = m->tab.w[a];
    for (int b = 0; b < m->n; ++b) {
      g.tab.V[a][b] = m->tab.V[a][b];
      g.tab.Dh[a][b] = m->tab.Dh[a][b];
    }
  }
  fe_status s = FE_OK;
  if (d->geom_mode == FE_GEOM_STORED) {
    // per cell and quadrature point, whatever the storage layout of the vectors
    s = fe_dalloc((void**)&m->geo64, m->ncells * n3 * FE_GEO_COMPS * sizeof(double), st,
                  "geometry");
    g.geo = m->geo64;
  } else if (d->geom_mode == FE_GEOM_RECOMPUTE) {
    s = fe_dalloc((void**)&m->xyz64, m->ncells * n3 * 3 * sizeof(double), st, "coordinates");
    g.xyz = m->xyz64;
  }
  if (s == FE_OK && d->geom_mode != FE_GEOM_AFFINE) {
    switch (m->n) {
      case 2: s = launch_geometry<2>(g, st); break;
      case 3: s = launch_geometry<3>(g, st); break;
      case 4: s = launch_geometry<4>(g, st); break;
      case 5: s = launch_geometry<5>(g, st); break;
      case 6: s = launch_geometry<6>(g, st); break;
      case 7: s = launch_geometry<7>(g, st); break;
      case 8: s = launch_geometry<8>(g, st); break;
    }
  }
  if (s == FE_OK) s = fe_cuda_check(cudaStreamSynchronize(st), "geometry synchronize");
  if (s == FE_OK) s = fe_ensure_geometry(m, FE_F64, false);
  if (s != FE_OK) {
    cudaStreamSynchronize(st);
    free_mesh(m, st);
    return s;
  }
  *out = m;
  return FE_OK;
}

extern "C" fe_status fe_mesh_destroy(fe_mesh* m) {
  if (!m) return FE_OK;
  FeDeviceGuard device_guard;
  device_guard.set(m->d.device);
  cudaDeviceSynchronize();  // the mesh may have been used on any stream
  free_mesh(m, nullptr);
  cudaDeviceSynchronize();
  fe_pool_trim();
  return FE_OK;
}

extern "C" fe_status fe_mesh_layout(const fe_mesh* m, fe_layout* out) {
  if (!m || !out) {
    fe_set_error("fe_mesh_layout: null argument");
    return FE_ERR_INVALID;
  }
  out->n_cells = (long long)m->sgx * m->sgy * m->sgz;
  out->nodes_per_cell = (long long)m->sn * m->sn * m->sn;
  out->cellwise_len = m->ncw;
  out->unique_dofs = m->nu;
  out->layout_id = m->packed ? FE_LAYOUT_PACKED2 : FE_LAYOUT_CELLS;
  return FE_OK;
}

// ---------------------------------------------------------------------------------------------
// gather G: x_cell[e] = x_unique[global(e)]
// ---------------------------------------------------------------------------------------------
__global__ void k_gather(const double* __restrict__ xu, double* __restrict__ xc, long long ncw,
                         int n, int mx, int my) {
  const int p = n - 1, n3 = n * n * n;
  const long long Nx = (long long)mx * p + 1, Ny = (long long)my * p + 1;
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < ncw;
       e += (long long)gridDim.x * blockDim.x) {
    const long long cell = e / n3;
    const int loc = (int)(e - cell * n3);
    const int i = loc % n, j = (loc / n) % n, k = loc / (n * n);
    const long long cx = cell % mx, cy = (cell / mx) % my, cz = cell / ((long long)mx * my);
    xc[e] = xu[((cz * p + k) * Ny + (cy * p + j)) * Nx + (cx * p + i)];
  }
}

extern "C" fe_status fe_gather(const fe_mesh* m, const double* xu_host, double* xc_dev,
                               void* stream) {
  if (!m || !xu_host || !xc_dev || !fe_aligned(xc_dev)) {
    fe_set_error("fe_gather: null or misaligned argument");
    return FE_ERR_INVALID;
  }
  if (m->packed) {
    fe_set_error("fe_gather: FE_LAYOUT_CELLS meshes only");
    return FE_ERR_INVALID;
  }
  cudaStream_t st = (cudaStream_t)stream;
  double* tmp = nullptr;
  FE_CUDA(cudaMallocAsync(&tmp, m->nu * sizeof(double), st), "fe_gather: cudaMallocAsync");
  fe_status s = fe_cuda_check(
      cudaMemcpyAsync(tmp, xu_host, m->nu * sizeof(double), cudaMemcpyHostToDevice, st),
      "fe_gather: copy");
  if (s == FE_OK) {
    k_gather<<<grid_for(m->ncw, 256), 256, 0, st>>>(tmp, xc_dev, m->ncw, m->n, m->d.mx, m->d.my);
    s = fe_cuda_check(cudaGetLastError(), "fe_gather: launch");
  }
  cudaFreeAsync(tmp, st);
  if (s == FE_OK) s = fe_cuda_check(cudaStreamSynchronize(st), "fe_gather: synchronize");
  return s;
}
