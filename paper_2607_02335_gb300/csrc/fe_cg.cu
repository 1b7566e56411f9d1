// fe_cg.cu -- conjugate gradients on cell-wise data (Sec. 3.2, Algorithm "Communication-Free
// (Flexible) PCG") with the Jacobi preconditioner P = D_cell^{-1} S (Sec. 3.3).
//
// Every vector of the iteration is cell-wise: u, p, z primal (continuous), r, q dual.  The only
// inter-element step is the DSS inside the preconditioner; every scalar is a duality pairing of
// one dual and one primal vector (Lemma "Duality Pairing Identity"), so the iterates equal those
// of CG on the assembled system (Theorem "Equivalence of Communication-Free FCG").
//
// One iteration is a fixed launch sequence captured once into a CUDA graph:
//   q = A p;  <q,p> -> alpha;  u += alpha p, r -= alpha q;  w = S r;
//   z = D^{-1} w (0 on Dirichlet nodes) with sum w^2/mult, <r,z> (and <q,z> for FCG) -> beta;
//   p = z + beta p.
// alpha, beta, the residual and the stop flag stay in device memory; every kernel returns at once
// when the flag is set, so the host replays the graph several times between two reads of the flag.
// Convergence (unspecified in the paper): ||G^T r||_2 / ||G^T b||_2 <= rtol over free nodes, with
// ||G^T r||^2 = sum_e (S r)_e^2 / mult_e.
//
// Mixed precision: FP32 PCG with FP64 reliable updates (solve_reliable), or FP64 FCG whose variable
// preconditioner is an FP32 PCG solve (solve_fcg_outer).
#include <cmath>
#include <cstring>
#include <new>

#include "fe_cgcore.h"
#include "fe_vec.cuh"

namespace {

// ---- element-wise kernels -------------------------------------------------------------------
// 1/multiplicity per cell-wise node (0 on Dirichlet nodes).  A slab's bottom / top nodes have a
// copy in the neighbouring slab when nbr_lo / nbr_hi; `mask` holds the FE_DIR_* Dirichlet faces.
__global__ void k_invmult(float* __restrict__ out, long long ncells, int n, int mx, int my, int mz,
                          int mask, int nbr_lo, int nbr_hi) {
  const int n3 = n * n * n, p = n - 1;
  const int lane = threadIdx.x & 31;
  const long long warp = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const long long nwarps = ((long long)gridDim.x * blockDim.x) >> 5;
  for (long long c = warp; c < ncells; c += nwarps) {
    const int cx = (int)(c % mx), cy = (int)((c / mx) % my), cz = (int)(c / ((long long)mx * my));
    for (int l = lane; l < n3; l += 32) {
      const int i = l % n, j = (l / n) % n, k = l / (n * n);
      const int gx = cx * p + i, gy = cy * p + j, gz = cz * p + k;
      int mult = 1;
      if (gx % p == 0 && gx > 0 && gx < mx * p) mult *= 2;
      if (gy % p == 0 && gy > 0 && gy < my * p) mult *= 2;
      if (gz % p == 0 && ((gz > 0 && gz < mz * p) || (gz == 0 && nbr_lo) || (gz == mz * p && nbr_hi)))
        mult *= 2;
      const bool bnd = ((mask & FE_DIR_XY) && (gx == 0 || gx == mx * p || gy == 0 || gy == my * p)) ||
                       ((mask & FE_DIR_ZLO) && gz == 0) || ((mask & FE_DIR_ZHI) && gz == mz * p);
      out[c * n3 + l] = bnd ? 0.0f : 1.0f / (float)mult;
    }
  }
}

__global__ void k_invdiag(const double* __restrict__ d, const float* __restrict__ invmult,
                          double* __restrict__ inv64, float* __restrict__ inv32, long long n) {
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < n;
       e += (long long)gridDim.x * blockDim.x) {
    const double v = invmult[e] == 0.0f ? 0.0 : 1.0 / d[e];
    inv64[e] = v;
    inv32[e] = (float)v;
  }
}

// r = b - q
__global__ void k_residual(const double* __restrict__ b, const double* __restrict__ q,
                           double* __restrict__ r, long long n) {
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < n;
       e += (long long)gridDim.x * blockDim.x)
    r[e] = b[e] - q[e];
}

// largest |v| as the bit pattern of a non-negative double (whose order is the values' order)
__global__ void k_absmax_bits(const double* __restrict__ v, long long n,
                              unsigned long long* __restrict__ out) {
  unsigned long long m = 0;
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < n;
       e += (long long)gridDim.x * blockDim.x)
    m = max(m, (unsigned long long)__double_as_longlong(v[e]) & 0x7FFFFFFFFFFFFFFFull);
  for (int off = 16; off > 0; off >>= 1) m = max(m, __shfl_down_sync(0xffffffffu, m, off));
  if ((threadIdx.x & 31) == 0) atomicMax(out, m);
}

__global__ void k_scale_vec(const double* src, double* dst, double s, long long n) {
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < n;
       e += (long long)gridDim.x * blockDim.x)
    dst[e] = s * src[e];
}

// Inner right-hand side r32 = s * (S r) / mult, d32 = 0.  The dual residual r is unassembled: the
// copies of a node hold partial integrals that cancel when summed, so near convergence single
// copies are orders of magnitude larger than G^T r.  Rounding them to FP32 would destroy the
// assembled value; the residual is therefore assembled in FP64 first (w = S r) and its value is
// split evenly over the copies.  G^T r32 = s G^T r, and every pairing with a continuous vector is
// unchanged (Lemma "Duality Pairing Identity").
__global__ void k_to_inner(const double* __restrict__ w, const float* __restrict__ invmult,
                           float* __restrict__ r32, float* __restrict__ d32, double s, long long n) {
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < n;
       e += (long long)gridDim.x * blockDim.x) {
    r32[e] = (float)(s * w[e] * (double)invmult[e]);
    d32[e] = 0.0f;
  }
}

// x += d / s
__global__ void k_correct(double* __restrict__ x, const float* __restrict__ d, double inv_s,
                          long long n) {
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < n;
       e += (long long)gridDim.x * blockDim.x)
    x[e] += inv_s * (double)d[e];
}

// Elements per thread whose loads a two-input streaming kernel (<q,p>, the p update) issues
// together: eight FP32 elements keep as many bytes in flight per thread as four FP64 ones.
template <class S>
__host__ __device__ constexpr int stream_u() {
  return sizeof(S) == 4 ? 2 * RED_U : RED_U;
}

// u += alpha p ; r -= alpha q, and the new r also into w (the DSS then works on w in place).
// keep_r = 0 leaves r unwritten: with redistribution the preconditioner overwrites r with
// (S r)/mult before anything reads it, so the store would be dead traffic.  Launched on a
// resident grid (RED_BLOCKS CTAs); each thread issues the loads of RED_U of its grid-stride
// elements before their stores (the arrays are distinct): one element at a time, on a grid of
// 2432 CTAs, the kernel ran at 5.4 of the HBM's 6.7 TB/s.
template <class S, class U>
__global__ void k_update_ur(U* __restrict__ u, S* __restrict__ r, S* __restrict__ w,
                            const S* __restrict__ p, const S* __restrict__ q,
                            const CgScal* __restrict__ sc, long long n, int keep_r) {
  if (*(volatile const int*)&sc->done) return;
  const double a = sc->alpha;
  auto step = [&](long long e, U ue, S pe, S qe, S rq) {
    u[e] = (U)((double)ue + a * (double)pe);
    const S re = (S)((double)rq - a * (double)qe);
    if (keep_r) r[e] = re;
    w[e] = re;
  };
  const long long stride = (long long)gridDim.x * blockDim.x;
  long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  for (; e + (RED_U - 1) * stride < n; e += RED_U * stride) {
    U uv[RED_U];
    S pv[RED_U], qv[RED_U], rv[RED_U];
#pragma unroll
    for (int k = 0; k < RED_U; ++k) {
      const long long f = e + k * stride;
      uv[k] = u[f], pv[k] = p[f], qv[k] = q[f], rv[k] = r[f];
    }
#pragma unroll
    for (int k = 0; k < RED_U; ++k) step(e + k * stride, uv[k], pv[k], qv[k], rv[k]);
  }
  for (; e < n; e += stride) step(e, u[e], p[e], q[e], r[e]);
}

template <>
__global__ void k_update_ur<float, float>(float* __restrict__ u, float* __restrict__ r,
                                          float* __restrict__ w, const float* __restrict__ p,
                                          const float* __restrict__ q,
                                          const CgScal* __restrict__ sc, long long n, int keep_r) {
  if (*(volatile const int*)&sc->done) return;
  const float a = (float)sc->alpha;
  auto step = [&](long long e, float ue, float pe, float qe, float rq) {
    u[e] = fmaf(a, pe, ue);
    const float re = fmaf(-a, qe, rq);
    if (keep_r) r[e] = re;
    w[e] = re;
  };
  const long long stride = (long long)gridDim.x * blockDim.x;
  long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  for (; e + (RED_U - 1) * stride < n; e += RED_U * stride) {
    float uv[RED_U], pv[RED_U], qv[RED_U], rv[RED_U];
#pragma unroll
    for (int k = 0; k < RED_U; ++k) {
      const long long f = e + k * stride;
      uv[k] = u[f], pv[k] = p[f], qv[k] = q[f], rv[k] = r[f];
    }
#pragma unroll
    for (int k = 0; k < RED_U; ++k) step(e + k * stride, uv[k], pv[k], qv[k], rv[k]);
  }
  for (; e < n; e += stride) step(e, u[e], p[e], q[e], r[e]);
}

// p = z + c p (host scalar): the search direction kept across a reliable update
__global__ void k_keep_direction(float* __restrict__ p, const float* __restrict__ z, float c,
                                 long long n) {
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < n;
       e += (long long)gridDim.x * blockDim.x)
    p[e] = fmaf(c, p[e], z[e]);
}

// p = z + beta p (stream_u elements' loads in flight per thread, on a resident grid)
template <class S>
__global__ void k_update_p(S* __restrict__ p, const S* __restrict__ z, const CgScal* __restrict__ sc,
                           long long n) {
  if (*(volatile const int*)&sc->done) return;
  const S b = (S)sc->beta;
  constexpr int PU = stream_u<S>();
  const long long stride = (long long)gridDim.x * blockDim.x;
  long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  for (; e + (PU - 1) * stride < n; e += PU * stride) {
    S zv[PU], pv[PU];
#pragma unroll
    for (int k = 0; k < PU; ++k) zv[k] = z[e + k * stride], pv[k] = p[e + k * stride];
#pragma unroll
    for (int k = 0; k < PU; ++k) p[e + k * stride] = zv[k] + b * pv[k];
  }
  for (; e < n; e += stride) p[e] = z[e] + b * p[e];
}

template <class S>
__device__ __forceinline__ dw prod_dw(S a, S b);
template <>
__device__ __forceinline__ dw prod_dw<double>(double a, double b) {
  return dw_mul(dw_from_double(a), dw_from_double(b));
}
template <>
__device__ __forceinline__ dw prod_dw<float>(float a, float b) {
  const float p = __fmul_rn(a, b);
  return {p, __fmaf_rn(a, b, -p)};
}

// A thread's running sum of products in a pairing: float vectors in double-word (exact products);
// double vectors in binary64 FMAs on the FP64 pipe, one per product, which costs less than
// converting both factors to double-word (the conversions were the kernels' issue bound)
template <class S>
struct Acc;
template <>
struct Acc<float> {
  dw v = {0.0f, 0.0f};
  __device__ __forceinline__ void add_prod(float a, float b) { v = dw_add(v, prod_dw<float>(a, b)); }
  __device__ __forceinline__ dw value() const { return v; }
};
template <>
struct Acc<double> {
  double v = 0.0;
  __device__ __forceinline__ void add_prod(double a, double b) { v = fma(a, b, v); }
  __device__ __forceinline__ dw value() const { return dw_from_double(v); }
};
// double-word for both: the preconditioner kernel already spends its FP64-pipe share on z = w /
// diag (measured: binary64 FMAs for <r,z> there made it slower, 165 -> 202 us at Q3 64^3)
template <class S>
struct AccDw {
  dw v = {0.0f, 0.0f};
  __device__ __forceinline__ void add_prod(S a, S b) { v = dw_add(v, prod_dw<S>(a, b)); }
  __device__ __forceinline__ dw value() const { return v; }
};

// partial of <q, p>  (slot 0)
template <class S>
__global__ void __launch_bounds__(RED_THREADS)
    k_qp(const S* __restrict__ q, const S* __restrict__ p, double* __restrict__ partials,
         const CgScal* __restrict__ sc, long long n) {
  if (*(volatile const int*)&sc->done) return;
  __shared__ dw sh[32];
  Acc<S> acc;
  constexpr long long STRIDE = (long long)RED_BLOCKS * RED_THREADS;
  constexpr int QU = stream_u<S>();
  long long e = (long long)blockIdx.x * RED_THREADS + threadIdx.x;
  // QU elements' loads in flight before their products join the accumulator, in the same order
  for (; e + (QU - 1) * STRIDE < n; e += QU * STRIDE) {
    S qv[QU], pv[QU];
#pragma unroll
    for (int u = 0; u < QU; ++u) {
      qv[u] = q[e + u * STRIDE];
      pv[u] = p[e + u * STRIDE];
    }
#pragma unroll
    for (int u = 0; u < QU; ++u) acc.add_prod(qv[u], pv[u]);
  }
  for (; e < n; e += STRIDE) acc.add_prod(q[e], p[e]);
  const dw accv = block_reduce_dw(acc.value(), sh);
  if (threadIdx.x == 0) partials[blockIdx.x] = dw_to_double(accv);
}

// z = w * invdiag (when z != null); partials: slot 0 sum w^2 invmult, slot 1 <r,z>, slot 2 <q,z>
// With `redistribute` the dual residual is replaced by its assembled value split evenly over the
// copies, r = (S r) / mult (0 on Dirichlet nodes): the same G^T r and the same pairings with
// continuous vectors, without the cancelling per-copy parts that FP32 cannot hold.
template <class S>
__global__ void __launch_bounds__(RED_THREADS)
    k_precond(const S* __restrict__ w, S* __restrict__ r, const S* __restrict__ q,
              const S* __restrict__ invdiag, const float* __restrict__ invmult, S* __restrict__ z,
              double* __restrict__ partials, const CgScal* __restrict__ sc, long long n,
              int check_done, int redistribute) {
  if (check_done && *(volatile const int*)&sc->done) return;
  __shared__ dw sh[32];
  dw a0 = {0.0f, 0.0f};
  AccDw<S> a1, a2;
  auto body = [&](long long e, S we, float im, S idg, S rv, S qv) {
    const dw w2 = prod_dw<S>(we, we);
    a0 = dw_add(a0, {w2.h * im, w2.l * im});  // im: a power of two or zero, exact scaling
    if (z) {
      const S ze = we * idg;
      z[e] = ze;
      S re;
      if (redistribute) {
        re = we * (S)im;
        r[e] = re;
      } else {
        re = rv;
      }
      a1.add_prod(re, ze);
      if (q) a2.add_prod(qv, ze);
    }
  };
  constexpr long long STRIDE = (long long)RED_BLOCKS * RED_THREADS;
  long long e = (long long)blockIdx.x * RED_THREADS + threadIdx.x;
  // RED_U elements' loads in flight before they join the accumulators, in the same order
  for (; e + (RED_U - 1) * STRIDE < n; e += RED_U * STRIDE) {
    S wv[RED_U], idg[RED_U], rv[RED_U], qv[RED_U];
    float im[RED_U];
#pragma unroll
    for (int u = 0; u < RED_U; ++u) {
      const long long f = e + u * STRIDE;
      wv[u] = w[f];
      im[u] = invmult[f];
      idg[u] = z ? invdiag[f] : S(0);
      rv[u] = (z && !redistribute) ? r[f] : S(0);
      qv[u] = (z && q) ? q[f] : S(0);
    }
#pragma unroll
    for (int u = 0; u < RED_U; ++u) body(e + u * STRIDE, wv[u], im[u], idg[u], rv[u], qv[u]);
  }
  for (; e < n; e += STRIDE)
    body(e, w[e], invmult[e], z ? invdiag[e] : S(0), (z && !redistribute) ? r[e] : S(0),
         (z && q) ? q[e] : S(0));
  a0 = block_reduce_dw(a0, sh);
  if (threadIdx.x == 0) partials[0 * RED_BLOCKS + blockIdx.x] = dw_to_double(a0);
  if (z) {
    const dw v1 = block_reduce_dw(a1.value(), sh);
    if (threadIdx.x == 0) partials[1 * RED_BLOCKS + blockIdx.x] = dw_to_double(v1);
    if (q) {
      const dw v2 = block_reduce_dw(a2.value(), sh);
      if (threadIdx.x == 0) partials[2 * RED_BLOCKS + blockIdx.x] = dw_to_double(v2);
    }
  }
}

__device__ double sum_slot(const double* partials, int slot, dw* sh) {
  dw acc = {0.0f, 0.0f};
  for (int b = threadIdx.x; b < RED_BLOCKS; b += RED_THREADS)
    acc = dw_add(acc, dw_from_double(partials[slot * RED_BLOCKS + b]));
  acc = block_reduce_dw(acc, sh);
  return dw_to_double(acc);  // valid in thread 0
}

// alpha = <r,z>/<q,p>
__global__ void __launch_bounds__(RED_THREADS)
    k_fin_alpha(const double* __restrict__ partials, CgScal* __restrict__ sc, double* hist) {
  if (*(volatile const int*)&sc->done) return;
  __shared__ dw sh[32];
  const double qp = sum_slot(partials, 0, sh);
  if (threadIdx.x == 0) {
    sc->qp = qp;
    if (!(qp > 0.0) || !isfinite(qp) || !isfinite(sc->rz)) {
      sc->status = FE_ERR_BREAKDOWN;
      sc->done = 1;
    } else {
      sc->alpha = sc->rz / qp;
      if (hist) hist[3 * sc->iter + 0] = sc->alpha;
    }
  }
}

// residual norm, convergence test and beta
__global__ void __launch_bounds__(RED_THREADS)
    k_fin_beta(const double* __restrict__ partials, CgScal* __restrict__ sc, double rtol, int mode,
               int flexible, double* hist) {
  if ((mode == FIN_ITER || mode == FIN_OUTER) && *(volatile const int*)&sc->done) return;
  __shared__ dw sh[32];
  const double rn2 = sum_slot(partials, 0, sh);
  const double rz = (mode == FIN_INIT_R || mode == FIN_ITER) ? sum_slot(partials, 1, sh) : 0.0;
  const double qz = (mode == FIN_ITER && flexible) ? sum_slot(partials, 2, sh) : 0.0;
  if (threadIdx.x != 0) return;
  const int k = sc->iter;
  fin_scalars(sc, rn2, rz, qz, rtol < 0.0 ? sc->rtol : rtol, mode, flexible);
  if (hist && mode == FIN_ITER) {
    hist[3 * k + 2] = sc->relres;
    if (!sc->done) hist[3 * k + 1] = sc->beta;
  }
}

// z = d / s (FP64 primal correction from the FP32 inner solve)
__global__ void k_from_inner(double* __restrict__ z, const float* __restrict__ d, double inv_s,
                             long long n) {
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < n;
       e += (long long)gridDim.x * blockDim.x)
    z[e] = inv_s * (double)d[e];
}

// partials: slot 1 <r, z>, slot 2 <q, z> (q may be null)
__global__ void __launch_bounds__(RED_THREADS)
    k_zpairs(const double* __restrict__ r, const double* __restrict__ q,
             const double* __restrict__ z, double* __restrict__ partials, long long n) {
  __shared__ dw sh[32];
  dw a1 = {0.0f, 0.0f}, a2 = {0.0f, 0.0f};
  for (long long e = (long long)blockIdx.x * RED_THREADS + threadIdx.x; e < n;
       e += (long long)RED_BLOCKS * RED_THREADS) {
    const double ze = z[e];
    a1 = dw_add(a1, prod_dw<double>(r[e], ze));
    if (q) a2 = dw_add(a2, prod_dw<double>(q[e], ze));
  }
  a1 = block_reduce_dw(a1, sh);
  if (threadIdx.x == 0) partials[1 * RED_BLOCKS + blockIdx.x] = dw_to_double(a1);
  if (q) {
    a2 = block_reduce_dw(a2, sh);
    if (threadIdx.x == 0) partials[2 * RED_BLOCKS + blockIdx.x] = dw_to_double(a2);
  }
}

// outer FCG scalars: init rz = <r,z>; iteration beta = -<q,z>/<q,p>, rz = <r,z>
__global__ void __launch_bounds__(RED_THREADS)
    k_fin_fcg(const double* __restrict__ partials, CgScal* __restrict__ sc, int init) {
  __shared__ dw sh[32];
  const double rz = sum_slot(partials, 1, sh);
  const double qz = init ? 0.0 : sum_slot(partials, 2, sh);
  if (threadIdx.x != 0) return;
  if (!init) sc->beta = -qz / sc->qp;
  sc->rz = rz;
}

unsigned grid_for(long long n) {
  long long b = (n + 255) / 256;
  if (b > 152LL * 16) b = 152LL * 16;
  return (unsigned)(b < 1 ? 1 : b);
}

// ---- workspace -------------------------------------------------------------------------------
}  // namespace

static void free_work(CgWork* w, cudaStream_t st) {
  if (!w) return;
  for (int f = 0; f < 2; ++f) {
    if (w->g64[f]) cudaGraphExecDestroy(w->g64[f]);
    if (w->g32[f]) cudaGraphExecDestroy(w->g32[f]);
  }
  void* bufs[] = {w->x, w->r, w->z, w->p, w->q, w->w, w->bs, w->invdiag64, w->partials, w->hist,
                  w->r32, w->z32, w->p32, w->q32, w->w32, w->d32, w->invdiag32, w->invmult, w->sc};
  for (void* b : bufs) fe_dfree(b, st);
  cudaFreeHost(w->hsc);
  if (w->st) cudaStreamDestroy(w->st);
  delete w;
}

fe_status fe_launch_invmult(const fe_mesh* m, float* out, cudaStream_t st) {
  k_invmult<<<grid_for(m->ncells * 32), 256, 0, st>>>(out, m->ncells, m->n, m->d.mx, m->d.my,
                                                      m->d.mz, fe_dir_mask(m), m->nbr_lo,
                                                      m->nbr_hi);
  return fe_cuda_check(cudaGetLastError(), "invmult launch");
}

fe_status fe_cg_get_work(const fe_mesh* cm, bool mixed, CgWork** out) {
  fe_mesh* m = const_cast<fe_mesh*>(cm);
  CgWork* w = static_cast<CgWork*>(m->cg_work);
  if (!w) {
    w = new (std::nothrow) CgWork();
    if (!w) {
      fe_set_error("fe_cg_solve: host allocation failed");
      return FE_ERR_OOM;
    }
    m->cg_work = w;
    m->cg_free = [](void* p, cudaStream_t st) { free_work(static_cast<CgWork*>(p), st); };
    const long long n = m->ncw;
    w->n = n;
    FE_CUDA(cudaStreamCreateWithFlags(&w->st, cudaStreamNonBlocking), "cg stream");
    double** d[] = {&w->x, &w->r, &w->z, &w->p, &w->q, &w->w, &w->bs, &w->invdiag64};
    for (double** v : d) FE_TRY(fe_dalloc((void**)v, n * sizeof(double), w->st, "cg vector"));
    FE_TRY(fe_dalloc((void**)&w->invdiag32, n * sizeof(float), w->st, "cg vector"));
    FE_TRY(fe_dalloc((void**)&w->invmult, n * sizeof(float), w->st, "cg vector"));
    FE_TRY(fe_dalloc((void**)&w->partials, (size_t)RED_BLOCKS * RED_SLOTS * sizeof(double), w->st,
                     "cg partials"));
    FE_TRY(fe_dalloc((void**)&w->sc, 2 * sizeof(CgScal), w->st, "cg scalars"));
    FE_CUDA(cudaMallocHost(&w->hsc, 2 * sizeof(CgScal)), "cudaMallocHost cg scalars");
    FE_TRY(fe_launch_invmult(m, w->invmult, w->st));
  }
  if (mixed && !w->r32) {
    float** f[] = {&w->r32, &w->z32, &w->p32, &w->q32, &w->w32, &w->d32};
    for (float** v : f) FE_TRY(fe_dalloc((void**)v, w->n * sizeof(float), w->st, "cg fp32 vector"));
  }
  *out = w;
  return FE_OK;
}

fe_status fe_cg_ensure_diag(const fe_mesh* m, CgWork* w, int op) {
  if (w->diag_op == op) return FE_OK;
  // w->q as scratch for the assembled diagonal
  FE_TRY(fe_launch_diag(m, op, w->q, w->st));
  k_invdiag<<<grid_for(w->n), 256, 0, w->st>>>(w->q, w->invmult, w->invdiag64, w->invdiag32, w->n);
  FE_CUDA(cudaGetLastError(), "invdiag launch");
  w->diag_op = op;
  return FE_OK;
}

namespace {

// the operator of the FP32 inner solve: FP32, or 16-bit operands with FP32 accumulation
fe_status launch_inner_apply(const ApplyLaunch& L, const CgWork* w) {
  return w->inner_prec == FE_F32 ? fe_launch_apply_f32(L) : fe_launch_apply_lowp(L, w->inner_prec);
}

// one PCG iteration on vectors of type S, solution of type U, scalars sc
template <class S, class U>
fe_status enqueue_iteration(const fe_mesh* m, CgWork* w, int op, bool flexible, U* u, S* r, S* z,
                            S* p, S* q, S* wv, const S* invdiag, CgScal* sc, double* hist) {
  const long long n = w->n;
  ApplyLaunch L{m, op, p, q, w->st, &sc->done};
  if (sizeof(S) == 8)
    FE_TRY(fe_launch_apply_f64dw(L));
  else
    FE_TRY(launch_inner_apply(L, w));
  // FP32 iterations redistribute: r = (S r)/mult is formed by the preconditioner
  const int redistribute = sizeof(S) == 4 ? 1 : 0;
  k_qp<S><<<RED_BLOCKS, RED_THREADS, 0, w->st>>>(q, p, w->partials, sc, n);
  k_fin_alpha<<<1, RED_THREADS, 0, w->st>>>(w->partials, sc, hist);
  k_update_ur<S, U><<<RED_BLOCKS, RED_THREADS, 0, w->st>>>(u, r, wv, p, q, sc, n, !redistribute);
  FE_TRY(fe_launch_dss(m, sizeof(S) == 8 ? FE_F64 : FE_F32, wv, w->st));
  k_precond<S><<<RED_BLOCKS, RED_THREADS, 0, w->st>>>(wv, r, flexible ? q : nullptr, invdiag,
                                                      w->invmult, z, w->partials, sc, n, 1,
                                                      redistribute);
  k_fin_beta<<<1, RED_THREADS, 0, w->st>>>(w->partials, sc, -1.0, FIN_ITER, flexible ? 1 : 0, hist);
  k_update_p<S><<<RED_BLOCKS, RED_THREADS, 0, w->st>>>(p, z, sc, n);
  return fe_cuda_check(cudaGetLastError(), "cg iteration launch");
}

// the iteration graph; its stopping tolerance is read from sc->rtol at every replay
template <class S, class U>
fe_status build_graph(const fe_mesh* m, CgWork* w, int op, bool flexible, U* u, S* r, S* z, S* p,
                      S* q, S* wv, const S* invdiag, CgScal* sc, double* hist,
                      cudaGraphExec_t* exec) {
  cudaGraph_t g = nullptr;
  {  // one uncaptured apply first, so that per-kernel attributes are set outside the capture
    ApplyLaunch L{m, op, p, q, w->st, &sc->done};
    FE_TRY(sizeof(S) == 8 ? fe_launch_apply_f64dw(L) : launch_inner_apply(L, w));
  }
  FE_CUDA(cudaStreamBeginCapture(w->st, cudaStreamCaptureModeThreadLocal), "begin capture");
  fe_status s = enqueue_iteration<S, U>(m, w, op, flexible, u, r, z, p, q, wv, invdiag, sc, hist);
  cudaError_t e = cudaStreamEndCapture(w->st, &g);
  if (s != FE_OK) {
    if (g) cudaGraphDestroy(g);
    return s;
  }
  FE_CUDA(e, "end capture");
  e = cudaGraphInstantiate(exec, g, 0);
  cudaGraphDestroy(g);
  return fe_cuda_check(e, "graph instantiate");
}

// run graph replays until the flag is set; returns the host copy of the scalars
fe_status run_until_done(CgWork* w, cudaGraphExec_t exec, int slot, CgScal* out) {
  const int batch = 8;
  for (;;) {
    for (int b = 0; b < batch; ++b) FE_CUDA(cudaGraphLaunch(exec, w->st), "graph launch");
    FE_CUDA(cudaMemcpyAsync(&w->hsc[slot], &w->sc[slot], sizeof(CgScal), cudaMemcpyDeviceToHost,
                            w->st),
            "scalar readback");
    FE_CUDA(cudaStreamSynchronize(w->st), "cg synchronize");
    if (w->hsc[slot].done) break;
  }
  *out = w->hsc[slot];
  return FE_OK;
}

// fresh scalars of a run; rtol is the stopping tolerance the replayed iteration graphs read
fe_status set_scal(CgWork* w, int slot, int maxit, int stall_limit, double rtol) {
  CgScal s;
  std::memset(&s, 0, sizeof(s));
  s.maxit = maxit;
  s.stall_limit = stall_limit;
  s.rtol = rtol;
  w->hsc[slot] = s;
  return fe_cuda_check(
      cudaMemcpyAsync(&w->sc[slot], &w->hsc[slot], sizeof(CgScal), cudaMemcpyHostToDevice, w->st),
      "scalar upload");
}

fe_status read_scal(CgWork* w, int slot, CgScal* out) {
  FE_CUDA(cudaMemcpyAsync(&w->hsc[slot], &w->sc[slot], sizeof(CgScal), cudaMemcpyDeviceToHost, w->st),
          "scalar readback");
  FE_CUDA(cudaStreamSynchronize(w->st), "cg synchronize");
  *out = w->hsc[slot];
  return FE_OK;
}

// ||G^T v||^2 / bnorm into slot's scalars: w = S v, precond kernel without z
template <class S>
fe_status residual_norm(const fe_mesh* m, CgWork* w, const S* v, S* wv, CgScal* sc, int mode) {
  FE_CUDA(cudaMemcpyAsync(wv, v, w->n * sizeof(S), cudaMemcpyDeviceToDevice, w->st), "cg copy");
  FE_TRY(fe_launch_dss(m, sizeof(S) == 8 ? FE_F64 : FE_F32, wv, w->st));
  k_precond<S><<<RED_BLOCKS, RED_THREADS, 0, w->st>>>(wv, nullptr, nullptr, nullptr, w->invmult,
                                                      nullptr, w->partials, sc, w->n, 0, 0);
  k_fin_beta<<<1, RED_THREADS, 0, w->st>>>(w->partials, sc, 0.0, mode, 0, nullptr);
  return fe_cuda_check(cudaGetLastError(), "residual norm launch");
}

// initial preconditioned residual: w = S r, z = D^{-1} w, <r,z>, relres; p = z
template <class S>
fe_status init_direction(const fe_mesh* m, CgWork* w, S* r, S* z, S* p, S* wv, const S* invdiag,
                         CgScal* sc, double rtol) {
  FE_CUDA(cudaMemcpyAsync(wv, r, w->n * sizeof(S), cudaMemcpyDeviceToDevice, w->st), "cg copy");
  FE_TRY(fe_launch_dss(m, sizeof(S) == 8 ? FE_F64 : FE_F32, wv, w->st));
  k_precond<S><<<RED_BLOCKS, RED_THREADS, 0, w->st>>>(wv, r, nullptr, invdiag, w->invmult, z,
                                                      w->partials, sc, w->n, 0, sizeof(S) == 4 ? 1 : 0);
  k_fin_beta<<<1, RED_THREADS, 0, w->st>>>(w->partials, sc, rtol, FIN_INIT_R, 0, nullptr);
  FE_CUDA(cudaMemcpyAsync(p, z, w->n * sizeof(S), cudaMemcpyDeviceToDevice, w->st), "cg copy");
  return fe_cuda_check(cudaGetLastError(), "init launch");
}

// Inner FP32 PCG on A d = s S(r)/mult with s = 1/||G^T r|| (w must hold S r in FP64, rnorm2
// its squared norm).  Returns the inner iteration count in *iters and the scale s.
fe_status inner_solve(const fe_mesh* m, CgWork* w, int op, int flex, double rnorm2, double irtol,
                      int maxit, int* iters, double* s_out) {
  const long long n = w->n;
  const double s = 1.0 / sqrt(rnorm2);
  k_to_inner<<<grid_for(n), 256, 0, w->st>>>(w->w, w->invmult, w->r32, w->d32, s, n);
  FE_TRY(set_scal(w, 1, maxit, 20, irtol));
  FE_TRY(residual_norm<float>(m, w, w->r32, w->w32, &w->sc[1], FIN_INIT_B));
  FE_TRY(init_direction<float>(m, w, w->r32, w->z32, w->p32, w->w32, w->invdiag32, &w->sc[1], irtol));
  CgScal h;
  FE_TRY(read_scal(w, 1, &h));
  if (!h.done) {
    if (!w->g32[flex])
      FE_TRY((build_graph<float, float>(m, w, op, flex, w->d32, w->r32, w->z32, w->p32, w->q32,
                                        w->w32, w->invdiag32, &w->sc[1], nullptr, &w->g32[flex])));
    FE_TRY(run_until_done(w, w->g32[flex], 1, &h));
  }
  *iters = h.iter;
  *s_out = s;
  if (h.status == FE_ERR_BREAKDOWN && h.iter == 0) {
    fe_set_error("fe_cg_solve: inner breakdown");
    return FE_ERR_BREAKDOWN;
  }
  return FE_OK;
}

// FP64 flexible CG whose preconditioner is an FP32 PCG solve: z = P(r) = d / s.  P consumes r only
// through S r = G (G^T r) and returns a continuous vector, the consistency the Equivalence theorem
// asks of a (variable) preconditioner; FCG (Notay) absorbs the variation between applications.
fe_status solve_fcg_outer(const fe_mesh* m, CgWork* w, int op, const double* b, double bnorm2,
                          const fe_cg_opts* opts, fe_cg_result* res, fe_status* status) {
  const long long n = w->n;
  const double irtol = opts->inner_rtol > 0.0 ? opts->inner_rtol : 1e-2;
  CgScal h;
  int total = 0, outer = 0, its = 0;
  double s = 1.0;
  // r = b - A x ; ||G^T r||
  {
    ApplyLaunch L{m, op, w->x, w->q, w->st, nullptr};
    FE_TRY(fe_launch_apply_f64dw(L));
  }
  k_residual<<<grid_for(n), 256, 0, w->st>>>(b, w->q, w->r, n);
  FE_TRY(residual_norm<double>(m, w, w->r, w->w, &w->sc[0], FIN_NORM));
  FE_TRY(read_scal(w, 0, &h));
  res->rel_res = sqrt(h.rnorm2 / bnorm2);
  if (res->rel_res <= opts->rtol) {
    *status = FE_OK;
    return FE_OK;
  }
  // z = P(r), p = z, rz = <r, z>
  FE_TRY(inner_solve(m, w, op, 0, h.rnorm2, irtol, opts->maxit, &its, &s));
  total += its;
  k_from_inner<<<grid_for(n), 256, 0, w->st>>>(w->z, w->d32, 1.0 / s, n);
  k_zpairs<<<RED_BLOCKS, RED_THREADS, 0, w->st>>>(w->r, nullptr, w->z, w->partials, n);
  k_fin_fcg<<<1, RED_THREADS, 0, w->st>>>(w->partials, &w->sc[0], 1);
  FE_CUDA(cudaMemcpyAsync(w->p, w->z, n * sizeof(double), cudaMemcpyDeviceToDevice, w->st), "copy");
  *status = FE_ERR_NOT_CONVERGED;
  while (total < opts->maxit) {
    ApplyLaunch L{m, op, w->p, w->q, w->st, nullptr};
    FE_TRY(fe_launch_apply_f64dw(L));
    k_qp<double><<<RED_BLOCKS, RED_THREADS, 0, w->st>>>(w->q, w->p, w->partials, &w->sc[0], n);
    k_fin_alpha<<<1, RED_THREADS, 0, w->st>>>(w->partials, &w->sc[0], nullptr);
    k_update_ur<double, double><<<RED_BLOCKS, RED_THREADS, 0, w->st>>>(
        w->x, w->r, w->w, w->p, w->q, &w->sc[0], n, 1);
    FE_TRY(residual_norm<double>(m, w, w->r, w->w, &w->sc[0], FIN_NORM));
    FE_TRY(read_scal(w, 0, &h));
    ++outer;
    res->rel_res = h.relres;
    if (h.done) {  // breakdown flagged by k_fin_alpha
      *status = (fe_status)h.status;
      break;
    }
    if (!std::isfinite(h.relres)) {
      *status = FE_ERR_BREAKDOWN;
      break;
    }
    if (h.relres <= opts->rtol) {
      *status = FE_OK;
      break;
    }
    FE_TRY(inner_solve(m, w, op, 0, h.rnorm2, irtol, opts->maxit - total, &its, &s));
    total += its;
    k_from_inner<<<grid_for(n), 256, 0, w->st>>>(w->z, w->d32, 1.0 / s, n);
    k_zpairs<<<RED_BLOCKS, RED_THREADS, 0, w->st>>>(w->r, w->q, w->z, w->partials, n);
    k_fin_fcg<<<1, RED_THREADS, 0, w->st>>>(w->partials, &w->sc[0], 0);
    k_update_p<double><<<RED_BLOCKS, RED_THREADS, 0, w->st>>>(w->p, w->z, &w->sc[0], n);
    FE_CUDA(cudaGetLastError(), "fcg launch");
  }
  res->iters = total;
  res->outer_iters = outer;
  return FE_OK;
}

// FP32 PCG with FP64 reliable updates (residual replacement; Sleijpen & van der Vorst 1996, the
// mixed-precision form of Clark et al. 2010): the iteration runs on FP32 vectors and the FP32
// operator; whenever its recursive residual has dropped by the factor delta since the last
// replacement, the correction accumulated in FP32 is added to the FP64 solution, the true residual
// b - A x is formed with the FP64 operator and replaces the recursive one (assembled in FP64 and
// split evenly over the copies of each node, scaled to unit norm), and the search direction is
// kept: p = P r' + beta p with beta = <r', P r'> / <r_{k-1}, z_{k-1}>.  Keeping p keeps the
// Krylov space, so the iteration count stays near that of FP64 PCG, while every step but the few
// replacements runs in FP32.  The FP64 residual of the final iterate decides convergence.
fe_status solve_reliable(const fe_mesh* m, CgWork* w, int op, const double* b, double bnorm2,
                         const fe_cg_opts* opts, fe_cg_result* res, fe_status* status) {
  const long long n = w->n;
  const double delta = opts->inner_rtol > 0.0 ? opts->inner_rtol : 0.1;
  int total = 0, outer = 0;
  double s_old = 0.0, rz_old = 0.0;  // scale and <r, z> (scaled units) when the FP32 run stopped
  bool have_p = false;
  CgScal h;
  for (;;) {
    // true FP64 residual of the current iterate; w = S r for the inner right-hand side
    ApplyLaunch L{m, op, w->x, w->q, w->st, nullptr};
    FE_TRY(fe_launch_apply_f64dw(L));
    k_residual<<<grid_for(n), 256, 0, w->st>>>(b, w->q, w->r, n);
    FE_TRY(residual_norm<double>(m, w, w->r, w->w, &w->sc[0], FIN_NORM));
    FE_TRY(read_scal(w, 0, &h));
    const double rel = sqrt(h.rnorm2 / bnorm2);
    res->rel_res = rel;
    if (rel <= opts->rtol) {
      *status = FE_OK;
      break;
    }
    if (!std::isfinite(rel)) {
      *status = FE_ERR_BREAKDOWN;
      break;
    }
    if (total >= opts->maxit) {
      *status = FE_ERR_NOT_CONVERGED;
      break;
    }
    // run the FP32 iteration down to delta, or to just below the outer target
    const double irtol = std::max(delta, 0.5 * opts->rtol / rel);
    FE_TRY(set_scal(w, 1, opts->maxit - total, 0, irtol));
    // r32 = s (S r) / mult, d32 = 0
    const double s = 1.0 / sqrt(h.rnorm2);
    k_to_inner<<<grid_for(n), 256, 0, w->st>>>(w->w, w->invmult, w->r32, w->d32, s, n);
    FE_TRY(residual_norm<float>(m, w, w->r32, w->w32, &w->sc[1], FIN_INIT_B));
    if (!have_p) {
      FE_TRY(init_direction<float>(m, w, w->r32, w->z32, w->p32, w->w32, w->invdiag32, &w->sc[1],
                                   irtol));
      FE_TRY(read_scal(w, 1, &h));
    } else {
      // z = P r', <r', z>; p = z + beta p in the new scale (p and rz_old were in units of s_old)
      FE_CUDA(cudaMemcpyAsync(w->w32, w->r32, n * sizeof(float), cudaMemcpyDeviceToDevice, w->st),
              "cg copy");
      FE_TRY(fe_launch_dss(m, FE_F32, w->w32, w->st));
      k_precond<float><<<RED_BLOCKS, RED_THREADS, 0, w->st>>>(w->w32, w->r32, nullptr, w->invdiag32,
                                                              w->invmult, w->z32, w->partials,
                                                              &w->sc[1], n, 0, 1);
      k_fin_beta<<<1, RED_THREADS, 0, w->st>>>(w->partials, &w->sc[1], irtol, FIN_INIT_R, 0, nullptr);
      FE_TRY(read_scal(w, 1, &h));
      const double ratio = s / s_old;
      const double beta = h.rz / (rz_old * ratio * ratio);
      k_keep_direction<<<grid_for(n), 256, 0, w->st>>>(w->p32, w->z32, (float)(beta * ratio), n);
      FE_CUDA(cudaGetLastError(), "keep direction launch");
    }
    if (!h.done) {
      if (!w->g32[0])
        FE_TRY((build_graph<float, float>(m, w, op, false, w->d32, w->r32, w->z32, w->p32, w->q32,
                                          w->w32, w->invdiag32, &w->sc[1], nullptr, &w->g32[0])));
      FE_TRY(run_until_done(w, w->g32[0], 1, &h));
    }
    if (h.status == FE_ERR_BREAKDOWN) {
      *status = FE_ERR_BREAKDOWN;
      break;
    }
    total += h.iter;
    ++outer;
    s_old = s;
    rz_old = h.rz;  // <r_{k-1}, z_{k-1}>: the run stopped before its last beta
    have_p = h.iter > 0 || have_p;
    if (h.iter == 0 && !have_p) {  // converged in FP32 before any step: nothing to add
      *status = FE_ERR_NOT_CONVERGED;
      break;
    }
    k_correct<<<grid_for(n), 256, 0, w->st>>>(w->x, w->d32, 1.0 / s, n);
    FE_CUDA(cudaGetLastError(), "correction launch");
  }
  res->iters = total;
  res->outer_iters = outer;
  return FE_OK;
}

}  // namespace

fe_status fe_launch_absmax(const double* v, long long n, unsigned long long* out, cudaStream_t st) {
  FE_CUDA(cudaMemsetAsync(out, 0, sizeof(*out), st), "absmax");
  k_absmax_bits<<<grid_for(n), 256, 0, st>>>(v, n, out);
  return fe_cuda_check(cudaGetLastError(), "absmax launch");
}

bool fe_scale_of_max(double mx, double* s) {
  if (!std::isfinite(mx)) return false;
  *s = mx > 0.0 ? std::ldexp(1.0, -std::ilogb(mx)) : 1.0;
  return true;
}

fe_status fe_cg_rhs_scale(CgWork* w, const double* b, long long n, double* s) {
  unsigned long long* d = reinterpret_cast<unsigned long long*>(w->partials);
  FE_TRY(fe_launch_absmax(b, n, d, w->st));
  unsigned long long bits = 0;
  FE_CUDA(cudaMemcpyAsync(&bits, d, sizeof(bits), cudaMemcpyDeviceToHost, w->st), "rhs scale");
  FE_CUDA(cudaStreamSynchronize(w->st), "rhs scale");
  double mx;
  std::memcpy(&mx, &bits, sizeof(mx));
  if (!fe_scale_of_max(mx, s)) {
    fe_set_error("cg: the right-hand side holds a non-finite value");
    return FE_ERR_INVALID;
  }
  return FE_OK;
}

fe_status fe_cg_scale(const double* src, double* dst, double s, long long n, cudaStream_t st) {
  k_scale_vec<<<grid_for(n), 256, 0, st>>>(src, dst, s, n);
  return fe_cuda_check(cudaGetLastError(), "cg scale launch");
}

extern "C" fe_status fe_cg_solve(const fe_mesh* m, const double* b, double* x,
                                 const fe_cg_opts* opts, fe_cg_result* res, void* stream) {
  if (!m || !b || !x || !opts || !res) {
    fe_set_error("fe_cg_solve: null argument");
    return FE_ERR_INVALID;
  }
  if (!fe_aligned(b) || !fe_aligned(x)) {
    fe_set_error("fe_cg_solve: vectors must be 16-byte aligned");
    return FE_ERR_INVALID;
  }
  const bool lowp = opts->mixed == FE_BF16_F32ACC || opts->mixed == FE_F16_F32ACC;
  if (opts->maxit < 1 || !(opts->rtol >= 0.0) ||
      (opts->mixed != 0 && opts->mixed != FE_F32 && !lowp)) {
    fe_set_error("fe_cg_solve: invalid options (maxit %d, rtol %g, mixed %d)", opts->maxit,
                 opts->rtol, opts->mixed);
    return FE_ERR_INVALID;
  }
  if (m->packed || m->mzg > 0) {
    fe_set_error("fe_cg_solve: FE_LAYOUT_CELLS meshes only (slabs: fe_slab_cg_solve)");
    return FE_ERR_INVALID;
  }
  if (lowp && m->d.geom_mode != FE_GEOM_STORED) {
    fe_set_error("fe_cg_solve: a 16-bit inner operator needs FE_GEOM_STORED geometry");
    return FE_ERR_INVALID;
  }
  std::memset(res, 0, sizeof(*res));
  FeDeviceGuard device_guard;
  FE_CUDA(device_guard.set(m->d.device), "cudaSetDevice");
  const bool mixed = opts->mixed != 0;
  const int op = FE_LAPLACE;
  CgWork* w = nullptr;
  FE_TRY(fe_cg_get_work(m, mixed, &w));
  FE_CUDA(cudaStreamSynchronize((cudaStream_t)stream), "cg: caller stream");
  FE_TRY(fe_ensure_geometry(m, FE_F64, false));
  if (mixed) {
    FE_TRY(fe_ensure_geometry(m, FE_F32, false));
    if (lowp) FE_TRY(fe_ensure_geometry(m, opts->mixed, false));
    w->inner_prec = opts->mixed;
    if (w->g32_prec != w->inner_prec) {  // the inner graphs bake the operator in
      for (int f = 0; f < 2; ++f)
        if (w->g32[f]) {
          cudaGraphExecDestroy(w->g32[f]);
          w->g32[f] = nullptr;
        }
      w->g32_prec = w->inner_prec;
    }
  }
  FE_TRY(fe_cg_ensure_diag(m, w, op));
  const long long n = w->n;
  const int flex = opts->flexible ? 1 : 0;
  if (opts->history && (!w->hist || w->hist_cap < opts->maxit)) {
    fe_dfree(w->hist, w->st);
    w->hist = nullptr;
    FE_TRY(fe_dalloc((void**)&w->hist, 3 * (size_t)opts->maxit * sizeof(double), w->st, "history"));
    w->hist_cap = opts->maxit;
    for (int f = 0; f < 2; ++f)
      if (w->g64[f]) {
        cudaGraphExecDestroy(w->g64[f]);
        w->g64[f] = nullptr;
      }
  }
  double* hist = opts->history ? w->hist : nullptr;
  if (w->g64_hist != hist) {  // graphs bake the history pointer in
    for (int f = 0; f < 2; ++f)
      if (w->g64[f]) {
        cudaGraphExecDestroy(w->g64[f]);
        w->g64[f] = nullptr;
      }
    w->g64_hist = hist;
  }

  // the system scaled by an exact power of two (fe_cg_rhs_scale): b := sb b, u := sb x, ||G^T b||
  double sb = 1.0;
  FE_TRY(fe_cg_rhs_scale(w, b, n, &sb));
  FE_TRY(fe_cg_scale(b, w->bs, sb, n, w->st));
  FE_TRY(fe_cg_scale(x, w->x, sb, n, w->st));
  b = w->bs;
  FE_TRY(set_scal(w, 0, opts->maxit, 0, opts->rtol));
  FE_TRY(residual_norm<double>(m, w, b, w->w, &w->sc[0], FIN_INIT_B));
  CgScal h;
  FE_TRY(read_scal(w, 0, &h));
  const double bnorm2 = h.bnorm2;
  if (!(bnorm2 > 0.0)) {  // zero right-hand side: the solution is zero
    FE_CUDA(cudaMemsetAsync(x, 0, n * sizeof(double), w->st), "cg zero");
    FE_CUDA(cudaStreamSynchronize(w->st), "cg synchronize");
    res->iters = 0;
    res->outer_iters = 0;
    res->rel_res = 0.0;
    res->status = FE_OK;
    return FE_OK;
  }
  fe_status status = FE_OK;

  if (!mixed) {
    // r = b - A u, z = P r, p = z
    ApplyLaunch L{m, op, w->x, w->q, w->st, nullptr};
    FE_TRY(fe_launch_apply_f64dw(L));
    k_residual<<<grid_for(n), 256, 0, w->st>>>(b, w->q, w->r, n);
    FE_TRY(init_direction<double>(m, w, w->r, w->z, w->p, w->w, w->invdiag64, &w->sc[0], opts->rtol));
    FE_TRY(read_scal(w, 0, &h));
    if (!h.done) {
      if (!w->g64[flex])
        FE_TRY((build_graph<double, double>(m, w, op, flex, w->x, w->r, w->z, w->p, w->q,
                                            w->w, w->invdiag64, &w->sc[0], hist, &w->g64[flex])));
      FE_TRY(run_until_done(w, w->g64[flex], 0, &h));
    }
    res->iters = h.iter;
    res->outer_iters = 1;
    res->rel_res = h.relres;
    status = (fe_status)h.status;
    if (hist && h.iter > 0)
      FE_CUDA(cudaMemcpy(opts->history, hist, 3 * (size_t)h.iter * sizeof(double),
                         cudaMemcpyDeviceToHost),
              "history readback");
  } else if (flex || lowp) {
    // 16-bit inner operators are too coarse to keep a direction across reliable updates (Q3 64^3
    // to 1e-10: bf16 diverged, fp16 needed 3658 iterations at inner_rtol 0.3 against 1013 for
    // FP32), so they precondition FCG
    FE_TRY(solve_fcg_outer(m, w, op, b, bnorm2, opts, res, &status));
  } else {
    FE_TRY(solve_reliable(m, w, op, b, bnorm2, opts, res, &status));
  }
  FE_TRY(fe_cg_scale(w->x, x, 1.0 / sb, n, w->st));  // 1/sb: a power of two, exact
  FE_CUDA(cudaStreamSynchronize(w->st), "cg synchronize");
  res->status = status;
  if (status == FE_ERR_NOT_CONVERGED) fe_set_error("fe_cg_solve: not converged");
  if (status == FE_ERR_BREAKDOWN) fe_set_error("fe_cg_solve: breakdown");
  return status;
}
