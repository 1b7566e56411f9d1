// fe_batch.cu -- many independent solves advanced together (batched CG, and the engine of the
// request server).
//
// Each problem keeps its own mesh, geometry and cell-wise state; the engine advances all active
// problems in lockstep.  Every CG iteration applies the operators of all problems in ONE
// persistent launch over a work list of (problem, cell-tile) items with a per-item degree switch
// into the degree-templated cell kernel; the vector kernels run over lists of (problem, chunk)
// items, and per-problem scalars are reduced one CTA per problem over that problem's chunk
// partials in a fixed order.  A problem's arithmetic therefore never depends on which other
// problems share the launch: its result is bitwise the same alone and in a mix.
//
// Precisions: FP64 Jacobi-PCG (double-word apply), or the mixed scheme of fe_cg_solve with
// mixed = FE_F32: FP32 Jacobi-PCG with FP64 reliable updates (every run of FP32 iterations ends
// with the FP32 correction added to the FP64 solution, the true residual b - A x formed in FP64
// and put in place of the recursive one, and the search direction kept).  The phases (FP64
// replacement, FP32 iterations) are global: a problem whose FP32 run ends early waits for the
// others, which changes nothing in its own sequence of operations.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <mutex>
#include <new>
#include <vector>

#include "fe_apply_launch.cuh"
#include "fe_batch.h"
#include "fe_vec.cuh"

namespace {

constexpr int BT = 256;            // threads of every batched CTA
constexpr long long CHUNK = 4096;  // elements per vector work item (small batches still fill the GPU)

// ---- 1D tables of every degree, in constant memory -------------------------------------------
template <class V>
struct AllTabs {
  Tab1D<2, V> t2;
  Tab1D<3, V> t3;
  Tab1D<4, V> t4;
  Tab1D<5, V> t5;
  Tab1D<6, V> t6;
  Tab1D<7, V> t7;
  Tab1D<8, V> t8;
};
__constant__ AllTabs<dw> c_tabs_dw;
__constant__ AllTabs<float> c_tabs_f32;

template <int N, class V>
__device__ __forceinline__ const Tab1D<N, V>& tab_of();
#define FE_TAB_OF(NN)                                                            \
  template <>                                                                    \
  __device__ __forceinline__ const Tab1D<NN, dw>& tab_of<NN, dw>() {             \
    return c_tabs_dw.t##NN;                                                      \
  }                                                                              \
  template <>                                                                    \
  __device__ __forceinline__ const Tab1D<NN, float>& tab_of<NN, float>() {       \
    return c_tabs_f32.t##NN;                                                     \
  }
FE_TAB_OF(2)
FE_TAB_OF(3)
FE_TAB_OF(4)
FE_TAB_OF(5)
FE_TAB_OF(6)
FE_TAB_OF(7)
FE_TAB_OF(8)
#undef FE_TAB_OF

std::mutex g_tab_mu;
bool g_tab_ready[64] = {};

fe_status ensure_tables(int dev) {
  std::lock_guard<std::mutex> lock(g_tab_mu);
  if (dev < 0 || dev >= 64) return FE_ERR_INVALID;
  if (g_tab_ready[dev]) return FE_OK;
  AllTabs<dw> tdw;
  AllTabs<float> t32;
  HostTab h[8];
  for (int p = 1; p <= 7; ++p) fe_host_tables(p, &h[p]);
  tdw.t2 = make_tab<2, dw>(h[1]);
  tdw.t3 = make_tab<3, dw>(h[2]);
  tdw.t4 = make_tab<4, dw>(h[3]);
  tdw.t5 = make_tab<5, dw>(h[4]);
  tdw.t6 = make_tab<6, dw>(h[5]);
  tdw.t7 = make_tab<7, dw>(h[6]);
  tdw.t8 = make_tab<8, dw>(h[7]);
  t32.t2 = make_tab<2, float>(h[1]);
  t32.t3 = make_tab<3, float>(h[2]);
  t32.t4 = make_tab<4, float>(h[3]);
  t32.t5 = make_tab<5, float>(h[4]);
  t32.t6 = make_tab<6, float>(h[5]);
  t32.t7 = make_tab<7, float>(h[6]);
  t32.t8 = make_tab<8, float>(h[7]);
  FE_CUDA(cudaMemcpyToSymbol(c_tabs_dw, &tdw, sizeof(tdw)), "batch tables");
  FE_CUDA(cudaMemcpyToSymbol(c_tabs_f32, &t32, sizeof(t32)), "batch tables");
  g_tab_ready[dev] = true;
  return FE_OK;
}

// ---- work items ------------------------------------------------------------------------------
struct Tile {
  int prob;
  int pad;
  long long cell0;
};
struct Chunk {
  int prob;
  int pad;
  long long lo, hi;
};
struct DssRow {  // one row of interfaces of one problem (see kb_dss)
  int prob, row;
};

// ---- persistent apply ------------------------------------------------------------------------
template <int N, class V>
__device__ __forceinline__ void apply_item(const BProb& P, int prec, int src, long long cell0,
                                           unsigned char* sm) {
  CellArgs<N, V> a;
  if (prec == FE_F64) {
    a.x = reinterpret_cast<const typename NT<V>::SV*>(src ? P.x64 : P.p64);
    a.y = reinterpret_cast<typename NT<V>::SV*>(P.q64);
    a.geo = reinterpret_cast<const typename NT<V>::GV*>(P.geodw);
  } else {
    a.x = reinterpret_cast<const typename NT<V>::SV*>(P.p32);
    a.y = reinterpret_cast<typename NT<V>::SV*>(P.q32);
    a.geo = reinterpret_cast<const typename NT<V>::GV*>(P.geo32);
  }
  a.ncells = P.ncells;
  a.cell_base = 0;
  a.geo_cell0 = 0;
  a.mx = P.mx;
  a.my = P.my;
  a.mz = P.mz;
  a.dirichlet = P.dirichlet;
  for (int c = 0; c < 4; ++c) {
    if constexpr (sizeof(V) == sizeof(dw))
      a.aff[c] = dw_from_double(P.aff[c]);
    else
      a.aff[c] = (V)P.aff[c];
  }
  constexpr int stride = Cfg<N>::TILE + Cfg<N>::CS;
  if (P.affine)
    apply_cells<N, V, FE_LAPLACE, GEOM_AFFINE_K>(a, tab_of<N, V>(), cell0, sm, stride);
  else
    apply_cells<N, V, FE_LAPLACE, GEOM_STORED_K>(a, tab_of<N, V>(), cell0, sm, stride);
}

// register budget of the persistent apply: 3 CTAs per SM for the unrolled double-word degrees, 4
// for the rolled ones (its CTA is wider than the tile and walks many tiles; the one-layer apply's
// per-degree budgets were measured on the one-layer kernel)
template <int N, class V>
__host__ __device__ constexpr int batch_minb() {
  return std::is_same<V, dw>::value ? (N < FE_ROLL_MINN ? 3 : 4) : 1;
}

// persistent apply over the tiles [lo, hi) of one degree (tiles are grouped by degree), each kernel
// compiled for its own degree: registers and shared memory of that degree, not of the largest.
// The next work item is claimed before the current tile's apply (its atomic round trip overlaps
// the apply) and published through a double-buffered shared slot.
template <int N, class V>
__global__ void __launch_bounds__(BT, (batch_minb<N, V>()))
    kb_apply_n(const BProb* __restrict__ probs, const Tile* __restrict__ tiles, long long lo,
               long long hi, int slot, int prec, int src, unsigned long long* counter) {
  extern __shared__ __align__(16) unsigned char sm[];
  __shared__ long long item[2];  // written one tile ahead by thread 0
  if (threadIdx.x == 0) item[0] = lo + (long long)atomicAdd(counter, 1ULL);
  __syncthreads();
  int buf = 0;
  long long it = item[0];
  while (it < hi) {  // uniform: every thread reads the same item
    unsigned long long nxt = 0;
    if (threadIdx.x == 0) nxt = atomicAdd(counter, 1ULL);  // consumed after this tile
    const Tile T = tiles[it];
    const BProb& P = probs[T.prob];
    if (!*(volatile const int*)&P.sc[slot].done)  // uniform over the CTA
      apply_item<N, V>(P, prec, src, T.cell0, sm);
    if (threadIdx.x == 0) item[buf ^ 1] = lo + (long long)nxt;
    __syncthreads();  // the shared-memory tile is free and the next item visible
    buf ^= 1;
    it = item[buf];
  }
}

template <int N, class V>
constexpr size_t tile_bytes() {
  return (size_t)apply_narr<V>(FE_LAPLACE) * (Cfg<N>::TILE + Cfg<N>::CS) * Sm<V>::BYTES;
}

// ---- vector kernels over chunks ----------------------------------------------------------------
template <class S>
__device__ __forceinline__ S* vec(const BProb& P, int which);
// which: 0 x/d, 1 r, 2 z, 3 p, 4 q, 5 w
template <>
__device__ __forceinline__ double* vec<double>(const BProb& P, int which) {
  switch (which) {
    case 0: return P.x64;
    case 1: return P.r64;
    case 2: return P.z64;
    case 3: return P.p64;
    case 4: return P.q64;
    case 5: return P.w64;
    default: return const_cast<double*>(P.b64);
  }
}
template <>
__device__ __forceinline__ float* vec<float>(const BProb& P, int which) {
  switch (which) {
    case 0: return P.d32;
    case 1: return P.r32;
    case 2: return P.z32;
    case 3: return P.p32;
    case 4: return P.q32;
    default: return P.w32;
  }
}

template <class S>
__device__ __forceinline__ dw prod2(S a, S b);
template <>
__device__ __forceinline__ dw prod2<double>(double a, double b) {
  return dw_mul(dw_from_double(a), dw_from_double(b));
}
template <>
__device__ __forceinline__ dw prod2<float>(float a, float b) {
  const float p = __fmul_rn(a, b);
  return {p, __fmaf_rn(a, b, -p)};
}

// partials[chunk*4 + 0] = sum q p
template <class S>
__global__ void __launch_bounds__(BT)
    kb_qp(const BProb* __restrict__ probs, const Chunk* __restrict__ chunks, int nchunks, int slot,
          double* __restrict__ partials) {
  __shared__ dw sh[32];
  for (int c = blockIdx.x; c < nchunks; c += gridDim.x) {
    const Chunk C = chunks[c];
    const BProb& P = probs[C.prob];
    if (*(volatile const int*)&P.sc[slot].done) continue;
    const S* q = vec<S>(P, 4);
    const S* p = vec<S>(P, 3);
    // float: double-word sums of exact products; double: binary64 FMAs (one FP64-pipe operation
    // per product costs less than converting both factors to double-word)
    dw acc = {0.0f, 0.0f};
    double acc64 = 0.0;
    auto add = [&](S a, S b) {
      if constexpr (sizeof(S) == 8)
        acc64 = fma(a, b, acc64);
      else
        acc = dw_add(acc, prod2<S>(a, b));
    };
    long long e = C.lo + threadIdx.x;
    for (; e + (RED_U - 1) * BT < C.hi; e += RED_U * BT) {  // loads first, same order
      S qv[RED_U], pv[RED_U];
#pragma unroll
      for (int u = 0; u < RED_U; ++u) qv[u] = q[e + u * BT], pv[u] = p[e + u * BT];
#pragma unroll
      for (int u = 0; u < RED_U; ++u) add(qv[u], pv[u]);
    }
    for (; e < C.hi; e += BT) add(q[e], p[e]);
    if constexpr (sizeof(S) == 8) acc = dw_from_double(acc64);
    acc = block_reduce_dw(acc, sh);
    if (threadIdx.x == 0) partials[(size_t)c * 4 + 0] = dw_to_double(acc);
  }
}

// u += alpha p ; r -= alpha q ; w = r.  keep_r = 0 leaves r unwritten: with redistribution the
// preconditioner overwrites r with (S r)/mult before anything reads it.
template <class S>
__global__ void __launch_bounds__(BT)
    kb_update_ur(const BProb* __restrict__ probs, const Chunk* __restrict__ chunks, int nchunks,
                 int slot, int keep_r) {
  for (int c = blockIdx.x; c < nchunks; c += gridDim.x) {
    const Chunk C = chunks[c];
    const BProb& P = probs[C.prob];
    if (*(volatile const int*)&P.sc[slot].done) continue;
    const double a = P.sc[slot].alpha;
    S* u = vec<S>(P, 0);
    S* r = vec<S>(P, 1);
    const S* p = vec<S>(P, 3);
    const S* q = vec<S>(P, 4);
    S* w = vec<S>(P, 5);
    // FP32 state: FP32 arithmetic (the FP64 pipe is slow).  RED_U elements' loads are issued
    // before their stores (the vectors are distinct arrays)
    auto step = [&](long long e, S ue, S pe, S qe, S rq) {
      S re;
      if constexpr (sizeof(S) == 4) {
        const float af = (float)a;
        u[e] = fmaf(af, pe, ue);
        re = fmaf(-af, qe, rq);
      } else {
        u[e] = fma(a, pe, ue);
        re = fma(-a, qe, rq);
      }
      if (keep_r) r[e] = re;
      w[e] = re;
    };
    long long e = C.lo + threadIdx.x;
    for (; e + (RED_U - 1) * BT < C.hi; e += RED_U * BT) {
      S uv[RED_U], pv[RED_U], qv[RED_U], rv[RED_U];
#pragma unroll
      for (int k = 0; k < RED_U; ++k) {
        const long long f = e + k * BT;
        uv[k] = u[f], pv[k] = p[f], qv[k] = q[f], rv[k] = r[f];
      }
#pragma unroll
      for (int k = 0; k < RED_U; ++k) step(e + k * BT, uv[k], pv[k], qv[k], rv[k]);
    }
    for (; e < C.hi; e += BT) step(e, u[e], p[e], q[e], r[e]);
  }
}

// structured DSS pass of one axis over rows of interfaces of every problem, one warp per row:
// x-pass row (cz, cy) with items (interface, face node), y-pass row (cz, interface) and z-pass row
// (interface, cy) with items (cx, face node); node counts are compile-time, so the index
// arithmetic inside a row is multiplications and shifts.  Pairs of one pass are disjoint.
template <class S, int N>
__device__ __forceinline__ void dss_row(S* __restrict__ v, int axis, int row, int mx, int my,
                                        int lane) {
  constexpr int P = N - 1, N2 = N * N, N3 = N2 * N;
  long long first, rstep;
  int items, lstep, locL0, locR0, sa, sb;
  if (axis == 0) {
    first = (long long)row * mx;
    items = (mx - 1) * N2;
    lstep = 1;
    rstep = 1;
    locL0 = P, locR0 = 0, sa = N, sb = N2;
  } else if (axis == 1) {
    const int cz = row / (my - 1), u = row - cz * (my - 1);
    first = ((long long)cz * my + u) * mx;
    items = mx * N2;
    lstep = 1;
    rstep = mx;
    locL0 = P * N, locR0 = 0, sa = 1, sb = N2;
  } else {
    const int u = row / my, cy = row - u * my;
    first = ((long long)u * my + cy) * mx;
    items = mx * N2;
    lstep = 1;
    rstep = (long long)mx * my;
    locL0 = P * N2, locR0 = 0, sa = 1, sb = N;
  }
  // RED_U pairs' loads in flight before their stores (pairs of a pass are disjoint)
  auto addr = [&](int it, S*& pl, S*& pr) {
    const int g = it / N2, f = it - g * N2, fb = f / N, fa = f - fb * N;
    const long long L = first + (long long)g * lstep;
    const int off = fa * sa + fb * sb;
    pl = v + L * N3 + locL0 + off;
    pr = v + (L + rstep) * N3 + locR0 + off;
  };
  int it = lane;
  for (; it + (RED_U - 1) * 32 < items; it += RED_U * 32) {
    S *pl[RED_U], *pr[RED_U], l[RED_U], r[RED_U];
#pragma unroll
    for (int k = 0; k < RED_U; ++k) {
      addr(it + k * 32, pl[k], pr[k]);
      l[k] = *pl[k];
      r[k] = *pr[k];
    }
#pragma unroll
    for (int k = 0; k < RED_U; ++k) {
      const S sum = l[k] + r[k];
      *pl[k] = sum;
      *pr[k] = sum;
    }
  }
  for (; it < items; it += 32) {
    S *pl, *pr;
    addr(it, pl, pr);
    const S sum = *pl + *pr;
    *pl = sum;
    *pr = sum;
  }
}

template <class S>
__global__ void __launch_bounds__(BT)
    kb_dss(const BProb* __restrict__ probs, const DssRow* __restrict__ rows, int nrows, int slot,
           int axis) {
  const int lane = threadIdx.x & 31;
  const int warps = gridDim.x * (BT / 32);
  for (int w = blockIdx.x * (BT / 32) + (threadIdx.x >> 5); w < nrows; w += warps) {
    const DssRow R = rows[w];
    const BProb& P = probs[R.prob];
    if (*(volatile const int*)&P.sc[slot].done) continue;  // uniform over the warp
    S* v = vec<S>(P, 5);
    switch (P.n) {
      case 2: dss_row<S, 2>(v, axis, R.row, P.mx, P.my, lane); break;
      case 3: dss_row<S, 3>(v, axis, R.row, P.mx, P.my, lane); break;
      case 4: dss_row<S, 4>(v, axis, R.row, P.mx, P.my, lane); break;
      case 5: dss_row<S, 5>(v, axis, R.row, P.mx, P.my, lane); break;
      case 6: dss_row<S, 6>(v, axis, R.row, P.mx, P.my, lane); break;
      case 7: dss_row<S, 7>(v, axis, R.row, P.mx, P.my, lane); break;
      case 8: dss_row<S, 8>(v, axis, R.row, P.mx, P.my, lane); break;
    }
  }
}

// z = w * invdiag (mode & 1), r = w * invmult (mode & 2, redistribute); partials slot 0 sum w^2/mult,
// slot 1 <r,z>, slot 2 <q,z> (mode & 4)
template <class S>
__global__ void __launch_bounds__(BT)
    kb_precond(const BProb* __restrict__ probs, const Chunk* __restrict__ chunks, int nchunks,
               int slot, int mode, double* __restrict__ partials) {
  __shared__ dw sh[32];
  for (int c = blockIdx.x; c < nchunks; c += gridDim.x) {
    const Chunk C = chunks[c];
    const BProb& P = probs[C.prob];
    if (*(volatile const int*)&P.sc[slot].done) continue;
    const S* w = vec<S>(P, 5);
    S* r = vec<S>(P, 1);
    S* z = vec<S>(P, 2);
    const S* q = vec<S>(P, 4);
    const S* idg = (sizeof(S) == 8) ? (const S*)P.invdiag64 : (const S*)P.invdiag32;
    dw a0 = {0.0f, 0.0f}, a1 = {0.0f, 0.0f}, a2 = {0.0f, 0.0f};
    auto body = [&](long long e, S we, float im, S dg, S rv, S qv) {
      const dw w2 = prod2<S>(we, we);
      a0 = dw_add(a0, {w2.h * im, w2.l * im});
      if (mode & 1) {
        const S ze = we * dg;
        z[e] = ze;
        S re;
        if (mode & 2) {
          re = we * (S)im;
          r[e] = re;
        } else {
          re = rv;
        }
        a1 = dw_add(a1, prod2<S>(re, ze));
        if (mode & 4) a2 = dw_add(a2, prod2<S>(qv, ze));
      }
    };
    long long e = C.lo + threadIdx.x;
    for (; e + (RED_U - 1) * BT < C.hi; e += RED_U * BT) {  // loads first, same order
      S wv[RED_U], dv[RED_U], rv[RED_U], qv[RED_U];
      float im[RED_U];
#pragma unroll
      for (int u = 0; u < RED_U; ++u) {
        const long long f = e + u * BT;
        wv[u] = w[f];
        im[u] = P.invmult[f];
        dv[u] = (mode & 1) ? idg[f] : S(0);
        rv[u] = ((mode & 1) && !(mode & 2)) ? r[f] : S(0);
        qv[u] = ((mode & 1) && (mode & 4)) ? q[f] : S(0);
      }
#pragma unroll
      for (int u = 0; u < RED_U; ++u) body(e + u * BT, wv[u], im[u], dv[u], rv[u], qv[u]);
    }
    for (; e < C.hi; e += BT)
      body(e, w[e], P.invmult[e], (mode & 1) ? idg[e] : S(0),
           ((mode & 1) && !(mode & 2)) ? r[e] : S(0), ((mode & 1) && (mode & 4)) ? q[e] : S(0));
    a0 = block_reduce_dw(a0, sh);
    if (threadIdx.x == 0) partials[(size_t)c * 4 + 0] = dw_to_double(a0);
    if (mode & 1) {
      a1 = block_reduce_dw(a1, sh);
      if (threadIdx.x == 0) partials[(size_t)c * 4 + 1] = dw_to_double(a1);
      if (mode & 4) {
        a2 = block_reduce_dw(a2, sh);
        if (threadIdx.x == 0) partials[(size_t)c * 4 + 2] = dw_to_double(a2);
      }
    }
  }
}

// p = z + beta p
template <class S>
__global__ void __launch_bounds__(BT)
    kb_update_p(const BProb* __restrict__ probs, const Chunk* __restrict__ chunks, int nchunks,
                int slot) {
  for (int c = blockIdx.x; c < nchunks; c += gridDim.x) {
    const Chunk C = chunks[c];
    const BProb& P = probs[C.prob];
    if (*(volatile const int*)&P.sc[slot].done) continue;
    const S b = (S)P.sc[slot].beta;
    S* p = vec<S>(P, 3);
    const S* z = vec<S>(P, 2);
    long long e = C.lo + threadIdx.x;
    for (; e + (RED_U - 1) * BT < C.hi; e += RED_U * BT) {  // loads before stores
      S zv[RED_U], pv[RED_U];
#pragma unroll
      for (int k = 0; k < RED_U; ++k) zv[k] = z[e + k * BT], pv[k] = p[e + k * BT];
#pragma unroll
      for (int k = 0; k < RED_U; ++k) p[e + k * BT] = zv[k] + b * pv[k];
    }
    for (; e < C.hi; e += BT) p[e] = z[e] + b * p[e];
  }
}

// dst = src (which -> which)
template <class S>
__global__ void __launch_bounds__(BT)
    kb_copy(const BProb* __restrict__ probs, const Chunk* __restrict__ chunks, int nchunks, int slot,
            int dst, int src) {
  for (int c = blockIdx.x; c < nchunks; c += gridDim.x) {
    const Chunk C = chunks[c];
    const BProb& P = probs[C.prob];
    if (*(volatile const int*)&P.sc[slot].done) continue;
    S* d = vec<S>(P, dst);
    const S* s = vec<S>(P, src);
    for (long long e = C.lo + threadIdx.x; e < C.hi; e += BT) d[e] = s[e];
  }
}

// inner start: r32 = s (S r64) / mult with s = 1/sqrt(rnorm2) (w64 holds S r64), d32 = 0
__global__ void __launch_bounds__(BT)
    kb_to_inner(const BProb* __restrict__ probs, const Chunk* __restrict__ chunks, int nchunks) {
  for (int c = blockIdx.x; c < nchunks; c += gridDim.x) {
    const Chunk C = chunks[c];
    const BProb& P = probs[C.prob];
    if (*(volatile const int*)&P.sc[0].done) continue;
    const double s = 1.0 / sqrt(P.sc[0].rnorm2);
    for (long long e = C.lo + threadIdx.x; e < C.hi; e += BT) {
      P.r32[e] = (float)(s * P.w64[e] * (double)P.invmult[e]);
      P.d32[e] = 0.0f;
    }
  }
}

// reliable update: x64 += d32 / s (s = 1/||G^T r|| of the run's residual)
__global__ void __launch_bounds__(BT)
    kb_correct(const BProb* __restrict__ probs, const Chunk* __restrict__ chunks, int nchunks) {
  for (int c = blockIdx.x; c < nchunks; c += gridDim.x) {
    const Chunk C = chunks[c];
    const BProb& P = probs[C.prob];
    if (*(volatile const int*)&P.sc[0].done) continue;
    const double inv_s = sqrt(P.sc[0].rnorm2);
    for (long long e = C.lo + threadIdx.x; e < C.hi; e += BT) P.x64[e] += inv_s * (double)P.d32[e];
  }
}

// start of a run: p32 = z32 (a problem's first run) or p32 = z32 + c p32, the direction of the
// previous run kept in the new scale: c = beta (s/s_old) with beta = <r', z'> / (rz_old
// (s/s_old)^2), rz_old = <r_{k-1}, z_{k-1}> in the old scale (sc[0].rz_new), s_old in sc[0].qz
__global__ void __launch_bounds__(BT)
    kb_keep_direction(const BProb* __restrict__ probs, const Chunk* __restrict__ chunks, int nchunks) {
  for (int c = blockIdx.x; c < nchunks; c += gridDim.x) {
    const Chunk C = chunks[c];
    const BProb& P = probs[C.prob];
    if (*(volatile const int*)&P.sc[0].done) continue;
    if (P.sc[0].pad) {  // first run: p = z (the buffer's old contents are not read)
      for (long long e = C.lo + threadIdx.x; e < C.hi; e += BT) P.p32[e] = P.z32[e];
      continue;
    }
    const double ratio = (1.0 / sqrt(P.sc[0].rnorm2)) / P.sc[0].qz;
    const float cf = (float)(P.sc[1].rz / (P.sc[0].rz_new * ratio));
    for (long long e = C.lo + threadIdx.x; e < C.hi; e += BT) P.p32[e] = fmaf(cf, P.p32[e], P.z32[e]);
  }
}

// ---- per-problem finishing kernels (one CTA per problem) --------------------------------------
__device__ double sum_chunks(const double* partials, int c0, int c1, int slot, dw* sh) {
  dw acc = {0.0f, 0.0f};
  for (int c = c0 + threadIdx.x; c < c1; c += BT)
    acc = dw_add(acc, dw_from_double(partials[(size_t)c * 4 + slot]));
  acc = block_reduce_dw(acc, sh);
  return dw_to_double(acc);
}

__global__ void __launch_bounds__(BT)
    kb_fin_alpha(BProb* __restrict__ probs, int slot, const double* __restrict__ partials) {
  __shared__ dw sh[32];
  BProb& P = probs[blockIdx.x];
  CgScal* sc = &P.sc[slot];
  if (*(volatile int*)&sc->done) return;
  const double qp = sum_chunks(partials, P.chunk0, P.chunk1, 0, sh);
  if (threadIdx.x != 0) return;
  sc->qp = qp;
  if (!(qp > 0.0) || !isfinite(qp) || !isfinite(sc->rz)) {
    sc->status = FE_ERR_BREAKDOWN;
    sc->done = 1;
  } else {
    sc->alpha = sc->rz / qp;
  }
}

// mode: FIN_INIT_B, FIN_INIT_R, FIN_ITER, FIN_NORM, FIN_OUTER (fe_cgcore.h); tolerances and the
// FCG switch are per problem (slot 0: the outer or FP64 solve, slot 1: the inner FP32 solve)
__global__ void __launch_bounds__(BT)
    kb_fin_beta(BProb* __restrict__ probs, int slot, int mode, const double* __restrict__ partials) {
  __shared__ dw sh[32];
  BProb& P = probs[blockIdx.x];
  CgScal* sc = &P.sc[slot];
  if (*(volatile int*)&sc->done) return;
  const int flexible = slot == 0 ? P.flexible : 0;
  const double rtol = slot == 0 ? P.rtol : sc->rtol;
  const double rn2 = sum_chunks(partials, P.chunk0, P.chunk1, 0, sh);
  const double rz = (mode == FIN_INIT_R || mode == FIN_ITER) ? sum_chunks(partials, P.chunk0, P.chunk1, 1, sh) : 0.0;
  const double qz = (mode == FIN_ITER && flexible) ? sum_chunks(partials, P.chunk0, P.chunk1, 2, sh) : 0.0;
  if (threadIdx.x != 0) return;
  fin_scalars(sc, rn2, rz, qz, rtol, mode, flexible);
}

// reset the inner scalars for a new inner solve (done mirrors the outer state)
__global__ void kb_reset_inner(BProb* __restrict__ probs, int nprob) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= nprob) return;
  const int maxit = probs[i].maxit;
  CgScal* o = &probs[i].sc[0];
  CgScal* in = &probs[i].sc[1];
  const int spent = in->stall_total;  // inner iterations so far
  if (!o->done && spent >= maxit) {
    o->status = FE_ERR_NOT_CONVERGED;
    o->done = 1;
  }
  CgScal s;
  memset(&s, 0, sizeof(s));
  s.maxit = maxit - spent > 0 ? maxit - spent : 1;
  s.stall_total = spent;
  s.done = o->done;
  // run the FP32 iterations down to delta, or to just below the outer target
  s.rtol = fmax(probs[i].irtol, 0.5 * probs[i].rtol / o->relres);
  *in = s;
}

// end of a run: keep <r_{k-1}, z_{k-1}> (the run stopped before its last beta) and the scale
__global__ void kb_save_run(BProb* __restrict__ probs, int nprob) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= nprob) return;
  CgScal* o = &probs[i].sc[0];
  if (o->done) return;
  o->rz_new = probs[i].sc[1].rz;
  o->qz = 1.0 / sqrt(o->rnorm2);
  o->pad = 0;
}

// accumulate the finished inner iteration count
__global__ void kb_count_inner(BProb* __restrict__ probs, int nprob) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= nprob) return;
  CgScal* in = &probs[i].sc[1];
  if (!probs[i].sc[0].done) in->stall_total += in->iter;
}

// r = b - q
__global__ void __launch_bounds__(BT)
    kb_residual(const BProb* __restrict__ probs, const Chunk* __restrict__ chunks, int nchunks) {
  for (int c = blockIdx.x; c < nchunks; c += gridDim.x) {
    const Chunk C = chunks[c];
    const BProb& P = probs[C.prob];
    if (*(volatile const int*)&P.sc[0].done) continue;
    for (long long e = C.lo + threadIdx.x; e < C.hi; e += BT) P.r64[e] = P.b64[e] - P.q64[e];
  }
}

// fresh scalars for a solve
__global__ void kb_init_scal(BProb* __restrict__ probs, int nprob) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= nprob) return;
  const int maxit = probs[i].maxit;
  CgScal s;
  memset(&s, 0, sizeof(s));
  s.maxit = maxit;
  probs[i].sc[1] = s;
  s.pad = 1;  // first outer direction still to come
  probs[i].sc[0] = s;
}

// contiguous copy of every problem's two scalar records, for one readback
__global__ void kb_gather_sc(const BProb* __restrict__ probs, int nprob, CgScal* __restrict__ out) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= nprob) return;
  out[2 * i] = probs[i].sc[0];
  out[2 * i + 1] = probs[i].sc[1];
}

unsigned grid_chunks(int n) { return (unsigned)std::max(1, std::min(n, 152 * 8)); }

}  // namespace

// ---------------------------------------------------------------------------------------------
// host engine
// ---------------------------------------------------------------------------------------------
fe_status fe_batch_build(FeBatch* B) {
  const int np = (int)B->hp.size();
  std::vector<Tile> tiles_n[FE_MAXN + 1];
  std::vector<Chunk> vch;
  std::vector<DssRow> dch[3];
  for (int i = 0; i < np; ++i) {
    BProb& P = B->hp[i];
    const int n = P.n;
    int cpb = 0;
    switch (n) {
      case 2: cpb = Cfg<2>::CPB; break;
      case 3: cpb = Cfg<3>::CPB; break;
      case 4: cpb = Cfg<4>::CPB; break;
      case 5: cpb = Cfg<5>::CPB; break;
      case 6: cpb = Cfg<6>::CPB; break;
      case 7: cpb = Cfg<7>::CPB; break;
      case 8: cpb = Cfg<8>::CPB; break;
    }
    if (!B->active[i]) {
      P.chunk0 = P.chunk1 = (int)vch.size();
      continue;
    }
    for (long long c = 0; c < P.ncells; c += cpb) tiles_n[n].push_back({i, 0, c});
    P.chunk0 = (int)vch.size();
    for (long long e = 0; e < P.ncw; e += CHUNK) vch.push_back({i, 0, e, std::min(P.ncw, e + CHUNK)});
    P.chunk1 = (int)vch.size();
    // rows of interfaces per axis: x (cz, cy) if mx > 1; y (cz, interface); z (interface, cy)
    const int rows[3] = {P.mx > 1 ? P.my * P.mz : 0, P.mz * (P.my - 1), (P.mz - 1) * P.my};
    for (int a = 0; a < 3; ++a)
      for (int r = 0; r < rows[a]; ++r) dch[a].push_back({i, r});
  }
  // tiles grouped by degree: one persistent apply launch per degree present
  std::vector<Tile> tiles;
  for (int nn = 0; nn <= FE_MAXN; ++nn) {
    B->tile_lo[nn] = (long long)tiles.size();
    tiles.insert(tiles.end(), tiles_n[nn].begin(), tiles_n[nn].end());
    B->tile_hi[nn] = (long long)tiles.size();
  }
  B->ntiles = (long long)tiles.size();
  B->nvch = (int)vch.size();
  for (int a = 0; a < 3; ++a) B->ndch[a] = (int)dch[a].size();
  auto up = [&](void** dst, size_t* cap, const void* src, size_t bytes) -> fe_status {
    if (bytes > *cap) {
      fe_dfree(*dst, B->st);
      *dst = nullptr;
      const size_t nb = std::max<size_t>(bytes + bytes / 2, 256);
      FE_TRY(fe_dalloc(dst, nb, B->st, "batch work list"));
      *cap = nb;
    }
    if (bytes) FE_CUDA(cudaMemcpyAsync(*dst, src, bytes, cudaMemcpyHostToDevice, B->st), "batch upload");
    return FE_OK;
  };
  FE_TRY(up(&B->d_tiles, &B->cap_tiles, tiles.data(), tiles.size() * sizeof(Tile)));
  FE_TRY(up(&B->d_vch, &B->cap_vch, vch.data(), vch.size() * sizeof(Chunk)));
  for (int a = 0; a < 3; ++a)
    FE_TRY(up(&B->d_dch[a], &B->cap_dch[a], dch[a].data(), dch[a].size() * sizeof(DssRow)));
  FE_TRY(up((void**)&B->d_probs, &B->cap_probs, B->hp.data(), np * sizeof(BProb)));
  const size_t pbytes = std::max<size_t>(1, vch.size()) * 4 * sizeof(double);
  if (pbytes > B->cap_partials) {
    fe_dfree(B->d_partials, B->st);
    B->d_partials = nullptr;
    FE_TRY(fe_dalloc((void**)&B->d_partials, pbytes + pbytes / 2, B->st, "batch partials"));
    B->cap_partials = pbytes + pbytes / 2;
  }
  if (!B->d_counter)
    FE_TRY(fe_dalloc((void**)&B->d_counter, 64 * sizeof(unsigned long long), B->st, "counter"));
  FE_TRY(up((void**)&B->d_sc, &B->cap_sc, nullptr, 0));
  if (B->cap_sc < 2 * np * sizeof(CgScal)) {
    fe_dfree(B->d_sc, B->st);
    B->d_sc = nullptr;
    B->cap_sc = 2 * (size_t)np * sizeof(CgScal) + 64 * sizeof(CgScal);
    FE_TRY(fe_dalloc((void**)&B->d_sc, B->cap_sc, B->st, "batch scalar gather"));
  }
  return FE_OK;
}

template <int N, class V>
static fe_status launch_apply_degree(FeBatch* B, int slot, int src) {
  const long long lo = B->tile_lo[N], hi = B->tile_hi[N];
  if (hi <= lo) return FE_OK;
  const size_t smem = tile_bytes<N, V>();
  static int per_sm_dev[64] = {};  // resident CTAs per SM, per device (attribute set once)
  int dev = 0;
  FE_CUDA(cudaGetDevice(&dev), "cudaGetDevice");
  int per_sm = (dev >= 0 && dev < 64) ? per_sm_dev[dev] : 0;
  if (per_sm == 0) {
    FE_CUDA(cudaFuncSetAttribute(kb_apply_n<N, V>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)smem),
            "batch apply attribute");
    FE_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kb_apply_n<N, V>, BT, smem),
            "occupancy");
    per_sm = std::max(1, per_sm);
    if (dev >= 0 && dev < 64) per_sm_dev[dev] = per_sm;
  }
  const long long grid = std::min<long long>(hi - lo, 152LL * per_sm);
  kb_apply_n<N, V><<<(unsigned)grid, BT, smem, B->st>>>(
      B->d_probs, (const Tile*)B->d_tiles, lo, hi, slot, std::is_same<V, dw>::value ? FE_F64 : FE_F32,
      src, B->d_counter + N);
  return fe_cuda_check(cudaGetLastError(), "batch apply launch");
}

template <class S>
static fe_status launch_apply_batched(FeBatch* B, int slot, int src = 0) {
  using V = typename std::conditional<sizeof(S) == 8, dw, float>::type;
  FE_CUDA(cudaMemsetAsync(B->d_counter, 0, (FE_MAXN + 1) * sizeof(unsigned long long), B->st),
          "counter reset");
  FE_TRY((launch_apply_degree<2, V>(B, slot, src)));
  FE_TRY((launch_apply_degree<3, V>(B, slot, src)));
  FE_TRY((launch_apply_degree<4, V>(B, slot, src)));
  FE_TRY((launch_apply_degree<5, V>(B, slot, src)));
  FE_TRY((launch_apply_degree<6, V>(B, slot, src)));
  FE_TRY((launch_apply_degree<7, V>(B, slot, src)));
  return launch_apply_degree<8, V>(B, slot, src);
}

template <class S>
static fe_status launch_dss_batched(FeBatch* B, int slot) {
  for (int axis = 2; axis >= 0; --axis)
    if (B->ndch[axis] > 0)
      kb_dss<S><<<grid_chunks((B->ndch[axis] + BT / 32 - 1) / (BT / 32)), BT, 0, B->st>>>(
          B->d_probs, (const DssRow*)B->d_dch[axis], B->ndch[axis], slot, axis);
  return fe_cuda_check(cudaGetLastError(), "batch dss launch");
}

// one PCG iteration of every active problem on vectors of type S, scalars `slot`
template <class S>
fe_status fe_batch_iteration(FeBatch* B, int slot, int redistribute) {
  const int flexible = slot == 0 ? B->any_flexible : 0;
  const int np = (int)B->hp.size();
  const unsigned g = grid_chunks(B->nvch);
  const Chunk* ch = (const Chunk*)B->d_vch;
  FE_TRY(launch_apply_batched<S>(B, slot));
  kb_qp<S><<<g, BT, 0, B->st>>>(B->d_probs, ch, B->nvch, slot, B->d_partials);
  kb_fin_alpha<<<np, BT, 0, B->st>>>(B->d_probs, slot, B->d_partials);
  kb_update_ur<S><<<g, BT, 0, B->st>>>(B->d_probs, ch, B->nvch, slot, !redistribute);
  FE_TRY(launch_dss_batched<S>(B, slot));
  kb_precond<S><<<g, BT, 0, B->st>>>(B->d_probs, ch, B->nvch, slot,
                                     1 | (redistribute ? 2 : 0) | (flexible ? 4 : 0), B->d_partials);
  kb_fin_beta<<<np, BT, 0, B->st>>>(B->d_probs, slot, FIN_ITER, B->d_partials);
  kb_update_p<S><<<g, BT, 0, B->st>>>(B->d_probs, ch, B->nvch, slot);
  return fe_cuda_check(cudaGetLastError(), "batch iteration launch");
}
template fe_status fe_batch_iteration<double>(FeBatch*, int, int);
template fe_status fe_batch_iteration<float>(FeBatch*, int, int);

// w = S(src) and the norm (and, with init_dir, z = D^{-1} w, p = z, <r,z>) of every active problem
template <class S>
fe_status fe_batch_norm(FeBatch* B, int slot, int src, int mode, int redistribute) {
  const int np = (int)B->hp.size();
  const unsigned g = grid_chunks(B->nvch);
  const Chunk* ch = (const Chunk*)B->d_vch;
  kb_copy<S><<<g, BT, 0, B->st>>>(B->d_probs, ch, B->nvch, slot, 5, src);
  FE_TRY(launch_dss_batched<S>(B, slot));
  const int pm = (mode == FIN_INIT_R) ? (1 | (redistribute ? 2 : 0)) : 0;
  kb_precond<S><<<g, BT, 0, B->st>>>(B->d_probs, ch, B->nvch, slot, pm, B->d_partials);
  kb_fin_beta<<<np, BT, 0, B->st>>>(B->d_probs, slot, mode, B->d_partials);
  if (mode == FIN_INIT_R) kb_copy<S><<<g, BT, 0, B->st>>>(B->d_probs, ch, B->nvch, slot, 3, 2);
  return fe_cuda_check(cudaGetLastError(), "batch norm launch");
}
template fe_status fe_batch_norm<double>(FeBatch*, int, int, int, int);
template fe_status fe_batch_norm<float>(FeBatch*, int, int, int, int);

fe_status fe_batch_read(FeBatch* B) {
  const int np = (int)B->hp.size();
  if (np == 0) return FE_OK;
  kb_gather_sc<<<(np + 127) / 128, 128, 0, B->st>>>(B->d_probs, np, B->d_sc);
  FE_CUDA(cudaMemcpyAsync(B->hsc, B->d_sc, 2 * np * sizeof(CgScal), cudaMemcpyDeviceToHost, B->st),
          "batch scalar readback");
  return fe_cuda_check(cudaStreamSynchronize(B->st), "batch synchronize");
}

// start of an FP32 run for every unconverged problem: r32 = s (S r)/mult, z32 = P r32, <r32, z32>,
// and the direction (first run: p = z; later: the previous direction kept, kb_keep_direction)
fe_status fe_batch_inner_start(FeBatch* B) {
  const int np = (int)B->hp.size();
  const unsigned g = grid_chunks(B->nvch);
  const Chunk* ch = (const Chunk*)B->d_vch;
  kb_reset_inner<<<(np + 127) / 128, 128, 0, B->st>>>(B->d_probs, np);
  kb_to_inner<<<g, BT, 0, B->st>>>(B->d_probs, ch, B->nvch);
  FE_TRY(fe_batch_norm<float>(B, 1, 1, FIN_INIT_B, 0));
  kb_copy<float><<<g, BT, 0, B->st>>>(B->d_probs, ch, B->nvch, 1, 5, 1);
  FE_TRY(launch_dss_batched<float>(B, 1));
  kb_precond<float><<<g, BT, 0, B->st>>>(B->d_probs, ch, B->nvch, 1, 1 | 2, B->d_partials);
  kb_fin_beta<<<np, BT, 0, B->st>>>(B->d_probs, 1, FIN_INIT_R, B->d_partials);
  kb_keep_direction<<<g, BT, 0, B->st>>>(B->d_probs, ch, B->nvch);
  return fe_cuda_check(cudaGetLastError(), "batch run start");
}

// end of an FP32 run (the reliable update): x += d / s, r = b - A x in FP64, ||G^T r||, convergence
fe_status fe_batch_inner_finish(FeBatch* B) {
  const int np = (int)B->hp.size();
  const unsigned g = grid_chunks(B->nvch);
  const Chunk* ch = (const Chunk*)B->d_vch;
  kb_count_inner<<<(np + 127) / 128, 128, 0, B->st>>>(B->d_probs, np);
  kb_save_run<<<(np + 127) / 128, 128, 0, B->st>>>(B->d_probs, np);
  kb_correct<<<g, BT, 0, B->st>>>(B->d_probs, ch, B->nvch);
  FE_TRY(launch_apply_batched<double>(B, 0, 1));  // q = A x
  kb_residual<<<g, BT, 0, B->st>>>(B->d_probs, ch, B->nvch);
  FE_TRY(fe_batch_norm<double>(B, 0, 1, FIN_NORM, 0));
  kb_fin_beta<<<np, BT, 0, B->st>>>(B->d_probs, 0, FIN_OUTER, B->d_partials);
  return fe_cuda_check(cudaGetLastError(), "batch reliable update");
}

fe_status fe_batch_prepare() {
  int dev = 0;
  FE_CUDA(cudaGetDevice(&dev), "cudaGetDevice");
  return ensure_tables(dev);
}

FeBatch::~FeBatch() {
  if (st) cudaStreamSynchronize(st);
  fe_dfree(d_probs, st);
  fe_dfree(d_tiles, st);
  fe_dfree(d_vch, st);
  for (int a = 0; a < 3; ++a) fe_dfree(d_dch[a], st);
  fe_dfree(d_partials, st);
  fe_dfree(d_counter, st);
  fe_dfree(d_sc, st);
  if (st) cudaStreamSynchronize(st);
  cudaFreeHost(hsc);
  if (st && own_stream) cudaStreamDestroy(st);
}

fe_status fe_batch_fill(FeBatch* B, int i, const fe_mesh* m, CgWork* w, const double* b,
                        const fe_cg_opts* opts) {
  BProb& P = B->hp[i];
  std::memset(&P, 0, sizeof(P));
  P.rtol = opts->rtol;
  P.irtol = opts->inner_rtol > 0.0 ? opts->inner_rtol : 0.1;
  P.maxit = opts->maxit;
  P.flexible = (opts->mixed == 0 && opts->flexible) ? 1 : 0;
  P.n = m->n;
  P.affine = m->d.geom_mode == FE_GEOM_AFFINE;
  P.ncells = m->ncells;
  P.ncw = m->ncw;
  P.mx = m->d.mx;
  P.my = m->d.my;
  P.mz = m->d.mz;
  P.dirichlet = fe_dir_mask(m);
  const double hx = 1.0 / m->d.mx, hy = 1.0 / m->d.my, hz = 1.0 / m->d.mz, det = hx * hy * hz;
  P.aff[0] = det / (hx * hx);
  P.aff[1] = det / (hy * hy);
  P.aff[2] = det / (hz * hz);
  P.aff[3] = det;
  P.geodw = m->geodw;
  P.geo32 = m->geo32;
  P.x64 = w->x;
  P.r64 = w->r;
  P.z64 = w->z;
  P.p64 = w->p;
  P.q64 = w->q;
  P.w64 = w->w;
  P.b64 = b;
  P.d32 = w->d32;
  P.r32 = w->r32;
  P.z32 = w->z32;
  P.p32 = w->p32;
  P.q32 = w->q32;
  P.w32 = w->w32;
  P.invdiag64 = w->invdiag64;
  P.invdiag32 = w->invdiag32;
  P.invmult = w->invmult;
  P.sc = w->sc;
  return FE_OK;
}

fe_status fe_batch_setup(FeBatch* B) {
  const int np = (int)B->hp.size();
  const unsigned g = grid_chunks(B->nvch);
  const Chunk* ch = (const Chunk*)B->d_vch;
  kb_init_scal<<<(np + 127) / 128, 128, 0, B->st>>>(B->d_probs, np);
  FE_TRY(fe_batch_norm<double>(B, 0, 6, FIN_INIT_B, 0));  // ||G^T b||
  FE_TRY(launch_apply_batched<double>(B, 0, 1));               // q = A x
  kb_residual<<<g, BT, 0, B->st>>>(B->d_probs, ch, B->nvch);
  return fe_cuda_check(cudaGetLastError(), "batch setup");
}

bool fe_batch_all_done(FeBatch* B, int slot) {
  for (size_t i = 0; i < B->hp.size(); ++i)
    if (B->active[i] && !B->hsc[2 * i + slot].done) return false;
  return true;
}

fe_status fe_batch_start(FeBatch* B, bool mixed) {
  FE_TRY(fe_batch_setup(B));
  if (!mixed) return fe_batch_norm<double>(B, 0, 1, FIN_INIT_R, 0);
  FE_TRY(fe_batch_norm<double>(B, 0, 1, FIN_NORM, 0));
  const int np = (int)B->hp.size();
  kb_fin_beta<<<np, BT, 0, B->st>>>(B->d_probs, 0, FIN_OUTER, B->d_partials);  // converged at x0?
  return fe_cuda_check(cudaGetLastError(), "batch start");
}

// after a read-back: converged problems leave the work lists, so the launches of the following
// iterations walk the unconverged problems' tiles and chunks only
static fe_status drop_converged(FeBatch* B) {
  bool changed = false;
  for (size_t i = 0; i < B->hp.size(); ++i)
    if (B->active[i] && B->hsc[2 * i].done) {
      B->active[i] = 0;
      changed = true;
    }
  return changed ? fe_batch_build(B) : FE_OK;
}

fe_status fe_batch_solve(FeBatch* B, const fe_cg_opts* opts) {
  const int batch = 8;
  const bool mixed = opts->mixed == FE_F32;
  FE_TRY(fe_batch_start(B, mixed));
  if (!mixed) {
    FE_TRY(fe_batch_read(B));
    while (!fe_batch_all_done(B, 0)) {
      FE_TRY(drop_converged(B));
      for (int k = 0; k < batch; ++k) FE_TRY(fe_batch_iteration<double>(B, 0, 0));
      FE_TRY(fe_batch_read(B));
    }
    return FE_OK;
  }
  // mixed: FP32 PCG runs between FP64 reliable updates, each problem on its own: after every
  // round of iterations the problems whose run has ended take their reliable update in a batch of
  // their own and leave converged or start their next run (the running batch's kernels skip a
  // problem whose run has ended), so a round costs the iterations it runs, not the longest run
  FE_TRY(fe_batch_read(B));
  FE_TRY(drop_converged(B));
  if (fe_batch_all_done(B, 0)) return FE_OK;
  FE_TRY(fe_batch_inner_start(B));
  auto subset = [&](const std::vector<int>& idx, FeBatch& J) -> fe_status {
    J.st = B->st;
    J.own_stream = false;
    J.hp.resize(idx.size());
    for (size_t k = 0; k < idx.size(); ++k) J.hp[k] = B->hp[idx[k]];
    J.active.assign(idx.size(), 1);
    FE_CUDA(cudaMallocHost(&J.hsc, 2 * idx.size() * sizeof(CgScal)), "batch scalars");
    J.cap_hsc = 2 * idx.size();
    return fe_batch_build(&J);
  };
  for (;;) {
    for (int k = 0; k < batch; ++k) FE_TRY(fe_batch_iteration<float>(B, 1, 1));
    FE_TRY(fe_batch_read(B));
    std::vector<int> ended;
    for (size_t i = 0; i < B->hp.size(); ++i)
      if (B->active[i] && B->hsc[2 * i + 1].done) ended.push_back((int)i);
    if (ended.empty()) continue;
    std::vector<int> cont;
    bool left = false;
    {
      FeBatch J;
      FE_TRY(subset(ended, J));
      FE_TRY(fe_batch_inner_finish(&J));
      FE_TRY(fe_batch_read(&J));
      for (size_t k = 0; k < ended.size(); ++k) {
        if (J.hsc[2 * k].done) {
          B->active[ended[k]] = 0;
          left = true;
        } else {
          cont.push_back(ended[k]);
        }
      }
    }
    if (!cont.empty()) {
      FeBatch K;
      FE_TRY(subset(cont, K));
      FE_TRY(fe_batch_inner_start(&K));
    }
    if (left) {
      bool any = false;
      for (size_t i = 0; i < B->hp.size(); ++i) any |= B->active[i] != 0;
      if (!any) break;
      FE_TRY(fe_batch_build(B));
    }
  }
  return FE_OK;
}

extern "C" fe_status fe_cg_solve_batched(int nprob, const fe_mesh* const* meshes,
                                         const double* const* b, double* const* x,
                                         const fe_cg_opts* opts, fe_cg_result* res, void* stream) {
  if (nprob < 1 || !meshes || !b || !x || !opts || !res) {
    fe_set_error("fe_cg_solve_batched: null argument or nprob < 1");
    return FE_ERR_INVALID;
  }
  if (opts->maxit < 1 || !(opts->rtol >= 0.0) || (opts->mixed != 0 && opts->mixed != FE_F32)) {
    fe_set_error("fe_cg_solve_batched: invalid options");
    return FE_ERR_INVALID;
  }
  for (int i = 0; i < nprob; ++i) {
    if (!meshes[i] || !b[i] || !x[i] || !fe_aligned(b[i]) || !fe_aligned(x[i])) {
      fe_set_error("fe_cg_solve_batched: problem %d: null or misaligned argument", i);
      return FE_ERR_INVALID;
    }
    if (meshes[i]->d.geom_mode == FE_GEOM_RECOMPUTE || meshes[i]->packed || meshes[i]->mzg > 0 ||
        meshes[i]->d.device != meshes[0]->d.device) {
      fe_set_error("fe_cg_solve_batched: problem %d: needs whole meshes with stored/affine geometry "
                   "on one device", i);
      return FE_ERR_INVALID;
    }
    for (int j = 0; j < i; ++j)
      if (meshes[j] == meshes[i]) {
        fe_set_error("fe_cg_solve_batched: mesh %d appears twice", i);
        return FE_ERR_INVALID;
      }
  }
  FeDeviceGuard device_guard;
  FE_CUDA(device_guard.set(meshes[0]->d.device), "cudaSetDevice");
  FE_CUDA(cudaStreamSynchronize((cudaStream_t)stream), "caller stream");
  const bool mixed = opts->mixed == FE_F32;
  FE_TRY(fe_batch_prepare());
  FeBatch B;
  FE_CUDA(cudaStreamCreateWithFlags(&B.st, cudaStreamNonBlocking), "batch stream");
  B.hp.resize(nprob);
  B.active.assign(nprob, 1);
  FE_CUDA(cudaMallocHost(&B.hsc, 2 * nprob * sizeof(CgScal)), "batch scalars");
  B.cap_hsc = 2 * nprob;
  std::vector<double> sb(nprob, 1.0);
  for (int i = 0; i < nprob; ++i) {
    CgWork* w = nullptr;
    FE_TRY(fe_cg_get_work(meshes[i], mixed, &w));
    FE_TRY(fe_ensure_geometry(meshes[i], FE_F64, false));
    if (mixed) FE_TRY(fe_ensure_geometry(meshes[i], FE_F32, false));
    FE_TRY(fe_cg_ensure_diag(meshes[i], w, FE_LAPLACE));
    // each problem scaled by its own exact power of two (fe_cg_rhs_scale), undone on x at the end
    const long long ncw = meshes[i]->ncw;
    FE_TRY(fe_cg_rhs_scale(w, b[i], ncw, &sb[i]));
    FE_TRY(fe_cg_scale(b[i], w->bs, sb[i], ncw, w->st));
    FE_TRY(fe_cg_scale(x[i], w->x, sb[i], ncw, w->st));
    FE_CUDA(cudaStreamSynchronize(w->st), "workspace set-up");
    FE_TRY(fe_batch_fill(&B, i, meshes[i], w, w->bs, opts));
  }
  B.any_flexible = (!mixed && opts->flexible) ? 1 : 0;
  FE_TRY(fe_batch_build(&B));
  FE_TRY(fe_batch_solve(&B, opts));
  FE_TRY(fe_batch_read(&B));
  fe_status worst = FE_OK;
  for (int i = 0; i < nprob; ++i) {
    FE_TRY(fe_cg_scale(B.hp[i].x64, x[i], 1.0 / sb[i], meshes[i]->ncw, B.st));
    const CgScal& o = B.hsc[2 * i];
    const CgScal& in = B.hsc[2 * i + 1];
    res[i].status = (fe_status)o.status;
    res[i].rel_res = o.relres;
    res[i].iters = mixed ? in.stall_total : o.iter;
    res[i].outer_iters = mixed ? o.iter : 1;
    if (o.status != FE_OK && worst == FE_OK) worst = (fe_status)o.status;
  }
  FE_CUDA(cudaStreamSynchronize(B.st), "batch synchronize");
  if (worst != FE_OK) fe_set_error("fe_cg_solve_batched: some problems did not converge");
  return worst;
}
