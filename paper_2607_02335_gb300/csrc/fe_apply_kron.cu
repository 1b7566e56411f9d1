// fe_apply_kron.cu -- the operator with 16-bit operands on the tensor cores (n <= 4).
//
// For n <= 4 the whole cell operator is a pair of small dense products (Eq. (mass_operator),
// Eq. (laplace_operator)): the gradient at the n^3 Gauss points is G x with G = [Dh (x) V (x) V;
// V (x) Dh (x) V; V (x) V (x) Dh] (3 n^3 x n^3), the metric multiplies each point's three
// components, and y = G^T t.  Mass: B = V (x) V (x) V, y = B^T (w detJ B x).  Written as matrix
// products over a batch of cells (rows = cells, K = nodes or point components), they map onto
// mma.sync m16n8k16 with 16-bit A and B operands and FP32 accumulation: a warp takes 16 cells,
// the cells' x in its A fragments, G (or B) from a fragment-ordered copy in shared memory, and
// the accumulators of the first product become the A fragments of the second after the metric
// scaling, without leaving registers.  Every operand of a product is a 16-bit value (x, the
// Kronecker entries formed in FP32 from the FP64 1D rules and rounded once, the scaled point
// values); the metric product and all accumulation are FP32.
//
// Index maps (chosen so that the four lanes holding one cell's row touch contiguous memory):
//  - x, k-step kk, fragment column c (0..15): node 16 kk + 4 ((c & 7) >> 1) + 2 (c >> 3) + (c & 1),
//    so lane t of a cell loads nodes 16 kk + 4 t + {0,1,2,3} (one 16-byte load per k-step);
//  - first-product column r (0..7) of n-tile nt, point group g (Laplace nt = 3 g + component,
//    mass nt = g), GC groups per chunk: point 8 GC (g / GC) + 2 GC (r >> 1) + 2 (g % GC) + (r & 1),
//    so lane t holds 2 GC consecutive points of each chunk (one load per metric entry);
//  - output column r of n-tile nb: node 16 (nb >> 1) + 4 (r >> 1) + 2 (nb & 1) + (r & 1) when
//    the output n-tiles come in pairs (one 16-byte store per pair), node 8 nb + r otherwise.
#include <cstdlib>
#include <cstring>

#include "fe_internal.h"

#ifndef FE_KRON_BIG_WARPS
#define FE_KRON_BIG_WARPS 4
#endif
#ifndef FE_KRON_BIG_MINB
#define FE_KRON_BIG_MINB 2
#endif

namespace {

template <int N, int OP>
struct Kron {
  static constexpr int NP = N * N * N;
  static constexpr int KS = (NP + 15) / 16;                        // k-steps of G x
  static constexpr int NG = (NP + 7) / 8;                          // groups of 8 points
  static constexpr int GC = NG >= 2 ? 2 : 1;                       // groups per chunk
  static constexpr int NCH = NG / GC;                              // chunks
  static constexpr int COMP = OP == FE_LAPLACE ? 3 : 1;            // components per point
  static constexpr int NTF = COMP * NG;                            // n-tiles of G x
  static constexpr int NTC = COMP * GC;                            // ... of one chunk
  static constexpr int KSC = (NTC + 1) / 2;                        // k-steps of G^T t per chunk
  static constexpr int NTB = (NP + 7) / 8;                         // n-tiles of the output
  static constexpr bool PAIRED = NTB % 2 == 0;
  // B fragments of two n-tiles side by side (one 16-byte shared load for two products)
  static constexpr bool PAIRF = NTF % 2 == 0 && NTC % 2 == 0;
  static constexpr bool PAIRB = NTB % 2 == 0;
  static constexpr int FWORDS = KS * NTF * 64;                     // 32-bit words of G
  static constexpr int BWORDS = NCH * KSC * NTB * 64;              // ... of G^T
  static constexpr int WORDS = FWORDS + BWORDS;
  // Q3 Laplace: 2 CTAs of 4 warps per SM with 219 registers a thread (x fragments, output
  // accumulators, a chunk's accumulators and metric, and the next phase's loads in flight), the
  // fastest of the shapes measured at Q3 96^3 (8 warps at 219 registers 0.265 ms; 12 at 168 with
  // spills 0.310 ms; 16 at 128 with spills 0.371 ms); the others fit 128 registers
  static constexpr bool BIG = OP == FE_LAPLACE && N == 4;
  static constexpr int WARPS = BIG ? FE_KRON_BIG_WARPS : 8;
  static constexpr int MINB = BIG ? FE_KRON_BIG_MINB : 2;
  static constexpr int THREADS = WARPS * 32;
  static_assert(NG % GC == 0, "whole chunks");
  static_assert(NTC % 2 == 0 || NCH == 1, "chunks end on a k-step");
};

struct KronArgs {
  const float* x;
  float* y;
  const unsigned short* geo;  // [cell][7][n^3] 16-bit metric, scaled by 1 / oscale
  long long ncells;
  int mx, my, mz, dirichlet;
  float oscale;
  const int* skip;
  const unsigned* tab;         // fragment tables of the operator (k_kron_tables)
  float V[FE_MAXN][FE_MAXN];   // V[q][i] = l_i(s_q)
  float Dh[FE_MAXN][FE_MAXN];  // Dh[q][i] = l_i'(s_q)
};

__device__ __forceinline__ int x_node(int kk, int c) {
  return 16 * kk + 4 * ((c & 7) >> 1) + 2 * (c >> 3) + (c & 1);
}
template <int N, int OP>
__device__ __forceinline__ int point_of(int nt, int r) {
  using K = Kron<N, OP>;
  const int g = nt / K::COMP;
  return 8 * K::GC * (g / K::GC) + 2 * K::GC * (r >> 1) + 2 * (g % K::GC) + (r & 1);
}
template <int N, int OP>
__device__ __forceinline__ int out_node(int nb, int r) {
  if constexpr (Kron<N, OP>::PAIRED)
    return 16 * (nb >> 1) + 4 * (r >> 1) + 2 * (nb & 1) + (r & 1);
  else
    return 8 * nb + r;
}

// entry of the (component comp of the) gradient matrix, or of B for mass, at point q, node nd
template <int N, int OP>
__device__ float kron_entry(const KronArgs& a, int comp, int q, int nd) {
  const int qx = q % N, qy = (q / N) % N, qz = q / (N * N);
  const int i = nd % N, j = (nd / N) % N, k = nd / (N * N);
  const float fx = (OP == FE_LAPLACE && comp == 0) ? a.Dh[qx][i] : a.V[qx][i];
  const float fy = (OP == FE_LAPLACE && comp == 1) ? a.Dh[qy][j] : a.V[qy][j];
  const float fz = (OP == FE_LAPLACE && comp == 2) ? a.Dh[qz][k] : a.V[qz][k];
  return fx * fy * fz;
}

template <bool BF>
__device__ __forceinline__ unsigned pack16(float lo, float hi) {
  if constexpr (BF) {
    const __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);
    return *reinterpret_cast<const unsigned*>(&v);
  } else {
    const __half2 v = __floats2half2_rn(lo, hi);
    return *reinterpret_cast<const unsigned*>(&v);
  }
}
template <bool BF>
__device__ __forceinline__ float unpack16(unsigned short b) {
  if constexpr (BF)
    return __uint_as_float((unsigned)b << 16);
  else
    return __half2float(__ushort_as_half(b));
}

template <bool BF>
__device__ __forceinline__ void mma16816(float (&d)[4], const unsigned (&a)[4], unsigned b0,
                                         unsigned b1) {
  if constexpr (BF)
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, "
        "{%8,%9}, {%0,%1,%2,%3};"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
  else
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.f16.f16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, "
        "{%8,%9}, {%0,%1,%2,%3};"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

// Fragment-ordered tables: word ((f * 32 + lane) * 2 + b) holds register b of lane's B fragment
// of fragment f, or, with fragments paired, word (((f >> 1) * 32 + lane) * 2 + (f & 1)) * 2 + b.
// B fragment (16 x 8, k x col): register b, half h holds k = 2 (lane & 3) + 8 b + h,
// col = lane >> 2.  Forward f = kk * NTF + nt; backward f = (ch * KSC + ks) * NTB + nb.
template <int N, int OP, bool BF>
__device__ unsigned table_word(const KronArgs& a, int w) {
  using K = Kron<N, OP>;
  const bool fwd = w < K::FWORDS;
  const int ww = fwd ? w : w - K::FWORDS;
  const bool pair = fwd ? K::PAIRF : K::PAIRB;
  const int b = ww & 1;
  const int lane = pair ? (ww >> 2) & 31 : (ww >> 1) & 31;
  const int f = pair ? 2 * (ww >> 7) + ((ww >> 1) & 1) : ww >> 6;
  float v[2];
#pragma unroll
  for (int h = 0; h < 2; ++h) {
    const int kl = 2 * (lane & 3) + 8 * b + h, col = lane >> 2;
    float e = 0.0f;
    if (fwd) {
      const int kk = f / K::NTF, nt = f % K::NTF;
      const int nd = x_node(kk, kl), q = point_of<N, OP>(nt, col);
      if (nd < K::NP && q < K::NP) e = kron_entry<N, OP>(a, nt % K::COMP, q, nd);
    } else {
      const int nb = f % K::NTB, cks = f / K::NTB, ch = cks / K::KSC, ks = cks % K::KSC;
      const int ntc = 2 * ks + (kl >> 3);  // n-tile within the chunk
      const int nt = ch * K::NTC + ntc;
      const int q = point_of<N, OP>(nt, kl & 7), nd = out_node<N, OP>(nb, col);
      if (ntc < K::NTC && q < K::NP && nd < K::NP) e = kron_entry<N, OP>(a, nt % K::COMP, q, nd);
    }
    v[h] = e;
  }
  return pack16<BF>(v[0], v[1]);
}

// the tables of one (n, operator, 16-bit format), once per mesh
template <int N, int OP, bool BF>
__global__ void k_kron_tables(const KronArgs a, unsigned* out) {
  using K = Kron<N, OP>;
  for (int w = blockIdx.x * blockDim.x + threadIdx.x; w < K::WORDS; w += gridDim.x * blockDim.x)
    out[w] = table_word<N, OP, BF>(a, w);
}

// faces of a node: bit 0 x = 0, 1 x = n-1, 2 y = 0, 3 y = n-1, 4 z = 0, 5 z = n-1
template <int N>
__device__ __forceinline__ unsigned node_faces(int nd) {
  const int i = nd % N, j = (nd / N) % N, k = nd / (N * N);
  return (i == 0 ? 1u : 0u) | (i == N - 1 ? 2u : 0u) | (j == 0 ? 4u : 0u) | (j == N - 1 ? 8u : 0u) |
         (k == 0 ? 16u : 0u) | (k == N - 1 ? 32u : 0u);
}
__device__ __forceinline__ unsigned cell_faces(const KronArgs& a, long long c) {
  if (!a.dirichlet) return 0u;
  const long long cxy = (long long)a.mx * a.my;
  const int cz = (int)(c / cxy), rem = (int)(c - (long long)cz * cxy);
  const int cy = rem / a.mx, cx = rem - cy * a.mx;
  unsigned f = 0;
  if (a.dirichlet & FE_DIR_XY)
    f |= (cx == 0 ? 1u : 0u) | (cx == a.mx - 1 ? 2u : 0u) | (cy == 0 ? 4u : 0u) |
         (cy == a.my - 1 ? 8u : 0u);
  if ((a.dirichlet & FE_DIR_ZLO) && cz == 0) f |= 16u;
  if ((a.dirichlet & FE_DIR_ZHI) && cz == a.mz - 1) f |= 32u;
  return f;
}

template <int N, int OP, bool BF>
__global__ void __launch_bounds__(Kron<N, OP>::THREADS, Kron<N, OP>::MINB) k_apply_kron(const KronArgs a) {
  using K = Kron<N, OP>;
  constexpr int NE = OP == FE_LAPLACE ? 6 : 1;  // metric entries per point
  constexpr int NPT = 2 * K::GC;                // points of a chunk per lane and cell
  if (a.skip && *(volatile const int*)a.skip) return;  // uniform over the grid
  extern __shared__ __align__(16) unsigned tab[];
  static_assert(K::WORDS % 4 == 0, "16-byte table copy");
  for (int w = threadIdx.x; w < K::WORDS / 4; w += blockDim.x)
    reinterpret_cast<uint4*>(tab)[w] = __ldg(reinterpret_cast<const uint4*>(a.tab) + w);
  __syncthreads();
  const unsigned* ftab = tab;
  const unsigned* btab = tab + K::FWORDS;

  const int lane = threadIdx.x & 31, t = lane & 3, gid = lane >> 2;
  // Dirichlet: for every face, the bits of this lane's input nodes (4 kk + u) and output nodes
  // (4 j + u paired, 2 nb + e otherwise) on it
  unsigned short fin16[6] = {0, 0, 0, 0, 0, 0}, fout16[6] = {0, 0, 0, 0, 0, 0};
  if (a.dirichlet) {
#pragma unroll
    for (int kk = 0; kk < K::KS; ++kk)
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const int nd = 16 * kk + 4 * t + u;
        const unsigned fc = nd < K::NP ? node_faces<N>(nd) : 0u;
#pragma unroll
        for (int f = 0; f < 6; ++f)
          if (fc & (1u << f)) fin16[f] |= (unsigned short)(1u << (4 * kk + u));
      }
#pragma unroll
    for (int nb = 0; nb < K::NTB; ++nb)
#pragma unroll
      for (int e = 0; e < 2; ++e) {
        const int nd = out_node<N, OP>(nb, 2 * t + e);
        const int bit = K::PAIRED ? 4 * (nb >> 1) + 2 * (nb & 1) + e : 2 * nb + e;
        const unsigned fc = nd < K::NP ? node_faces<N>(nd) : 0u;
#pragma unroll
        for (int f = 0; f < 6; ++f)
          if (fc & (1u << f)) fout16[f] |= (unsigned short)(1u << bit);
      }
  }
  auto face_mask = [&](const unsigned short (&fm)[6], unsigned faces) {
    unsigned m = 0;
#pragma unroll
    for (int f = 0; f < 6; ++f)
      if (faces & (1u << f)) m |= fm[f];
    return m;
  };

  const long long ntasks = (a.ncells + 15) / 16;
  const long long wstride = (long long)gridDim.x * K::WARPS;
  long long task = (long long)blockIdx.x * K::WARPS + (threadIdx.x >> 5);
  if (task >= ntasks) return;  // uniform over the warp

  // The loads of the next phase are issued as soon as their registers are free: the next task's
  // x after the last first product, the next chunk's metric after the scaling.  A cell past the
  // end (ragged last task, or the task after a warp's last) reads cell 0 and is zeroed.
  unsigned ax[K::KS][4];
  unsigned gw[2][NE][NPT / 2];  // metric, two 16-bit values per word, lower point in the low half
  auto load_x = [&](long long tk) {
    const long long cA = tk * 16 + gid, cB = cA + 8;
    const bool vA = cA < a.ncells, vB = cB < a.ncells;
    const long long lA = vA ? cA : 0, lB = vB ? cB : 0;
    const unsigned mA = vA ? face_mask(fin16, cell_faces(a, cA)) : ~0u;
    const unsigned mB = vB ? face_mask(fin16, cell_faces(a, cB)) : ~0u;
#pragma unroll
    for (int kk = 0; kk < K::KS; ++kk) {
      float xa[4] = {0.f, 0.f, 0.f, 0.f}, xb[4] = {0.f, 0.f, 0.f, 0.f};
      const int nd0 = 16 * kk + 4 * t;
      if constexpr (K::NP % 4 == 0) {
        if (nd0 < K::NP) {
          const float4 va = __ldcs(reinterpret_cast<const float4*>(a.x + lA * K::NP + nd0));
          const float4 vb = __ldcs(reinterpret_cast<const float4*>(a.x + lB * K::NP + nd0));
          xa[0] = va.x, xa[1] = va.y, xa[2] = va.z, xa[3] = va.w;
          xb[0] = vb.x, xb[1] = vb.y, xb[2] = vb.z, xb[3] = vb.w;
        }
      } else {
#pragma unroll
        for (int u = 0; u < 4; ++u)
          if (nd0 + u < K::NP) {
            xa[u] = __ldcs(a.x + lA * K::NP + nd0 + u);
            xb[u] = __ldcs(a.x + lB * K::NP + nd0 + u);
          }
      }
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        if (mA & (1u << (4 * kk + u))) xa[u] = 0.f;
        if (mB & (1u << (4 * kk + u))) xb[u] = 0.f;
      }
      ax[kk][0] = pack16<BF>(xa[0], xa[1]);
      ax[kk][1] = pack16<BF>(xb[0], xb[1]);
      ax[kk][2] = pack16<BF>(xa[2], xa[3]);
      ax[kk][3] = pack16<BF>(xb[2], xb[3]);
    }
  };
  auto load_gw = [&](long long tk, int ch) {
    const int p0 = 8 * K::GC * ch + NPT * t;
#pragma unroll
    for (int s = 0; s < 2; ++s) {
      const long long c = tk * 16 + gid + 8 * s;
      const bool v = c < a.ncells;
      const long long l = v ? c : 0;
#pragma unroll
      for (int e = 0; e < NE; ++e) {
        const int comp = OP == FE_LAPLACE ? e : 6;
        const unsigned short* gp = a.geo + (l * FE_GEO_COMPS + comp) * K::NP + p0;
#pragma unroll
        for (int w = 0; w < NPT / 2; ++w) gw[s][e][w] = 0u;
        if constexpr (K::NP % 4 == 0 && NPT == 4) {
          const uint2 w = __ldcs(reinterpret_cast<const uint2*>(gp));
          gw[s][e][0] = w.x, gw[s][e][1] = w.y;
        } else if constexpr (K::NP % 2 == 0 && NPT == 2) {
          gw[s][e][0] = __ldcs(reinterpret_cast<const unsigned*>(gp));
        } else {
#pragma unroll
          for (int u = 0; u < NPT; ++u)
            if (p0 + u < K::NP) gw[s][e][u >> 1] |= (unsigned)__ldcs(gp + u) << (16 * (u & 1));
        }
#pragma unroll
        for (int w = 0; w < NPT / 2; ++w) gw[s][e][w] = v ? gw[s][e][w] : 0u;
      }
    }
  };

  load_x(task);
  load_gw(task, 0);
  for (; task < ntasks; task += wstride) {
    const long long next = task + wstride;
    float out[K::NTB][4];
#pragma unroll
    for (int nb = 0; nb < K::NTB; ++nb) out[nb][0] = out[nb][1] = out[nb][2] = out[nb][3] = 0.f;

#pragma unroll
    for (int ch = 0; ch < K::NCH; ++ch) {
      // first product for the chunk's n-tiles
      float acc[K::NTC][4];
#pragma unroll
      for (int j = 0; j < K::NTC; ++j) acc[j][0] = acc[j][1] = acc[j][2] = acc[j][3] = 0.f;
      if constexpr (K::PAIRF) {
#pragma unroll
        for (int j = 0; j < K::NTC; j += 2) {
          const int nt = ch * K::NTC + j;
#pragma unroll
          for (int kk = 0; kk < K::KS; ++kk) {
            const uint4 bf =
                reinterpret_cast<const uint4*>(ftab)[((kk * K::NTF + nt) >> 1) * 32 + lane];
            mma16816<BF>(acc[j], ax[kk], bf.x, bf.y);
            mma16816<BF>(acc[j + 1], ax[kk], bf.z, bf.w);
          }
        }
      } else {
#pragma unroll
        for (int j = 0; j < K::NTC; ++j) {
          const int nt = ch * K::NTC + j;
#pragma unroll
          for (int kk = 0; kk < K::KS; ++kk) {
            const uint2 bf = reinterpret_cast<const uint2*>(ftab)[(kk * K::NTF + nt) * 32 + lane];
            mma16816<BF>(acc[j], ax[kk], bf.x, bf.y);
          }
        }
      }
      if (ch == K::NCH - 1) load_x(next);  // x of this task is no longer needed
      // metric: accumulator (row s, column 2 t + e) of group gl is point p0 + 2 gl + e
#pragma unroll
      for (int gl = 0; gl < K::GC; ++gl)
#pragma unroll
        for (int s = 0; s < 2; ++s)
#pragma unroll
          for (int e = 0; e < 2; ++e) {
            const int u = 2 * gl + e, r = 2 * s + e;
            auto gm = [&](int e2) {
              return unpack16<BF>((unsigned short)(gw[s][e2][u >> 1] >> (16 * (u & 1))));
            };
            if constexpr (OP == FE_LAPLACE) {
              const float gx = acc[3 * gl][r], gy = acc[3 * gl + 1][r], gz = acc[3 * gl + 2][r];
              const float mxx = gm(0), myy = gm(1), mzz = gm(2), mxy = gm(3), mxz = gm(4),
                          myz = gm(5);
              acc[3 * gl][r] = fmaf(mxx, gx, fmaf(mxy, gy, mxz * gz));
              acc[3 * gl + 1][r] = fmaf(mxy, gx, fmaf(myy, gy, myz * gz));
              acc[3 * gl + 2][r] = fmaf(mxz, gx, fmaf(myz, gy, mzz * gz));
            } else {
              acc[gl][r] *= gm(0);
            }
          }
      if (ch + 1 < K::NCH)
        load_gw(task, ch + 1);
      else
        load_gw(next, 0);
      // second product: k-step ks of the chunk takes its n-tiles 2 ks and 2 ks + 1 as A
#pragma unroll
      for (int ks = 0; ks < K::KSC; ++ks) {
        unsigned af[4];
        af[0] = pack16<BF>(acc[2 * ks][0], acc[2 * ks][1]);
        af[1] = pack16<BF>(acc[2 * ks][2], acc[2 * ks][3]);
        if (2 * ks + 1 < K::NTC) {
          af[2] = pack16<BF>(acc[2 * ks + 1][0], acc[2 * ks + 1][1]);
          af[3] = pack16<BF>(acc[2 * ks + 1][2], acc[2 * ks + 1][3]);
        } else {
          af[2] = af[3] = 0u;
        }
        const int f0 = (ch * K::KSC + ks) * K::NTB;
        if constexpr (K::PAIRB) {
#pragma unroll
          for (int nb = 0; nb < K::NTB; nb += 2) {
            const uint4 bf = reinterpret_cast<const uint4*>(btab)[((f0 + nb) >> 1) * 32 + lane];
            mma16816<BF>(out[nb], af, bf.x, bf.y);
            mma16816<BF>(out[nb + 1], af, bf.z, bf.w);
          }
        } else {
#pragma unroll
          for (int nb = 0; nb < K::NTB; ++nb) {
            const uint2 bf = reinterpret_cast<const uint2*>(btab)[(f0 + nb) * 32 + lane];
            mma16816<BF>(out[nb], af, bf.x, bf.y);
          }
        }
      }
    }

    // y: scale back, Dirichlet rows, store
    const long long cA = task * 16 + gid, cB = cA + 8;
    const bool vA = cA < a.ncells, vB = cB < a.ncells;
    const unsigned oA = vA ? face_mask(fout16, cell_faces(a, cA)) : 0u;
    const unsigned oB = vB ? face_mask(fout16, cell_faces(a, cB)) : 0u;
#pragma unroll
    for (int s = 0; s < 2; ++s) {
      const long long c = s ? cB : cA;
      if (!(s ? vB : vA)) continue;
      const unsigned om = s ? oB : oA;
      float* yc = a.y + c * K::NP;
      if constexpr (K::PAIRED) {
#pragma unroll
        for (int j = 0; j < K::NTB / 2; ++j) {
          float v[4] = {out[2 * j][2 * s], out[2 * j][2 * s + 1], out[2 * j + 1][2 * s],
                        out[2 * j + 1][2 * s + 1]};
#pragma unroll
          for (int u = 0; u < 4; ++u) v[u] = (om & (1u << (4 * j + u))) ? 0.f : v[u] * a.oscale;
          const int nd0 = 16 * j + 4 * t;
          if constexpr (K::NP % 4 == 0) {
            __stcs(reinterpret_cast<float4*>(yc + nd0), make_float4(v[0], v[1], v[2], v[3]));
          } else {
#pragma unroll
            for (int u = 0; u < 4; ++u)
              if (nd0 + u < K::NP) __stcs(yc + nd0 + u, v[u]);
          }
        }
      } else {
#pragma unroll
        for (int nb = 0; nb < K::NTB; ++nb) {
          float v[2] = {out[nb][2 * s], out[nb][2 * s + 1]};
#pragma unroll
          for (int e = 0; e < 2; ++e) v[e] = (om & (1u << (2 * nb + e))) ? 0.f : v[e] * a.oscale;
          const int nd0 = 8 * nb + 2 * t;
          if (nd0 + 1 < K::NP)
            __stcs(reinterpret_cast<float2*>(yc + nd0), make_float2(v[0], v[1]));
        }
      }
    }
  }
}

void fill_args(KronArgs& a, const fe_mesh* m, int op) {
  std::memset(&a, 0, sizeof(a));
  a.ncells = m->ncells;
  a.mx = m->d.mx;
  a.my = m->d.my;
  a.mz = m->d.mz;
  a.dirichlet = fe_dir_mask(m);
  a.oscale = 1.0f / m->gscale[op == FE_LAPLACE ? 0 : 1];
  for (int q = 0; q < m->n; ++q)
    for (int i = 0; i < m->n; ++i) {
      a.V[q][i] = (float)m->tab.V[q][i];
      a.Dh[q][i] = (float)m->tab.Dh[q][i];
    }
}

template <int N, int OP, bool BF>
fe_status build_tables(fe_mesh* m, unsigned** out) {
  using K = Kron<N, OP>;
  KronArgs a;
  fill_args(a, m, OP);
  FE_TRY(fe_dalloc((void**)out, (size_t)K::WORDS * sizeof(unsigned), m->st, "tensor-core tables"));
  k_kron_tables<N, OP, BF><<<(K::WORDS + 255) / 256, 256, 0, m->st>>>(a, *out);
  return fe_cuda_check(cudaGetLastError(), "tensor-core tables");
}

template <int N, bool BF>
fe_status build_both(fe_mesh* m, unsigned** lap, unsigned** mass) {
  FE_TRY((build_tables<N, FE_LAPLACE, BF>(m, lap)));
  return build_tables<N, FE_MASS, BF>(m, mass);
}

template <int N, int OP, bool BF>
fe_status launch_kron(const ApplyLaunch& L, const unsigned short* geo, const unsigned* tab) {
  using K = Kron<N, OP>;
  const fe_mesh* m = L.m;
  KronArgs a;
  fill_args(a, m, OP);
  a.x = static_cast<const float*>(L.x);
  a.y = static_cast<float*>(L.y);
  a.geo = geo;
  a.skip = L.skip;
  a.tab = tab;
  auto kern = k_apply_kron<N, OP, BF>;
  const size_t smem = (size_t)K::WORDS * sizeof(unsigned);
  static int slots[64] = {};  // resident CTAs on the whole device, per device
  int dev = 0;
  FE_CUDA(cudaGetDevice(&dev), "cudaGetDevice");
  int resident = (dev >= 0 && dev < 64) ? slots[dev] : 0;
  if (resident == 0) {
    FE_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem),
            "kron smem attribute");
    int per_sm = 0, sms = 0;
    FE_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, K::THREADS, smem),
            "occupancy");
    FE_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev), "SM count");
    resident = (per_sm > 0 ? per_sm : 1) * sms;
    if (dev >= 0 && dev < 64) slots[dev] = resident;
  }
  const long long ntasks = (m->ncells + 15) / 16;
  const long long need = (ntasks + K::WARPS - 1) / K::WARPS;
  const long long blocks = need < resident ? need : resident;
  if (blocks > 0) kern<<<(unsigned)blocks, K::THREADS, smem, L.st>>>(a);
  return fe_cuda_check(cudaGetLastError(), "kron apply launch");
}

template <int N, bool BF>
fe_status launch_kron_op(const ApplyLaunch& L, const unsigned short* geo, unsigned* const* tab) {
  return L.op == FE_LAPLACE ? launch_kron<N, FE_LAPLACE, BF>(L, geo, tab[0])
                            : launch_kron<N, FE_MASS, BF>(L, geo, tab[1]);
}

}  // namespace

bool fe_kron_eligible(const fe_mesh* m) {
  return m->n >= 2 && m->n <= 4 && !m->packed && m->d.geom_mode == FE_GEOM_STORED;
}

bool fe_kron_supported(const fe_mesh* m) {
  if (const char* e = std::getenv("FE_LOWP_FMA"))
    if (std::atoi(e) != 0) return false;
  return fe_kron_eligible(m);
}

fe_status fe_kron_build_tables(fe_mesh* m, int prec) {
  const int k = prec == FE_BF16_F32ACC ? 0 : 1;
  if (!fe_kron_eligible(m) || m->kron_tab[k][0]) return FE_OK;
  unsigned** t = m->kron_tab[k];
  switch (m->n) {
    case 2: FE_TRY((k == 0 ? build_both<2, true>(m, &t[0], &t[1]) : build_both<2, false>(m, &t[0], &t[1]))); break;
    case 3: FE_TRY((k == 0 ? build_both<3, true>(m, &t[0], &t[1]) : build_both<3, false>(m, &t[0], &t[1]))); break;
    case 4: FE_TRY((k == 0 ? build_both<4, true>(m, &t[0], &t[1]) : build_both<4, false>(m, &t[0], &t[1]))); break;
  }
  return fe_cuda_check(cudaStreamSynchronize(m->st), "tensor-core tables");
}

fe_status fe_launch_apply_kron(const ApplyLaunch& L, int prec) {
  const fe_mesh* m = L.m;
  const bool bf = prec == FE_BF16_F32ACC;
  const unsigned short* geo = m->geo16[bf ? 0 : 1];
  unsigned* const* tab = m->kron_tab[bf ? 0 : 1];
  if (!geo || !tab[0] || !tab[1]) {
    fe_set_error("apply: the 16-bit metric or the tensor-core tables of this mesh are missing");
    return FE_ERR_INVALID;
  }
  switch (m->n) {
    case 2: FE_TRY((bf ? launch_kron_op<2, true>(L, geo, tab) : launch_kron_op<2, false>(L, geo, tab))); break;
    case 3: FE_TRY((bf ? launch_kron_op<3, true>(L, geo, tab) : launch_kron_op<3, false>(L, geo, tab))); break;
    case 4: FE_TRY((bf ? launch_kron_op<4, true>(L, geo, tab) : launch_kron_op<4, false>(L, geo, tab))); break;
    default:
      fe_set_error("apply: tensor-core kernels cover n = 2..4, not %d", m->n);
      return FE_ERR_INVALID;
  }
  if (!L.assemble) return FE_OK;
  if (L.brick_out) {  // nothing was summed in the kernel: the caller runs the full passes
    L.brick_out[0] = L.brick_out[1] = 1;
    return FE_OK;
  }
  return fe_launch_dss(m, FE_F32, L.y, L.st);
}
