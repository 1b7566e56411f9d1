// fe_apply_kernel.cuh -- sum-factorized cell-wise operator apply (one template, three
// arithmetics).
//
// Per cell K the kernel computes y_K = A_K x_K, the unassembled dual output of the local
// operator (Sec. 3.1), with the sum factorization of Sec. 2.3 extended to general
// per-quadrature-point geometry:
//   Laplace  y_K = (V^T x V^T x V^T) [ sum_a D_a^T ( G (D_x u_q, D_y u_q, D_z u_q) )_a ],
//            u_q = (V x V x V) x_K,  G = w_q detJ J^{-1} J^{-T}    (Eq. (laplace_operator))
//   mass     y_K = (V^T x V^T x V^T) (w_q detJ) (V x V x V) x_K   (Eq. (mass_operator))
// V interpolates from the n GLL nodes to the n Gauss points of a direction, D is the
// collocation derivative at the Gauss points.
//
// Thread mapping.  A CTA owns CPB consecutive cells and n^2 threads per cell.  Thread t of a cell
// owns one 1D line of the cell's n^3 tensor per phase: the z-line (i,j) = (t % n, t / n) while
// data sits in registers (global load/store, pointwise geometry, z sweeps), the x-line
// (j,k) = (t % n, t / n) and the y-line (i,k) = (t % n, t / n) for the x and y sweeps, which
// read and write the cell's tile in shared memory.  Rows of the tile are padded to n+1 entries,
// which keeps the line accesses of a warp free of bank conflicts (double-word values are stored
// as interleaved hi/lo pairs, one 64-bit access each).
//
// Every 1D contraction uses the even-odd form of the matrix (the reflection symmetry of the GLL
// nodes and Gauss points; the even-odd decomposition named in Sec. 2.3 "Initial performance
// measurements"), which halves the multiply-adds.
// Up to n = FE_ROLL_MINN - 1 all loops unroll with compile-time indices, so the 1D tables (kernel
// parameters) are read from the constant bank as instruction operands; from n = FE_ROLL_MINN on
// the double-word and FP64 kernels keep the output loop of each contraction a run-time loop
// (apply_cells_rolled), because fully unrolled they no longer fit the instruction cache.
#pragma once
#include <type_traits>

#include "fe_internal.h"

template <int N>
struct Cfg {
  static constexpr int N2 = N * N;
  static constexpr int N3 = N * N * N;
  static constexpr int CPB = (256 / N2) > 0 ? (256 / N2) : 1;  // cells per CTA
  static constexpr int THREADS = CPB * N2;
  static constexpr int RS = N + 1;      // padded row stride in shared memory
  static constexpr int PS = N * RS;     // plane stride
  static constexpr int CS = N * PS;     // cell stride
  static constexpr int TILE = CPB * CS; // elements per array per CTA
};

// shared-memory view of one array of the tile
template <class V>
struct Sm;
template <>
struct Sm<double> {
  double* p;
  __device__ __forceinline__ Sm(unsigned char* base, int, int arr, int tile)
      : p(reinterpret_cast<double*>(base) + (size_t)arr * tile) {}
  __device__ __forceinline__ double get(int e) const { return p[e]; }
  __device__ __forceinline__ void put(int e, double v) const { p[e] = v; }
  static constexpr int BYTES = 8;
};
template <>
struct Sm<float> {
  float* p;
  __device__ __forceinline__ Sm(unsigned char* base, int, int arr, int tile)
      : p(reinterpret_cast<float*>(base) + (size_t)arr * tile) {}
  __device__ __forceinline__ float get(int e) const { return p[e]; }
  __device__ __forceinline__ void put(int e, float v) const { p[e] = v; }
  static constexpr int BYTES = 4;
};
template <class W>
struct Sm16 {  // 16-bit-operand values kept as floats
  float* p;
  __device__ __forceinline__ Sm16(unsigned char* base, int, int arr, int tile)
      : p(reinterpret_cast<float*>(base) + (size_t)arr * tile) {}
  __device__ __forceinline__ W get(int e) const { return {p[e]}; }
  __device__ __forceinline__ void put(int e, W v) const { p[e] = v.v; }
  static constexpr int BYTES = 4;
};
template <>
struct Sm<bfv> : Sm16<bfv> {
  using Sm16<bfv>::Sm16;
};
template <>
struct Sm<hfv> : Sm16<hfv> {
  using Sm16<hfv>::Sm16;
};
template <>
struct Sm<dw> {  // hi and lo interleaved: one 64-bit shared-memory access per value
  float2* p;
  __device__ __forceinline__ Sm(unsigned char* base, int, int arr, int tile)
      : p(reinterpret_cast<float2*>(base) + (size_t)arr * tile) {}
  __device__ __forceinline__ dw get(int e) const {
    const float2 v = p[e];
    return {v.x, v.y};
  }
  __device__ __forceinline__ void put(int e, dw v) const { p[e] = make_float2(v.h, v.l); }
  static constexpr int BYTES = 8;
};

// One 1D contraction of a line in even-odd form (the EO comment in fe_internal.h):
// put(q, value) receives output q.  ROLLED: the output pairs are a run-time loop (outputs must
// go to shared memory); otherwise everything unrolls and put may write a register array.
template <int N, class V, int SIG, int ROLLED, class Put>
__device__ __forceinline__ void eo_line(const EO<N, V>& t, const V (&in)[N], Put put) {
  using T = NT<V>;
  constexpr int H = N / 2, MID = N / 2;
  V e[H], o[H];
#pragma unroll
  for (int r = 0; r < H; ++r) {
    e[r] = T::addk(in[r], in[N - 1 - r]);
    o[r] = T::subk(in[r], in[N - 1 - r]);
  }
  if constexpr (N & 1) {
    V acc;
    if constexpr (SIG > 0) {
      acc = T::prod(t.mm, in[MID]);
#pragma unroll
      for (int r = 0; r < H; ++r) acc = T::mac(acc, t.cr[r], e[r]);
    } else {
      acc = T::prod(t.cr[0], o[0]);
#pragma unroll
      for (int r = 1; r < H; ++r) acc = T::mac(acc, t.cr[r], o[r]);
    }
    put(MID, T::keep(acc));
  }
  auto pair = [&](int q) {
    V a = T::prod(t.A[q][0], e[0]);
#pragma unroll
    for (int r = 1; r < H; ++r) a = T::mac(a, t.A[q][r], e[r]);
    if constexpr (N & 1) a = T::mac(a, t.cm[q], in[MID]);
    V b = T::prod(t.B[q][0], o[0]);
#pragma unroll
    for (int r = 1; r < H; ++r) b = T::mac(b, t.B[q][r], o[r]);
    put(q, T::addk(a, b));
    put(N - 1 - q, SIG > 0 ? T::subk(a, b) : T::subk(b, a));
  };
  if constexpr (ROLLED > 0) {
    constexpr int kUnroll = ROLLED;  // output pairs per loop iteration
#pragma unroll(kUnroll)
    for (int q = 0; q < H; ++q) pair(q);
  } else {
#pragma unroll
    for (int q = 0; q < H; ++q) pair(q);
  }
}

// Derivative at the n Gauss points of a line from the n-1 differences d_s = x_{s+1} - x_s of its
// nodal values, in the even-odd form of B' (EOB in fe_arith.h); put(q, value) receives output q.
template <int N, class V, int ROLLED, class Put>
__device__ __forceinline__ void eob_line(const EOB<N, V>& t, const V (&d)[N - 1], Put put) {
  using T = NT<V>;
  using E = EOB<N, V>;
  constexpr int NI = E::NI, HI = E::HI, HO = E::HO;
  V e[E::HA], o[E::HA];
#pragma unroll
  for (int s = 0; s < HI; ++s) {
    e[s] = T::addk(d[s], d[NI - 1 - s]);
    o[s] = T::subk(d[s], d[NI - 1 - s]);
  }
  if constexpr (N & 1) {  // middle output (no middle difference for odd n)
    V acc = T::prod(t.cr[0], e[0]);
#pragma unroll
    for (int s = 1; s < HI; ++s) acc = T::mac(acc, t.cr[s], e[s]);
    put(N / 2, T::keep(acc));
  }
  auto pair = [&](int q) {
    V a;
    if constexpr (HI > 0) {
      a = T::prod(t.A[q][0], e[0]);
#pragma unroll
      for (int s = 1; s < HI; ++s) a = T::mac(a, t.A[q][s], e[s]);
      if constexpr (NI & 1) a = T::mac(a, t.cm[q], d[NI / 2]);
      V b = T::prod(t.B[q][0], o[0]);
#pragma unroll
      for (int s = 1; s < HI; ++s) b = T::mac(b, t.B[q][s], o[s]);
      put(q, T::addk(a, b));
      put(N - 1 - q, T::subk(a, b));
    } else {  // n = 2: one difference, a constant derivative
      a = T::keep(T::prod(t.cm[q], d[0]));
      put(q, a);
      put(N - 1 - q, a);
    }
  };
  if constexpr (ROLLED > 0) {
    constexpr int kUnroll = ROLLED;
#pragma unroll(kUnroll)
    for (int q = 0; q < HO; ++q) pair(q);
  } else {
#pragma unroll
    for (int q = 0; q < HO; ++q) pair(q);
  }
}

// Exponent shift of the FP64 path: the CTA's inputs enter the double-word arithmetic scaled by
// 2^-sh, sh = (binary exponent of the largest finite |x| of the CTA), and every output is scaled
// back by 2^sh.  Powers of two are exact, so the result is the same operator applied to x; the
// scaling keeps every intermediate double-word value (and its low part) inside the float range
// whatever the magnitude of x.  Scaled values below 2^-74 (of the CTA's largest) are flushed to
// zero.  All threads of the CTA call it; it holds a __syncthreads.
template <int N>
__device__ __forceinline__ int cta_exp_shift(const double (&xr)[N]) {
  __shared__ unsigned s_wmax[32];
  unsigned em = 0;
#pragma unroll
  for (int k = 0; k < N; ++k) {
    unsigned e = ((unsigned)__double2hiint(xr[k]) >> 20) & 0x7FFu;
    em = max(em, e == 0x7FFu ? 0u : e);  // infinities and NaNs keep their own value
  }
  const unsigned warp = threadIdx.x >> 5;
  const unsigned lanes = min(32u, blockDim.x - warp * 32u);
  em = __reduce_max_sync(lanes == 32u ? 0xFFFFFFFFu : ((1u << lanes) - 1u), em);
  if ((threadIdx.x & 31u) == 0u) s_wmax[warp] = em;
  __syncthreads();
  unsigned m = 0;
  const unsigned nw = (blockDim.x + 31u) >> 5;
  for (unsigned w = 0; w < nw; ++w) m = max(m, s_wmax[w]);
  return (int)m - 1023;
}

// Reference gradient at the Gauss points from differences of the stored inputs (the FP64 path:
// binary64 inputs into double-word differences; also written for float values): component a is
// B'_a (the derivative from the differences along axis a) followed by V along the two other axes.
// Every value the sweeps carry is of the size of a difference of neighbouring nodal values, not of
// x itself, so the rounding of the sweeps does not meet the cancellation of the derivative (a
// smooth field's Laplacian).  Three phases, each the same contraction on three lines of the thread
// (an axis loop, not unrolled, which keeps the kernel's code within the instruction cache):
//   1  B' on the x-, y- and z-line of the inputs (raw tile)  -> s1, s2, s0
//   2  V  along z of s1 and s2, along x of s0
//   3  V  along y of s1, along x of s2, along y of s0
// On return s1, s2, s0 hold d/dx, d/dy, d/dz of u at the Gauss points and sh the exponent shift
// (FP64 path; 0 otherwise).
template <int N, class V, int RU>
__device__ __forceinline__ void diff_gradient(const typename NT<V>::SV (&xr)[N],
                                              const Sm<typename NT<V>::SV>& raw, const Sm<V>& s0,
                                              const Sm<V>& s1, const Sm<V>& s2, int cb, int la,
                                              int lb, const Tab1D<N, V>& tab, int& sh) {
  constexpr bool DW = std::is_same<V, dw>::value;
  using SV = typename NT<V>::SV;
  constexpr int RS = Cfg<N>::RS, PS = Cfg<N>::PS;
  const int bx = cb + lb * PS + la * RS, by = cb + lb * PS + la, bz = cb + lb * RS + la;
#pragma unroll
  for (int k = 0; k < N; ++k) raw.put(bz + k * PS, xr[k]);
  if constexpr (DW)
    sh = cta_exp_shift<N>(xr);  // its barrier also publishes the raw tile
  else
    __syncthreads();
#pragma unroll 1
  for (int ax = 0; ax < 3; ++ax) {
    const int base = ax == 0 ? bx : (ax == 1 ? by : bz);
    const int st = ax == 0 ? 1 : (ax == 1 ? RS : PS);
    const Sm<V> o = ax == 0 ? s1 : (ax == 1 ? s2 : s0);
    SV dd[N - 1];
#pragma unroll
    for (int r = 0; r < N - 1; ++r) dd[r] = raw.get(base + (r + 1) * st) - raw.get(base + r * st);
    V d[N - 1];
#pragma unroll
    for (int r = 0; r < N - 1; ++r) {
      if constexpr (DW)
        d[r] = dw_from_double_ftz(dd[r], sh);
      else
        d[r] = dd[r];
    }
    eob_line<N, V, RU>(tab.eB, d, [&](int q, V v) { o.put(base + q * st, v); });
  }
  __syncthreads();
#pragma unroll 1
  for (int ax = 0; ax < 6; ++ax) {
    if (ax == 3) __syncthreads();
    const Sm<V> o = (ax == 0 || ax == 3) ? s1 : ((ax == 1 || ax == 4) ? s2 : s0);
    const int base = ax < 2 ? bz : ((ax == 2 || ax == 4) ? bx : by);
    const int st = ax < 2 ? PS : ((ax == 2 || ax == 4) ? 1 : RS);
    V in[N];
#pragma unroll
    for (int r = 0; r < N; ++r) in[r] = o.get(base + r * st);
    eo_line<N, V, 1, RU>(tab.eV, in, [&](int q, V v) { o.put(base + q * st, v); });
  }
  __syncthreads();
}

// register line -> register line
template <int N, class V, int SIG>
__device__ __forceinline__ void eo_regs(const EO<N, V>& t, const V (&in)[N], V (&out)[N]) {
  eo_line<N, V, SIG, 0>(t, in, [&](int q, V v) { out[q] = v; });
}

// line access in the padded tile: x-line (a=j, b=k), y-line (a=i, b=k), z-line (a=i, b=j)
template <int N>
__device__ __forceinline__ int xl(int a, int b, int r) { return b * Cfg<N>::PS + a * Cfg<N>::RS + r; }
template <int N>
__device__ __forceinline__ int yl(int a, int b, int r) { return b * Cfg<N>::PS + r * Cfg<N>::RS + a; }
template <int N>
__device__ __forceinline__ int zl(int a, int b, int r) { return r * Cfg<N>::PS + b * Cfg<N>::RS + a; }

// in-place 1D sweep of every line along one axis of the tile, by the line-owning thread
template <int N, class V, int AX, int SIG>
__device__ __forceinline__ void tile_sweep(const Sm<V>& s, int cbase, int a, int b,
                                           const EO<N, V>& M) {
  V in[N];
#pragma unroll
  for (int r = 0; r < N; ++r)
    in[r] = s.get(cbase + (AX == 0 ? xl<N>(a, b, r) : yl<N>(a, b, r)));
  eo_line<N, V, SIG, 0>(M, in, [&](int q, V v) {
    s.put(cbase + (AX == 0 ? xl<N>(a, b, q) : yl<N>(a, b, q)), v);
  });
}

// Everything an apply needs except the 1D tables.
template <int N, class V>
struct CellArgs {
  const typename NT<V>::SV* x;
  typename NT<V>::SV* y;
  const typename NT<V>::GV* geo;  // [cell - geo_cell0][7][N3]: w detJ J^-1 J^-T (xx,..,yz), w detJ
  long long ncells;               // cells at or above this index are not touched
  long long cell_base;            // first cell of the launch (k_apply)
  long long geo_cell0;            // cell whose metric is geo[0] (a chunk's scratch in recompute mode)
  int mx, my, mz;
  int dirichlet;  // FE_DIR_* mask of the Dirichlet faces (0: none)
  V aff[4];      // affine mode: detJ/h_x^2, detJ/h_y^2, detJ/h_z^2, detJ
  float oscale;  // 16-bit operand types: 1 / (power-of-two scale of the stored metric)
};

template <int N, class V>
struct ApplyArgs {
  CellArgs<N, V> c;
  const int* skip;  // optional device flag: the whole launch returns at once when *skip != 0
  int zchunk;       // MODE_BRICKZ: z-layers per CTA
  Tab1D<N, V> tab;
};

// MODE_BRICKZ state of one thread between the layers of its chunk: the stored value of the top
// node (k = n-1) of its z-line in the previous layer, whose store waits for the pair sum with the
// bottom node of the same line in the next layer.
template <class SV>
struct ZCarry {
  SV top;
  bool pending;  // top waits for this layer
  bool last;     // this layer is the chunk's last: its top node is stored at once
};

enum { GEOM_STORED_K = 0, GEOM_AFFINE_K = 2 };

// ---------------------------------------------------------------------------------------------
// Assembled applies (FE_ASSEMBLE): a CTA owns a BX x BY brick of cells in one z-layer and sums the
// copies on the x- and y-interfaces inside the brick in shared memory before it stores y (the
// fused part of the structured DSS of Sec. 4.1); the DSS passes that follow only visit the
// interfaces between bricks (and all z-interfaces).  Every node has at most one copy pair per
// axis, and the per-axis pair sums commute, so the order of the intra- and inter-brick sums does
// not change the assembled value.
// ---------------------------------------------------------------------------------------------
template <int N>
struct Brick;
template <> struct Brick<2> { static constexpr int BX = 8, BY = 8; };
template <> struct Brick<3> { static constexpr int BX = 7, BY = 4; };
template <> struct Brick<4> { static constexpr int BX = 4, BY = 4; };
template <> struct Brick<5> { static constexpr int BX = 5, BY = 2; };
template <> struct Brick<6> { static constexpr int BX = 3, BY = 2; };
template <> struct Brick<7> { static constexpr int BX = 2, BY = 2; };
template <> struct Brick<8> { static constexpr int BX = 2, BY = 2; };

struct CellPos {
  long long cell;
  int cx, cy, cz;
  bool active;
};

// Tile placement modes of an apply launch.  MODE_BRICKZ: a CTA walks a chunk of z-layers of one
// brick column, one MODE_BRICK tile per layer, and sums the z-interfaces inside the chunk itself.
enum { MODE_CELLS = 0, MODE_BRICK = 1, MODE_PACKED = 2, MODE_BRICKZ = 3 };
// 2^3-packed storage units (Sec. 2.2): 8 cells per unit, whole units per CTA
template <int N>
struct Packed {
  static constexpr int P = N - 1, NU = 2 * N - 1, NU3 = NU * NU * NU;
  static constexpr int UPB = Cfg<N>::CPB / 8;  // units per CTA
};

// Cell of tile slot cl.  MODE_CELLS: cells cell0 + cl (below ncells).  MODE_BRICK: cell0 is the
// brick index over (bricks along x, bricks along y, z-layers).  MODE_PACKED: cell0 is the first
// storage unit of the CTA; slot cl is sub-cell cl % 8 (x fastest) of unit cell0 + cl / 8.
template <int N, int MODE, class A>
__device__ __forceinline__ CellPos cell_pos(const A& a, long long cell0, int cl) {
  CellPos c;
  if constexpr (MODE == MODE_PACKED) {
    const int ux_n = a.mx / 2, uy_n = a.my / 2;
    const long long u = cell0 + cl / 8;
    const int sub = cl % 8;
    c.cx = (int)(u % ux_n) * 2 + (sub & 1);
    c.cy = (int)((u / ux_n) % uy_n) * 2 + ((sub >> 1) & 1);
    c.cz = (int)(u / ((long long)ux_n * uy_n)) * 2 + ((sub >> 2) & 1);
    c.active = cl / 8 < Packed<N>::UPB && u < a.ncells / 8;
    c.cell = ((long long)c.cz * a.my + c.cy) * a.mx + c.cx;
  } else if constexpr (MODE == MODE_BRICK || MODE == MODE_BRICKZ) {  // brick index < 2^31
    constexpr int BX = Brick<N>::BX, BY = Brick<N>::BY;
    const unsigned nbx = (unsigned)(a.mx + BX - 1) / BX, nby = (unsigned)(a.my + BY - 1) / BY;
    const unsigned b = (unsigned)cell0, rb = b / nbx;
    c.cx = (int)(b - rb * nbx) * BX + cl % BX;
    c.cy = (int)(rb % nby) * BY + cl / BX;
    c.cz = (int)(rb / nby);
    c.active = cl < BX * BY && c.cx < a.mx && c.cy < a.my;
    c.cell = ((long long)c.cz * a.my + c.cy) * a.mx + c.cx;
  } else {  // cell coordinates only where the Dirichlet masks need them (64-bit divisions)
    c.cell = cell0 + cl;
    c.active = cl < Cfg<N>::CPB && c.cell < a.ncells;
    c.cx = c.cy = c.cz = 0;
    if (a.dirichlet && c.active) {
      c.cx = (int)(c.cell % a.mx);
      c.cy = (int)((c.cell / a.mx) % a.my);
      c.cz = (int)(c.cell / ((long long)a.mx * a.my));
    }
  }
  return c;
}

// Intra-brick interface sums on the output tile s (all threads of the CTA call it).  x-faces:
// (slot, i = n-1) + (slot+1, i = 0) at (j, k) = (la, lb); y-faces: (slot, j = n-1) +
// (slot+BX, j = 0) at (i, k) = (la, lb).
template <int N, class V, class A>
__device__ __forceinline__ void brick_sums(const Sm<V>& s, int cb, int cl, int la, int lb,
                                           const A& a, long long cell0) {
  using C = Cfg<N>;
  constexpr int BX = Brick<N>::BX, BY = Brick<N>::BY;
  const int dx = cl % BX, dy = cl / BX;
  const int mx = a.mx, my = a.my;
  const CellPos c = cell_pos<N, MODE_BRICK>(a, cell0, cl);  // recomputed: nothing held across sweeps
  if (c.active && dx < BX - 1 && c.cx + 1 < mx) {
    const int eL = cb + lb * C::PS + la * C::RS + (N - 1);
    const int eR = cb + C::CS + lb * C::PS + la * C::RS;
    const V v = NT<V>::add(s.get(eL), s.get(eR));
    s.put(eL, v);
    s.put(eR, v);
  }
  __syncthreads();
  if (c.active && dy < BY - 1 && c.cy + 1 < my) {
    const int eL = cb + lb * C::PS + (N - 1) * C::RS + la;
    const int eR = cb + BX * C::CS + lb * C::PS + la;
    const V v = NT<V>::add(s.get(eL), s.get(eR));
    s.put(eL, v);
    s.put(eR, v);
  }
  __syncthreads();
}

// ---------------------------------------------------------------------------------------------
// High degrees: the same sweeps with the output index of every 1D contraction as a run-time loop.
// Fully unrolled n x n contractions in double-word arithmetic outgrow the instruction cache from
// n ~ 6 on (the unrolled kernel then waits on instruction fetch); here each sweep is one unrolled
// n-term dot product per output, the coefficients come from the constant bank with a
// warp-uniform index, and every output goes straight to the shared-memory tile.
// ---------------------------------------------------------------------------------------------
#ifndef FE_PREFETCH_MASS_MAXN  // mass: fetch w detJ of the z-line at the start up to this n
#define FE_PREFETCH_MASS_MAXN 6
#endif
#ifndef FE_ROLL_MINN
#define FE_ROLL_MINN 5
#endif
// single-float arithmetics (FP32, 16-bit operands) stay unrolled at every degree: a float
// contraction is a fraction of the double-word one, the unrolled kernels fit the instruction cache,
// and they ran faster (FP32 Laplace at 32^3 Q7 0.113 against 0.138 ms, 48^3 Q5 0.171 against 0.210)
#ifndef FE_ROLL_MINN_F32
#define FE_ROLL_MINN_F32 9
#endif
template <class V>
__host__ __device__ constexpr int roll_minn() {
  return (std::is_same<V, dw>::value || std::is_same<V, double>::value) ? FE_ROLL_MINN
                                                                         : FE_ROLL_MINN_F32;
}

// s[base + q * stride] = (M in)_q, R output pairs per loop iteration
template <int N, class V, int SIG, int R>
__device__ __forceinline__ void sweep_rolled(const EO<N, V>& M, const V (&in)[N], const Sm<V>& s,
                                             int base, int stride) {
  eo_line<N, V, SIG, R>(M, in, [&](int q, V v) { s.put(base + q * stride, v); });
}

// Output pairs per loop iteration of the run-time contraction loops (measured, double-word, GB300):
// all of them (the loop unrolled) except the Laplace kernels at n = 6 and 8, where the unrolled
// loops ran 7.5% slower (n = 6) and no faster (n = 8: equal at 32^3 cells, 10% slower at 16^3);
// unrolled, the mass kernels gain 5-16% at n = 5..8 and the Laplace kernels 6% at n = 5 and 7.
template <int N, int OP>
__host__ __device__ constexpr int roll_unroll() {
  return (OP == FE_LAPLACE && (N == 6 || N == 8)) ? 1 : N / 2;
}

// Arrays of the shared-memory tile: Laplace 3 (the FP64 path a fourth for the binary64 inputs
// that are differenced), mass 1.
template <class V>
__host__ __device__ constexpr int apply_narr(int op) {
  return op == FE_LAPLACE ? (std::is_same<V, dw>::value ? 4 : 3) : 1;
}

template <int N, class V, int OP, int GEOM, int MODE>
__device__ __forceinline__ void apply_cells_rolled(const CellArgs<N, V>& a, const Tab1D<N, V>& tab,
                                                   long long cell0, unsigned char* smraw,
                                                   int tile_stride) {
  constexpr int RU = roll_unroll<N, OP>();
  using T = NT<V>;
  using C = Cfg<N>;
  constexpr int N2 = C::N2, N3 = C::N3, RS = C::RS, PS = C::PS;
  constexpr int NARR = (OP == FE_LAPLACE) ? 3 : 1;
  const Sm<V> s0(smraw, NARR, 0, tile_stride);
  const Sm<V> s1(smraw, NARR, NARR > 1 ? 1 : 0, tile_stride);
  const Sm<V> s2(smraw, NARR, NARR > 2 ? 2 : 0, tile_stride);

  const int t = threadIdx.x;
  const int cl = t / N2;
  const int lt = t - cl * N2;
  const int la = lt % N, lb = lt / N;
  const int cb = cl * C::CS;
  const CellPos pos = cell_pos<N, MODE>(a, cell0, cl);
  const long long cell = pos.cell;
  const bool active = pos.active;
  const long long gbase = cell * N3;
  // line starts in the tile: x-line (j=la, k=lb), y-line (i=la, k=lb), z-line (i=la, j=lb)
  const int bx = cb + lb * PS + la * RS, by = cb + lb * PS + la, bz = cb + lb * RS + la;

  bool bnd_line = false, bnd_k0 = false, bnd_k1 = false;
  if (a.dirichlet && active) {
    const int cx = pos.cx, cy = pos.cy, cz = pos.cz;
    bnd_line = (cx == 0 && la == 0) || (cx == a.mx - 1 && la == N - 1) || (cy == 0 && lb == 0) ||
               (cy == a.my - 1 && lb == N - 1);
    bnd_k0 = (a.dirichlet & FE_DIR_ZLO) && cz == 0;
    bnd_k1 = (a.dirichlet & FE_DIR_ZHI) && cz == a.mz - 1;
  }
  auto masked = [&](int k) { return bnd_line || (k == 0 && bnd_k0) || (k == N - 1 && bnd_k1); };
  auto load_line = [&](const Sm<V>& s, int base, int stride, V (&v)[N]) {
#pragma unroll
    for (int r = 0; r < N; ++r) v[r] = s.get(base + r * stride);
  };

  // FP64 path: binary64 inputs until they are differenced, CTA exponent shift (as apply_cells)
  constexpr bool DW = std::is_same<V, dw>::value;
  // FP64 path: Laplace gradient from differences of the binary64 inputs (diff_gradient)
  constexpr bool DIFF = DW && OP == FE_LAPLACE;
  using SV = typename NT<V>::SV;
  int sh = 0;
  V in[N];
  SV xr[(DW || DIFF) ? N : 1];
  if constexpr (DW || DIFF) {
#pragma unroll
    for (int k = 0; k < N; ++k) {
      const SV v = active ? __ldcs(a.x + gbase + k * N2 + lt) : SV(0);
      xr[k] = masked(k) ? SV(0) : v;
    }
  } else {
#pragma unroll
    for (int k = 0; k < N; ++k) {
      V v = active ? T::load_stream(a.x + gbase + k * N2 + lt) : T::zero();
      in[k] = masked(k) ? T::zero() : v;
    }
  }
  constexpr bool PREF_M = (OP == FE_MASS) && (GEOM == GEOM_STORED_K) && (N <= FE_PREFETCH_MASS_MAXN);
  V jpre[PREF_M ? N : 1];
  if constexpr (PREF_M) {
    const typename NT<V>::GV* g6 =
        a.geo + (size_t)(cell - a.geo_cell0) * (FE_GEO_COMPS * N3) + 6 * N3 + lt;
#pragma unroll
    for (int k = 0; k < N; ++k) jpre[k] = active ? T::geo(g6 + k * N2) : T::zero();
  }
  if constexpr (DIFF) {
    diff_gradient<N, V, RU>(xr, Sm<SV>(smraw, 4, 3, tile_stride), s0, s1, s2, cb, la, lb, tab, sh);
  } else {
    if constexpr (DW) {
      sh = cta_exp_shift<N>(xr);
#pragma unroll
      for (int k = 0; k < N; ++k) in[k] = dw_from_double_ftz(xr[k], sh);
    }
    sweep_rolled<N, V, 1, RU>(tab.eV, in, s0, bz, PS);  // z
    __syncthreads();
    load_line(s0, bx, 1, in);
    sweep_rolled<N, V, 1, RU>(tab.eV, in, s0, bx, 1);  // x
    __syncthreads();
    load_line(s0, by, RS, in);
    sweep_rolled<N, V, 1, RU>(tab.eV, in, s0, by, RS);  // y
    __syncthreads();
    if constexpr (OP == FE_LAPLACE) {
      V inz[N];
      load_line(s0, bz, PS, inz);
      load_line(s0, bx, 1, in);
      sweep_rolled<N, V, -1, RU>(tab.eD, in, s1, bx, 1);  // d/dx -> s1
      load_line(s0, by, RS, in);
      sweep_rolled<N, V, -1, RU>(tab.eD, in, s2, by, RS);  // d/dy -> s2
      __syncthreads();
      sweep_rolled<N, V, -1, RU>(tab.eD, inz, s0, bz, PS);  // d/dz -> s0 (own z-line)
    }
  }

  if constexpr (OP == FE_LAPLACE) {
    // pointwise metric on the own z-line: g = G grad u
    const typename NT<V>::GV* gp = a.geo + (size_t)(cell - a.geo_cell0) * (FE_GEO_COMPS * N3) + lt;
#pragma unroll
    for (int k = 0; k < N; ++k) {
      const int e = bz + k * PS;
      const V dx = s1.get(e), dy = s2.get(e), dz = s0.get(e);
      V gxx, gyy, gzz, gxy, gxz, gyz;
      if constexpr (GEOM == GEOM_AFFINE_K) {
        const V wq = T::mul(T::mul(tab.W_[la], tab.W_[lb]), tab.W_[k]);
        s1.put(e, T::mul(T::mul(wq, a.aff[0]), dx));
        s2.put(e, T::mul(T::mul(wq, a.aff[1]), dy));
        s0.put(e, T::mul(T::mul(wq, a.aff[2]), dz));
      } else {
        if (active) {
          gxx = T::geo(gp + 0 * N3 + k * N2);
          gyy = T::geo(gp + 1 * N3 + k * N2);
          gzz = T::geo(gp + 2 * N3 + k * N2);
          gxy = T::geo(gp + 3 * N3 + k * N2);
          gxz = T::geo(gp + 4 * N3 + k * N2);
          gyz = T::geo(gp + 5 * N3 + k * N2);
        } else {
          gxx = gyy = gzz = gxy = gxz = gyz = T::zero();
        }
        const V gx = T::keep(T::mac(T::mac(T::prod(gxx, dx), gxy, dy), gxz, dz));
        const V gy = T::keep(T::mac(T::mac(T::prod(gxy, dx), gyy, dy), gyz, dz));
        const V gz = T::keep(T::mac(T::mac(T::prod(gxz, dx), gyz, dy), gzz, dz));
        s1.put(e, gx);
        s2.put(e, gy);
        s0.put(e, gz);
      }
    }
    __syncthreads();
    // transposed derivatives, each in place on its own array
    load_line(s1, bx, 1, in);
    sweep_rolled<N, V, -1, RU>(tab.eDT, in, s1, bx, 1);
    load_line(s2, by, RS, in);
    sweep_rolled<N, V, -1, RU>(tab.eDT, in, s2, by, RS);
    load_line(s0, bz, PS, in);
    sweep_rolled<N, V, -1, RU>(tab.eDT, in, s0, bz, PS);
    __syncthreads();
#pragma unroll
    for (int k = 0; k < N; ++k) {
      const int e = bz + k * PS;
      in[k] = T::add(T::add(s0.get(e), s1.get(e)), s2.get(e));
    }
  } else {
#pragma unroll
    for (int k = 0; k < N; ++k) {
      const V uq = s0.get(bz + k * PS);
      V jw;
      if constexpr (GEOM == GEOM_AFFINE_K) {
        jw = T::mul(T::mul(T::mul(tab.W_[la], tab.W_[lb]), tab.W_[k]), a.aff[3]);
      } else if constexpr (PREF_M) {
        jw = jpre[k];
      } else {
        jw = active ? T::geo(a.geo + (size_t)(cell - a.geo_cell0) * (FE_GEO_COMPS * N3) + 6 * N3 +
                             k * N2 + lt)
                    : T::zero();
      }
      in[k] = T::mul(jw, uq);
    }
  }

  // transposed interpolation: z from registers, then x and y in place
  sweep_rolled<N, V, 1, RU>(tab.eVT, in, s0, bz, PS);
  __syncthreads();
  load_line(s0, bx, 1, in);
  sweep_rolled<N, V, 1, RU>(tab.eVT, in, s0, bx, 1);
  __syncthreads();
  load_line(s0, by, RS, in);
  sweep_rolled<N, V, 1, RU>(tab.eVT, in, s0, by, RS);
  __syncthreads();
  if constexpr (MODE == MODE_BRICK) brick_sums<N, V>(s0, cb, cl, la, lb, a, cell0);
  if (active) {
#pragma unroll
    for (int k = 0; k < N; ++k) {
      V v = s0.get(bz + k * PS);
      if (masked(k)) v = T::zero();
      if constexpr (T::LOWP) v.v *= a.oscale;
      T::store(a.y + gbase + k * N2 + lt, v, sh);
    }
  }
}

// The cells cell0 .. cell0 + CPB - 1 (those below ncells), applied by the CTA's first CPB*n^2
// threads.  Threads beyond that (a CTA wider than the tile, as in the batched persistent kernel)
// work on a spare slot of the tile that nobody reads and still reach every barrier; the caller
// then sizes each array tile_stride = TILE + CS.
template <int N, class V, int OP, int GEOM, int MODE = MODE_CELLS>
__device__ __forceinline__ void apply_cells(const CellArgs<N, V>& a, const Tab1D<N, V>& tab,
                                            long long cell0, unsigned char* smraw,
                                            int tile_stride,
                                            ZCarry<typename NT<V>::SV>* zc = nullptr) {
  static_assert(MODE != MODE_PACKED || N < FE_ROLL_MINN, "packed units: unrolled degrees only");
  static_assert(MODE != MODE_BRICKZ || (N < FE_ROLL_MINN && !NT<V>::LOWP),
                "z-carry bricks: unrolled degrees, FP64 / double-word / FP32 values");
  if constexpr (N >= roll_minn<V>() && MODE != MODE_PACKED) {
    apply_cells_rolled<N, V, OP, GEOM, MODE>(a, tab, cell0, smraw, tile_stride);
    return;
  }
  using T = NT<V>;
  using C = Cfg<N>;
  constexpr int N2 = C::N2, N3 = C::N3;
  constexpr int NARR = (OP == FE_LAPLACE) ? 3 : 1;
  const Sm<V> s0(smraw, NARR, 0, tile_stride);
  const Sm<V> s1(smraw, NARR, NARR > 1 ? 1 : 0, tile_stride);
  const Sm<V> s2(smraw, NARR, NARR > 2 ? 2 : 0, tile_stride);

  const int t = threadIdx.x;
  const int cl = t / N2;
  const int lt = t - cl * N2;
  const int la = lt % N, lb = lt / N;  // line coordinates (a, b) of this thread
  const int cb = cl * C::CS;           // this cell's offset in the tile
  const CellPos pos = cell_pos<N, MODE>(a, cell0, cl);
  const long long cell = pos.cell;
  const bool active = pos.active;
  const long long gbase = cell * N3;

  // Dirichlet masks of this thread's z-line (i = la, j = lb)
  bool bnd_line = false;  // the whole z-line lies on the x- or y-boundary
  bool bnd_k0 = false, bnd_k1 = false;
  if (a.dirichlet && active) {
    const int cx = pos.cx, cy = pos.cy, cz = pos.cz;
    bnd_line = (cx == 0 && la == 0) || (cx == a.mx - 1 && la == N - 1) || (cy == 0 && lb == 0) ||
               (cy == a.my - 1 && lb == N - 1);
    bnd_k0 = (a.dirichlet & FE_DIR_ZLO) && cz == 0;
    bnd_k1 = (a.dirichlet & FE_DIR_ZHI) && cz == a.mz - 1;
  }
  auto masked = [&](int k) { return bnd_line || (k == 0 && bnd_k0) || (k == N - 1 && bnd_k1); };

  // ---- load x (z-line owner, coalesced) and interpolate along z in registers
  // (packed: the sub-cell's z-line inside its storage unit of (2n-1)^3 nodes)
  auto xaddr = [&](int k) -> long long {
    if constexpr (MODE == MODE_PACKED) {
      constexpr int P = Packed<N>::P, NU = Packed<N>::NU;
      const int sub = cl % 8;
      return (cell0 + cl / 8) * Packed<N>::NU3 +
             ((long long)(((sub >> 2) & 1) * P + k) * NU + ((sub >> 1) & 1) * P + lb) * NU +
             (sub & 1) * P + la;
    } else {
      return gbase + k * N2 + lt;
    }
  };
  // FP64 path (double-word values): the inputs stay binary64 until they are differenced, and the
  // CTA's values are scaled by a power of two (cta_exp_shift)
  constexpr bool DW = std::is_same<V, dw>::value;
  // FP64 path: Laplace gradient from differences of the binary64 inputs (diff_gradient)
  constexpr bool DIFF = DW && OP == FE_LAPLACE;
  using SV = typename NT<V>::SV;
  int sh = 0;
  V u[N], w[N];
  SV xr[(DW || DIFF) ? N : 1];
  if constexpr (DW || DIFF) {
#pragma unroll
    for (int k = 0; k < N; ++k) {
      const SV v = active ? __ldcs(a.x + xaddr(k)) : SV(0);
      xr[k] = masked(k) ? SV(0) : v;
    }
  } else {
#pragma unroll
    for (int k = 0; k < N; ++k) {
      V v = active ? T::load_stream(a.x + xaddr(k)) : T::zero();
      u[k] = masked(k) ? T::zero() : v;
    }
  }
  // low degrees: issue the metric loads now so that their latency hides behind the sweeps
#ifndef FE_PREFETCH_MAXN
#define FE_PREFETCH_MAXN 4
#endif
  constexpr bool PREF = (OP == FE_LAPLACE) && (GEOM == GEOM_STORED_K) && (N <= FE_PREFETCH_MAXN);
  V gpre[PREF ? 6 * N : 1];
  // mass: the N values of w detJ on the z-line are always fetched up front
  constexpr bool PREF_M = (OP == FE_MASS) && (GEOM == GEOM_STORED_K) && (N <= FE_PREFETCH_MASS_MAXN);
  V jpre[PREF_M ? N : 1];
  if constexpr (PREF_M) {
    const typename NT<V>::GV* g6 =
        a.geo + (size_t)(cell - a.geo_cell0) * (FE_GEO_COMPS * N3) + 6 * N3 + lt;
#pragma unroll
    for (int k = 0; k < N; ++k) jpre[k] = active ? T::geo(g6 + k * N2) : T::zero();
  }
  if constexpr (PREF) {
    const typename NT<V>::GV* g0 = a.geo + (size_t)(cell - a.geo_cell0) * (FE_GEO_COMPS * N3) + lt;
#pragma unroll
    for (int k = 0; k < N; ++k)
#pragma unroll
      for (int c = 0; c < 6; ++c) gpre[c * N + k] = active ? T::geo(g0 + c * N3 + k * N2) : T::zero();
  }
  if constexpr (DIFF) {
    diff_gradient<N, V, 0>(xr, Sm<SV>(smraw, 4, 3, tile_stride), s0, s1, s2, cb, la, lb, tab, sh);
    // s1, s2, s0: d/dx, d/dy, d/dz of u at the Gauss points
#pragma unroll
    for (int k = 0; k < N; ++k) u[k] = s0.get(cb + zl<N>(la, lb, k));
  } else {
    if constexpr (DW) {
      sh = cta_exp_shift<N>(xr);
#pragma unroll
      for (int k = 0; k < N; ++k) u[k] = dw_from_double_ftz(xr[k], sh);
    }
    eo_regs<N, V, 1>(tab.eV, u, w);
#pragma unroll
    for (int k = 0; k < N; ++k) s0.put(cb + zl<N>(la, lb, k), w[k]);
    __syncthreads();
    tile_sweep<N, V, 0, 1>(s0, cb, la, lb, tab.eV);  // x
    __syncthreads();
    tile_sweep<N, V, 1, 1>(s0, cb, la, lb, tab.eV);  // y
    __syncthreads();
    // s0 now holds u at the Gauss points
    if constexpr (OP == FE_LAPLACE) {
      // ---- reference gradient at the Gauss points (collocation derivative)
      V in[N], out[N];
#pragma unroll
      for (int r = 0; r < N; ++r) in[r] = s0.get(cb + xl<N>(la, lb, r));
      eo_regs<N, V, -1>(tab.eD, in, out);
#pragma unroll
      for (int r = 0; r < N; ++r) s1.put(cb + xl<N>(la, lb, r), out[r]);
#pragma unroll
      for (int r = 0; r < N; ++r) in[r] = s0.get(cb + yl<N>(la, lb, r));
      eo_regs<N, V, -1>(tab.eD, in, out);
#pragma unroll
      for (int r = 0; r < N; ++r) s2.put(cb + yl<N>(la, lb, r), out[r]);
#pragma unroll
      for (int r = 0; r < N; ++r) in[r] = s0.get(cb + zl<N>(la, lb, r));
      eo_regs<N, V, -1>(tab.eD, in, u);  // u := d/dz along the z-line
      __syncthreads();
    }
  }

  if constexpr (OP == FE_LAPLACE) {
    // ---- pointwise metric: g = G grad u (z-line owner)
#pragma unroll
    for (int k = 0; k < N; ++k) {
      const int e = cb + zl<N>(la, lb, k);
      const V dx = s1.get(e), dy = s2.get(e), dz = u[k];
      V gxx, gyy, gzz, gxy, gxz, gyz;
      if constexpr (GEOM == GEOM_AFFINE_K) {
        const int q1 = la, q2 = lb;
        const V wq = T::mul(T::mul(tab.W_[q1], tab.W_[q2]), tab.W_[k]);
        gxx = T::mul(wq, a.aff[0]);
        gyy = T::mul(wq, a.aff[1]);
        gzz = T::mul(wq, a.aff[2]);
        V gx = T::mul(gxx, dx), gy = T::mul(gyy, dy), gz = T::mul(gzz, dz);
        s1.put(e, gx);
        s2.put(e, gy);
        u[k] = gz;
      } else {
        if constexpr (PREF) {
          gxx = gpre[0 * N + k];
          gyy = gpre[1 * N + k];
          gzz = gpre[2 * N + k];
          gxy = gpre[3 * N + k];
          gxz = gpre[4 * N + k];
          gyz = gpre[5 * N + k];
        } else {
          const typename NT<V>::GV* gp =
              a.geo + (size_t)(cell - a.geo_cell0) * (FE_GEO_COMPS * N3) + k * N2 + lt;
          if (active) {
            gxx = T::geo(gp + 0 * N3);
            gyy = T::geo(gp + 1 * N3);
            gzz = T::geo(gp + 2 * N3);
            gxy = T::geo(gp + 3 * N3);
            gxz = T::geo(gp + 4 * N3);
            gyz = T::geo(gp + 5 * N3);
          } else {
            gxx = gyy = gzz = gxy = gxz = gyz = T::zero();
          }
        }
        const V gx = T::keep(T::mac(T::mac(T::prod(gxx, dx), gxy, dy), gxz, dz));
        const V gy = T::keep(T::mac(T::mac(T::prod(gxy, dx), gyy, dy), gyz, dz));
        const V gz = T::keep(T::mac(T::mac(T::prod(gxz, dx), gyz, dy), gzz, dz));
        s1.put(e, gx);
        s2.put(e, gy);
        u[k] = gz;
      }
    }
    __syncthreads();
    // ---- transposed derivative: t = D^T gx (x) + D^T gy (y) + D^T gz (z)
    tile_sweep<N, V, 0, -1>(s1, cb, la, lb, tab.eDT);
    tile_sweep<N, V, 1, -1>(s2, cb, la, lb, tab.eDT);
    eo_regs<N, V, -1>(tab.eDT, u, w);
    __syncthreads();
#pragma unroll
    for (int k = 0; k < N; ++k) {
      const int e = cb + zl<N>(la, lb, k);
      u[k] = T::add(T::add(w[k], s1.get(e)), s2.get(e));
    }
  } else {
    // ---- mass: pointwise w detJ
#pragma unroll
    for (int k = 0; k < N; ++k) {
      const V uq = s0.get(cb + zl<N>(la, lb, k));
      V jw;
      if constexpr (GEOM == GEOM_AFFINE_K) {
        jw = T::mul(T::mul(T::mul(tab.W_[la], tab.W_[lb]), tab.W_[k]), a.aff[3]);
      } else if constexpr (PREF_M) {
        jw = jpre[k];
      } else {
        jw = active ? T::geo(a.geo + (size_t)(cell - a.geo_cell0) * (FE_GEO_COMPS * N3) + 6 * N3 +
                             k * N2 + lt)
                    : T::zero();
      }
      u[k] = T::mul(jw, uq);
    }
  }

  // ---- transposed interpolation: z in registers, then x and y in the tile
  eo_regs<N, V, 1>(tab.eVT, u, w);
#pragma unroll
  for (int k = 0; k < N; ++k) s0.put(cb + zl<N>(la, lb, k), w[k]);
  __syncthreads();
  tile_sweep<N, V, 0, 1>(s0, cb, la, lb, tab.eVT);
  __syncthreads();
  tile_sweep<N, V, 1, 1>(s0, cb, la, lb, tab.eVT);
  __syncthreads();
  if constexpr (MODE == MODE_BRICK || MODE == MODE_BRICKZ) brick_sums<N, V>(s0, cb, cl, la, lb, a, cell0);
  if constexpr (MODE == MODE_BRICKZ) {
    // The z-interface with the previous layer of the chunk: the structured DSS's z-pass pair sum
    // (lower + upper copy), formed on the stored values, so the result is that of the pass.
    // The x/y sums inside the brick came first, as they do before the pass.
    if (active) {
      using SV = typename NT<V>::SV;
      SV bottom = T::to_sv(masked(0) ? T::zero() : s0.get(cb + zl<N>(la, lb, 0)), sh);
      if (zc->pending) {
        bottom = zc->top + bottom;
        T::store_sv(a.y + gbase - (long long)a.mx * a.my * N3 + (N - 1) * N2 + lt, bottom);
      }
      T::store_sv(a.y + gbase + lt, bottom);
#pragma unroll
      for (int k = 1; k < N - 1; ++k) {
        V v = s0.get(cb + zl<N>(la, lb, k));
        if (masked(k)) v = T::zero();
        T::store(a.y + gbase + k * N2 + lt, v, sh);
      }
      const SV top = T::to_sv(masked(N - 1) ? T::zero() : s0.get(cb + zl<N>(la, lb, N - 1)), sh);
      if (zc->last) {
        T::store_sv(a.y + gbase + (N - 1) * N2 + lt, top);
        zc->pending = false;
      } else {
        zc->top = top;
        zc->pending = true;
      }
    }
    return;
  }
  if constexpr (MODE == MODE_PACKED) {
    // unit-internal assembly: sum the copies on the x-, y- and z-interfaces between the unit's
    // sub-cells in the tile (as the structured DSS passes do, z then y then x), then every stored
    // node is written once, by the sub-cell with the lowest index along each axis that holds it
    constexpr int P = Packed<N>::P, NU = Packed<N>::NU;
    const int sub = cl % 8, sx = sub & 1, sy = (sub >> 1) & 1, sz = (sub >> 2) & 1;
    auto pair_sum = [&](int eL, int eR) {
      const V v = T::add(s0.get(eL), s0.get(eR));
      s0.put(eL, v);
      s0.put(eR, v);
    };
    if (active && sz == 0)  // z-interface: (k = P of sz 0) + (k = 0 of sz 1), thread (i, j)
      pair_sum(cb + zl<N>(la, lb, P), cb + 4 * C::CS + zl<N>(la, lb, 0));
    __syncthreads();
    if (active && sy == 0)  // y-interface, thread (i, k) = (la, lb)
      pair_sum(cb + zl<N>(la, P, lb), cb + 2 * C::CS + zl<N>(la, 0, lb));
    __syncthreads();
    if (active && sx == 0)  // x-interface, thread (j, k) = (la, lb)
      pair_sum(cb + zl<N>(P, la, lb), cb + 1 * C::CS + zl<N>(0, la, lb));
    __syncthreads();
    if (active && (sx == 0 || la > 0) && (sy == 0 || lb > 0)) {
      typename NT<V>::SV* yu = a.y + (cell0 + cl / 8) * Packed<N>::NU3 +
                               (long long)(sy * P + lb) * NU + sx * P + la;
#pragma unroll
      for (int k = 0; k < N; ++k) {
        if (sz == 1 && k == 0) continue;
        V v = s0.get(cb + zl<N>(la, lb, k));
        if (masked(k)) v = T::zero();
        if constexpr (T::LOWP) v.v *= a.oscale;
        T::store(yu + (long long)(sz * P + k) * NU * NU, v, sh);
      }
    }
    return;
  }
  if (active) {
#pragma unroll
    for (int k = 0; k < N; ++k) {
      V v = s0.get(cb + zl<N>(la, lb, k));
      if (masked(k)) v = T::zero();
      if constexpr (T::LOWP) v.v *= a.oscale;
      T::store(a.y + gbase + k * N2 + lt, v, sh);
    }
  }
}

// Resident CTAs per SM the one-layer kernels are compiled for: the double-word kernels are held
// to the register budget of 3 (Laplace, unrolled degrees: 80 registers; n = 3: 4), 4 (Laplace,
// rolled: 64; n = 7: 3, n = 8: 5) or 6 (mass: 40; up to n = 4: 8, n = 6: 5) CTAs per SM; the rest
// are left to the compiler.
// n = 3 double-word Laplace: 4 CTAs per SM (64 registers, no spills); its kernel waits on shared
// memory rather than on issue, and the extra CTA took Q2 48^3 from 0.0887 to 0.0846 ms (assembled
// 0.1184 to 0.1133 ms)
#ifndef FE_DW_LAPLACE_MINB_N3
#define FE_DW_LAPLACE_MINB_N3 4
#endif
// n = 8 double-word Laplace: 5 CTAs per SM (51 registers, no spills): Q7 32^3 0.621 -> 0.601 ms
#ifndef FE_DW_LAPLACE_MINB_N8
#define FE_DW_LAPLACE_MINB_N8 5
#endif
// n = 7 Laplace at 3 CTAs per SM and n = 6 mass at 5: the budgets of 4 and 6 spilled (100 and 16
// bytes); Q6 32^3 Laplace 0.443 -> 0.437 ms, Q5 40^3 mass 0.171 -> 0.168 ms
#ifndef FE_DW_LAPLACE_MINB_N7
#define FE_DW_LAPLACE_MINB_N7 3
#endif
#ifndef FE_DW_MASS_MINB_N6
#define FE_DW_MASS_MINB_N6 5
#endif
// double-word mass up to n = 4: 8 CTAs per SM (32 registers): Q3 96^3 0.580 -> 0.566 ms, Q2 48^3
// assembled 0.0641 -> 0.0611 ms; from n = 5 on 32 registers spill, and 6 CTAs stay
#ifndef FE_DW_MASS_MINB_LOW
#define FE_DW_MASS_MINB_LOW 8
#endif
template <int N, class V, int OP>
__host__ __device__ constexpr int apply_minb() {
  return std::is_same<V, dw>::value
             ? (OP == FE_LAPLACE
                    ? (N == 3 ? FE_DW_LAPLACE_MINB_N3
                              : (N < FE_ROLL_MINN ? 3
                                                  : (N == 8 ? FE_DW_LAPLACE_MINB_N8
                                                            : (N == 7 ? FE_DW_LAPLACE_MINB_N7 : 4))))
                    : (N <= 4 ? FE_DW_MASS_MINB_LOW : (N == 6 ? FE_DW_MASS_MINB_N6 : 6)))
             : 1;
}
#ifdef FE_MINB
#define FE_APPLY_BOUNDS __launch_bounds__(Cfg<N>::THREADS, FE_MINB)
#else
#define FE_APPLY_BOUNDS __launch_bounds__(Cfg<N>::THREADS, (apply_minb<N, V, OP>()))
#endif
// z-carry bricks: held to a register budget for 3 CTAs per SM (Laplace, as the one-layer brick
// kernel; left to itself the compiler gives the layer loop 98 registers, 2 CTAs per SM) or 6
// (mass, whose one-layer kernel needs 32 registers)
#ifndef FE_ZCARRY_MINB_LAPLACE
#define FE_ZCARRY_MINB_LAPLACE 3
#endif
#ifndef FE_ZCARRY_MINB_MASS
#define FE_ZCARRY_MINB_MASS 6
#endif
template <int N, class V, int OP, int GEOM, int MODE>
__global__ void FE_APPLY_BOUNDS k_apply(const __grid_constant__ ApplyArgs<N, V> a) {
  extern __shared__ __align__(16) unsigned char smraw[];
  if (a.skip && *(volatile const int*)a.skip) return;  // uniform over the grid
  long long cell0;
  if constexpr (MODE == MODE_BRICK)
    cell0 = (long long)blockIdx.x;
  else if constexpr (MODE == MODE_PACKED)
    cell0 = (long long)blockIdx.x * Packed<N>::UPB;
  else
    cell0 = a.c.cell_base + (long long)blockIdx.x * Cfg<N>::CPB;
  apply_cells<N, V, OP, GEOM, MODE>(a.c, a.tab, cell0, smraw, Cfg<N>::TILE);
}

// MODE_BRICKZ: blockIdx.x = chunk * (bricks per layer) + brick column; the CTA applies the layers
// [z0, z1) of its column one after the other
template <int N, class V, int OP, int GEOM>
__global__ void __launch_bounds__(Cfg<N>::THREADS,
                                  OP == FE_LAPLACE ? FE_ZCARRY_MINB_LAPLACE : FE_ZCARRY_MINB_MASS)
    k_apply_zcarry(const __grid_constant__ ApplyArgs<N, V> a) {
  extern __shared__ __align__(16) unsigned char smraw[];
  if (a.skip && *(volatile const int*)a.skip) return;  // uniform over the grid
  constexpr int BX = Brick<N>::BX, BY = Brick<N>::BY;
  const unsigned per_layer =
      (unsigned)((a.c.mx + BX - 1) / BX) * (unsigned)((a.c.my + BY - 1) / BY);
  const unsigned col = blockIdx.x % per_layer, chunk = blockIdx.x / per_layer;
  const int z0 = (int)chunk * a.zchunk;
  const int z1 = z0 + a.zchunk < a.c.mz ? z0 + a.zchunk : a.c.mz;
  ZCarry<typename NT<V>::SV> zc;
  zc.pending = false;
  for (int cz = z0; cz < z1; ++cz) {
    zc.last = cz == z1 - 1;
    apply_cells<N, V, OP, GEOM, MODE_BRICKZ>(a.c, a.tab, (long long)cz * per_layer + col, smraw,
                                             Cfg<N>::TILE, &zc);
    __syncthreads();  // the next layer refills the tile
  }
}

template <int N, class V>
inline size_t apply_smem_bytes(int op) {
  return (size_t)apply_narr<V>(op) * Cfg<N>::TILE * Sm<V>::BYTES;
}
