// fe_recompute.cuh -- metric terms formed on the fly from cell-wise nodal coordinates
// (FE_GEOM_RECOMPUTE).
//
// Sec. 2.3 defines the isoparametric map of a cell through its GLL-node coordinates; the
// Laplace apply needs G = w detJ J^-1 J^-T and the mass apply w detJ at every Gauss point.
// In the recompute mode only the coordinates are kept in HBM (3 values per cell node).  The apply
// walks the mesh in chunks of cells sized to stay in L2: k_recompute forms the metric of one
// chunk into a scratch buffer and the stored-metric apply consumes it right away, so HBM carries
// the coordinates instead of the metric.
//
// The coordinates are stored as offsets from the cell's first node: the derivative sums then
// work on values of the size of the cell rather than of the domain, and do not cancel.
// Thread mapping: one thread per node (then per Gauss point) of a cell, floor(256 / n^3) cells per
// CTA.  J is obtained as in the apply's gradient: interpolation to the Gauss points along x, y, z,
// then the Gauss-point collocation derivative along each direction.
#pragma once
#include "fe_apply_kernel.cuh"

template <int N>
struct GeoCfg {
  static constexpr int N2 = N * N, N3 = N2 * N;
  static constexpr int CPB = N3 >= 256 ? 1 : 256 / N3;
  static constexpr int THREADS = CPB * N3;
};

template <int N, class V>
struct RecomputeArgs {
  const typename NT<V>::GV* xyz;  // [cell][3][N3] offsets from the cell's first node
  typename NT<V>::GV* geo;        // [cell - cell0][7][N3]
  long long cell0, cell_end;
  const int* skip;
  Tab1D<N, V> tab;
};

__device__ __forceinline__ void geo_put(float2* p, dw v) { *p = make_float2(v.h, v.l); }
__device__ __forceinline__ void geo_put(double* p, double v) { *p = v; }
__device__ __forceinline__ void geo_put(float* p, float v) { *p = v; }

template <int N, class V>
constexpr size_t recompute_smem_bytes() {
  return (size_t)GeoCfg<N>::CPB * 6 * GeoCfg<N>::N3 * sizeof(V);
}

template <int N, class V, int OP>
__global__ void __launch_bounds__(GeoCfg<N>::THREADS)
    k_recompute(const __grid_constant__ RecomputeArgs<N, V> a) {
  using G = GeoCfg<N>;
  using T = NT<V>;
  constexpr int N2 = G::N2, N3 = G::N3;
  extern __shared__ __align__(16) unsigned char smraw[];
  if (a.skip && *(volatile const int*)a.skip) return;
  const int cl = threadIdx.x / N3, t = threadIdx.x % N3;
  const int i = t % N, j = (t / N) % N, k = t / N2;
  const long long cell = a.cell0 + (long long)blockIdx.x * G::CPB + cl;
  const bool active = cell < a.cell_end;
  V* s0 = reinterpret_cast<V*>(smraw) + (size_t)cl * 6 * N3;
  V* s1 = s0 + 3 * N3;
#pragma unroll
  for (int c = 0; c < 3; ++c)
    s0[c * N3 + t] = active ? T::geo(a.xyz + (size_t)cell * 3 * N3 + c * N3 + t) : T::zero();
  __syncthreads();
  // interpolation to the Gauss points: x (s0 -> s1), y (s1 -> s0), z (s0 -> s1)
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    V acc = T::zero();
#pragma unroll
    for (int r = 0; r < N; ++r)
      acc = T::mac12(acc, a.tab.V_[i][r], s0[c * N3 + (k * N + j) * N + r]);
    s1[c * N3 + t] = T::keep(acc);
  }
  __syncthreads();
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    V acc = T::zero();
#pragma unroll
    for (int r = 0; r < N; ++r)
      acc = T::mac12(acc, a.tab.V_[j][r], s1[c * N3 + (k * N + r) * N + i]);
    s0[c * N3 + t] = T::keep(acc);
  }
  __syncthreads();
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    V acc = T::zero();
#pragma unroll
    for (int r = 0; r < N; ++r)
      acc = T::mac12(acc, a.tab.V_[k][r], s0[c * N3 + (r * N + j) * N + i]);
    s1[c * N3 + t] = T::fin(acc);
  }
  __syncthreads();
  // J[c][b] = d x_c / d xi_b by collocation at the Gauss points
  V J[3][3];
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    V d0 = T::zero(), d1 = T::zero(), d2 = T::zero();
#pragma unroll
    for (int r = 0; r < N; ++r) {
      d0 = T::mac12(d0, a.tab.D_[i][r], s1[c * N3 + (k * N + j) * N + r]);
      d1 = T::mac12(d1, a.tab.D_[j][r], s1[c * N3 + (k * N + r) * N + i]);
      d2 = T::mac12(d2, a.tab.D_[k][r], s1[c * N3 + (r * N + j) * N + i]);
    }
    J[c][0] = T::fin(d0);
    J[c][1] = T::fin(d1);
    J[c][2] = T::fin(d2);
  }
  if (!active) return;
  auto dp = [](V p, V q, V r, V s) { return T::sub(T::mul(p, q), T::mul(r, s)); };
  // first column of the adjugate, enough for the determinant
  const V A00 = dp(J[1][1], J[2][2], J[1][2], J[2][1]);
  const V A10 = dp(J[1][2], J[2][0], J[1][0], J[2][2]);
  const V A20 = dp(J[1][0], J[2][1], J[1][1], J[2][0]);
  const V det = T::add(T::add(T::mul(J[0][0], A00), T::mul(J[0][1], A10)), T::mul(J[0][2], A20));
  const V w3 = T::mul(T::mul(a.tab.W_[i], a.tab.W_[j]), a.tab.W_[k]);
  typename NT<V>::GV* out = a.geo + (size_t)(cell - a.cell0) * (FE_GEO_COMPS * N3) + t;
  if constexpr (OP == FE_MASS) {
    geo_put(out + 6 * N3, T::mul(w3, det));
  } else {
    // G = w detJ J^-1 J^-T = (w / detJ) adj(J) adj(J)^T
    const V A01 = dp(J[0][2], J[2][1], J[0][1], J[2][2]);
    const V A11 = dp(J[0][0], J[2][2], J[0][2], J[2][0]);
    const V A21 = dp(J[0][1], J[2][0], J[0][0], J[2][1]);
    const V A02 = dp(J[0][1], J[1][2], J[0][2], J[1][1]);
    const V A12 = dp(J[0][2], J[1][0], J[0][0], J[1][2]);
    const V A22 = dp(J[0][0], J[1][1], J[0][1], J[1][0]);
    const V sc = T::mul(w3, T::recip(det));
    auto row = [&](V p0, V p1, V p2, V q0, V q1, V q2) {
      return T::mul(sc, T::add(T::add(T::mul(p0, q0), T::mul(p1, q1)), T::mul(p2, q2)));
    };
    geo_put(out + 0 * N3, row(A00, A01, A02, A00, A01, A02));
    geo_put(out + 1 * N3, row(A10, A11, A12, A10, A11, A12));
    geo_put(out + 2 * N3, row(A20, A21, A22, A20, A21, A22));
    geo_put(out + 3 * N3, row(A00, A01, A02, A10, A11, A12));
    geo_put(out + 4 * N3, row(A00, A01, A02, A20, A21, A22));
    geo_put(out + 5 * N3, row(A10, A11, A12, A20, A21, A22));
  }
}
