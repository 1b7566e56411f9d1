// fe_manufactured.cu -- manufactured right-hand side and L2 error on the device (FP64).
//
// Poisson problem -Laplace(u) = f on the unit cube, u = 0 on the boundary:
//   FE_RHS_SINE       u = sin(pi x) sin(pi y) sin(pi z),  f = 3 pi^2 u
//   FE_RHS_QUADRATIC  u = x(1-x) y(1-y) z(1-z),           f = 2 [y(1-y) z(1-z) + ...]
// Load vector (dual, unassembled): b_K,i = sum_q w_q detJ(q) f(x(xi_q)) phi_i(xi_q), the right-hand
// side b~ of Eq. (constrained_system).  L2 error: sum_K sum_q w_q detJ (u_h - u)^2 with an
// (n+2)-point Gauss rule.  One CTA per cell; coordinates, Jacobians and field values at the
// quadrature points by sum factorization in shared memory.
#include <cmath>
#include <cstring>

#include "fe_vec.cuh"

namespace {

constexpr int MAXQ = FE_MAXN + 2;

struct QTab {            // 1D tables for NQ quadrature points
  double t[FE_MAXN];     // GLL nodes on [0,1]
  double w[MAXQ];        // Gauss weights on [0,1]
  double V[MAXQ][FE_MAXN];   // l_i(s_q)
  double Dh[MAXQ][FE_MAXN];  // l_i'(s_q)
};

struct ManArgs {
  const double* u;  // l2: cell-wise solution; rhs: unused
  double* out;      // rhs: cell-wise load vector; l2: per-cell error^2
  long long ncells;
  int mx, my, mz, kind;  // mz: layers of the whole mesh (a slab's cells start at layer z0)
  int z0;
  double amp;
  QTab tab;
};

__device__ __forceinline__ double exact_u(int kind, double x, double y, double z) {
  if (kind == 0) return sinpi(x) * sinpi(y) * sinpi(z);
  return x * (1.0 - x) * y * (1.0 - y) * z * (1.0 - z);
}
__device__ __forceinline__ double exact_f(int kind, double x, double y, double z) {
  const double pi = 3.14159265358979323846;
  if (kind == 0) return 3.0 * pi * pi * sinpi(x) * sinpi(y) * sinpi(z);
  const double a = x * (1.0 - x), b = y * (1.0 - y), c = z * (1.0 - z);
  return 2.0 * (b * c + a * c + a * b);
}

// Contract a field given at the N^3 nodes (smem, [N3]) to the NQ^3 points along one axis at a
// time.  in: [n0][n1][n2] with extents (rows) given per phase.  Generic helper for one thread per
// output point.
template <int N, int NQ, bool L2>
__global__ void __launch_bounds__(NQ* NQ* NQ) k_manufactured(const __grid_constant__ ManArgs a) {
  constexpr int N2 = N * N, N3 = N2 * N;
  constexpr int Q3 = NQ * NQ * NQ;
  // stage buffers, sized for the largest phase (NQ^3 points, 4 fields: x, y, z, u)
  extern __shared__ double sm[];
  double* sX = sm;               // [4][N3]     nodal x, y, z, u
  double* sA = sm + 4 * N3;      // [4][NQ*N*N] after x-contraction (V)
  double* sB = sA + 4 * NQ * N2; // [3][NQ*N*N] after x-contraction (Dh), coordinates only
  double* sC = sB + 3 * NQ * N2; // [4][NQ*NQ*N] V x, V y
  double* sD = sC + 4 * NQ * NQ * N;  // [3][NQ*NQ*N] V x, Dh y
  double* sE = sD + 3 * NQ * NQ * N;  // [3][NQ*NQ*N] Dh x, V y
  double* red = sE + 3 * NQ * NQ * N; // [Q3] per-point contributions (l2) / g values (rhs)
  const long long cell = blockIdx.x;
  const int t = threadIdx.x;
  const int cx = (int)(cell % a.mx), cy = (int)((cell / a.mx) % a.my),
            cz = a.z0 + (int)(cell / ((long long)a.mx * a.my));
  // nodes
  if (t < N3) {
    const int i = t % N, j = (t / N) % N, k = t / N2;
    const double X0 = (cx + a.tab.t[i]) / a.mx, X1 = (cy + a.tab.t[j]) / a.my,
                 X2 = (cz + a.tab.t[k]) / a.mz;
    const double s = a.amp * sinpi(X0) * sinpi(X1) * sinpi(X2);
    sX[0 * N3 + t] = X0 + s;
    sX[1 * N3 + t] = X1 + s;
    sX[2 * N3 + t] = X2 + s;
    sX[3 * N3 + t] = L2 ? a.u[cell * N3 + t] : 0.0;
  }
  __syncthreads();
  // x-contraction: point (q1, j, k)
  if (t < NQ * N2) {
    const int q1 = t % NQ, j = (t / NQ) % N, k = t / (NQ * N);
    for (int f = 0; f < 4; ++f) {
      double A = 0.0, B = 0.0;
#pragma unroll
      for (int r = 0; r < N; ++r) {
        const double v = sX[f * N3 + (k * N + j) * N + r];
        A = fma(a.tab.V[q1][r], v, A);
        if (f < 3) B = fma(a.tab.Dh[q1][r], v, B);
      }
      sA[f * NQ * N2 + t] = A;
      if (f < 3) sB[f * NQ * N2 + t] = B;
    }
  }
  __syncthreads();
  // y-contraction: point (q1, q2, k)
  if (t < NQ * NQ * N) {
    const int q1 = t % NQ, q2 = (t / NQ) % NQ, k = t / (NQ * NQ);
    for (int f = 0; f < 4; ++f) {
      double C = 0.0, D = 0.0, E = 0.0;
#pragma unroll
      for (int r = 0; r < N; ++r) {
        const int e = (k * N + r) * NQ + q1;
        C = fma(a.tab.V[q2][r], sA[f * NQ * N2 + e], C);
        if (f < 3) {
          D = fma(a.tab.Dh[q2][r], sA[f * NQ * N2 + e], D);
          E = fma(a.tab.V[q2][r], sB[f * NQ * N2 + e], E);
        }
      }
      sC[f * NQ * NQ * N + t] = C;
      if (f < 3) {
        sD[f * NQ * NQ * N + t] = D;
        sE[f * NQ * NQ * N + t] = E;
      }
    }
  }
  __syncthreads();
  // z-contraction: point (q1, q2, q3)
  double val = 0.0;
  if (t < Q3) {
    const int q1 = t % NQ, q2 = (t / NQ) % NQ, q3 = t / (NQ * NQ);
    double xq[4], J[3][3];
    for (int f = 0; f < 4; ++f) {
      double acc = 0.0;
#pragma unroll
      for (int r = 0; r < N; ++r) acc = fma(a.tab.V[q3][r], sC[f * NQ * NQ * N + (r * NQ + q2) * NQ + q1], acc);
      xq[f] = acc;
    }
    for (int c = 0; c < 3; ++c) {
      double j0 = 0.0, j1 = 0.0, j2 = 0.0;
#pragma unroll
      for (int r = 0; r < N; ++r) {
        const int e = (r * NQ + q2) * NQ + q1;
        j0 = fma(a.tab.V[q3][r], sE[c * NQ * NQ * N + e], j0);
        j1 = fma(a.tab.V[q3][r], sD[c * NQ * NQ * N + e], j1);
        j2 = fma(a.tab.Dh[q3][r], sC[c * NQ * NQ * N + e], j2);
      }
      J[c][0] = j0;
      J[c][1] = j1;
      J[c][2] = j2;
    }
    const double det = J[0][0] * (J[1][1] * J[2][2] - J[1][2] * J[2][1]) -
                       J[0][1] * (J[1][0] * J[2][2] - J[1][2] * J[2][0]) +
                       J[0][2] * (J[1][0] * J[2][1] - J[1][1] * J[2][0]);
    const double wd = a.tab.w[q1] * a.tab.w[q2] * a.tab.w[q3] * det;
    if (L2) {
      const double d = xq[3] - exact_u(a.kind, xq[0], xq[1], xq[2]);
      val = wd * d * d;
    } else {
      val = wd * exact_f(a.kind, xq[0], xq[1], xq[2]);
    }
  }
  if (L2) {
    // per-cell sum in a fixed order (tree over the block)
    red[t] = (t < Q3) ? val : 0.0;
    __syncthreads();
    for (int s = 1; s < (int)blockDim.x; s <<= 1) {
      if ((t % (2 * s)) == 0 && t + s < (int)blockDim.x) red[t] += red[t + s];
      __syncthreads();
    }
    if (t == 0) a.out[cell] = red[0];
    return;
  }
  // rhs: b_i = sum_q V[q1][i] V[q2][j] V[q3][k] g(q), transposed sweeps z, y, x (NQ == N)
  red[t] = val;
  __syncthreads();
  if (t < N3) {
    const int i = t % N, j = (t / N) % N, k = t / N2;
    // brute-force over the N^3 points per node is N^3 work; use three sweeps through smem
    double acc = 0.0;
#pragma unroll
    for (int q3 = 0; q3 < NQ; ++q3) acc = fma(a.tab.V[q3][k], red[(q3 * NQ + j) * NQ + i], acc);
    sC[t] = acc;  // (q1=i, q2=j, k)
  }
  __syncthreads();
  if (t < N3) {
    const int i = t % N, j = (t / N) % N, k = t / N2;
    double acc = 0.0;
#pragma unroll
    for (int q2 = 0; q2 < NQ; ++q2) acc = fma(a.tab.V[q2][j], sC[(k * NQ + q2) * NQ + i], acc);
    sD[t] = acc;  // (q1=i, j, k)
  }
  __syncthreads();
  if (t < N3) {
    const int i = t % N, j = (t / N) % N, k = t / N2;
    double acc = 0.0;
#pragma unroll
    for (int q1 = 0; q1 < NQ; ++q1) acc = fma(a.tab.V[q1][i], sD[(k * N + j) * NQ + q1], acc);
    a.out[cell * N3 + t] = acc;
  }
}

template <int N, int NQ, bool L2>
fe_status launch_man(const ManArgs& a, cudaStream_t st) {
  constexpr int N2 = N * N, N3 = N2 * N, Q3 = NQ * NQ * NQ;
  const size_t smem = sizeof(double) * (4 * N3 + 4 * NQ * N2 + 3 * NQ * N2 + 4 * NQ * NQ * N +
                                        3 * NQ * NQ * N + 3 * NQ * NQ * N + Q3);
  FE_CUDA(cudaFuncSetAttribute(k_manufactured<N, NQ, L2>,
                               cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem),
          "manufactured smem attribute");
  if (a.ncells > 0) k_manufactured<N, NQ, L2><<<(unsigned)a.ncells, Q3, smem, st>>>(a);
  return fe_cuda_check(cudaGetLastError(), "manufactured launch");
}

// 1D Gauss rule on [0,1] with nq points (Newton on Legendre), for the tables only
void gauss01(int nq, double* s, double* w) {
  const double pi = 3.14159265358979323846;
  for (int i = 0; i < nq; ++i) {
    double r = -std::cos(pi * (4.0 * i + 3.0) / (4.0 * nq + 2.0));
    for (int it = 0; it < 60; ++it) {
      double p0 = 1.0, p1 = r, dp0 = 0.0, dp1 = 1.0;
      for (int k = 1; k < nq; ++k) {
        const double p2 = ((2 * k + 1) * r * p1 - k * p0) / (k + 1);
        const double dp2 = dp0 + (2 * k + 1) * p1;
        p0 = p1;
        p1 = p2;
        dp0 = dp1;
        dp1 = dp2;
      }
      const double dr = p1 / dp1;
      r -= dr;
      if (std::fabs(dr) <= 1e-17) {
        s[i] = 0.5 * (r + 1.0);
        w[i] = 1.0 / ((1.0 - r * r) * dp1 * dp1);  // 0.5 * 2/((1-r^2) P'^2)
        break;
      }
      s[i] = 0.5 * (r + 1.0);
      w[i] = 1.0 / ((1.0 - r * r) * dp1 * dp1);
    }
  }
}

// Lagrange basis through the GLL nodes t and its derivative at s (barycentric)
void lagrange_row(int n, const double* t, double s, double* val, double* der) {
  for (int i = 0; i < n; ++i) {
    double v = 1.0, d = 0.0;
    for (int j = 0; j < n; ++j) {
      if (j == i) continue;
      double term = 1.0 / (t[i] - t[j]);
      for (int k = 0; k < n; ++k)
        if (k != i && k != j) term *= (s - t[k]) / (t[i] - t[k]);
      d += term;
      v *= (s - t[j]) / (t[i] - t[j]);
    }
    val[i] = v;
    der[i] = d;
  }
}

template <int N, bool L2>
fe_status run_man(const fe_mesh* m, int kind, const double* u, double* out, cudaStream_t st) {
  constexpr int NQ = L2 ? N + 2 : N;
  ManArgs a;
  std::memset(&a, 0, sizeof(a));
  a.u = u;
  a.out = out;
  a.ncells = m->ncells;
  a.mx = m->d.mx;
  a.my = m->d.my;
  a.mz = fe_mz_global(m);
  a.z0 = m->zoff;
  a.kind = kind;
  a.amp = m->d.deform_amp;
  double s[MAXQ], w[MAXQ];
  gauss01(NQ, s, w);
  for (int i = 0; i < N; ++i) a.tab.t[i] = m->tab.t[i];
  for (int q = 0; q < NQ; ++q) {
    a.tab.w[q] = w[q];
    lagrange_row(N, m->tab.t, s[q], a.tab.V[q], a.tab.Dh[q]);
  }
  return launch_man<N, NQ, L2>(a, st);
}

template <bool L2>
fe_status dispatch(const fe_mesh* m, int kind, const double* u, double* out, cudaStream_t st) {
  switch (m->n) {
    case 2: return run_man<2, L2>(m, kind, u, out, st);
    case 3: return run_man<3, L2>(m, kind, u, out, st);
    case 4: return run_man<4, L2>(m, kind, u, out, st);
    case 5: return run_man<5, L2>(m, kind, u, out, st);
    case 6: return run_man<6, L2>(m, kind, u, out, st);
    case 7: return run_man<7, L2>(m, kind, u, out, st);
    case 8: return run_man<8, L2>(m, kind, u, out, st);
  }
  fe_set_error("manufactured: bad n");
  return FE_ERR_INVALID;
}

__global__ void __launch_bounds__(RED_THREADS)
    k_sum_cells(const double* __restrict__ v, long long n, double* __restrict__ out) {
  __shared__ dw sh[32];
  dw acc = {0.0f, 0.0f};
  for (long long e = threadIdx.x; e < n; e += RED_THREADS) acc = dw_add(acc, dw_from_double(v[e]));
  acc = block_reduce_dw(acc, sh);
  if (threadIdx.x == 0) out[0] = dw_to_double(acc);
}

}  // namespace

extern "C" fe_status fe_rhs(const fe_mesh* m, int kind, double* b, void* stream) {
  if (!m || !b || !fe_aligned(b)) {
    fe_set_error("fe_rhs: null or misaligned argument");
    return FE_ERR_INVALID;
  }
  if (kind != FE_RHS_SINE && kind != FE_RHS_QUADRATIC) {
    fe_set_error("fe_rhs: unknown kind %d", kind);
    return FE_ERR_INVALID;
  }
  if (m->packed) {
    fe_set_error("fe_rhs: FE_LAYOUT_CELLS meshes only");
    return FE_ERR_INVALID;
  }
  FeDeviceGuard device_guard;
  FE_CUDA(device_guard.set(m->d.device), "cudaSetDevice");
  return dispatch<false>(m, kind, nullptr, b, (cudaStream_t)stream);
}

extern "C" fe_status fe_l2_error(const fe_mesh* m, int kind, const double* u, double* err,
                                 void* stream) {
  if (!m || !u || !err || !fe_aligned(u)) {
    fe_set_error("fe_l2_error: null or misaligned argument");
    return FE_ERR_INVALID;
  }
  if (kind != FE_RHS_SINE && kind != FE_RHS_QUADRATIC) {
    fe_set_error("fe_l2_error: unknown kind %d", kind);
    return FE_ERR_INVALID;
  }
  if (m->packed) {
    fe_set_error("fe_l2_error: FE_LAYOUT_CELLS meshes only");
    return FE_ERR_INVALID;
  }
  FeDeviceGuard device_guard;
  FE_CUDA(device_guard.set(m->d.device), "cudaSetDevice");
  cudaStream_t st = (cudaStream_t)stream;
  double* tmp = nullptr;
  FE_CUDA(cudaMallocAsync(&tmp, (m->ncells + 1) * sizeof(double), st), "fe_l2_error scratch");
  fe_status s = dispatch<true>(m, kind, u, tmp, st);
  if (s == FE_OK) {
    k_sum_cells<<<1, RED_THREADS, 0, st>>>(tmp, m->ncells, tmp + m->ncells);
    s = fe_cuda_check(cudaGetLastError(), "fe_l2_error sum");
  }
  double h = 0.0;
  if (s == FE_OK)
    s = fe_cuda_check(cudaMemcpyAsync(&h, tmp + m->ncells, sizeof(double), cudaMemcpyDeviceToHost, st),
                      "fe_l2_error readback");
  cudaFreeAsync(tmp, st);
  if (s == FE_OK) s = fe_cuda_check(cudaStreamSynchronize(st), "fe_l2_error synchronize");
  if (s == FE_OK) *err = sqrt(h);
  return s;
}
