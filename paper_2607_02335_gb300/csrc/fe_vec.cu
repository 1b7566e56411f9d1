// fe_vec.cu -- structured DSS, Jacobi diagonal, duality pairings and cell-wise vector kernels.
#include <cstring>

#include "fe_recompute.cuh"
#include "fe_vec.cuh"

// ---------------------------------------------------------------------------------------------
// Structured DSS (Sec. 4.1, Algorithm "Dimensionally-Split Structured Summation").  One launch
// per axis, in the order z, y, x.  Each thread owns one node pair of one interior interface
// (cell K_L with local index p along the axis, cell K_R with local index 0): it sums the two
// copies and writes the sum to both.  Pairs of one pass are disjoint, so no atomics are needed;
// because each pass sees the partial sums of the previous one, edge and vertex copies are
// assembled as a by-product.
// ---------------------------------------------------------------------------------------------
// stride s > 1: just the interfaces whose left (lower) cell index is s-1 mod s, the boundaries
// between bricks (x, y) or z-chunks (z) of s cells along that axis (nb = (m-1)/s per line)
// the node pair of work item e of one axis pass (cells L, R and local nodes locL, locR)
template <class S>
__device__ __forceinline__ void dss_pair(S* __restrict__ v, int axis, int n, int mx, int my,
                                         int stride, long long e) {
  const int p = n - 1, n2 = n * n, n3 = n2 * n;
  const int f = (int)(e % n2);
  const long long q = e / n2;
  const int fa = f % n, fb = f / n;
  long long L, R;
  int locL, locR;
  if (axis == 0) {  // faces normal to x
    const int nbx = (mx - 1) / stride;
    const long long u = q % nbx, r = q / nbx;
    L = r * mx + (u * stride + stride - 1);  // r = cz*my + cy
    R = L + 1;
    locL = (fb * n + fa) * n + p;
    locR = (fb * n + fa) * n + 0;
  } else if (axis == 1) {  // faces normal to y
    const int nby = (my - 1) / stride;
    const long long cx = q % mx, r = q / mx, u = r % nby, cz = r / nby;
    const long long cyL = u * stride + stride - 1;
    L = (cz * my + cyL) * mx + cx;
    R = L + mx;
    locL = (fb * n + p) * n + fa;
    locR = (fb * n + 0) * n + fa;
  } else {  // faces normal to z
    const long long mxy = (long long)mx * my, u = q / mxy;
    L = (u * stride + stride - 1) * mxy + (q - u * mxy);  // q = (u*my + cy)*mx + cx
    R = L + mxy;
    locL = (p * n + fb) * n + fa;
    locR = (0 * n + fb) * n + fa;
  }
  S* pl = v + L * n3 + locL;
  S* pr = v + R * n3 + locR;
  const S s = *pl + *pr;
  *pl = s;
  *pr = s;
}

template <class S>
__global__ void k_dss_pass(S* __restrict__ v, int axis, int n, int mx, int my, int stride,
                           long long nwork) {
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < nwork;
       e += (long long)gridDim.x * blockDim.x)
    dss_pair(v, axis, n, mx, my, stride, e);
}

// One axis pass over every block of a block-structured mesh in one launch: block b owns the work
// items [first[b], first[b+1]) and the cell-wise slice starting at cell off[b].
constexpr int DSS_MAXB = 32;
struct DssBlocks {
  int nb, stride;  // stride: brick size along this axis (x and y passes after a fused apply)
  int mx[DSS_MAXB], my[DSS_MAXB];
  long long off[DSS_MAXB], first[DSS_MAXB + 1];
};

template <class S>
__global__ void k_dss_pass_blocks(S* __restrict__ v, int axis, int n,
                                  const __grid_constant__ DssBlocks B) {
  const long long n3 = (long long)n * n * n;
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < B.first[B.nb];
       e += (long long)gridDim.x * blockDim.x) {
    int b = 0;
    while (e >= B.first[b + 1]) ++b;
    dss_pair(v + B.off[b] * n3, axis, n, B.mx[b], B.my[b], B.stride, e - B.first[b]);
  }
}

// The passes on one structured grid: one CTA per row of interfaces, the row's cell offsets formed
// once per CTA and the items of the row (interface along the row, face node) in 32-bit arithmetic
// with compile-time divisors.  Rows and items: x-pass row (cz, cy), items (u, node); y-pass row
// (cz, u), items (cx, node); z-pass row (u, cy), items (cx, node); u counts the interfaces visited
// along the axis (nb per line), the left cell of interface u has index u*stride + stride - 1.
// Each pair gets the sum of dss_pair.
template <class S, int N>
__global__ void __launch_bounds__(256) k_dss_row(S* __restrict__ v, int axis, int mx, int my,
                                                 int stride, int nb) {
  constexpr int P = N - 1, N2 = N * N, N3 = N2 * N;
  const long long r = blockIdx.x;
  long long first;  // left cell of the row's first item
  int items, lstep;  // items in the row; left-cell step from one item group to the next
  long long rstep;   // right cell - left cell
  int locL0, locR0, sa, sb;  // local node of face node (fa, fb): loc0 + fa*sa + fb*sb
  if (axis == 0) {
    first = r * mx + stride - 1;
    items = nb * N2;
    lstep = stride;
    rstep = 1;
    locL0 = P, locR0 = 0, sa = N, sb = N2;
  } else if (axis == 1) {
    const long long cz = r / nb, u = r - cz * nb;
    first = (cz * my + u * stride + stride - 1) * mx;
    items = mx * N2;
    lstep = 1;
    rstep = mx;
    locL0 = P * N, locR0 = 0, sa = 1, sb = N2;
  } else {
    const long long u = r / my, cy = r - u * my;
    first = ((u * stride + stride - 1) * my + cy) * mx;
    items = mx * N2;
    lstep = 1;
    rstep = (long long)mx * my;
    locL0 = P * N2, locR0 = 0, sa = 1, sb = N;
  }
  for (int it = threadIdx.x; it < items; it += blockDim.x) {
    const int g = it / N2, f = it - g * N2, fa = f % N, fb = f / N;
    const long long L = first + (long long)g * lstep;
    const int off = fa * sa + fb * sb;
    S* pl = v + L * N3 + locL0 + off;
    S* pr = v + (L + rstep) * N3 + locR0 + off;
    const S s = *pl + *pr;
    *pl = s;
    *pr = s;
  }
}

template <class S, int N>
static void launch_dss_rows(S* v, int axis, int mx, int my, int mz, int stride, cudaStream_t st) {
  const int nb = axis == 0 ? (mx - 1) / stride : axis == 1 ? (my - 1) / stride : (mz - 1) / stride;
  const long long rows = axis == 0 ? (long long)my * mz : axis == 1 ? (long long)mz * nb
                                                                    : (long long)nb * my;
  const int items = (axis == 0 ? nb : mx) * N * N;
  if (nb <= 0 || rows <= 0) return;
  const int threads = items >= 256 ? 256 : (items + 31) / 32 * 32;
  k_dss_row<S, N><<<(unsigned)rows, threads, 0, st>>>(v, axis, mx, my, stride, nb);
}

static unsigned grid_cap(long long n, int threads) {
  long long b = (n + threads - 1) / threads;
  if (b > 152LL * 32) b = 152LL * 32;
  if (b < 1) b = 1;
  return (unsigned)b;
}

template <class S>
static fe_status dss_t(const fe_mesh* m, S* v, int sx, int sy, cudaStream_t st, int axis_hi = 2,
                       int axis_lo = 0, int sz = 1) {
  // the storage grid: cells, or 2^3-packed units whose sides carry 2p+1 nodes
  const int n = m->sn, n2 = n * n;
  const int mx = m->sgx, my = m->sgy, mz = m->sgz;
  const int stride[3] = {sx, sy, sz};
  const long long work[3] = {(long long)((mx - 1) / sx) * my * mz * n2,
                             (long long)mx * ((my - 1) / sy) * mz * n2,
                             (long long)mx * my * ((mz - 1) / sz) * n2};
  for (int axis = axis_hi; axis >= axis_lo; --axis) {  // z, y, x
    if (work[axis] <= 0) continue;
    switch (n) {
      case 2: launch_dss_rows<S, 2>(v, axis, mx, my, mz, stride[axis], st); break;
      case 3: launch_dss_rows<S, 3>(v, axis, mx, my, mz, stride[axis], st); break;
      case 4: launch_dss_rows<S, 4>(v, axis, mx, my, mz, stride[axis], st); break;
      case 5: launch_dss_rows<S, 5>(v, axis, mx, my, mz, stride[axis], st); break;
      case 6: launch_dss_rows<S, 6>(v, axis, mx, my, mz, stride[axis], st); break;
      case 7: launch_dss_rows<S, 7>(v, axis, mx, my, mz, stride[axis], st); break;
      case 8: launch_dss_rows<S, 8>(v, axis, mx, my, mz, stride[axis], st); break;
      default:
        k_dss_pass<S><<<grid_cap(work[axis], 256), 256, 0, st>>>(v, axis, n, mx, my, stride[axis],
                                                                 work[axis]);
    }
  }
  return fe_cuda_check(cudaGetLastError(), "dss launch");
}

fe_status fe_launch_dss_strided(const fe_mesh* m, int prec, void* v, int bx, int by,
                                cudaStream_t st) {
  if (bx < 1 || by < 1) {
    fe_set_error("dss: bad brick %d x %d", bx, by);
    return FE_ERR_INVALID;
  }
  if (prec == FE_F64) return dss_t<double>(m, (double*)v, bx, by, st);
  if (prec == FE_F32) return dss_t<float>(m, (float*)v, bx, by, st);
  fe_set_error("dss: unsupported precision %d", prec);
  return FE_ERR_INVALID;
}

fe_status fe_launch_dss_axes(const fe_mesh* m, int prec, void* v, int bx, int by, int axis_hi,
                             int axis_lo, cudaStream_t st) {
  if (bx < 1 || by < 1 || axis_hi > 2 || axis_lo < 0) {
    fe_set_error("dss: bad brick %d x %d or axes %d..%d", bx, by, axis_hi, axis_lo);
    return FE_ERR_INVALID;
  }
  if (prec == FE_F64) return dss_t<double>(m, (double*)v, bx, by, st, axis_hi, axis_lo);
  if (prec == FE_F32) return dss_t<float>(m, (float*)v, bx, by, st, axis_hi, axis_lo);
  fe_set_error("dss: unsupported precision %d", prec);
  return FE_ERR_INVALID;
}

fe_status fe_launch_dss_strided3(const fe_mesh* m, int prec, void* v, int bx, int by, int bz,
                                 cudaStream_t st) {
  if (bx < 1 || by < 1 || bz < 1) {
    fe_set_error("dss: bad brick %d x %d x %d", bx, by, bz);
    return FE_ERR_INVALID;
  }
  if (prec == FE_F64) return dss_t<double>(m, (double*)v, bx, by, st, 2, 0, bz);
  if (prec == FE_F32) return dss_t<float>(m, (float*)v, bx, by, st, 2, 0, bz);
  fe_set_error("dss: unsupported precision %d", prec);
  return FE_ERR_INVALID;
}

fe_status fe_launch_dss(const fe_mesh* m, int prec, void* v, cudaStream_t st) {
  return fe_launch_dss_strided(m, prec, v, 1, 1, st);
}

template <class S>
static fe_status dss_blocks_t(const fe_mesh* const* blocks, const long long* off, int nb, S* v,
                              int sx, int sy, cudaStream_t st) {
  const int n = blocks[0]->n, n2 = n * n;
  for (int axis = 2; axis >= 0; --axis) {  // z, y, x
    DssBlocks B;
    std::memset(&B, 0, sizeof(B));
    B.nb = nb;
    B.stride = axis == 0 ? sx : (axis == 1 ? sy : 1);
    for (int b = 0; b < nb; ++b) {
      const int mx = blocks[b]->d.mx, my = blocks[b]->d.my, mz = blocks[b]->d.mz;
      B.mx[b] = mx;
      B.my[b] = my;
      B.off[b] = off[b];
      const long long w = axis == 0 ? (long long)((mx - 1) / sx) * my * mz * n2
                          : axis == 1 ? (long long)mx * ((my - 1) / sy) * mz * n2
                                      : (long long)mx * my * (mz - 1) * n2;
      B.first[b + 1] = B.first[b] + w;
    }
    if (B.first[nb] > 0)
      k_dss_pass_blocks<S><<<grid_cap(B.first[nb], 256), 256, 0, st>>>(v, axis, n, B);
  }
  return fe_cuda_check(cudaGetLastError(), "dss launch");
}

fe_status fe_launch_dss_blocks(const fe_mesh* const* blocks, const long long* off, int nb,
                               int prec, void* v, int sx, int sy, cudaStream_t st) {
  if (sx < 1 || sy < 1) {
    fe_set_error("dss: bad brick %d x %d", sx, sy);
    return FE_ERR_INVALID;
  }
  if (nb > DSS_MAXB) {  // one launch triple per block
    const size_t es = prec == FE_F64 ? sizeof(double) : sizeof(float);
    for (int b = 0; b < nb; ++b)
      FE_TRY(fe_launch_dss_strided(blocks[b], prec, (char*)v + (size_t)off[b] * blocks[b]->n3 * es,
                                   sx, sy, st));
    return FE_OK;
  }
  if (prec == FE_F64) return dss_blocks_t<double>(blocks, off, nb, (double*)v, sx, sy, st);
  if (prec == FE_F32) return dss_blocks_t<float>(blocks, off, nb, (float*)v, sx, sy, st);
  fe_set_error("dss: unsupported precision %d", prec);
  return FE_ERR_INVALID;
}

// ---------------------------------------------------------------------------------------------
// Jacobi diagonal (Sec. 3.3: D_cell = diag(G d)).  The local diagonal of A_K,
//   d_i = sum_q sum_ab G_ab(q) dphi_i/dxi_a(q) dphi_i/dxi_b(q)   (Laplace)
//   d_i = sum_q w_q detJ(q) phi_i(q)^2                          (mass),
// is a transposed sum factorization with squared 1D matrices (Dh^2, V^2, Dh*V): six terms for
// the symmetric G.  FP64, once per mesh and operator.  Then DSS assembles the copies and
// Dirichlet nodes get 1.
// ---------------------------------------------------------------------------------------------
struct DiagTab {
  double V2[FE_MAXN][FE_MAXN];   // V[q][i]^2
  double D2[FE_MAXN][FE_MAXN];   // Dh[q][i]^2
  double DV[FE_MAXN][FE_MAXN];   // Dh[q][i] V[q][i]
  double w[FE_MAXN];
};
struct DiagArgs {
  const double* geo;  // [cell - geo_cell0][7][N3]
  double* d;
  long long ncells, cell_base, geo_cell0;
  int op, affine;
  double aff[4];
  DiagTab tab;
};

template <int N>
__global__ void __launch_bounds__(Cfg<N>::THREADS) k_diag(const __grid_constant__ DiagArgs a) {
  using C = Cfg<N>;
  constexpr int N2 = C::N2, N3 = C::N3;
  extern __shared__ double dsm[];
  const int t = threadIdx.x, cl = t / N2, lt = t - cl * N2, la = lt % N, lb = lt / N;
  const int cb = cl * C::CS;
  const long long cell = a.cell_base + (long long)blockIdx.x * C::CPB + cl;
  const bool active = cell < a.ncells;
  // term t: (component, C1, C2, C3, factor)   matrices: 0 = V2, 1 = D2, 2 = DV
  const int nterms = (a.op == FE_LAPLACE) ? 6 : 1;
  const int comp[6] = {0, 1, 2, 3, 4, 5};
  const int m1[6] = {1, 0, 0, 2, 2, 0}, m2[6] = {0, 1, 0, 2, 0, 2}, m3[6] = {0, 0, 1, 0, 2, 2};
  const double fac[6] = {1, 1, 1, 2, 2, 2};
  double dsum[N];
#pragma unroll
  for (int k = 0; k < N; ++k) dsum[k] = 0.0;
  for (int term = 0; term < nterms; ++term) {
    const int c = (a.op == FE_LAPLACE) ? comp[term] : 6;
    const int M1 = (a.op == FE_LAPLACE) ? m1[term] : 0, M2 = (a.op == FE_LAPLACE) ? m2[term] : 0,
              M3 = (a.op == FE_LAPLACE) ? m3[term] : 0;
    const double (*T1)[FE_MAXN] = M1 == 0 ? a.tab.V2 : (M1 == 1 ? a.tab.D2 : a.tab.DV);
    const double (*T2)[FE_MAXN] = M2 == 0 ? a.tab.V2 : (M2 == 1 ? a.tab.D2 : a.tab.DV);
    const double (*T3)[FE_MAXN] = M3 == 0 ? a.tab.V2 : (M3 == 1 ? a.tab.D2 : a.tab.DV);
    double g[N];
#pragma unroll
    for (int q3 = 0; q3 < N; ++q3) {
      double v = 0.0;
      if (active) {
        if (a.affine) {
          const double wq = a.tab.w[la] * a.tab.w[lb] * a.tab.w[q3];
          v = (c == 6) ? wq * a.aff[3] : (c < 3 ? wq * a.aff[c] : 0.0);
        } else {
          v = a.geo[(size_t)(cell - a.geo_cell0) * FE_GEO_COMPS * N3 + (size_t)c * N3 + q3 * N2 + lt];
        }
      }
      g[q3] = v * fac[term];
    }
    // z: P(q1, q2, k) = sum_q3 T3[q3][k] g(q1, q2, q3)
#pragma unroll
    for (int k = 0; k < N; ++k) {
      double acc = 0.0;
#pragma unroll
      for (int q3 = 0; q3 < N; ++q3) acc = fma(T3[q3][k], g[q3], acc);
      dsm[cb + zl<N>(la, lb, k)] = acc;
    }
    __syncthreads();
    {  // x: line (q2 = la, k = lb), contract q1 -> i
      double in[N];
#pragma unroll
      for (int r = 0; r < N; ++r) in[r] = dsm[cb + xl<N>(la, lb, r)];
#pragma unroll
      for (int i = 0; i < N; ++i) {
        double acc = 0.0;
#pragma unroll
        for (int r = 0; r < N; ++r) acc = fma(T1[r][i], in[r], acc);
        dsm[cb + xl<N>(la, lb, i)] = acc;
      }
    }
    __syncthreads();
    {  // y: line (i = la, k = lb), contract q2 -> j
      double in[N];
#pragma unroll
      for (int r = 0; r < N; ++r) in[r] = dsm[cb + yl<N>(la, lb, r)];
#pragma unroll
      for (int j = 0; j < N; ++j) {
        double acc = 0.0;
#pragma unroll
        for (int r = 0; r < N; ++r) acc = fma(T2[r][j], in[r], acc);
        dsm[cb + yl<N>(la, lb, j)] = acc;
      }
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < N; ++k) dsum[k] += dsm[cb + zl<N>(la, lb, k)];
    __syncthreads();
  }
  if (active) {
#pragma unroll
    for (int k = 0; k < N; ++k) a.d[cell * N3 + k * N2 + lt] = dsum[k];
  }
}

template <int N>
static fe_status launch_diag_chunk(const DiagArgs& a, cudaStream_t st) {
  using C = Cfg<N>;
  const size_t smem = (size_t)C::TILE * sizeof(double);
  FE_CUDA(cudaFuncSetAttribute(k_diag<N>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem),
          "diag smem attribute");
  const long long blocks = (a.ncells - a.cell_base + C::CPB - 1) / C::CPB;
  if (blocks > 0) k_diag<N><<<(unsigned)blocks, C::THREADS, smem, st>>>(a);
  return fe_cuda_check(cudaGetLastError(), "diag launch");
}

// Recompute mode: the FP64 metric of one chunk of cells into the FP64 scratch, then the diagonal
// of that chunk.
template <int N>
static fe_status launch_diag_n(const fe_mesh* m, DiagArgs a, cudaStream_t st) {
  if (m->d.geom_mode != FE_GEOM_RECOMPUTE) return launch_diag_chunk<N>(a, st);
  using G = GeoCfg<N>;
  double* scratch = static_cast<double*>(m->rc_scratch[1]);
  if (!scratch || !m->xyz64) {
    fe_set_error("diag: recompute-mode buffers missing");
    return FE_ERR_INVALID;
  }
  const long long chunk = fe_rc_chunk_cells(N, m->ncells, sizeof(double));
  RecomputeArgs<N, double> r;
  std::memset(&r, 0, sizeof(r));
  r.xyz = m->xyz64;
  r.geo = scratch;
  for (int q = 0; q < N; ++q) {
    r.tab.W_[q] = m->tab.w[q];
    for (int i = 0; i < N; ++i) {
      r.tab.V_[q][i] = m->tab.V[q][i];
      r.tab.D_[q][i] = m->tab.D[q][i];
    }
  }
  a.geo = scratch;
  const long long total = m->ncells;
  for (long long c0 = 0; c0 < total; c0 += chunk) {
    const long long c1 = c0 + chunk < total ? c0 + chunk : total;
    r.cell0 = c0;
    r.cell_end = c1;
    const unsigned gb = (unsigned)((c1 - c0 + G::CPB - 1) / G::CPB);
    const size_t gs = recompute_smem_bytes<N, double>();
    if (a.op == FE_LAPLACE)
      k_recompute<N, double, FE_LAPLACE><<<gb, G::THREADS, gs, st>>>(r);
    else
      k_recompute<N, double, FE_MASS><<<gb, G::THREADS, gs, st>>>(r);
    FE_CUDA(cudaGetLastError(), "recompute kernel launch");
    a.cell_base = c0;
    a.geo_cell0 = c0;
    a.ncells = c1;
    FE_TRY(launch_diag_chunk<N>(a, st));
  }
  return FE_OK;
}

// Dirichlet nodes -> 1 (one warp per cell, lanes over the cell's nodes)
__global__ void k_dirichlet_fill(double* __restrict__ v, double val, long long ncells, int n, int mx,
                                 int my, int mz, int mask) {
  const int n3 = n * n * n, p = n - 1;
  const int lane = threadIdx.x & 31;
  const long long warp = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const long long nwarps = ((long long)gridDim.x * blockDim.x) >> 5;
  for (long long c = warp; c < ncells; c += nwarps) {
    const int cx = (int)(c % mx), cy = (int)((c / mx) % my), cz = (int)(c / ((long long)mx * my));
    if (cx != 0 && cx != mx - 1 && cy != 0 && cy != my - 1 && cz != 0 && cz != mz - 1) continue;
    for (int l = lane; l < n3; l += 32) {
      const int i = l % n, j = (l / n) % n, k = l / (n * n);
      if ((cx == 0 && i == 0) || (cx == mx - 1 && i == p) || (cy == 0 && j == 0) ||
          (cy == my - 1 && j == p) || ((mask & FE_DIR_ZLO) && cz == 0 && k == 0) ||
          ((mask & FE_DIR_ZHI) && cz == mz - 1 && k == p))
        v[c * n3 + l] = val;
    }
  }
}

fe_status fe_launch_diag(const fe_mesh* m, int op, double* d, cudaStream_t st) {
  DiagArgs a;
  std::memset(&a, 0, sizeof(a));
  a.geo = m->geo64;
  a.d = d;
  a.ncells = m->ncells;
  a.op = op;
  a.affine = m->d.geom_mode == FE_GEOM_AFFINE;
  const double hx = 1.0 / m->d.mx, hy = 1.0 / m->d.my, hz = 1.0 / fe_mz_global(m),
               det = hx * hy * hz;
  a.aff[0] = det / (hx * hx);
  a.aff[1] = det / (hy * hy);
  a.aff[2] = det / (hz * hz);
  a.aff[3] = det;
  for (int q = 0; q < m->n; ++q) {
    a.tab.w[q] = m->tab.w[q];
    for (int i = 0; i < m->n; ++i) {
      a.tab.V2[q][i] = m->tab.V[q][i] * m->tab.V[q][i];
      a.tab.D2[q][i] = m->tab.Dh[q][i] * m->tab.Dh[q][i];
      a.tab.DV[q][i] = m->tab.Dh[q][i] * m->tab.V[q][i];
    }
  }
  if (m->d.geom_mode == FE_GEOM_RECOMPUTE) FE_TRY(fe_ensure_geometry(m, FE_F64, true));
  if (!a.affine && !a.geo && m->d.geom_mode != FE_GEOM_RECOMPUTE) {
    fe_set_error("diag: the stored metric has been released");
    return FE_ERR_INVALID;
  }
  fe_status s;
  switch (m->n) {
    case 2: s = launch_diag_n<2>(m, a, st); break;
    case 3: s = launch_diag_n<3>(m, a, st); break;
    case 4: s = launch_diag_n<4>(m, a, st); break;
    case 5: s = launch_diag_n<5>(m, a, st); break;
    case 6: s = launch_diag_n<6>(m, a, st); break;
    case 7: s = launch_diag_n<7>(m, a, st); break;
    case 8: s = launch_diag_n<8>(m, a, st); break;
    default: fe_set_error("diag: bad n"); return FE_ERR_INVALID;
  }
  if (s != FE_OK) return s;
  FE_TRY(fe_launch_dss(m, FE_F64, d, st));
  if (m->d.dirichlet) {
    k_dirichlet_fill<<<grid_cap(m->ncells * 32, 256), 256, 0, st>>>(
        d, 1.0, m->ncells, m->n, m->d.mx, m->d.my, m->d.mz, fe_dir_mask(m));
    FE_TRY(fe_cuda_check(cudaGetLastError(), "dirichlet fill"));
  }
  return FE_OK;
}

// ---------------------------------------------------------------------------------------------
// Deterministic reductions.  A fixed grid of RED_BLOCKS CTAs strides over the vector; each thread
// accumulates its products in binary64 (the FP64 pipe: one fma per entry, the whole binary64
// range), the CTA reduces in a fixed shuffle tree and writes one partial per CTA, and a one-CTA
// kernel sums the partials in a fixed order.  The result depends only on the data, never on
// timing.
// ---------------------------------------------------------------------------------------------
// partials[block] = sum over the CTA's stride of a_e * b_e
template <class S>
__global__ void __launch_bounds__(RED_THREADS)
    k_pairing_partial(const S* __restrict__ a, const S* __restrict__ b, long long n,
                      double* __restrict__ partials) {
  __shared__ double sh[32];
  double acc = 0.0;
  for (long long e = (long long)blockIdx.x * RED_THREADS + threadIdx.x; e < n;
       e += (long long)RED_BLOCKS * RED_THREADS)
    acc = fma((double)__ldg(a + e), (double)__ldg(b + e), acc);
  acc = block_reduce_f64(acc, sh);
  if (threadIdx.x == 0) partials[blockIdx.x] = acc;
}

// out[0] = sum of the nparts partials in a fixed order
__global__ void __launch_bounds__(RED_THREADS)
    k_partials_sum64(const double* __restrict__ partials, int nparts, double* __restrict__ out) {
  __shared__ double sh[32];
  double acc = 0.0;
  for (int b = threadIdx.x; b < nparts; b += RED_THREADS) acc += partials[b];
  acc = block_reduce_f64(acc, sh);
  if (threadIdx.x == 0) out[0] = acc;
}

fe_status fe_ensure_reduction(const fe_mesh* cm) {
  fe_mesh* m = const_cast<fe_mesh*>(cm);
  if (!m->red) {
    FE_TRY(fe_dalloc((void**)&m->red, (size_t)RED_BLOCKS * RED_SLOTS * sizeof(double), m->st,
                     "reduction partials"));
    FE_CUDA(cudaStreamSynchronize(m->st), "reduction partials");
    m->red_len = RED_BLOCKS * RED_SLOTS;
  }
  return FE_OK;
}

fe_status fe_launch_pairing(const fe_mesh* m, int prec, const void* a, const void* b, double* out,
                            cudaStream_t st) {
  FE_TRY(fe_ensure_reduction(m));
  if (prec == FE_F64)
    k_pairing_partial<double><<<RED_BLOCKS, RED_THREADS, 0, st>>>((const double*)a, (const double*)b,
                                                                  m->ncw, m->red);
  else if (prec == FE_F32)
    k_pairing_partial<float><<<RED_BLOCKS, RED_THREADS, 0, st>>>((const float*)a, (const float*)b,
                                                                 m->ncw, m->red);
  else {
    fe_set_error("pairing: unsupported precision %d", prec);
    return FE_ERR_INVALID;
  }
  k_partials_sum64<<<1, RED_THREADS, 0, st>>>(m->red, RED_BLOCKS, out);
  return fe_cuda_check(cudaGetLastError(), "pairing launch");
}
