// fe_host.cu -- operator applies on host vectors in unique-node form.
//
// Cell-wise storage keeps one value per copy of a node (Sec. 2.2; (p+1)^3 / p^3 copies per node
// in the interior, 2.4x at Q3).  It is the device's working format, not what a host needs to send:
// the gather G of Sec. 2.1 rebuilds every copy from one value per node, and after the DSS every
// copy of a node holds the same sum, so one copy per node carries the whole result.  The host link
// therefore moves unique-node vectors only, and the expansion and selection run as kernels next to
// the apply:
//   x_unique --H2D--> expand (G) --> fe_apply with FE_ASSEMBLE --> select one copy --D2H--> y_unique
// y_unique = G^T A_D G x_unique, the assembled operator on the global node vector.
#include <cstdlib>

#include "fe_internal.h"

namespace {

// One CTA per row of cells along x (expand) or row of nodes along x (select): the row's
// coordinates and 64-bit offsets are formed once per CTA, the threads of the row use 32-bit
// arithmetic with compile-time divisors.

// Four elements per thread have their loads issued before their stores (HOST_U), and a select
// CTA takes SEL_ROWS node rows: one row each (a few hundred nodes) left the CTAs too short.
constexpr int HOST_U = 4;
constexpr int SEL_ROWS = 8;

// x_cell[e] = x_unique[global node of e], for the cells of row r = cz my + cy
template <int N>
__global__ void __launch_bounds__(256) k_expand(const double* __restrict__ xu,
                                                double* __restrict__ xc, int mx, int my) {
  constexpr int P = N - 1, N2 = N * N, N3 = N2 * N;
  const long long r = blockIdx.x;
  const int cy = (int)(r % my);
  const long long cz = r / my;
  const long long Nx = (long long)mx * P + 1, Ny = (long long)my * P + 1;
  const double* src = xu + (cz * P * Ny + (long long)cy * P) * Nx;  // node (0, cy p, cz p)
  double* dst = xc + r * mx * N3;
  const int len = mx * N3;
  auto from = [&](int e) {
    const int cx = e / N3, loc = e - cx * N3;
    const int k = loc / N2, j = (loc / N) % N, i = loc % N;
    return (k * Ny + j) * Nx + cx * P + i;
  };
  int e = threadIdx.x;
  for (; e + (HOST_U - 1) * (int)blockDim.x < len; e += HOST_U * blockDim.x) {
    double v[HOST_U];
#pragma unroll
    for (int u = 0; u < HOST_U; ++u) v[u] = __ldg(src + from(e + u * blockDim.x));
#pragma unroll
    for (int u = 0; u < HOST_U; ++u) dst[e + u * blockDim.x] = v[u];
  }
  for (; e < len; e += blockDim.x) dst[e] = __ldg(src + from(e));
}

// y_unique[g] for the node layers gz0 <= gz < gz0 + nrows, row r = (gz - gz0) Ny + gy: along z the
// copy in the lower cell (k = p) on a cell interface, so that a layer's nodes are final as soon as
// the cell layers below them are; along x and y the copy in the upper cell (all copies are equal
// once the DSS passes of the cell layer are done).  CTA b takes rows [b SEL_ROWS, (b+1) SEL_ROWS).
template <int N>
__global__ void __launch_bounds__(256) k_select(const double* __restrict__ yc,
                                                double* __restrict__ yu, int mx, int my, int gz0,
                                                long long nrows) {
  constexpr int P = N - 1, N3 = N * N * N;
  const int Nx = mx * P + 1, Ny = my * P + 1;
  const long long r0 = (long long)blockIdx.x * SEL_ROWS;
  const int rows = nrows - r0 < SEL_ROWS ? (int)(nrows - r0) : SEL_ROWS;
  const int len = rows * Nx;
  auto from = [&](int e) {
    const int rl = e / Nx, gx = e - rl * Nx;
    const long long r = r0 + rl;
    const int gy = (int)(r % Ny), gz = gz0 + (int)(r / Ny);
    const int cy = gy / P < my ? gy / P : my - 1;
    const int cz = (gz > 0 && gz % P == 0) ? gz / P - 1 : gz / P;
    const int j = gy - cy * P, k = gz - cz * P;
    const int cx = gx / P < mx ? gx / P : mx - 1;
    return (((long long)cz * my + cy) * mx + cx) * N3 + (k * N + j) * N + (gx - cx * P);
  };
  // rows r0.. of layer gz0 + r / Ny are contiguous in y_unique from (gz0 Ny + r0) Nx on
  double* dst = yu + ((long long)gz0 * Ny + r0) * Nx;
  int e = threadIdx.x;
  for (; e + (HOST_U - 1) * (int)blockDim.x < len; e += HOST_U * blockDim.x) {
    double v[HOST_U];
#pragma unroll
    for (int u = 0; u < HOST_U; ++u) v[u] = __ldg(yc + from(e + u * blockDim.x));
#pragma unroll
    for (int u = 0; u < HOST_U; ++u) dst[e + u * blockDim.x] = v[u];
  }
  for (; e < len; e += blockDim.x) dst[e] = __ldg(yc + from(e));
}

// expand the cell layers [z0, z1) (from node layers z0 p .. z1 p), or select the node layers
// [z0, z1)
template <int N>
fe_status launch_expand_select(const fe_mesh* m, bool expand, const double* src, double* dst,
                               int z0, int z1, cudaStream_t st) {
  const int mx = m->d.mx, my = m->d.my, p = m->p;
  if (z1 <= z0) return FE_OK;
  if (expand) {
    const long long row = (long long)(mx * p + 1) * (my * p + 1);
    k_expand<N><<<(unsigned)((long long)my * (z1 - z0)), 256, 0, st>>>(
        src + (long long)z0 * p * row, dst + (long long)z0 * mx * my * m->n3, mx, my);
  } else {
    const long long nrows = (long long)(my * p + 1) * (z1 - z0);
    k_select<N><<<(unsigned)((nrows + SEL_ROWS - 1) / SEL_ROWS), 256, 0, st>>>(src, dst, mx, my, z0,
                                                                             nrows);
  }
  return fe_cuda_check(cudaGetLastError(), expand ? "expand launch" : "select launch");
}

fe_status expand_select(const fe_mesh* m, bool expand, const double* src, double* dst, int z0,
                        int z1, cudaStream_t st) {
  switch (m->n) {
    case 2: return launch_expand_select<2>(m, expand, src, dst, z0, z1, st);
    case 3: return launch_expand_select<3>(m, expand, src, dst, z0, z1, st);
    case 4: return launch_expand_select<4>(m, expand, src, dst, z0, z1, st);
    case 5: return launch_expand_select<5>(m, expand, src, dst, z0, z1, st);
    case 6: return launch_expand_select<6>(m, expand, src, dst, z0, z1, st);
    case 7: return launch_expand_select<7>(m, expand, src, dst, z0, z1, st);
    case 8: return launch_expand_select<8>(m, expand, src, dst, z0, z1, st);
  }
  fe_set_error("host apply: bad n");
  return FE_ERR_INVALID;
}

// The cell layers [z0, z1) of m as a mesh of their own, sharing m's memory (never freed or grown):
// vectors and geometry start z0 mx my cells in; the layers' outer faces towards the rest of m are
// interfaces, not Dirichlet boundary.
void make_view(const fe_mesh* m, int z0, int z1, fe_mesh* v) {
  *v = *m;
  const long long cells0 = (long long)z0 * m->d.mx * m->d.my;
  const long long goff = cells0 * FE_GEO_COMPS * m->n3;
  v->d.mz = z1 - z0;
  v->sgz = z1 - z0;
  v->ncells = (long long)(z1 - z0) * m->d.mx * m->d.my;
  v->ncw = v->ncells * m->n3;
  v->nu = (long long)(m->d.mx * m->p + 1) * (m->d.my * m->p + 1) * ((long long)(z1 - z0) * m->p + 1);
  v->zoff = m->zoff + z0;
  v->mzg = fe_mz_global(m);
  v->nbr_lo = m->nbr_lo || z0 > 0;
  v->nbr_hi = m->nbr_hi || z1 < m->d.mz;
  v->geo64 = m->geo64 ? m->geo64 + goff : nullptr;
  v->geodw = m->geodw ? m->geodw + goff : nullptr;
  v->geo32 = m->geo32 ? m->geo32 + goff : nullptr;
  for (int k = 0; k < 2; ++k) v->geo16[k] = m->geo16[k] ? m->geo16[k] + goff : nullptr;
  v->xyz64 = nullptr;
  v->xyzdw = nullptr;
  v->xyz32 = nullptr;
  for (void*& r : v->rc_scratch) r = nullptr;
  for (int k = 0; k < 2; ++k) {
    v->diag64[k] = nullptr;
    v->invdiag32[k] = nullptr;
    v->invdiag64[k] = nullptr;
  }
  v->invmult64 = nullptr;
  v->red = nullptr;
  v->cg_work = nullptr;
  v->cg_free = nullptr;
  v->hs_xu = v->hs_xc = v->hs_yc = v->hs_yu[0] = v->hs_yu[1] = nullptr;
  v->hs_copy = v->hs_up = nullptr;
  for (cudaEvent_t& e : v->hs_ev) e = nullptr;
}

// chunks of z-layers of a host apply: about 32 MB of unique-node output each (at most 16); the
// environment variable FE_HOST_CHUNKS overrides the count
int host_chunks(const fe_mesh* m) {
  long long k = (m->nu * (long long)sizeof(double) + (16LL << 20)) / (32LL << 20);
  if (const char* force = std::getenv("FE_HOST_CHUNKS")) k = std::atoi(force);
  if (k > 16) k = 16;
  if (k > m->d.mz) k = m->d.mz;
  if (m->d.geom_mode == FE_GEOM_RECOMPUTE) k = 1;  // recompute scratch is per mesh, not per view
  return k < 1 ? 1 : (int)k;
}

fe_status ensure_staging(fe_mesh* m, int nout) {
  if (!m->hs_copy) {
    FE_CUDA(cudaStreamCreateWithFlags(&m->hs_copy, cudaStreamNonBlocking), "host apply stream");
    FE_CUDA(cudaStreamCreateWithFlags(&m->hs_up, cudaStreamNonBlocking), "host apply stream");
    for (cudaEvent_t& e : m->hs_ev)
      FE_CUDA(cudaEventCreateWithFlags(&e, cudaEventDisableTiming), "host apply event");
  }
  if (!m->hs_xu) {
    FE_TRY(fe_dalloc((void**)&m->hs_xu, m->nu * sizeof(double), m->st, "host apply staging"));
    FE_TRY(fe_dalloc((void**)&m->hs_xc, m->ncw * sizeof(double), m->st, "host apply staging"));
    FE_TRY(fe_dalloc((void**)&m->hs_yc, m->ncw * sizeof(double), m->st, "host apply staging"));
  }
  for (int k = 0; k < nout; ++k)
    if (!m->hs_yu[k])
      FE_TRY(fe_dalloc((void**)&m->hs_yu[k], m->nu * sizeof(double), m->st, "host apply staging"));
  return fe_cuda_check(cudaStreamSynchronize(m->st), "host apply staging");
}

}  // namespace

extern "C" fe_status fe_apply_host(const fe_mesh* cm, int nop, const fe_op* ops,
                                   const double* x_unique_host, double* const* y_unique_host,
                                   unsigned flags, void* stream) {
  if (!cm || !ops || !x_unique_host || !y_unique_host || nop < 1 || nop > 2) {
    fe_set_error("fe_apply_host: null argument or nop outside [1, 2]");
    return FE_ERR_INVALID;
  }
  for (int k = 0; k < nop; ++k)
    if (!y_unique_host[k] || (ops[k] != FE_LAPLACE && ops[k] != FE_MASS)) {
      fe_set_error("fe_apply_host: output %d null or operator %d unknown", k, (int)ops[k]);
      return FE_ERR_INVALID;
    }
  if (flags & ~FE_NATIVE_F64) {
    fe_set_error("fe_apply_host: flags 0x%x (only FE_NATIVE_F64 is accepted)", flags);
    return FE_ERR_INVALID;
  }
  if (cm->packed) {
    fe_set_error("fe_apply_host: FE_LAYOUT_CELLS meshes only");
    return FE_ERR_INVALID;
  }
  fe_mesh* m = const_cast<fe_mesh*>(cm);
  FeDeviceGuard device_guard;
  FE_CUDA(device_guard.set(m->d.device), "cudaSetDevice");
  FE_TRY(ensure_staging(m, nop));
  FE_TRY(fe_ensure_geometry(m, FE_F64, (flags & FE_NATIVE_F64) != 0));
  cudaStream_t st = (cudaStream_t)stream;
  const int mz = m->d.mz, p = m->p, K = host_chunks(m);
  const long long row = (long long)(m->d.mx * p + 1) * (m->d.my * p + 1);  // nodes per node layer
  const size_t rb = (size_t)row * sizeof(double);
  int zb[17];
  for (int c = 0; c <= K; ++c) zb[c] = (int)((long long)c * mz / K);
  cudaEvent_t* ev = m->hs_ev;  // [0] start, [1] done, [2 + c] uploads, [18 + 16 k + c] read-backs
  // the uploads follow what the caller's stream holds (an earlier call still expanding)
  FE_CUDA(cudaEventRecord(ev[0], st), "host apply event");
  FE_CUDA(cudaStreamWaitEvent(m->hs_up, ev[0], 0), "host apply wait");
  int up_end = 0;  // node layers uploaded
  for (int k = 0; k < nop; ++k) {
    int sel_end = 0;  // node layers selected
    for (int c = 0; c < K; ++c) {
      const int z0 = zb[c], z1 = zb[c + 1];
      fe_mesh view;
      if (k == 0) {  // x: the node layers this chunk's cells read, uploaded on their own stream
        const int need = z1 * p + 1;
        FE_CUDA(cudaMemcpyAsync(m->hs_xu + (size_t)up_end * row, x_unique_host + (size_t)up_end * row,
                                (size_t)(need - up_end) * rb, cudaMemcpyHostToDevice, m->hs_up),
                "fe_apply_host: input copy");
        up_end = need;
        FE_CUDA(cudaEventRecord(ev[2 + c], m->hs_up), "host apply event");
        FE_CUDA(cudaStreamWaitEvent(st, ev[2 + c], 0), "host apply wait");
        FE_TRY(expand_select(m, true, m->hs_xu, m->hs_xc, z0, z1, st));
      }
      // the chunk's assembled apply, DSS passes ordered as on the whole mesh: the z-pass inside
      // the chunk and across its lower interface, then the y- and x-passes of every layer whose
      // z-sums are complete (the chunk's last layer waits for the next chunk)
      make_view(m, z0, z1, &view);
      const long long cell0 = (long long)z0 * m->d.mx * m->d.my * m->n3;
      int brick[2] = {1, 1};
      // one chunk: the mesh itself (recompute-mode meshes keep their coordinates and scratch)
      ApplyLaunch L{K == 1 ? m : &view, (int)ops[k], m->hs_xc + cell0, m->hs_yc + cell0, st,
                    nullptr, true, brick};  // the kernels need 8-byte alignment only
      FE_TRY((flags & FE_NATIVE_F64) ? fe_launch_apply_f64native(L) : fe_launch_apply_f64dw(L));
      FE_TRY(fe_launch_dss_axes(&view, FE_F64, m->hs_yc + cell0, brick[0], brick[1], 2, 2, st));
      if (c > 0) {
        make_view(m, z0 - 1, z0 + 1, &view);
        FE_TRY(fe_launch_dss_axes(&view, FE_F64, m->hs_yc + cell0 - (long long)m->d.mx * m->d.my * m->n3,
                                  1, 1, 2, 2, st));
      }
      const int ylo = c > 0 ? z0 - 1 : 0, yhi = c < K - 1 ? z1 - 1 : z1;
      if (yhi > ylo) {
        make_view(m, ylo, yhi, &view);
        FE_TRY(fe_launch_dss_axes(&view, FE_F64,
                                  m->hs_yc + (long long)ylo * m->d.mx * m->d.my * m->n3, brick[0],
                                  brick[1], 1, 0, st));
      }
      // the node layers now final, read back on the copy stream under the next chunk's work
      const int sel_hi = c < K - 1 ? (z1 - 1) * p + 1 : mz * p + 1;
      if (sel_hi > sel_end) {
        FE_TRY(expand_select(m, false, m->hs_yc, m->hs_yu[k], sel_end, sel_hi, st));
        cudaEvent_t e = ev[18 + 16 * k + c];
        FE_CUDA(cudaEventRecord(e, st), "host apply event");
        FE_CUDA(cudaStreamWaitEvent(m->hs_copy, e, 0), "host apply wait");
        FE_CUDA(cudaMemcpyAsync(y_unique_host[k] + (size_t)sel_end * row,
                                m->hs_yu[k] + (size_t)sel_end * row,
                                (size_t)(sel_hi - sel_end) * rb, cudaMemcpyDeviceToHost, m->hs_copy),
                "fe_apply_host: output copy");
        sel_end = sel_hi;
      }
    }
  }
  // the caller's stream reaches the end of the call once the read-backs are done
  FE_CUDA(cudaEventRecord(ev[1], m->hs_copy), "host apply event");
  FE_CUDA(cudaStreamWaitEvent(st, ev[1], 0), "host apply wait");
  return FE_OK;
}
