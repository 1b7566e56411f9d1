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
#include "fe_internal.h"

namespace {

// One CTA per row of cells along x (expand) or row of nodes along x (select): the row's
// coordinates and 64-bit offsets are formed once per CTA, the threads of the row use 32-bit
// arithmetic with compile-time divisors.

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
  for (int e = threadIdx.x; e < len; e += blockDim.x) {
    const int cx = e / N3, loc = e - cx * N3;
    const int k = loc / N2, j = (loc / N) % N, i = loc % N;
    dst[e] = __ldg(src + (k * Ny + j) * Nx + cx * P + i);
  }
}

// y_unique[g] = the copy of node g in the lowest cell holding it (all copies are equal after the
// DSS), for the nodes of row r = gz Ny + gy
template <int N>
__global__ void __launch_bounds__(256) k_select(const double* __restrict__ yc,
                                                double* __restrict__ yu, int mx, int my, int mz) {
  constexpr int P = N - 1, N3 = N * N * N;
  const int Nx = mx * P + 1, Ny = my * P + 1;
  const long long r = blockIdx.x;
  const int gy = (int)(r % Ny), gz = (int)(r / Ny);
  const int cy = gy / P < my ? gy / P : my - 1, cz = gz / P < mz ? gz / P : mz - 1;
  const int j = gy - cy * P, k = gz - cz * P;
  const double* src = yc + ((long long)cz * my + cy) * mx * N3 + (k * N + j) * N;
  double* dst = yu + r * Nx;
  for (int gx = threadIdx.x; gx < Nx; gx += blockDim.x) {
    const int cx = gx / P < mx ? gx / P : mx - 1;
    dst[gx] = __ldg(src + (long long)cx * N3 + (gx - cx * P));
  }
}

template <int N>
fe_status launch_expand_select(const fe_mesh* m, bool expand, const double* src, double* dst,
                               cudaStream_t st) {
  const int mx = m->d.mx, my = m->d.my, mz = m->d.mz, p = m->p;
  if (expand)
    k_expand<N><<<(unsigned)((long long)my * mz), 256, 0, st>>>(src, dst, mx, my);
  else
    k_select<N><<<(unsigned)((long long)(my * p + 1) * (mz * p + 1)), 256, 0, st>>>(src, dst, mx,
                                                                                   my, mz);
  return fe_cuda_check(cudaGetLastError(), expand ? "expand launch" : "select launch");
}

fe_status expand_select(const fe_mesh* m, bool expand, const double* src, double* dst,
                        cudaStream_t st) {
  switch (m->n) {
    case 2: return launch_expand_select<2>(m, expand, src, dst, st);
    case 3: return launch_expand_select<3>(m, expand, src, dst, st);
    case 4: return launch_expand_select<4>(m, expand, src, dst, st);
    case 5: return launch_expand_select<5>(m, expand, src, dst, st);
    case 6: return launch_expand_select<6>(m, expand, src, dst, st);
    case 7: return launch_expand_select<7>(m, expand, src, dst, st);
    case 8: return launch_expand_select<8>(m, expand, src, dst, st);
  }
  fe_set_error("host apply: bad n");
  return FE_ERR_INVALID;
}

fe_status ensure_staging(fe_mesh* m, int nout) {
  if (!m->hs_copy) {
    FE_CUDA(cudaStreamCreateWithFlags(&m->hs_copy, cudaStreamNonBlocking), "host apply stream");
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
  FE_CUDA(cudaSetDevice(m->d.device), "cudaSetDevice");
  FE_TRY(ensure_staging(m, nop));
  cudaStream_t st = (cudaStream_t)stream;
  const size_t ubytes = (size_t)m->nu * sizeof(double);
  FE_CUDA(cudaMemcpyAsync(m->hs_xu, x_unique_host, ubytes, cudaMemcpyHostToDevice, st),
          "fe_apply_host: input copy");
  FE_TRY(expand_select(m, true, m->hs_xu, m->hs_xc, st));
  for (int k = 0; k < nop; ++k) {
    FE_TRY(fe_apply_impl(m, ops[k], FE_F64, m->hs_xc, m->hs_yc, FE_ASSEMBLE | flags, stream,
                         nullptr));
    FE_TRY(expand_select(m, false, m->hs_yc, m->hs_yu[k], st));
    // read-back on the copy stream, overlapping the next operator's apply
    FE_CUDA(cudaEventRecord(m->hs_ev[k], st), "host apply event");
    FE_CUDA(cudaStreamWaitEvent(m->hs_copy, m->hs_ev[k], 0), "host apply wait");
    FE_CUDA(cudaMemcpyAsync(y_unique_host[k], m->hs_yu[k], ubytes, cudaMemcpyDeviceToHost,
                            m->hs_copy),
            "fe_apply_host: output copy");
  }
  // the caller's stream reaches the end of the call once the read-backs are done
  FE_CUDA(cudaEventRecord(m->hs_ev[2], m->hs_copy), "host apply event");
  FE_CUDA(cudaStreamWaitEvent(st, m->hs_ev[2], 0), "host apply wait");
  return FE_OK;
}
