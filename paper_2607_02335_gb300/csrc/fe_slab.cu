// fe_slab.cu -- slab decomposition of a structured mesh: interface planes, the DSS with one plane
// exchange (Sec. 4.1's structured DSS across slabs), and PCG over slabs with one scalar collective
// per iteration.
//
// A slab is an fe_mesh of whole z-layers of a larger mesh (fe_mesh_create_impl with z0 < z1):
// geometry and Dirichlet faces follow the whole mesh, and its interface planes are summed with the
// neighbouring slab's copies by the caller's fe_comm.  The structured DSS runs its passes in the
// order z, y, x; across slabs the exchange sits between the z-pass and the y-pass, where an
// interface node's two z-copies (one per slab) form one pair: each slab adds the neighbour's copy
// to its own, and the y- and x-passes then proceed as on the whole mesh.  Every node therefore gets
// the same pair sums in the same order as with the whole mesh's DSS, bit for bit.
//
// PCG (Sec. 3.2 with the Jacobi preconditioner P = D^{-1} S of Sec. 3.3) in the single-reduction
// form of Chronopoulos and Gear (1989): with z = P r and s = A z,
//   gamma = <r,z>, delta = <s,z>, rho = sum w^2 / mult (w = S r),
//   beta = gamma / gamma_old, alpha = gamma / (delta - beta gamma / alpha_old),
//   p = z + beta p, q = s + beta q (= A p), x += alpha p, r -= alpha q,
// equal to the two-reduction iteration of fe_cg.cu in exact arithmetic.  All three pairings come
// after the DSS and the apply of one iteration, so the slabs exchange them in one allgather; every
// slab sums the gathered values in rank order and takes the same decisions.
#include <cmath>
#include <cstring>
#include <vector>

#include "fe_cgcore.h"
#include "fe_vec.cuh"

namespace {

unsigned grid_for(long long n) {
  long long b = (n + 255) / 256;
  if (b > 152LL * 16) b = 152LL * 16;
  return (unsigned)(b < 1 ? 1 : b);
}

// ---- interface planes --------------------------------------------------------------------------
// plane entry e = ((cy mx + cx) n + j) n + i  <->  node (i, j, k) of cell cell0 + cy mx + cx
template <class S>
__global__ void k_face_pack(const S* __restrict__ v, S* __restrict__ plane, long long cell0, int n,
                            int k, long long count) {
  const int n2 = n * n, n3 = n2 * n;
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < count;
       e += (long long)gridDim.x * blockDim.x) {
    const long long c = e / n2;
    const int ij = (int)(e - c * n2);
    plane[e] = v[(cell0 + c) * n3 + k * n2 + ij];
  }
}

template <class S>
__global__ void k_face_add(S* __restrict__ v, const S* __restrict__ plane, long long cell0, int n,
                           int k, long long count) {
  const int n2 = n * n, n3 = n2 * n;
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < count;
       e += (long long)gridDim.x * blockDim.x) {
    const long long c = e / n2;
    const int ij = (int)(e - c * n2);
    S* dst = v + (cell0 + c) * n3 + k * n2 + ij;
    *dst = *dst + plane[e];
  }
}

long long plane_len(const fe_mesh* m) { return (long long)m->d.mx * m->d.my * m->n * m->n; }

fe_status face_op(const fe_mesh* m, int prec, void* v, int side, void* plane, bool add,
                  cudaStream_t st) {
  const long long count = plane_len(m);
  const long long cell0 = side == 0 ? 0 : (long long)(m->d.mz - 1) * m->d.mx * m->d.my;
  const int k = side == 0 ? 0 : m->p;
  const unsigned g = grid_for(count);
  if (prec == FE_F64) {
    if (add)
      k_face_add<double><<<g, 256, 0, st>>>((double*)v, (const double*)plane, cell0, m->n, k, count);
    else
      k_face_pack<double><<<g, 256, 0, st>>>((const double*)v, (double*)plane, cell0, m->n, k, count);
  } else {
    if (add)
      k_face_add<float><<<g, 256, 0, st>>>((float*)v, (const float*)plane, cell0, m->n, k, count);
    else
      k_face_pack<float><<<g, 256, 0, st>>>((const float*)v, (float*)plane, cell0, m->n, k, count);
  }
  return fe_cuda_check(cudaGetLastError(), add ? "face add launch" : "face pack launch");
}

int slab_sides(const fe_mesh* m) { return (m->nbr_lo ? 1 : 0) | (m->nbr_hi ? 2 : 0); }

fe_status check_slab(const fe_mesh* m, const char* what) {
  if (!m) {
    fe_set_error("%s: null mesh", what);
    return FE_ERR_INVALID;
  }
  if (m->mzg <= 0) {
    fe_set_error("%s: not a slab (create it with fe_slab_create)", what);
    return FE_ERR_INVALID;
  }
  return FE_OK;
}

fe_status check_comm(const fe_mesh* m, const fe_comm* c, bool reduce, const char* what) {
  if (!c) {
    fe_set_error("%s: null comm", what);
    return FE_ERR_INVALID;
  }
  if (c->size < 1 || c->rank < 0 || c->rank >= c->size || (c->rank == 0) != !m->nbr_lo ||
      (c->rank == c->size - 1) != !m->nbr_hi) {
    fe_set_error("%s: comm rank %d of %d does not match the slab (neighbour below %d, above %d)",
                 what, c->rank, c->size, (int)m->nbr_lo, (int)m->nbr_hi);
    return FE_ERR_INVALID;
  }
  const int sides = slab_sides(m);
  if (sides && !c->exchange) {
    fe_set_error("%s: comm has no exchange callback", what);
    return FE_ERR_INVALID;
  }
  for (int s = 0; s < 2; ++s)
    if ((sides >> s) & 1) {
      if (!c->send[s] || !c->recv[s] || !fe_aligned(c->send[s]) || !fe_aligned(c->recv[s])) {
        fe_set_error("%s: comm plane buffers of side %d null or not 16-byte aligned", what, s);
        return FE_ERR_INVALID;
      }
    }
  if (reduce && (!c->red_send || !c->red_all || (c->size > 1 && !c->allgather))) {
    fe_set_error("%s: comm needs red_send, red_all and an allgather callback", what);
    return FE_ERR_INVALID;
  }
  return FE_OK;
}

// add the neighbours' copies of the interface planes to v
fe_status exchange_planes(const fe_mesh* m, int prec, void* v, const fe_comm* c, cudaStream_t st) {
  const int sides = slab_sides(m);
  if (!sides) return FE_OK;
  for (int s = 0; s < 2; ++s)
    if ((sides >> s) & 1) FE_TRY(face_op(m, prec, v, s, c->send[s], false, st));
  const int eb = prec == FE_F64 ? (int)sizeof(double) : (int)sizeof(float);
  if (c->exchange(c->ctx, sides, eb, plane_len(m), (void*)st) != 0) {
    fe_set_error("slab exchange callback failed");
    return FE_ERR_COMM;
  }
  for (int s = 0; s < 2; ++s)
    if ((sides >> s) & 1) FE_TRY(face_op(m, prec, v, s, c->recv[s], true, st));
  return FE_OK;
}

// the DSS of v over all slabs: the z-pass inside the slab, the plane exchange (which completes the
// z-pairs across the interfaces), then the y- and x-passes (between bricks of bx x by cells after a
// brick-fused apply).  Every node gets the pair sums of the whole mesh's DSS in the same order.
fe_status slab_dss_passes(const fe_mesh* m, int prec, void* v, int bx, int by, const fe_comm* c,
                          cudaStream_t st) {
  FE_TRY(fe_launch_dss_axes(m, prec, v, bx, by, 2, 2, st));
  FE_TRY(exchange_planes(m, prec, v, c, st));
  return fe_launch_dss_axes(m, prec, v, bx, by, 1, 0, st);
}

fe_status allgather(const fe_comm* c, int n, cudaStream_t st) {
  if (c->size == 1)
    return fe_cuda_check(cudaMemcpyAsync(c->red_all, c->red_send, n * sizeof(double),
                                         cudaMemcpyDeviceToDevice, st),
                         "allgather copy");
  if (c->allgather(c->ctx, n, (void*)st) != 0) {
    fe_set_error("slab allgather callback failed");
    return FE_ERR_COMM;
  }
  return FE_OK;
}

// ---- PCG kernels -------------------------------------------------------------------------------
__device__ __forceinline__ dw prod(double a, double b) {
  return dw_mul(dw_from_double(a), dw_from_double(b));
}

__global__ void k_sub(const double* __restrict__ b, const double* __restrict__ s,
                      double* __restrict__ r, long long n) {
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < n;
       e += (long long)gridDim.x * blockDim.x)
    r[e] = b[e] - s[e];
}

__global__ void k_invdiag(const double* __restrict__ d, const float* __restrict__ invmult,
                          double* __restrict__ inv, long long n) {
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < n;
       e += (long long)gridDim.x * blockDim.x)
    inv[e] = invmult[e] == 0.0f ? 0.0 : 1.0 / d[e];
}

// slot 0: sum w^2 / mult; with z: z = w / diag (0 on Dirichlet nodes), slot 1: <r, z>
__global__ void __launch_bounds__(RED_THREADS)
    k_precond(const double* __restrict__ w, const double* __restrict__ r,
              const double* __restrict__ invdiag, const float* __restrict__ invmult,
              double* __restrict__ z, double* __restrict__ partials, const CgScal* __restrict__ sc,
              long long n) {
  if (*(volatile const int*)&sc->done) return;
  __shared__ dw sh[32];
  dw a0 = {0.0f, 0.0f}, a1 = {0.0f, 0.0f};
  for (long long e = (long long)blockIdx.x * RED_THREADS + threadIdx.x; e < n;
       e += (long long)RED_BLOCKS * RED_THREADS) {
    const double we = w[e];
    const dw w2 = prod(we, we);
    const float im = invmult[e];  // a power of two or zero: exact scaling
    a0 = dw_add(a0, {w2.h * im, w2.l * im});
    if (z) {
      const double ze = we * invdiag[e];
      z[e] = ze;
      a1 = dw_add(a1, prod(r[e], ze));
    }
  }
  a0 = block_reduce_dw(a0, sh);
  if (threadIdx.x == 0) partials[blockIdx.x] = dw_to_double(a0);
  if (z) {
    a1 = block_reduce_dw(a1, sh);
    if (threadIdx.x == 0) partials[RED_BLOCKS + blockIdx.x] = dw_to_double(a1);
  }
}

// slot 2: <s, z>
__global__ void __launch_bounds__(RED_THREADS)
    k_dot(const double* __restrict__ s, const double* __restrict__ z, double* __restrict__ partials,
          const CgScal* __restrict__ sc, long long n) {
  if (*(volatile const int*)&sc->done) return;
  __shared__ dw sh[32];
  dw a = {0.0f, 0.0f};
  for (long long e = (long long)blockIdx.x * RED_THREADS + threadIdx.x; e < n;
       e += (long long)RED_BLOCKS * RED_THREADS)
    a = dw_add(a, prod(s[e], z[e]));
  a = block_reduce_dw(a, sh);
  if (threadIdx.x == 0) partials[2 * RED_BLOCKS + blockIdx.x] = dw_to_double(a);
}

// this slab's sums of the first `nslots` slots, in a fixed order, into red_send
__global__ void __launch_bounds__(RED_THREADS)
    k_local_sums(const double* __restrict__ partials, int nslots, double* __restrict__ red_send) {
  __shared__ dw sh[32];
  for (int s = 0; s < nslots; ++s) {
    dw acc = {0.0f, 0.0f};
    for (int b = threadIdx.x; b < RED_BLOCKS; b += RED_THREADS)
      acc = dw_add(acc, dw_from_double(partials[s * RED_BLOCKS + b]));
    acc = block_reduce_dw(acc, sh);
    if (threadIdx.x == 0) red_send[s] = dw_to_double(acc);
  }
}

// sums over the slabs in rank order, then the scalar logic (one thread)
__global__ void k_fin(const double* __restrict__ red_all, int size, int nslots, CgScal* sc,
                      double rtol, int mode, double* hist) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  if (mode == FIN_ITER && sc->done) return;
  dw acc[3] = {{0.0f, 0.0f}, {0.0f, 0.0f}, {0.0f, 0.0f}};
  for (int r = 0; r < size; ++r)
    for (int s = 0; s < nslots; ++s) acc[s] = dw_add(acc[s], dw_from_double(red_all[r * nslots + s]));
  const double rho = dw_to_double(acc[0]), gamma = dw_to_double(acc[1]),
               delta = dw_to_double(acc[2]);
  if (mode == FIN_INIT_B) {
    fin_scalars(sc, rho, 0.0, 0.0, rtol, FIN_INIT_B, 0);
    return;
  }
  const int k = sc->iter;
  const double alpha_used = sc->alpha;
  fin_scalars(sc, rho, gamma, 0.0, rtol, mode, 0);  // FIN_ITER: beta = gamma / gamma_old
  if (mode == FIN_ITER && hist) {
    hist[3 * k + 0] = alpha_used;
    hist[3 * k + 2] = sc->relres;
  }
  if (sc->done) return;
  double den = delta;
  if (mode == FIN_INIT_R)
    sc->beta = 0.0;
  else
    den = delta - sc->beta * gamma / alpha_used;
  if (!(den > 0.0) || !isfinite(den) || !isfinite(gamma)) {
    sc->status = FE_ERR_BREAKDOWN;
    sc->done = 1;
    return;
  }
  sc->alpha = gamma / den;
  if (mode == FIN_ITER && hist) hist[3 * k + 1] = sc->beta;
}

// p = z + beta p, q = s + beta q, x += alpha p, r -= alpha q
__global__ void k_update(double* __restrict__ x, double* __restrict__ r, double* __restrict__ p,
                         double* __restrict__ q, const double* __restrict__ z,
                         const double* __restrict__ s, const CgScal* __restrict__ sc, long long n) {
  if (*(volatile const int*)&sc->done) return;
  const double alpha = sc->alpha, beta = sc->beta;
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < n;
       e += (long long)gridDim.x * blockDim.x) {
    const double pe = z[e] + beta * p[e], qe = s[e] + beta * q[e];
    p[e] = pe;
    q[e] = qe;
    x[e] += alpha * pe;
    r[e] -= alpha * qe;
  }
}

struct SlabWork {
  double *r = nullptr, *w = nullptr, *z = nullptr, *s = nullptr, *p = nullptr, *q = nullptr,
         *invdiag = nullptr, *partials = nullptr, *hist = nullptr, *bs = nullptr;
  float* invmult = nullptr;
  CgScal* sc = nullptr;
  CgScal* hsc = nullptr;
  cudaStream_t st = nullptr;
  ~SlabWork() {
    void* bufs[] = {r, w, z, s, p, q, invdiag, partials, hist, bs, invmult, sc};
    for (void* b : bufs) fe_dfree(b, st);
    if (st) cudaStreamSynchronize(st);
    if (hsc) cudaFreeHost(hsc);
  }
};

// w = S r across the slabs, then the preconditioner and its pairings, s = A z and <s,z>, one
// allgather, and the scalar step `mode`
fe_status tail(const fe_mesh* m, SlabWork& W, const fe_comm* c, double rtol, int mode,
               double* hist) {
  const long long n = m->ncw;
  cudaStream_t st = W.st;
  FE_CUDA(cudaMemcpyAsync(W.w, W.r, n * sizeof(double), cudaMemcpyDeviceToDevice, st), "copy");
  FE_TRY(slab_dss_passes(m, FE_F64, W.w, 1, 1, c, st));
  k_precond<<<RED_BLOCKS, RED_THREADS, 0, st>>>(W.w, W.r, W.invdiag, W.invmult, W.z, W.partials,
                                                W.sc, n);
  FE_CUDA(cudaGetLastError(), "precond launch");
  ApplyLaunch L{m, FE_LAPLACE, W.z, W.s, st, &W.sc->done};
  FE_TRY(fe_launch_apply_f64dw(L));
  k_dot<<<RED_BLOCKS, RED_THREADS, 0, st>>>(W.s, W.z, W.partials, W.sc, n);
  k_local_sums<<<1, RED_THREADS, 0, st>>>(W.partials, 3, c->red_send);
  FE_CUDA(cudaGetLastError(), "pairing launch");
  FE_TRY(allgather(c, 3, st));
  k_fin<<<1, 32, 0, st>>>(c->red_all, c->size, 3, W.sc, rtol, mode, hist);
  return fe_cuda_check(cudaGetLastError(), "scalar launch");
}

fe_status read_scal(SlabWork& W, CgScal* out) {
  FE_CUDA(cudaMemcpyAsync(W.hsc, W.sc, sizeof(CgScal), cudaMemcpyDeviceToHost, W.st), "scal read");
  FE_CUDA(cudaStreamSynchronize(W.st), "scal synchronize");
  *out = *W.hsc;
  return FE_OK;
}

}  // namespace

extern "C" fe_status fe_slab_create(const fe_slab_desc* desc, void* stream, fe_mesh** out) {
  if (!desc || !out) {
    fe_set_error("fe_slab_create: null argument");
    return FE_ERR_INVALID;
  }
  if (desc->z1 <= 0) {
    fe_set_error("fe_slab_create: need 0 <= z0 < z1 <= mz (%d, %d)", desc->z0, desc->z1);
    return FE_ERR_INVALID;
  }
  return fe_mesh_create_impl(&desc->global, nullptr, stream, out, desc->z0, desc->z1);
}

extern "C" fe_status fe_slab_plane_len(const fe_mesh* m, long long* count) {
  FE_TRY(check_slab(m, "fe_slab_plane_len"));
  if (!count) {
    fe_set_error("fe_slab_plane_len: null argument");
    return FE_ERR_INVALID;
  }
  *count = plane_len(m);
  return FE_OK;
}

static fe_status face_call(const fe_mesh* m, fe_prec prec, const void* v, int side,
                           const void* plane, bool add, void* stream, const char* what) {
  FE_TRY(check_slab(m, what));
  if (!v || !plane || !fe_aligned(v) || !fe_aligned(plane) || (side != 0 && side != 1) ||
      (prec != FE_F64 && prec != FE_F32)) {
    fe_set_error("%s: null or misaligned vector, side not 0/1, or precision not FE_F64/FE_F32",
                 what);
    return FE_ERR_INVALID;
  }
  FeDeviceGuard device_guard;
  FE_CUDA(device_guard.set(m->d.device), "cudaSetDevice");
  return face_op(m, (int)prec, const_cast<void*>(v), side, const_cast<void*>(plane), add,
                 (cudaStream_t)stream);
}

extern "C" fe_status fe_slab_face_pack(const fe_mesh* m, fe_prec prec, const void* v, int side,
                                       void* plane, void* stream) {
  return face_call(m, prec, v, side, plane, false, stream, "fe_slab_face_pack");
}

extern "C" fe_status fe_slab_face_add(const fe_mesh* m, fe_prec prec, void* v, int side,
                                      const void* plane, void* stream) {
  return face_call(m, prec, v, side, plane, true, stream, "fe_slab_face_add");
}

extern "C" fe_status fe_slab_dss(const fe_mesh* m, fe_prec prec, const void* r, void* z,
                                 const fe_comm* comm, void* stream) {
  FE_TRY(check_slab(m, "fe_slab_dss"));
  FE_TRY(check_comm(m, comm, false, "fe_slab_dss"));
  if (!r || !z || !fe_aligned(r) || !fe_aligned(z) || (prec != FE_F64 && prec != FE_F32)) {
    fe_set_error("fe_slab_dss: null or misaligned vector, or precision not FE_F64/FE_F32");
    return FE_ERR_INVALID;
  }
  FeDeviceGuard device_guard;
  FE_CUDA(device_guard.set(m->d.device), "cudaSetDevice");
  cudaStream_t st = (cudaStream_t)stream;
  if (r != z)
    FE_CUDA(cudaMemcpyAsync(z, r, (size_t)m->ncw * (prec == FE_F64 ? 8 : 4),
                            cudaMemcpyDeviceToDevice, st),
            "fe_slab_dss copy");
  return slab_dss_passes(m, (int)prec, z, 1, 1, comm, st);
}

extern "C" fe_status fe_slab_apply(const fe_mesh* m, fe_op op, fe_prec prec, const void* x, void* y,
                                   unsigned flags, const fe_comm* comm, void* stream) {
  FE_TRY(check_slab(m, "fe_slab_apply"));
  if (!(flags & FE_ASSEMBLE)) return fe_apply(m, op, prec, x, y, flags, stream);
  FE_TRY(check_comm(m, comm, false, "fe_slab_apply"));
  int brick[2] = {1, 1};  // the kernel's in-brick sums; the passes follow here
  FE_TRY(fe_apply_impl(m, op, prec, x, y, flags, stream, brick));
  return slab_dss_passes(m, prec == FE_F64 ? FE_F64 : FE_F32, y, brick[0], brick[1], comm,
                         (cudaStream_t)stream);
}

extern "C" fe_status fe_slab_cg_solve(const fe_mesh* m, const double* b, double* x,
                                      const fe_cg_opts* opts, const fe_comm* comm,
                                      fe_cg_result* res, void* stream) {
  FE_TRY(check_slab(m, "fe_slab_cg_solve"));
  if (!b || !x || !opts || !res || !fe_aligned(b) || !fe_aligned(x)) {
    fe_set_error("fe_slab_cg_solve: null or misaligned argument");
    return FE_ERR_INVALID;
  }
  if (opts->maxit < 1 || !(opts->rtol >= 0.0) || opts->mixed != 0 || opts->flexible != 0) {
    fe_set_error("fe_slab_cg_solve: invalid options (maxit %d, rtol %g, mixed %d, flexible %d)",
                 opts->maxit, opts->rtol, opts->mixed, opts->flexible);
    return FE_ERR_INVALID;
  }
  FE_TRY(check_comm(m, comm, true, "fe_slab_cg_solve"));
  std::memset(res, 0, sizeof(*res));
  FeDeviceGuard device_guard;
  FE_CUDA(device_guard.set(m->d.device), "cudaSetDevice");
  FE_TRY(fe_ensure_geometry(m, FE_F64, false));
  const long long n = m->ncw;
  SlabWork W;
  W.st = (cudaStream_t)stream;
  cudaStream_t st = W.st;
  double** vecs[] = {&W.r, &W.w, &W.z, &W.s, &W.p, &W.q, &W.invdiag, &W.bs};
  for (double** v : vecs) FE_TRY(fe_dalloc((void**)v, n * sizeof(double), st, "slab cg vector"));
  FE_TRY(fe_dalloc((void**)&W.invmult, n * sizeof(float), st, "slab cg vector"));
  FE_TRY(fe_dalloc((void**)&W.partials, 3 * RED_BLOCKS * sizeof(double), st, "slab cg partials"));
  FE_TRY(fe_dalloc((void**)&W.sc, sizeof(CgScal), st, "slab cg scalars"));
  if (opts->history)
    FE_TRY(fe_dalloc((void**)&W.hist, 3 * (size_t)opts->maxit * sizeof(double), st, "history"));
  FE_CUDA(cudaMallocHost(&W.hsc, sizeof(CgScal)), "cudaMallocHost slab cg scalars");

  // 1 / multiplicity and the Jacobi diagonal assembled across the interfaces
  FE_TRY(fe_launch_invmult(m, W.invmult, st));
  FE_TRY(fe_launch_diag(m, FE_LAPLACE, W.w, st));
  FE_TRY(exchange_planes(m, FE_F64, W.w, comm, st));
  k_invdiag<<<grid_for(n), 256, 0, st>>>(W.w, W.invmult, W.invdiag, n);
  FE_CUDA(cudaMemsetAsync(W.p, 0, n * sizeof(double), st), "zero p");
  FE_CUDA(cudaMemsetAsync(W.q, 0, n * sizeof(double), st), "zero q");
  CgScal h;
  std::memset(&h, 0, sizeof(h));
  h.maxit = opts->maxit;
  FE_CUDA(cudaMemcpyAsync(W.sc, &h, sizeof(CgScal), cudaMemcpyHostToDevice, st), "scal init");

  // The system scaled by an exact power of two from the largest |b| over all slabs (as
  // fe_cg_solve: the pairings' double-word sums have FP32's exponent range): b := sb b, x := sb x
  double sb = 1.0;
  {
    unsigned long long* d = reinterpret_cast<unsigned long long*>(W.partials);
    FE_TRY(fe_launch_absmax(b, n, d, st));
    // the bits of a non-negative double are the double: one slot of the scalar allgather
    FE_CUDA(cudaMemcpyAsync(comm->red_send, d, sizeof(double), cudaMemcpyDeviceToDevice, st),
            "scale copy");
    FE_TRY(allgather(comm, 1, st));
    std::vector<double> all(comm->size > 0 ? comm->size : 1);
    FE_CUDA(cudaMemcpyAsync(all.data(), comm->red_all, all.size() * sizeof(double),
                            cudaMemcpyDeviceToHost, st),
            "scale readback");
    FE_CUDA(cudaStreamSynchronize(st), "scale readback");
    double mx = 0.0;
    for (double v : all) mx = v > mx || v != v ? v : mx;
    if (!fe_scale_of_max(mx, &sb)) {
      fe_set_error("fe_slab_cg_solve: the right-hand side holds a non-finite value");
      return FE_ERR_INVALID;
    }
    FE_TRY(fe_cg_scale(b, W.bs, sb, n, st));
    FE_TRY(fe_cg_scale(x, x, sb, n, st));
    b = W.bs;
  }

  // ||G^T b||^2 over the whole mesh
  FE_CUDA(cudaMemcpyAsync(W.w, b, n * sizeof(double), cudaMemcpyDeviceToDevice, st), "copy");
  FE_TRY(slab_dss_passes(m, FE_F64, W.w, 1, 1, comm, st));
  k_precond<<<RED_BLOCKS, RED_THREADS, 0, st>>>(W.w, nullptr, nullptr, W.invmult, nullptr,
                                                W.partials, W.sc, n);
  k_local_sums<<<1, RED_THREADS, 0, st>>>(W.partials, 1, comm->red_send);
  FE_CUDA(cudaGetLastError(), "norm launch");
  FE_TRY(allgather(comm, 1, st));
  k_fin<<<1, 32, 0, st>>>(comm->red_all, comm->size, 1, W.sc, opts->rtol, FIN_INIT_B, nullptr);
  FE_TRY(read_scal(W, &h));
  if (!(h.bnorm2 > 0.0)) {  // zero right-hand side on every slab: the solution is zero
    FE_CUDA(cudaMemsetAsync(x, 0, n * sizeof(double), st), "zero x");
    FE_CUDA(cudaStreamSynchronize(st), "synchronize");
    res->status = FE_OK;
    return FE_OK;
  }

  // r = b - A x, then z, s = A z and the first scalars
  {
    ApplyLaunch L{m, FE_LAPLACE, x, W.s, st, nullptr};
    FE_TRY(fe_launch_apply_f64dw(L));
    k_sub<<<grid_for(n), 256, 0, st>>>(b, W.s, W.r, n);
    FE_CUDA(cudaGetLastError(), "residual launch");
  }
  FE_TRY(tail(m, W, comm, opts->rtol, FIN_INIT_R, W.hist));
  FE_TRY(read_scal(W, &h));
  // Every slab reads the same flag after the same number of iterations (the scalars are equal
  // on all slabs), so the loops end together; iterations past convergence are no-ops.
  constexpr int CHECK_EVERY = 4;
  for (int it = 0; !h.done; ++it) {
    k_update<<<grid_for(n), 256, 0, st>>>(x, W.r, W.p, W.q, W.z, W.s, W.sc, n);
    FE_CUDA(cudaGetLastError(), "update launch");
    FE_TRY(tail(m, W, comm, opts->rtol, FIN_ITER, W.hist));
    if ((it + 1) % CHECK_EVERY == 0 || it + 1 >= opts->maxit) FE_TRY(read_scal(W, &h));
    if (!h.done && it + 1 >= opts->maxit) {  // the scalar step stops at maxit
      fe_set_error("fe_slab_cg_solve: iteration did not stop at maxit");
      return FE_ERR_CUDA;
    }
  }
  FE_TRY(fe_cg_scale(x, x, 1.0 / sb, n, st));  // 1/sb: a power of two, exact
  FE_CUDA(cudaStreamSynchronize(st), "synchronize");
  res->iters = h.iter;
  res->outer_iters = 1;
  res->rel_res = h.relres;
  res->status = (fe_status)h.status;
  if (opts->history && h.iter > 0)
    FE_CUDA(cudaMemcpy(opts->history, W.hist, 3 * (size_t)h.iter * sizeof(double),
                       cudaMemcpyDeviceToHost),
            "history readback");
  if (h.status == FE_ERR_NOT_CONVERGED) fe_set_error("fe_slab_cg_solve: not converged");
  if (h.status == FE_ERR_BREAKDOWN) fe_set_error("fe_slab_cg_solve: breakdown");
  return (fe_status)h.status;
}
