// fe_api.cu -- C-ABI entry points for the operator, DSS, diagonal and pairing calls.
#include "fe_vec.cuh"

static fe_status check_vec(const fe_mesh* m, const void* p, const char* what) {
  if (!p) {
    fe_set_error("%s: null pointer", what);
    return FE_ERR_INVALID;
  }
  if (!fe_aligned(p)) {
    fe_set_error("%s: pointer not 16-byte aligned", what);
    return FE_ERR_INVALID;
  }
  (void)m;
  return FE_OK;
}

// element size of the vectors of a call: double for FE_F64, float otherwise (the 16-bit operand
// formats keep float vectors)
static size_t elem_size(int prec) { return prec == FE_F64 ? sizeof(double) : sizeof(float); }

fe_status fe_apply_impl(const fe_mesh* m, fe_op op, fe_prec prec, const void* x, void* y,
                        unsigned flags, void* stream, int* brick_out) {
  if (!m) {
    fe_set_error("fe_apply: null mesh");
    return FE_ERR_INVALID;
  }
  FE_TRY(check_vec(m, x, "fe_apply x"));
  FE_TRY(check_vec(m, y, "fe_apply y"));
  if (op != FE_LAPLACE && op != FE_MASS) {
    fe_set_error("fe_apply: unknown operator %d", (int)op);
    return FE_ERR_INVALID;
  }
  if (prec != FE_F64 && prec != FE_F32 && prec != FE_BF16_F32ACC && prec != FE_F16_F32ACC) {
    fe_set_error("fe_apply: unknown precision %d", (int)prec);
    return FE_ERR_INVALID;
  }
  const bool lowp = prec == FE_BF16_F32ACC || prec == FE_F16_F32ACC;
  if (lowp && m->d.geom_mode != FE_GEOM_STORED) {
    fe_set_error("fe_apply: 16-bit contractions need FE_GEOM_STORED geometry");
    return FE_ERR_INVALID;
  }
  if (flags & ~(FE_ASSEMBLE | FE_NATIVE_F64)) {
    fe_set_error("fe_apply: unknown flags 0x%x", flags);
    return FE_ERR_INVALID;
  }
  const size_t bytes = (size_t)m->ncw * elem_size(prec);
  const char *xb = (const char*)x, *yb = (const char*)y;
  if (xb < yb + bytes && yb < xb + bytes) {
    fe_set_error("fe_apply: x and y overlap");
    return FE_ERR_INVALID;
  }
  FeDeviceGuard device_guard;
  FE_CUDA(device_guard.set(m->d.device), "cudaSetDevice");
  const bool native = (flags & FE_NATIVE_F64) && prec == FE_F64;
  FE_TRY(fe_ensure_geometry(m, prec, native));
  ApplyLaunch L{m, (int)op, x, y, (cudaStream_t)stream, nullptr, (flags & FE_ASSEMBLE) != 0,
                brick_out};
  if (prec == FE_F64)
    FE_TRY(native ? fe_launch_apply_f64native(L) : fe_launch_apply_f64dw(L));
  else if (lowp)
    FE_TRY(fe_launch_apply_lowp(L, (int)prec));
  else
    FE_TRY(fe_launch_apply_f32(L));
  return FE_OK;
}

extern "C" fe_status fe_apply(const fe_mesh* m, fe_op op, fe_prec prec, const void* x, void* y,
                              unsigned flags, void* stream) {
  return fe_apply_impl(m, op, prec, x, y, flags, stream, nullptr);
}

extern "C" fe_status fe_dss(const fe_mesh* m, fe_prec prec, const void* r, void* z, void* stream) {
  if (!m) {
    fe_set_error("fe_dss: null mesh");
    return FE_ERR_INVALID;
  }
  FE_TRY(check_vec(m, r, "fe_dss r"));
  FE_TRY(check_vec(m, z, "fe_dss z"));
  if (prec != FE_F64 && prec != FE_F32) {
    fe_set_error("fe_dss: precision %d not provided", (int)prec);
    return FE_ERR_INVALID;
  }
  FeDeviceGuard device_guard;
  FE_CUDA(device_guard.set(m->d.device), "cudaSetDevice");
  cudaStream_t st = (cudaStream_t)stream;
  if (r != z)
    FE_CUDA(cudaMemcpyAsync(z, r, (size_t)m->ncw * elem_size(prec), cudaMemcpyDeviceToDevice, st),
            "fe_dss copy");
  return fe_launch_dss(m, prec, z, st);
}

extern "C" fe_status fe_diag(const fe_mesh* m, fe_op op, double* d, void* stream) {
  if (!m) {
    fe_set_error("fe_diag: null mesh");
    return FE_ERR_INVALID;
  }
  FE_TRY(check_vec(m, d, "fe_diag d"));
  if (m->packed) {
    fe_set_error("fe_diag: FE_LAYOUT_CELLS meshes only");
    return FE_ERR_INVALID;
  }
  if (op != FE_LAPLACE && op != FE_MASS) {
    fe_set_error("fe_diag: unknown operator %d", (int)op);
    return FE_ERR_INVALID;
  }
  FeDeviceGuard device_guard;
  FE_CUDA(device_guard.set(m->d.device), "cudaSetDevice");
  return fe_launch_diag(m, (int)op, d, (cudaStream_t)stream);
}

extern "C" fe_status fe_pairing(const fe_mesh* m, fe_prec prec, const void* a, const void* b,
                                double* result_dev, void* stream) {
  if (!m || !result_dev) {
    fe_set_error("fe_pairing: null argument");
    return FE_ERR_INVALID;
  }
  FE_TRY(check_vec(m, a, "fe_pairing a"));
  FE_TRY(check_vec(m, b, "fe_pairing b"));
  FeDeviceGuard device_guard;
  FE_CUDA(device_guard.set(m->d.device), "cudaSetDevice");
  return fe_launch_pairing(m, (int)prec, a, b, result_dev, (cudaStream_t)stream);
}
