// fe_apply_h16.cu -- apply with 16-bit (bf16 or fp16) operands and FP32 accumulation (inner
// operator of mixed precision): the tensor-core kernels of fe_apply_kron.cu where they apply, the
// sum-factorized FMA-pipe kernels otherwise.
#include "fe_apply_launch.cuh"

fe_status fe_launch_apply_lowp(const ApplyLaunch& L, int prec) {
  if (fe_kron_supported(L.m)) return fe_launch_apply_kron(L, prec);
  if (prec == FE_BF16_F32ACC)
    return launch_apply_v<bfv>(L, reinterpret_cast<const unsigned short*>(L.m->geo16[0]), nullptr,
                               nullptr);
  if (prec == FE_F16_F32ACC)
    return launch_apply_v<hfv>(L, reinterpret_cast<const unsigned short*>(L.m->geo16[1]), nullptr,
                               nullptr);
  fe_set_error("apply: precision %d is not a 16-bit operand format", prec);
  return FE_ERR_INVALID;
}
