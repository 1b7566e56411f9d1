// fe_apply_f32.cu -- FP32 apply (inner operator of mixed-precision CG).
#include "fe_apply_launch.cuh"

fe_status fe_launch_apply_f32(const ApplyLaunch& L) {
  if (L.m->d.geom_mode == FE_GEOM_RECOMPUTE) {
    fe_set_error("apply: FE_GEOM_RECOMPUTE is not available");
    return FE_ERR_INVALID;
  }
  return launch_apply_v<float>(L, L.m->geo32);
}
