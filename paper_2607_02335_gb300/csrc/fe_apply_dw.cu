// fe_apply_dw.cu -- FP64-accurate apply in double-word arithmetic on the FP32 pipe.
#include "fe_apply_launch.cuh"

fe_status fe_launch_apply_f64dw(const ApplyLaunch& L) {
  if (L.m->d.geom_mode == FE_GEOM_RECOMPUTE) {
    fe_set_error("apply: FE_GEOM_RECOMPUTE is not available");
    return FE_ERR_INVALID;
  }
  return launch_apply_v<dw>(L, L.m->geodw);
}
