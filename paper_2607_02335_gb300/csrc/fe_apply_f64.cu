// fe_apply_f64.cu -- apply on the native FP64 pipe (cross-check variant, FE_NATIVE_F64).
#include "fe_apply_launch.cuh"

fe_status fe_launch_apply_f64native(const ApplyLaunch& L) {
  if (L.m->d.geom_mode == FE_GEOM_RECOMPUTE) {
    fe_set_error("apply: FE_GEOM_RECOMPUTE is not available");
    return FE_ERR_INVALID;
  }
  return launch_apply_v<double>(L, L.m->geo64);
}
