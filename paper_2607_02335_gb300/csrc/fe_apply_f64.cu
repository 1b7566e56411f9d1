// fe_apply_f64.cu -- apply on the native FP64 pipe (cross-check variant, FE_NATIVE_F64).
#include "fe_apply_launch.cuh"

fe_status fe_launch_apply_f64native(const ApplyLaunch& L) {
  return launch_apply_v<double>(L, L.m->geo64, L.m->xyz64, static_cast<double*>(L.m->rc_scratch[1]));
}
