// fe_apply_f32.cu -- FP32 apply (inner operator of mixed-precision CG).
#include "fe_apply_launch.cuh"

fe_status fe_launch_apply_f32(const ApplyLaunch& L) {
  return launch_apply_v<float>(L, L.m->geo32, L.m->xyz32, static_cast<float*>(L.m->rc_scratch[2]));
}
