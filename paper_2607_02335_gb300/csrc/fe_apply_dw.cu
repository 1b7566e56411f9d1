// fe_apply_dw.cu -- FP64-accurate apply in double-word arithmetic on the FP32 pipe.
#include "fe_apply_launch.cuh"

fe_status fe_launch_apply_f64dw(const ApplyLaunch& L) {
  return launch_apply_v<dw>(L, L.m->geodw, L.m->xyzdw, static_cast<float2*>(L.m->rc_scratch[0]));
}
