// fe_cg.cu -- conjugate gradients on cell-wise data.
#include "fe_vec.cuh"

extern "C" fe_status fe_cg_solve(const fe_mesh* m, const double* b, double* x,
                                 const fe_cg_opts* opts, fe_cg_result* res, void* stream) {
  (void)m; (void)b; (void)x; (void)opts; (void)res; (void)stream;
  fe_set_error("fe_cg_solve: not available in this build");
  return FE_ERR_INVALID;
}
