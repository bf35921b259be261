// FP32 instantiation of the tiled Godunov kernel: reconstruction, predictor and Riemann
// solve in FP32 (compiled with fast single-precision division and square root), state
// accumulation in FP64.
#include "godunov_impl.cuh"

namespace amr {
amr_status godunov_dispatch_fp32(const amr_tree *t, int level, const hydro_params *p, const double *u_old,
                                 double *u_new, double *reg, const double *dt, double *dt_next, cudaStream_t st)
{
    return dispatch_impl<float>(t, level, p, u_old, u_new, reg, dt, dt_next, st);
}
}  // namespace amr
