// FP64 instantiation of the tiled Godunov kernel: every operation of the scheme in FP64
// (the plain path; IEEE division and square root).
#include "godunov_impl.cuh"

namespace amr {
amr_status godunov_dispatch_fp64(const amr_tree *t, int level, const hydro_params *p, const double *u_old,
                                 double *u_new, double *reg, const double *dt, double *dt_next, cudaStream_t st)
{
    return dispatch_impl<double>(t, level, p, u_old, u_new, reg, dt, dt_next, st);
}
}  // namespace amr
