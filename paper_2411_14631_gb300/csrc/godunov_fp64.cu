// FP64 instantiation of the tiled Godunov kernel: every operation of the scheme in FP64
// (the plain path; IEEE division and square root).
#include "godunov_impl.cuh"

namespace amr {
amr_status godunov_dispatch_fp64(const amr_tree *t, int level, const hydro_params *p, const double *u_old,
                                 double *u_new, double *reg, const double *dt, double *dt_next, cudaStream_t st)
{
    return dispatch_impl<double>(t, level, p, u_old, u_new, reg, dt, dt_next, st);
}
amr_status harvest_dispatch(const amr_tree *t, const hydro_params *p, const double *u, const double *dt, double *out,
                            int64_t cap, int64_t stride, unsigned long long *count, cudaStream_t st)
{
    return harvest_impl(t, p, u, dt, out, cap, stride, count, st);
}
}  // namespace amr
