// Compile-time-sized DST-I tiles (Section 3.6), FP64 compute (the FP64 path).
#include "hs_dst_fast_launch.cuh"

hs_status hs_dst_fast_f64(const hs_plan_s *P, int axis, int tin, const void *in, int tout,
                          void *out, int mode, double scale, cudaStream_t s, double *aux) {
    const DstAxis &ax = P->axd[axis];
    if (tin == HS_T_F64 && tout == HS_T_F64 && mode == HS_MODE_WRITE)
        return launch_sized<double, double, double, HS_MODE_WRITE>(P, axis, ax, in, out, scale, s, aux);
    if (tin == HS_T_F64 && tout == HS_T_F64 && mode == HS_MODE_ADD)
        return launch_sized<double, double, double, HS_MODE_ADD>(P, axis, ax, in, out, scale, s, aux);
    return HS_ERR_UNSUPPORTED;
}
