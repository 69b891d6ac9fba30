// Compile-time-sized DST-I tiles (Section 3.6), FP32 compute: plain write / add modes.
#include "hs_dst_fast_launch.cuh"

hs_status hs_dst_fast_f32(const hs_plan_s *P, int axis, int tin, const void *in, int tout,
                          void *out, int mode, double scale, cudaStream_t s, double *aux) {
    const DstAxis &ax = P->axf[axis];
    if (tin == HS_T_F64 && tout == HS_T_F32 && mode == HS_MODE_WRITE)
        return launch_sized<float, double, float, HS_MODE_WRITE>(P, axis, ax, in, out, scale, s, aux);
    if (tin == HS_T_F32 && tout == HS_T_F32 && mode == HS_MODE_WRITE)
        return launch_sized<float, float, float, HS_MODE_WRITE>(P, axis, ax, in, out, scale, s, aux);
    if (tin == HS_T_F32 && tout == HS_T_F64 && mode == HS_MODE_WRITE)
        return launch_sized<float, float, double, HS_MODE_WRITE>(P, axis, ax, in, out, scale, s, aux);
    if (tin == HS_T_F32 && tout == HS_T_F64 && mode == HS_MODE_ADD)
        return launch_sized<float, float, double, HS_MODE_ADD>(P, axis, ax, in, out, scale, s, aux);
    return HS_ERR_UNSUPPORTED;
}
