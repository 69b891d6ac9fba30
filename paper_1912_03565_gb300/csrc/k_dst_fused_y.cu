// Fused DST tiles along y (FP32 compute, in-place FP32 passes of the mixed path).
#include "hs_dst_fused_launch.cuh"

hs_status hs_launch_dst_fused_y(const hs_plan_s *P, int tin, const void *in, int tout, void *out,
                                int mode, double scale, cudaStream_t s, double *aux) {
    const DstAxis &ax = P->axf[HS_AXIS_Y];
    if (tin == HS_T_F32 && tout == HS_T_F32 && mode == HS_MODE_WRITE)
        return fused_launch_sized<float, float, HS_AXIS_Y, HS_MODE_WRITE>(P, ax, in, out, scale, s, aux);
    return HS_ERR_UNSUPPORTED;
}
