// Fused DST tiles along x (FP32 compute): the modes of the mixed path.
#include "hs_dst_fused_launch.cuh"

hs_status hs_launch_dst_fused_x(const hs_plan_s *P, int tin, const void *in, int tout, void *out,
                                int mode, double scale, cudaStream_t s, double *aux) {
    const DstAxis &ax = P->axf[HS_AXIS_X];
    if (tin != HS_T_F32) return HS_ERR_UNSUPPORTED;
    if (tout == HS_T_F32 && mode == HS_MODE_WRITE)
        return fused_launch_sized<float, float, HS_AXIS_X, HS_MODE_WRITE>(P, ax, in, out, scale, s, aux);
    if (tout == HS_T_F64 && mode == HS_MODE_WRITE)
        return fused_launch_sized<float, double, HS_AXIS_X, HS_MODE_WRITE>(P, ax, in, out, scale, s, aux);
    if (tout == HS_T_DF && mode == HS_MODE_DF_SET)
        return fused_launch_sized<float, float, HS_AXIS_X, HS_MODE_DF_SET>(P, ax, in, out, scale, s, aux);
    if (tout == HS_T_DF && mode == HS_MODE_DF_ADD)
        return fused_launch_sized<float, float, HS_AXIS_X, HS_MODE_DF_ADD>(P, ax, in, out, scale, s, aux);
    if (tout == HS_T_DF && mode == HS_MODE_DF_FINAL)
        return fused_launch_sized<float, float, HS_AXIS_X, HS_MODE_DF_FINAL>(P, ax, in, out, scale, s, aux);
    return HS_ERR_UNSUPPORTED;
}
