// Compile-time-sized DST-I tiles (Section 3.6), FP32 compute: the double-float iterate modes
// of the refined mixed path.
#include "hs_dst_fast_launch.cuh"

hs_status hs_dst_fast_df(const hs_plan_s *P, int axis, int tin, const void *in, int tout,
                         void *out, int mode, double scale, cudaStream_t s, double *aux) {
    const DstAxis &ax = P->axf[axis];
    if (tin != HS_T_F32 || tout != HS_T_DF) return HS_ERR_UNSUPPORTED;
    if (mode == HS_MODE_DF_SET)
        return launch_sized<float, float, float, HS_MODE_DF_SET>(P, axis, ax, in, out, scale, s, aux);
    if (mode == HS_MODE_DF_ADD)
        return launch_sized<float, float, float, HS_MODE_DF_ADD>(P, axis, ax, in, out, scale, s, aux);
    if (mode == HS_MODE_DF_FINAL)
        return launch_sized<float, float, float, HS_MODE_DF_FINAL>(P, axis, ax, in, out, scale, s, aux);
    if (mode == HS_MODE_DF_FINAL_HI)
        return launch_sized<float, float, float, HS_MODE_DF_FINAL_HI>(P, axis, ax, in, out, scale, s, aux);
    return HS_ERR_UNSUPPORTED;
}
