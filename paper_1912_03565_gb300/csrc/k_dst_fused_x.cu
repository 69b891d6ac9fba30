// Fused DST-I tiles (Section 3.6) along x (FP32 compute): the modes of the mixed path.
#include "hs_dst_fused_launch.cuh"

namespace {

template <bool W>
hs_status launch_x(const hs_plan_s *P, int tin, const void *in, int tout, void *out, int mode,
                   double scale, cudaStream_t s, double *aux) {
    const DstAxis &ax = P->axf[HS_AXIS_X];
    if (tin != HS_T_F32) return HS_ERR_UNSUPPORTED;
    if (tout == HS_T_F32 && mode == HS_MODE_WRITE)
        return fused_launch_sized<float, float, HS_AXIS_X, HS_MODE_WRITE, W>(P, ax, in, out, scale, s, aux);
    if (tout == HS_T_F64 && mode == HS_MODE_WRITE)
        return fused_launch_sized<float, double, HS_AXIS_X, HS_MODE_WRITE, W>(P, ax, in, out, scale, s, aux);
    if (tout == HS_T_DF && mode == HS_MODE_DF_SET)
        return fused_launch_sized<float, float, HS_AXIS_X, HS_MODE_DF_SET, W>(P, ax, in, out, scale, s, aux);
    if (tout == HS_T_DF && mode == HS_MODE_DF_ADD)
        return fused_launch_sized<float, float, HS_AXIS_X, HS_MODE_DF_ADD, W>(P, ax, in, out, scale, s, aux);
    if (tout == HS_T_DF && mode == HS_MODE_DF_FINAL)
        return fused_launch_sized<float, float, HS_AXIS_X, HS_MODE_DF_FINAL, W>(P, ax, in, out, scale, s, aux);
    if (tout == HS_T_DF && mode == HS_MODE_DF_FINAL_HI)
        return fused_launch_sized<float, float, HS_AXIS_X, HS_MODE_DF_FINAL_HI, W>(P, ax, in, out, scale, s, aux);
    return HS_ERR_UNSUPPORTED;
}

}  // namespace

hs_status hs_launch_dst_fused_x(const hs_plan_s *P, int tin, const void *in, int tout, void *out,
                                int mode, double scale, cudaStream_t s, double *aux, int wide) {
    if (wide) return launch_x<true>(P, tin, in, tout, out, mode, scale, s, aux);
    return launch_x<false>(P, tin, in, tout, out, mode, scale, s, aux);
}

int hs_dst_fused_lines_x(int M, int wide) {
    DstAxis ax{};
    ax.M = M;
    int S = 0;
    const hs_status st =
        wide ? fused_launch_sized<float, float, HS_AXIS_X, HS_MODE_WRITE, true>(
                   nullptr, ax, nullptr, nullptr, 1.0, 0, nullptr, &S)
             : fused_launch_sized<float, float, HS_AXIS_X, HS_MODE_WRITE, false>(
                   nullptr, ax, nullptr, nullptr, 1.0, 0, nullptr, &S);
    return st == HS_OK ? S : 0;
}
