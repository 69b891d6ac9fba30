// Fused DST-I tiles (Section 3.6) along y (FP32 compute, in-place FP32 passes of the mixed path).
#include "hs_dst_fused_launch.cuh"

namespace {

template <bool W>
hs_status launch_y(const hs_plan_s *P, int tin, const void *in, int tout, void *out, int mode,
                   double scale, cudaStream_t s, double *aux) {
    const DstAxis &ax = P->axf[HS_AXIS_Y];
    if (tin == HS_T_F32 && tout == HS_T_F32 && mode == HS_MODE_WRITE)
        return fused_launch_sized<float, float, HS_AXIS_Y, HS_MODE_WRITE, W>(P, ax, in, out, scale, s, aux);
    return HS_ERR_UNSUPPORTED;
}

}  // namespace

hs_status hs_launch_dst_fused_y(const hs_plan_s *P, int tin, const void *in, int tout, void *out,
                                int mode, double scale, cudaStream_t s, double *aux, int wide) {
    if (wide) return launch_y<true>(P, tin, in, tout, out, mode, scale, s, aux);
    return launch_y<false>(P, tin, in, tout, out, mode, scale, s, aux);
}

int hs_dst_fused_lines_y(int M, int wide) {
    DstAxis ax{};
    ax.M = M;
    int S = 0;
    const hs_status st =
        wide ? fused_launch_sized<float, float, HS_AXIS_Y, HS_MODE_WRITE, true>(
                   nullptr, ax, nullptr, nullptr, 1.0, 0, nullptr, &S)
             : fused_launch_sized<float, float, HS_AXIS_Y, HS_MODE_WRITE, false>(
                   nullptr, ax, nullptr, nullptr, 1.0, 0, nullptr, &S);
    return st == HS_OK ? S : 0;
}
