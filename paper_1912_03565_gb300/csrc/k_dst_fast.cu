// Compile-time-sized DST-I kernels for the line lengths the solver meets most
// (N + 1 = M in {32, 64, 96, 128, 192, 256, 384, 512, 768, 1024}).
//
// Same algorithm as k_dst.cu (odd extension, length-M complex FFT of the
// packed line, X_k from W_k and W_{M-k}; Section 3.6's 2-D DST through FFTs), but
// every size, radix and stride is a template constant: the index arithmetic
// of the Stockham stages becomes shifts and multiplies, and each thread does
// one radix-R butterfly (R up to 16) in registers per stage, so a 256-point
// line takes two passes through shared memory instead of four.  In-register
// DFTs of size R = R1 R2 use the Cooley-Tukey split n = R2 n1 + n2,
// k = k1 + R1 k2 with the twiddles W_R^(n2 k1) taken from the 48th roots
// below (every R used divides 48).
#include "hs_internal.cuh"

int hs_dst_fast_size(int M) {
    switch (M) {
        case 32: case 64: case 96: case 128: case 192: case 256: case 384: case 512: case 768:
        case 1024:
            return 1;
        default:
            return 0;
    }
}

hs_status hs_launch_dst_fast(const hs_plan_s *P, int axis, int tc, int tin, const void *in,
                             int tout, void *out, int mode, double scale, cudaStream_t s,
                             double *aux) {
    if (tc == HS_T_F64) return hs_dst_fast_f64(P, axis, tin, in, tout, out, mode, scale, s, aux);
    if (mode == HS_MODE_DF_SET || mode == HS_MODE_DF_ADD || mode == HS_MODE_DF_FINAL ||
        mode == HS_MODE_DF_FINAL_HI)
        return hs_dst_fast_df(P, axis, tin, in, tout, out, mode, scale, s, aux);
    return hs_dst_fast_f32(P, axis, tin, in, tout, out, mode, scale, s, aux);
}
