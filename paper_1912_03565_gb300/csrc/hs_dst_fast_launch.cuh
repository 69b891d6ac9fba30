// Kernels and launchers of the compile-time-sized DST-I tiles (Section 3.6); included by one
// translation unit per group of output modes (k_dst_fast*.cu) so that the
// kernel instances compile in parallel.
#pragma once

#include "hs_tiles.cuh"

namespace {

using namespace hs_tiles;

template <typename Tc, typename Tin, typename Tout, int AXIS, int MODE, int M, int S, int... Rs>
__global__ void __launch_bounds__(256, (sizeof(Tc) == 4 ? 2 : 1))
dst_fast_kernel(const Tin *in, Tout *out, double *aux, const typename Cx<Tc>::t *roots_g,
                const typename Cx<Tc>::t *half_g, int Nx, int Ny, int Nz, Tc scale,
                const int *skip) {
    if (skip && *skip) return;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    dst_fast_tile<Tc, Tin, Tout, AXIS, MODE, M, S, false, Rs...>(
        in, out, aux, roots_g, half_g, Nx, Ny, Nz, scale, smem_raw, blockIdx.x, blockIdx.y);
}

template <typename Tc, typename Tin, typename Tout, int MODE, int M, int... Rs>
hs_status launch_m(const hs_plan_s *P, int axis, const DstAxis &ax, const void *in, void *out,
                   double scale, cudaStream_t st, double *aux) {
    typedef typename Cx<Tc>::t T2;
    const T2 *roots = static_cast<const T2 *>(ax.roots);
    const T2 *half = static_cast<const T2 *>(ax.half);
    if (axis == HS_AXIS_X) {
        constexpr int S = Lines<Tc, M, HS_AXIS_X>::value;
        constexpr size_t smem = fast_smem<Tc, M, S>();
        static_assert(smem <= 227 * 1024, "transform tile exceeds shared memory");
        auto k = dst_fast_kernel<Tc, Tin, Tout, HS_AXIS_X, MODE, M, S, Rs...>;
        if (cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) !=
            cudaSuccess)
            return HS_ERR_CUDA;
        const long nrows = (long)P->Ny * P->Nz;
        k<<<(unsigned)((nrows + S - 1) / S), 256, smem, st>>>(
            static_cast<const Tin *>(in), static_cast<Tout *>(out), aux, roots, half, P->Nx,
            P->Ny, P->Nz, (Tc)scale, P->cur_skip);
    } else {
        constexpr int S = Lines<Tc, M, HS_AXIS_Y>::value;
        constexpr size_t smem = fast_smem<Tc, M, S>();
        static_assert(smem <= 227 * 1024, "transform tile exceeds shared memory");
        auto k = dst_fast_kernel<Tc, Tin, Tout, HS_AXIS_Y, MODE, M, S, Rs...>;
        if (cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) !=
            cudaSuccess)
            return HS_ERR_CUDA;
        dim3 grid((unsigned)((P->Nx + S - 1) / S), (unsigned)P->Nz, 1);
        k<<<grid, 256, smem, st>>>(static_cast<const Tin *>(in), static_cast<Tout *>(out), aux,
                                   roots, half, P->Nx, P->Ny, P->Nz, (Tc)scale, P->cur_skip);
    }
    return cudaGetLastError() == cudaSuccess ? HS_OK : HS_ERR_CUDA;
}

template <typename Tc, typename Tin, typename Tout, int MODE>
hs_status launch_sized(const hs_plan_s *P, int axis, const DstAxis &ax, const void *in, void *out,
                       double scale, cudaStream_t st, double *aux) {
    switch (ax.M) {
        case 32: return launch_m<Tc, Tin, Tout, MODE, 32, 8, 4>(P, axis, ax, in, out, scale, st, aux);
        case 64: return launch_m<Tc, Tin, Tout, MODE, 64, 16, 4>(P, axis, ax, in, out, scale, st, aux);
        case 96: return launch_m<Tc, Tin, Tout, MODE, 96, 16, 6>(P, axis, ax, in, out, scale, st, aux);
        case 128: return launch_m<Tc, Tin, Tout, MODE, 128, 16, 8>(P, axis, ax, in, out, scale, st, aux);
        case 192: return launch_m<Tc, Tin, Tout, MODE, 192, 16, 12>(P, axis, ax, in, out, scale, st, aux);
        case 256: return launch_m<Tc, Tin, Tout, MODE, 256, 16, 16>(P, axis, ax, in, out, scale, st, aux);
        case 384: return launch_m<Tc, Tin, Tout, MODE, 384, 16, 8, 3>(P, axis, ax, in, out, scale, st, aux);
        case 512: return launch_m<Tc, Tin, Tout, MODE, 512, 16, 16, 2>(P, axis, ax, in, out, scale, st, aux);
        case 768: return launch_m<Tc, Tin, Tout, MODE, 768, 16, 16, 3>(P, axis, ax, in, out, scale, st, aux);
        case 1024: return launch_m<Tc, Tin, Tout, MODE, 1024, 16, 16, 4>(P, axis, ax, in, out, scale, st, aux);
        default: return HS_ERR_UNSUPPORTED;
    }
}

}  // namespace
