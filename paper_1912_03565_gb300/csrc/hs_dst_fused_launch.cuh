// Kernels and launcher of the fused DST-I tiles (Section 3.6; hs_dst_fused.cuh); included by
// one translation unit per axis.
#pragma once

#include "hs_dst_fused.cuh"

namespace {

using namespace hs_tiles;

template <typename Tin, typename Tout, int AXIS, int MODE, int M, int S, int R1, int RL,
          int... Rmid>
__global__ void __launch_bounds__(256, 2)
dst_fused_kernel(const Tin *in, Tout *out, double *aux, const float2 *roots_g,
                 const float2 *half_g, int Nx, int Ny, int Nz, float scale, const int *skip) {
    if (skip && *skip) return;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    dst_fused_tile<Tin, Tout, AXIS, MODE, M, S, false, R1, RL, Rmid...>(
        in, out, aux, roots_g, half_g, Nx, Ny, Nz, scale, smem_raw, blockIdx.x, blockIdx.y);
}

// Lines per CTA of the fused tiles: as the staged tiles, or twice as many
// (WIDE) when the stages run in place and the one buffer still fits.
template <bool WIDE, int AXIS, int M, int R1, int RL, int... Rmid>
struct FusedLines {
    static constexpr int base = Lines<float, M, AXIS>::value;
    static constexpr bool can = fused_inplace<AXIS, M, 2 * base, R1, RL, Rmid...>() &&
                                fused_smem<AXIS, M, 2 * base, R1, RL, Rmid...>() <= 227 * 1024;
    static constexpr int value = (WIDE && can) ? 2 * base : base;
};

template <typename Tin, typename Tout, int AXIS, int MODE, bool WIDE, int M, int R1, int RL,
          int... Rmid>
hs_status fused_launch_m(const hs_plan_s *P, const DstAxis &ax, const void *in, void *out,
                         double scale, cudaStream_t st, double *aux, int *probe) {
    constexpr int S = FusedLines<WIDE, AXIS, M, R1, RL, Rmid...>::value;
    if (WIDE && S == Lines<float, M, AXIS>::value) return HS_ERR_UNSUPPORTED;
    if (probe) {   // lines per CTA only, nothing launched
        *probe = S;
        return HS_OK;
    }
    constexpr size_t smem = fused_smem<AXIS, M, S, R1, RL, Rmid...>();
    static_assert(smem <= 227 * 1024, "transform tile exceeds shared memory");
    static_assert(R1 * RL * (1 * ... * Rmid) == M, "radices must multiply to M");
    auto k = dst_fused_kernel<Tin, Tout, AXIS, MODE, M, S, R1, RL, Rmid...>;
    if (cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) !=
        cudaSuccess)
        return HS_ERR_CUDA;
    const float2 *roots = static_cast<const float2 *>(ax.roots);
    const float2 *half = static_cast<const float2 *>(ax.half);
    dim3 grid;
    if (AXIS == HS_AXIS_X)
        grid = dim3((unsigned)(((long)P->Ny * P->Nz + S - 1) / S), 1, 1);
    else
        grid = dim3((unsigned)((P->Nx + S - 1) / S), (unsigned)P->Nz, 1);
    k<<<grid, 256, smem, st>>>(static_cast<const Tin *>(in), static_cast<Tout *>(out), aux,
                               roots, half, P->Nx, P->Ny, P->Nz, (float)scale, P->cur_skip);
    return cudaGetLastError() == cudaSuccess ? HS_OK : HS_ERR_CUDA;
}

// Radices per length: first R1, last RL (M / RL lanes per line in the last
// stage: at most 32 and a divisor of 32, for the shuffle pairing of x-lines).
template <typename Tin, typename Tout, int AXIS, int MODE, bool WIDE = false>
hs_status fused_launch_sized(const hs_plan_s *P, const DstAxis &ax, const void *in, void *out,
                             double scale, cudaStream_t st, double *aux, int *probe = nullptr) {
#define HS_F(...) return fused_launch_m<Tin, Tout, AXIS, MODE, WIDE, __VA_ARGS__>(P, ax, in, out, scale, st, aux, probe)
    switch (ax.M) {
        case 32: HS_F(32, 8, 4);
        case 64: HS_F(64, 16, 4);
        case 96: HS_F(96, 16, 6);
        case 128: HS_F(128, 16, 8);
        case 192: HS_F(192, 16, 12);
        case 256: HS_F(256, 16, 16);
        case 384: HS_F(384, 16, 12, 2);
        case 512: HS_F(512, 16, 16, 2);
        case 768: HS_F(768, 16, 24, 2);
        case 1024:
            if constexpr (AXIS == HS_AXIS_Y) {
                HS_F(1024, 16, 16, 4);
            } else {
                HS_F(1024, 16, 32, 2);   // 32 lanes per line: a length-32 last stage
            }
        default: return HS_ERR_UNSUPPORTED;
    }
#undef HS_F
}

}  // namespace
