// Two-pass DST-I along y for long lines (M = N + 1 in {512, 768, 1024}; FP32).
//
// The transform is the one of the other DST kernels (odd extension packed as M
// complex points z_n = e_{2n} + i e_{2n+1}, a length-M FFT W_k, then
// X_k = [(W_{M-k}.y - W_k.y) + cos(pi k/M)(W_k.x - W_{M-k}.x)
//        + sin(pi k/M)(W_k.y + W_{M-k}.y)] / 4; Section 3.6's DST by FFT), but the
// FFT is split as M = M1 M2 (n = n1 + M1 n2, k = k2 + M2 k1):
//   W_{k2 + M2 k1} = sum_{n1} W_M1^{n1 k1} [ W_M^{n1 k2} sum_{n2} z_{n1 + M1 n2} W_M2^{n2 k2} ].
// Pass 1: one thread per (column, n1) reads its M2 points straight from the
// column, does the inner DFT in registers and the twiddle, and writes the
// complex intermediate T[k2][n1] of its column.  Pass 2: one warp per k2 does
// the outer DFT over n1 for 32 columns; k2 and M2 - k2 sit in the same CTA, so
// W_k and its partner W_{M-k} meet in shared memory for the final step.  A
// warp always covers 32 adjacent columns, so every global access is a whole
// 128-byte row segment: a single-pass kernel holds whole 1024-point lines in
// shared memory and fits only 12 columns (48-byte segments) and one CTA per SM.
#include "hs_tiles.cuh"

namespace {

using namespace hs_tiles;

constexpr int TP_M1 = 32;   // outer length (pass 2)
constexpr int TP_W = 8;     // warps per CTA

// In-register DFT of length 32 (forward, natural order in and out) as 4 x 8:
// the length-4 and length-8 DFTs use the constant 48th roots (4 and 8 divide
// 48, 32 does not); the twiddles W_32^(n2 k1) between them come from the
// line's table of M-th roots, W_32^m = W_M^(m M / 32).
__device__ __forceinline__ void dft32_rt(float2 *x, const float2 *__restrict__ roots, int stride) {
    float2 y[32];
#pragma unroll
    for (int n2 = 0; n2 < 8; ++n2) {
        float2 t[4];
#pragma unroll
        for (int n1 = 0; n1 < 4; ++n1) t[n1] = x[8 * n1 + n2];
        Dft<float, 4>::run(t);
#pragma unroll
        for (int k1 = 0; k1 < 4; ++k1) {
            float2 a = t[k1];
            if (n2 * k1 != 0) {
                const float2 r = __ldg(roots + n2 * k1 * stride);
                a = make_float2(a.x * r.x - a.y * r.y, a.x * r.y + a.y * r.x);
            }
            y[n2 * 4 + k1] = a;
        }
    }
#pragma unroll
    for (int k1 = 0; k1 < 4; ++k1) {
        float2 t[8];
#pragma unroll
        for (int n2 = 0; n2 < 8; ++n2) t[n2] = y[n2 * 4 + k1];
        Dft<float, 8>::run(t);
#pragma unroll
        for (int k2 = 0; k2 < 8; ++k2) x[k1 + 4 * k2] = t[k2];
    }
}

// Length-R DFT in registers: the constant-root DFTs where R divides 48, else 32.
template <int R>
__device__ __forceinline__ void dft_any(float2 *v, const float2 *roots, int M) {
    if constexpr (R == 32)
        dft32_rt(v, roots, M / 32);
    else
        Dft<float, R>::run(v);
}

// Pass 1.  grid (ceil(Nx / 32), Nz, M1 / 8); block 256 = 32 columns x 8 values of n1.
template <int M, int M2>
__global__ void __launch_bounds__(256) dst_y_pass1(const float *__restrict__ in,
                                                   float2 *__restrict__ tmp,
                                                   const float2 *__restrict__ roots, int Nx,
                                                   int Ny, const int *skip) {
    if (skip && *skip) return;
    constexpr int M1 = TP_M1;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int p = blockIdx.x * 32 + lane;
    const int l = blockIdx.y;
    const int n1 = blockIdx.z * TP_W + w;
    if (p >= Nx) return;   // no barrier or shuffle below
    const float *col = in + (size_t)l * Ny * Nx + p;
    auto ext = [&](int m) -> float {
        if (m == 0 || m == M) return 0.f;
        if (m < M) return __ldg(col + (size_t)(m - 1) * Nx);
        return -__ldg(col + (size_t)(2 * M - m - 1) * Nx);
    };
    float2 v[M2];
#pragma unroll
    for (int n2 = 0; n2 < M2; ++n2) {
        const int n = n1 + M1 * n2;
        v[n2].x = ext(2 * n);
        v[n2].y = ext(2 * n + 1);
    }
    dft_any<M2>(v, roots, M);   // v[k2] = sum_n2 z_{n1 + M1 n2} W_M2^{n2 k2}
    float2 *t = tmp + (size_t)l * M * Nx + p;
#pragma unroll
    for (int k2 = 0; k2 < M2; ++k2) {
        const float2 r = __ldg(roots + n1 * k2);   // W_M^{n1 k2}, n1 k2 < M
        const float2 a = v[k2];
        t[(size_t)(k2 * M1 + n1) * Nx] = make_float2(a.x * r.x - a.y * r.y, a.x * r.y + a.y * r.x);
    }
}

// Pass 2.  grid (ceil(Nx / 32), Nz, ceil((M2/2 + 1) / 4)); block 256: warps 0-3
// take k2 = 4 z + w, warps 4-7 the partners M2 - k2 (mod M2).
template <int M, int M2>
__global__ void __launch_bounds__(256) dst_y_pass2(const float2 *__restrict__ tmp,
                                                   float *__restrict__ out,
                                                   const float2 *__restrict__ roots,
                                                   const float2 *__restrict__ half, int Nx,
                                                   int Ny, float scale, const int *skip) {
    if (skip && *skip) return;
    constexpr int M1 = TP_M1;
    constexpr int N = M - 1;
    extern __shared__ float2 ws_raw[];   // [warp][k1][column]: 8 x 32 x 32 float2 = 64 KB
    float2(*ws)[M1][32] = reinterpret_cast<float2(*)[M1][32]>(ws_raw);
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int p = blockIdx.x * 32 + lane;
    const int l = blockIdx.y;
    const int base = blockIdx.z * 4 + (w & 3);           // k2 of warps 0-3
    const int k2 = w < 4 ? base : (M2 - base) % M2;      // partner for warps 4-7
    const bool valid = base <= M2 / 2;
    const bool pin = p < Nx;
    float2 v[M1];
    if (valid && pin) {
        const float2 *t = tmp + (size_t)l * M * Nx + (size_t)k2 * M1 * Nx + p;
#pragma unroll
        for (int n1 = 0; n1 < M1; ++n1) v[n1] = __ldg(t + (size_t)n1 * Nx);
    } else {
#pragma unroll
        for (int n1 = 0; n1 < M1; ++n1) v[n1] = make_float2(0.f, 0.f);
    }
    dft_any<M1>(v, roots, M);   // v[k1] = W_{k2 + M2 k1}
#pragma unroll
    for (int k1 = 0; k1 < M1; ++k1) ws[w][k1][lane] = v[k1];
    __syncthreads();
    // outputs: warps 0-3 for k2, warps 4-7 for the partner (unless self-paired)
    const bool self = (k2 == 0) || (2 * k2 == M2);
    if (!valid || !pin || (w >= 4 && self)) return;
    const int pw = self ? w : (w ^ 4);   // warp holding W_{M-k}
    const float q = scale * 0.25f;
    float *o = out + (size_t)l * N * Nx + p;
#pragma unroll 4
    for (int k1 = 0; k1 < M1; ++k1) {
        const int k = k2 + M2 * k1;
        if (k == 0) continue;
        // partner M - k: for k2 > 0 it is (M2 - k2) + M2 (M1 - 1 - k1), for k2 = 0 it is
        // M2 (M1 - k1)
        const int pk1 = k2 == 0 ? (M1 - k1) % M1 : M1 - 1 - k1;
        const float2 Wk = v[k1];
        const float2 Wm = ws[pw][pk1][lane];
        const float2 cs = __ldg(half + k);
        o[(size_t)(k - 1) * Nx] = ((Wm.y - Wk.y) + cs.x * (Wk.x - Wm.x) + cs.y * (Wk.y + Wm.y)) * q;
    }
}

template <int M, int M2>
hs_status launch_tp(const hs_plan_s *P, const float *in, float *out, float2 *tmp, double scale,
                    cudaStream_t s) {
    static_assert(TP_M1 * M2 == M, "M = 32 M2");
    const DstAxis &ax = P->axf[HS_AXIS_Y];
    const float2 *roots = static_cast<const float2 *>(ax.roots);
    const float2 *half = static_cast<const float2 *>(ax.half);
    const unsigned gx = (unsigned)((P->Nx + 31) / 32);
    dst_y_pass1<M, M2><<<dim3(gx, P->Nz, TP_M1 / TP_W), 256, 0, s>>>(in, tmp, roots, P->Nx,
                                                                      P->Ny, P->cur_skip);
    constexpr int smem = TP_W * TP_M1 * 32 * (int)sizeof(float2);
    if (cudaFuncSetAttribute(dst_y_pass2<M, M2>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             smem) != cudaSuccess)
        return HS_ERR_CUDA;
    dst_y_pass2<M, M2><<<dim3(gx, P->Nz, (M2 / 2 + 1 + 3) / 4), 256, smem, s>>>(
        tmp, out, roots, half, P->Nx, P->Ny, (float)scale, P->cur_skip);
    return cudaGetLastError() == cudaSuccess ? HS_OK : HS_ERR_CUDA;
}

}  // namespace

int hs_dst_twopass_size(int M) { return M == 512 || M == 768 || M == 1024; }

hs_status hs_launch_dst_twopass_y(const hs_plan_s *P, const float *in, float *out, double scale,
                                  cudaStream_t s) {
    float2 *tmp = static_cast<float2 *>(P->d_ytmp);
    if (!tmp) return HS_ERR_INVALID_ARG;
    switch (P->axf[HS_AXIS_Y].M) {
        case 512: return launch_tp<512, 16>(P, in, out, tmp, scale, s);
        case 768: return launch_tp<768, 24>(P, in, out, tmp, scale, s);
        case 1024: return launch_tp<1024, 32>(P, in, out, tmp, scale, s);
        default: return HS_ERR_UNSUPPORTED;
    }
}
