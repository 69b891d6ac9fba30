// DCT-I of lines of M + 1 nodes (FP64): the transform of a side axis with
// u_n = 0 on both faces, whose modes cos(pi p i / M), p = 0..M, diagonalise
// the reflected second difference (Section 3.6's separation with cosines in
// place of sines).
//
// Same FFT as the sine transform (k_dst_fast.cu): the line is extended to 2M
// reals, here evenly (e_m = x_m for m <= M, e_2M-m = x_m), packed as M complex
// points z_n = e_2n + i e_2n+1, transformed by the compile-time Stockham stages,
// and unpacked.  With W_k the packed FFT, the even extension's DFT is real:
//   E_k = [(W_k.x + W_M-k.x) - sin(pi k/M)(W_k.x - W_M-k.x)
//          + cos(pi k/M)(W_k.y + W_M-k.y)] / 2,     k = 0..M (indices mod M),
// and X_k = sum_i w_i x_i cos(pi k i / M) = E_k / 2 (w_0 = w_M = 1/2).  The
// inverse is the same transform scaled by 2 / M.
#include "hs_tiles.cuh"

namespace {

using namespace hs_tiles;

// AXIS X: lines are contiguous rows of M + 1 values, nrows of them.
// AXIS Y: in each of the planes [M + 1][nx], the columns; grid (ceil(nx / S), planes).
template <int AXIS, int M, int S, int... Rs>
__global__ void __launch_bounds__(256, 1)
dct_kernel(const double *in, double *out, const double2 *roots_g, const double2 *half_g,
           long nrows, int nx, double scale) {
    constexpr int L = M + 1;
    constexpr int LS = LineStride<M>::value;
    constexpr int NT = 256;
    constexpr int ITER = (S * L + NT - 1) / NT;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    double2 *roots = reinterpret_cast<double2 *>(smem_raw);
    double2 *half = roots + M;
    double2 *buf0 = half + (M + 1);
    double2 *buf1 = buf0 + S * LS;
    for (int t = threadIdx.x; t < M; t += NT) roots[t] = roots_g[t];
    for (int t = threadIdx.x; t <= M; t += NT) half[t] = half_g[t];
    double *z = reinterpret_cast<double *>(buf0);

    size_t base;
    int nvalid;
    double v[ITER];
    // every global load of the tile before any store (the transform runs in place)
    if (AXIS == HS_AXIS_X) {
        const long row0 = (long)blockIdx.x * S;
        base = (size_t)row0 * L;
        nvalid = (int)min((long)S, nrows - row0);
        const int nel = nvalid * L;
#pragma unroll
        for (int it = 0; it < ITER; ++it) {
            const int e = threadIdx.x + it * NT;
            v[it] = e < nel ? in[base + e] : 0.0;
        }
    } else {
        const int p0 = blockIdx.x * S;
        base = (size_t)blockIdx.y * L * nx + p0;
        nvalid = min(S, nx - p0);
#pragma unroll
        for (int it = 0; it < ITER; ++it) {
            const int e = threadIdx.x + it * NT;
            const int j = e / S, s = e - j * S;
            v[it] = (e < S * L && s < nvalid) ? in[base + (size_t)j * nx + s] : 0.0;
        }
    }
#pragma unroll
    for (int it = 0; it < ITER; ++it) {
        const int e = threadIdx.x + it * NT;
        if (e < S * L) {
            int s, i;
            if (AXIS == HS_AXIS_X) {
                s = e / L;
                i = e - s * L;
            } else {
                i = e / S;
                s = e - i * S;
            }
            double *zl = z + s * 2 * LS;
            zl[ZPAD(i)] = v[it];
            if (i >= 1 && i <= M - 1) zl[ZPAD(2 * M - i)] = v[it];
        }
    }
    __syncthreads();

    double2 *src = buf0, *dst = buf1;
    fstages<double, M, S, 1, Rs...>(src, dst, roots);

    const double q = scale * 0.25;
    auto coef = [&](int s, int k) {
        const int a = k == M ? 0 : k, b = k == 0 ? 0 : M - k;
        const double2 Wk = src[s * LS + PAD(a)];
        const double2 Wm = src[s * LS + PAD(b)];
        const double2 cs = half[k];
        return ((Wk.x + Wm.x) - cs.y * (Wk.x - Wm.x) + cs.x * (Wk.y + Wm.y)) * q;
    };
    if (AXIS == HS_AXIS_X) {
        const int nel = nvalid * L;
#pragma unroll
        for (int it = 0; it < ITER; ++it) {
            const int e = threadIdx.x + it * NT;
            if (e < nel) {
                const int s = e / L;
                out[base + e] = coef(s, e - s * L);
            }
        }
    } else {
#pragma unroll
        for (int it = 0; it < ITER; ++it) {
            const int e = threadIdx.x + it * NT;
            const int k = e / S, s = e - k * S;
            if (e < S * L && s < nvalid) out[base + (size_t)k * nx + s] = coef(s, k);
        }
    }
}

template <int M, int... Rs>
hs_status launch_dct_m(int axis, const double *in, double *out, const double2 *roots,
                       const double2 *half, long nrows, int nx, int nplanes, double scale,
                       cudaStream_t st) {
    if (axis == HS_AXIS_X) {
        constexpr int S = Lines<double, M, HS_AXIS_X>::value;
        constexpr size_t smem = fast_smem<double, M, S>();
        static_assert(smem <= 227 * 1024, "transform tile exceeds shared memory");
        auto k = dct_kernel<HS_AXIS_X, M, S, Rs...>;
        if (cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) !=
            cudaSuccess)
            return HS_ERR_CUDA;
        k<<<(unsigned)((nrows + S - 1) / S), 256, smem, st>>>(in, out, roots, half, nrows, nx,
                                                              scale);
    } else {
        constexpr int S = Lines<double, M, HS_AXIS_Y>::value;
        constexpr size_t smem = fast_smem<double, M, S>();
        static_assert(smem <= 227 * 1024, "transform tile exceeds shared memory");
        auto k = dct_kernel<HS_AXIS_Y, M, S, Rs...>;
        if (cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) !=
            cudaSuccess)
            return HS_ERR_CUDA;
        k<<<dim3((unsigned)((nx + S - 1) / S), (unsigned)nplanes, 1), 256, smem, st>>>(
            in, out, roots, half, nrows, nx, scale);
    }
    return cudaGetLastError() == cudaSuccess ? HS_OK : HS_ERR_CUDA;
}

}  // namespace

hs_status hs_launch_dct(int axis, int M, const double *in, double *out, const void *roots,
                        const void *half, long nrows, int nx, int nplanes, double scale,
                        cudaStream_t s) {
    const double2 *r = static_cast<const double2 *>(roots);
    const double2 *h = static_cast<const double2 *>(half);
#define HS_D(M_, ...) return launch_dct_m<M_, __VA_ARGS__>(axis, in, out, r, h, nrows, nx, nplanes, scale, s)
    switch (M) {
        case 32: HS_D(32, 8, 4);
        case 64: HS_D(64, 16, 4);
        case 96: HS_D(96, 16, 6);
        case 128: HS_D(128, 16, 8);
        case 192: HS_D(192, 16, 12);
        case 256: HS_D(256, 16, 16);
        case 384: HS_D(384, 16, 8, 3);
        case 512: HS_D(512, 16, 16, 2);
        case 768: HS_D(768, 16, 16, 3);
        case 1024: HS_D(1024, 16, 16, 4);
        default: return HS_ERR_UNSUPPORTED;
    }
#undef HS_D
}
