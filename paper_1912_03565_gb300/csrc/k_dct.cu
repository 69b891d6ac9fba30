// DCT-I of lines of M + 1 nodes (FP64; compiled FFT lengths, direct sums for the
// others): the transform of a side axis with
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

// Runtime-sized DCT-I (any M, for the lengths without a compiled FFT): direct
// sums X_k = sum_i w_i x_i cos(pi k i / M), w_0 = w_M = 1/2, with the argument
// reduced exactly (k i mod 2M) into the table of cos(pi m / M), m = 0..M.  One
// CTA owns S whole lines, read into shared memory before any output is written
// (so the transform may run in place); O(M^2) FP64 operations per line.
constexpr int GDCT_S = 8;

template <int AXIS>
__global__ void __launch_bounds__(256)
dct_generic_kernel(const double *in, double *out, const double2 *half_g, int M, long nrows,
                   int nx, double scale) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int L = M + 1;
    double *cs = reinterpret_cast<double *>(smem_raw);   // [M + 1]: cos(pi m / M)
    double *x = cs + L;                                   // [GDCT_S][L], weights applied
    for (int t = threadIdx.x; t < L; t += blockDim.x) cs[t] = half_g[t].x;
    size_t base;
    int nvalid;
    if (AXIS == HS_AXIS_X) {
        const long r0 = (long)blockIdx.x * GDCT_S;
        nvalid = (int)min((long)GDCT_S, nrows - r0);
        base = (size_t)r0 * L;
        for (int e = threadIdx.x; e < nvalid * L; e += blockDim.x) {
            const int s = e / L, i = e - s * L;
            x[s * L + i] = (i == 0 || i == M ? 0.5 : 1.0) * in[base + e];
        }
    } else {
        const int p0 = blockIdx.x * GDCT_S;
        nvalid = min(GDCT_S, nx - p0);
        base = (size_t)blockIdx.y * L * nx + p0;
        for (int e = threadIdx.x; e < GDCT_S * L; e += blockDim.x) {
            const int i = e / GDCT_S, s = e - i * GDCT_S;
            if (s < nvalid)
                x[s * L + i] = (i == 0 || i == M ? 0.5 : 1.0) * in[base + (size_t)i * nx + s];
        }
    }
    __syncthreads();
    const int twoM = 2 * M;
    for (int e = threadIdx.x; e < nvalid * L; e += blockDim.x) {
        int s, k;
        if (AXIS == HS_AXIS_X) {
            s = e / L;
            k = e - s * L;
        } else {   // consecutive threads take consecutive columns: coalesced stores
            k = e / nvalid;
            s = e - k * nvalid;
        }
        const double *xs = x + s * L;
        double acc = 0.0;
        int m = 0;   // k i mod 2M
        for (int i = 0; i < L; ++i) {
            acc = fma(xs[i], cs[m <= M ? m : twoM - m], acc);
            m += k;
            if (m >= twoM) m -= twoM;
        }
        if (AXIS == HS_AXIS_X)
            out[base + (size_t)s * L + k] = scale * acc;
        else
            out[base + (size_t)k * nx + s] = scale * acc;
    }
}

}  // namespace

// DCT-I for a length without a compiled FFT (direct sums; see dct_generic_kernel).
hs_status hs_launch_dct_generic(int axis, int M, const double *in, double *out, const void *half,
                                long nrows, int nx, int nplanes, double scale, cudaStream_t s) {
    if (M < 1) return HS_ERR_INVALID_ARG;
    const size_t smem = sizeof(double) * ((size_t)(M + 1) * (1 + GDCT_S));
    if (smem > 227 * 1024) return HS_ERR_UNSUPPORTED;
    const double2 *h = static_cast<const double2 *>(half);
    if (axis == HS_AXIS_X) {
        if (cudaFuncSetAttribute(dct_generic_kernel<HS_AXIS_X>,
                                 cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
            return HS_ERR_CUDA;
        dct_generic_kernel<HS_AXIS_X><<<(unsigned)((nrows + GDCT_S - 1) / GDCT_S), 256, smem, s>>>(
            in, out, h, M, nrows, nx, scale);
    } else {
        if (cudaFuncSetAttribute(dct_generic_kernel<HS_AXIS_Y>,
                                 cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
            return HS_ERR_CUDA;
        dct_generic_kernel<HS_AXIS_Y>
            <<<dim3((unsigned)((nx + GDCT_S - 1) / GDCT_S), (unsigned)nplanes, 1), 256, smem, s>>>(
                in, out, h, M, nrows, nx, scale);
    }
    return cudaGetLastError() == cudaSuccess ? HS_OK : HS_ERR_CUDA;
}

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
        default: return hs_launch_dct_generic(axis, M, in, out, half, nrows, nx, nplanes, scale, s);
    }
#undef HS_D
}
