// DCT-I of lines of M + 1 nodes (FP64; compiled FFT lengths through one complex
// FFT of M/2 points, direct sums for the others): the transform of a side axis
// with u_n = g on both faces, whose modes cos(pi p i / M), p = 0..M, diagonalise
// the reflected second difference (Section 3.6's separation with cosines in
// place of sines),
//     X_k = sum_{j=0..M} w_j x_j cos(pi j k / M),   w_0 = w_M = 1/2;
// the inverse is the same transform scaled by 2 / M.
//
// Half-length formulation (a standard real-data form of the DCT-I): with
// s_j = sin(pi j / M),
//     y_j = (1/2 - s_j) x_j + (1/2 + s_j) x_{M-j},   j = 0..M-1,
// the part (x_j + x_{M-j}) / 2 is even about M/2 and -s_j (x_j - x_{M-j}) odd, so
// Y = DFT_M(y) has
//     Re Y_k = X_{2k},   Im Y_k = X_{2k-1} - X_{2k+1}   (k = 0..M/2),
// and Y comes from the M/2-point complex FFT Z of z_m = y_{2m} + i y_{2m+1} as in the
// half-length sine transform (k_dst_half.cu).  The odd outputs are the running
// sum X_{2k+1} = X_1 - sum_{k'=1..k} Im Y_k', from X_1 = sum_j w_j x_j cos(pi j / M)
// taken directly (one dot product per line).  Values are kept doubled (2 Y_k,
// 2 X_1) and the factor scale / 2 is applied at the store.
#include "hs_tiles.cuh"

namespace {

using namespace hs_tiles;

template <int M, int AXIS>
struct DctHalfLines {
    static constexpr int base = 4096 / M > 0 ? 4096 / M : 1;
    static constexpr int value = (AXIS == HS_AXIS_Y && base < 8) ? 8 : base;
};

template <int M, int S>
constexpr size_t dct_half_smem() {
    // rootsH[M/2] + wk[M/2 + 1] + cpm[M] (double2), cs[M + 1] + x1[S] (double),
    // 2 buffers of S lines (each also holds a line of M + 1 reals)
    return sizeof(double2) * ((size_t)M / 2 + (M / 2 + 1) + M +
                              (size_t)2 * S * LineStride<M / 2>::value) +
           sizeof(double) * ((size_t)M + 1 + S);
}

// AXIS X: lines are contiguous rows of M + 1 values, nrows of them.
// AXIS Y: in each of the planes [M + 1][nx], the columns; grid (ceil(nx / S), planes).
template <int AXIS, int M, int S, int... Rs>
__global__ void __launch_bounds__(256, 2)
dct_half_kernel(const double *in, double *out, const double2 *__restrict__ roots_g,
                const double2 *__restrict__ half_g, long nrows, int nx, double scale) {
    constexpr int H = M / 2;
    constexpr int L = M + 1;
    constexpr int LS = LineStride<H>::value;
    constexpr int NT = 256;
    constexpr int ITER = (S * L + NT - 1) / NT;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    double2 *rootsH = reinterpret_cast<double2 *>(smem_raw);
    double2 *wk = rootsH + H;          // [H + 1]
    double2 *cpm = wk + (H + 1);       // [M]
    double2 *buf0 = cpm + M;
    double2 *buf1 = buf0 + S * LS;
    double *cs = reinterpret_cast<double *>(buf1 + S * LS);   // [M + 1]: cos(pi j / M)
    double *x1 = cs + L;                                       // [S]: 2 X_1 of each line
    for (int t = threadIdx.x; t < H; t += NT) rootsH[t] = roots_g[2 * t];   // e^{-2 pi i t / H}
    for (int t = threadIdx.x; t <= H; t += NT) wk[t] = roots_g[t];          // e^{-2 pi i t / M}
    for (int t = threadIdx.x; t < M; t += NT) {   // 1/2 -+ sin(pi t / M)
        const double sn = half_g[t].y;
        cpm[t] = make_double2(0.5 - sn, 0.5 + sn);
    }
    for (int t = threadIdx.x; t < L; t += NT) cs[t] = half_g[t].x;

    // ---- load (every global load of the tile before any shared store; the
    // transform runs in place): x_0..x_M of line s into the real array buf1 + s LS
    size_t base;
    int nvalid;
    double v[ITER];
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
            reinterpret_cast<double *>(buf1 + s * LS)[i] = v[it];
        }
    }
    __syncthreads();

    // ---- pre-processing: z_m = y_{2m} + i y_{2m+1} into buf0; 2 X_1 per line
    for (int t = threadIdx.x; t < S * H; t += NT) {
        const int s = t / H;
        const int m = t - s * H;
        const double *xr = reinterpret_cast<const double *>(buf1 + s * LS);
        const double2 c0 = cpm[2 * m], c1 = cpm[2 * m + 1];
        const double y0 = fma(c0.x, xr[2 * m], c0.y * xr[M - 2 * m]);
        const double y1 = fma(c1.x, xr[2 * m + 1], c1.y * xr[M - 2 * m - 1]);
        buf0[s * LS + PAD(m)] = make_double2(y0, y1);
    }
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    for (int s = warp; s < S; s += NT / 32) {
        const double *xr = reinterpret_cast<const double *>(buf1 + s * LS);
        double acc = 0.0;
        for (int j = lane; j < L; j += 32) {
            const double w = (j == 0 || j == M) ? 1.0 : 2.0;   // 2 w_j
            acc = fma(w * xr[j], cs[j], acc);
        }
#pragma unroll
        for (int d = 16; d > 0; d >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, d);
        if (lane == 0) x1[s] = acc;
    }
    __syncthreads();

    double2 *src = buf0, *dst = buf1;
    fstages<double, H, S, 1, Rs...>(src, dst, rootsH);

    // ---- post-processing, one warp per line: lane l takes the KL consecutive
    // k = KL l .. KL l + KL - 1 of 0..H - 1 (the last lane with work also takes
    // k = H); even outputs 2 X_{2k} = 2 Re Y_k, odd outputs by a per-lane prefix
    // sum and a warp scan of a_0 = 2 X_1, a_k = -2 Im Y_k
    constexpr int KL = (H + 31) / 32;
    for (int s = warp; s < S; s += NT / 32) {
        const double2 *Z = src + s * LS;
        double *Xr = reinterpret_cast<double *>(dst + s * LS);   // 2 X_k at index k
        double pre[KL];
        double run = 0.0;
#pragma unroll
        for (int c = 0; c < KL; ++c) {
            const int k = lane * KL + c;
            if (k < H) {
                const double2 A = Z[PAD(k)];
                const double2 B = Z[PAD(k == 0 ? 0 : H - k)];   // conj(B) enters
                const double p = A.x + B.x, q = A.y - B.y, r = A.y + B.y, t = A.x - B.x;
                const double2 w = wk[k];   // (cos, -sin)
                Xr[2 * k] = fma(w.x, r, fma(w.y, t, p));         // 2 X_{2k} = 2 Re Y_k
                run += (k == 0) ? x1[s] : -fma(w.y, r, fma(-w.x, t, q));
            }
            pre[c] = run;
        }
        if (lane == 0) {   // k = H: Y_H = Z_0.x - Z_0.y
            const double2 A = Z[PAD(0)];
            Xr[M] = 2.0 * (A.x - A.y);
        }
        double tot = run;
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            const double o = __shfl_up_sync(0xffffffffu, tot, d);
            if (lane >= d) tot += o;
        }
        double before = __shfl_up_sync(0xffffffffu, tot, 1);
        if (lane == 0) before = 0.0;
#pragma unroll
        for (int c = 0; c < KL; ++c) {
            const int k = lane * KL + c;
            if (k < H) Xr[2 * k + 1] = before + pre[c];   // 2 X_{2k+1}
        }
    }
    __syncthreads();

    // ---- store: scale X (Xr holds 2 X)
    const double hs = 0.5 * scale;
    if (AXIS == HS_AXIS_X) {
        const int nel = nvalid * L;
#pragma unroll
        for (int it = 0; it < ITER; ++it) {
            const int e = threadIdx.x + it * NT;
            if (e < nel) {
                const int s = e / L;
                out[base + e] = hs * reinterpret_cast<const double *>(dst + s * LS)[e - s * L];
            }
        }
    } else {
#pragma unroll
        for (int it = 0; it < ITER; ++it) {
            const int e = threadIdx.x + it * NT;
            const int k = e / S, s = e - k * S;
            if (e < S * L && s < nvalid)
                out[base + (size_t)k * nx + s] = hs * reinterpret_cast<const double *>(dst + s * LS)[k];
        }
    }
}

template <int M, int... Rs>
hs_status launch_dct_m(int axis, const double *in, double *out, const double2 *roots,
                       const double2 *half, long nrows, int nx, int nplanes, double scale,
                       cudaStream_t st) {
    if (axis == HS_AXIS_X) {
        constexpr int S = DctHalfLines<M, HS_AXIS_X>::value;
        constexpr size_t smem = dct_half_smem<M, S>();
        static_assert(smem <= 227 * 1024, "transform tile exceeds shared memory");
        auto k = dct_half_kernel<HS_AXIS_X, M, S, Rs...>;
        if (cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) !=
            cudaSuccess)
            return HS_ERR_CUDA;
        k<<<(unsigned)((nrows + S - 1) / S), 256, smem, st>>>(in, out, roots, half, nrows, nx,
                                                              scale);
    } else {
        constexpr int S = DctHalfLines<M, HS_AXIS_Y>::value;
        constexpr size_t smem = dct_half_smem<M, S>();
        static_assert(smem <= 227 * 1024, "transform tile exceeds shared memory");
        auto k = dct_half_kernel<HS_AXIS_Y, M, S, Rs...>;
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
    switch (M) {   // radices of the M/2-point FFT
        case 32: HS_D(32, 16);
        case 64: HS_D(64, 8, 4);
        case 96: HS_D(96, 16, 3);
        case 128: HS_D(128, 16, 4);
        case 192: HS_D(192, 16, 6);
        case 256: HS_D(256, 16, 8);
        case 384: HS_D(384, 16, 12);
        case 512: HS_D(512, 16, 16);
        case 768: HS_D(768, 16, 8, 3);
        case 1024: HS_D(1024, 16, 16, 2);
        default: return hs_launch_dct_generic(axis, M, in, out, half, nrows, nx, nplanes, scale, s);
    }
#undef HS_D
}
