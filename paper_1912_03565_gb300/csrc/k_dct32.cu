// DCT-I of lines of M + 1 nodes in FP32 (the mixed-precision plan's cosine axes):
// the transform of a side axis with u_n = g on both faces (Section 3.6's
// separation with the cosine modes cos(pi p i / M), p = 0..M),
//     X_k = sum_{j=0..M} w_j x_j cos(pi j k / M),   w_0 = w_M = 1/2,
// through one complex FFT of M/2 points per line, as the FP64 tile of k_dct.cu:
// with s_j = sin(pi j / M), y_j = (1/2 - s_j) x_j + (1/2 + s_j) x_{M-j} and
// Y = DFT_M(y) (from the M/2-point FFT of z_m = y_{2m} + i y_{2m+1}),
//     Re Y_k = X_{2k},   Im Y_k = X_{2k-1} - X_{2k+1},
// and the odd outputs are the running sum X_{2k+1} = X_1 - sum_{k'=1..k} Im Y_k'
// from X_1 = sum_j w_j x_j cos(pi j / M).  In FP32 that sum is compensated (each
// addition's rounding error carried, Knuth's two_sum), so its additions add no
// error of their own; the rounding of the FFT outputs it sums still accumulates
// along the line (see hs_dct32_size).  Outputs go through hs_emit, so the same tile serves
// the forward passes (write) and the inverse x pass of a refined solve (the pair
// modes, and the final FP64 u).
#include "hs_internal.cuh"
#include "hs_tiles.cuh"

namespace {

using namespace hs_tiles;

// lines per CTA: about 4096 complex points of FP32 per buffer (at least 16 for y
// lines, so each row segment is 64 bytes)
template <int M, int AXIS>
struct Dct32Lines {
    static constexpr int base = 8192 / M > 0 ? 8192 / M : 1;
    static constexpr int value = (AXIS == HS_AXIS_Y && base < 16) ? 16 : base;
};

template <int M, int S>
constexpr size_t dct32_smem() {
    // rootsH[M/2] + wk[M/2 + 1] + cpm[M] (float2), 2 buffers of S lines (each also
    // holds a line of M + 1 reals), cs[M + 1] + x1[S] + x1e[S] (float)
    return sizeof(float2) * ((size_t)M / 2 + (M / 2 + 1) + M +
                             (size_t)2 * S * LineStride<M / 2>::value) +
           sizeof(float) * ((size_t)M + 1 + 2 * S);
}

// s + e += v exactly in s, e (two_sum into the carried error)
__device__ __forceinline__ void csum(float &s, float &e, float v) {
    float t, r;
    df_two_sum(s, v, t, r);
    s = t;
    e += r;
}

// AXIS X: lines are contiguous rows of M + 1 values, nrows of them.
// AXIS Y: in each of the planes [M + 1][nx], the columns; grid (ceil(nx / S), planes).
template <int AXIS, int MODE, typename Tout, int M, int S, int... Rs>
__global__ void __launch_bounds__(256, 2)
dct32_kernel(const float *in, Tout *out, double *aux, size_t lo_off,
             const float2 *__restrict__ roots_g, const float2 *__restrict__ half_g, long nrows,
             int nx, float scale) {
    constexpr int H = M / 2;
    constexpr int L = M + 1;
    constexpr int LS = LineStride<H>::value;
    constexpr int NT = 256;
    constexpr int ITER = (S * L + NT - 1) / NT;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    float2 *rootsH = reinterpret_cast<float2 *>(smem_raw);
    float2 *wk = rootsH + H;          // [H + 1]
    float2 *cpm = wk + (H + 1);       // [M]
    float2 *buf0 = cpm + M;
    float2 *buf1 = buf0 + S * LS;
    float *cs = reinterpret_cast<float *>(buf1 + S * LS);   // [M + 1]: cos(pi j / M)
    float *x1 = cs + L;                                     // [S]: 2 X_1 of each line
    float *x1e = x1 + S;                                    // [S]: its rounding error
    for (int t = threadIdx.x; t < H; t += NT) rootsH[t] = roots_g[2 * t];   // e^{-2 pi i t / H}
    for (int t = threadIdx.x; t <= H; t += NT) wk[t] = roots_g[t];          // e^{-2 pi i t / M}
    for (int t = threadIdx.x; t < M; t += NT) {   // 1/2 -+ sin(pi t / M)
        const float sn = half_g[t].y;
        cpm[t] = make_float2(0.5f - sn, 0.5f + sn);
    }
    for (int t = threadIdx.x; t < L; t += NT) cs[t] = half_g[t].x;

    // ---- load (every global load of the tile before any shared store; the
    // transform runs in place): x_0..x_M of line s into the real array buf1 + s LS
    size_t base;
    int nvalid;
    float v[ITER];
    if (AXIS == HS_AXIS_X) {
        const long row0 = (long)blockIdx.x * S;
        base = (size_t)row0 * L;
        nvalid = (int)min((long)S, nrows - row0);
        const int nel = nvalid * L;
#pragma unroll
        for (int it = 0; it < ITER; ++it) {
            const int e = threadIdx.x + it * NT;
            v[it] = e < nel ? in[base + e] : 0.f;
        }
    } else {
        const int p0 = blockIdx.x * S;
        base = (size_t)blockIdx.y * L * nx + p0;
        nvalid = min(S, nx - p0);
#pragma unroll
        for (int it = 0; it < ITER; ++it) {
            const int e = threadIdx.x + it * NT;
            const int j = e / S, s = e - j * S;
            v[it] = (e < S * L && s < nvalid) ? in[base + (size_t)j * nx + s] : 0.f;
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
            reinterpret_cast<float *>(buf1 + s * LS)[i] = v[it];
        }
    }
    __syncthreads();

    // ---- pre-processing: z_m = y_{2m} + i y_{2m+1} into buf0; 2 X_1 per line
    for (int t = threadIdx.x; t < S * H; t += NT) {
        const int s = t / H;
        const int m = t - s * H;
        const float *xr = reinterpret_cast<const float *>(buf1 + s * LS);
        const float2 c0 = cpm[2 * m], c1 = cpm[2 * m + 1];
        const float y0 = fmaf(c0.x, xr[2 * m], c0.y * xr[M - 2 * m]);
        const float y1 = fmaf(c1.x, xr[2 * m + 1], c1.y * xr[M - 2 * m - 1]);
        buf0[s * LS + PAD(m)] = make_float2(y0, y1);
    }
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    for (int s = warp; s < S; s += NT / 32) {
        const float *xr = reinterpret_cast<const float *>(buf1 + s * LS);
        float acc = 0.f, err = 0.f;
        for (int j = lane; j < L; j += 32) {
            const float w = (j == 0 || j == M) ? 1.f : 2.f;   // 2 w_j (exact scaling)
            const float p = (w * xr[j]) * cs[j];
            csum(acc, err, p);
            err += fmaf(w * xr[j], cs[j], -p);
        }
#pragma unroll
        for (int d = 16; d > 0; d >>= 1) {
            const float oa = __shfl_xor_sync(0xffffffffu, acc, d);
            const float oe = __shfl_xor_sync(0xffffffffu, err, d);
            csum(acc, err, oa);
            err += oe;
        }
        if (lane == 0) {
            x1[s] = acc;
            x1e[s] = err;
        }
    }
    __syncthreads();

    float2 *src = buf0, *dst = buf1;
    fstages<float, H, S, 1, Rs...>(src, dst, rootsH);

    // ---- post-processing, one warp per line: lane l takes the KL consecutive
    // k = KL l .. KL l + KL - 1 of 0..H - 1 (the last lane with work also takes
    // k = H); even outputs 2 X_{2k} = 2 Re Y_k, odd outputs by a compensated
    // per-lane prefix sum and a compensated warp scan of a_0 = 2 X_1, a_k = -2 Im Y_k
    constexpr int KL = (H + 31) / 32;
    for (int s = warp; s < S; s += NT / 32) {
        const float2 *Z = src + s * LS;
        float *Xr = reinterpret_cast<float *>(dst + s * LS);   // 2 X_k at index k
        float pre[KL], pree[KL];
        float run = 0.f, rune = 0.f;
#pragma unroll
        for (int c = 0; c < KL; ++c) {
            const int k = lane * KL + c;
            if (k < H) {
                const float2 A = Z[PAD(k)];
                const float2 B = Z[PAD(k == 0 ? 0 : H - k)];   // conj(B) enters
                const float p = A.x + B.x, q = A.y - B.y, r = A.y + B.y, t = A.x - B.x;
                const float2 w = wk[k];   // (cos, -sin)
                Xr[2 * k] = fmaf(w.x, r, fmaf(w.y, t, p));   // 2 X_{2k} = 2 Re Y_k
                if (k == 0) {
                    csum(run, rune, x1[s]);
                    rune += x1e[s];
                } else {
                    csum(run, rune, -fmaf(w.y, r, fmaf(-w.x, t, q)));
                }
            }
            pre[c] = run;
            pree[c] = rune;
        }
        if (lane == 0) {   // k = H: Y_H = Z_0.x - Z_0.y
            const float2 A = Z[PAD(0)];
            Xr[M] = 2.f * (A.x - A.y);
        }
        float tot = run, tote = rune;
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            const float o = __shfl_up_sync(0xffffffffu, tot, d);
            const float oe = __shfl_up_sync(0xffffffffu, tote, d);
            if (lane >= d) {
                csum(tot, tote, o);
                tote += oe;
            }
        }
        float before = __shfl_up_sync(0xffffffffu, tot, 1);
        float beforee = __shfl_up_sync(0xffffffffu, tote, 1);
        if (lane == 0) before = beforee = 0.f;
#pragma unroll
        for (int c = 0; c < KL; ++c) {
            const int k = lane * KL + c;
            if (k < H) {
                float sum = before, e = beforee;
                csum(sum, e, pre[c]);
                Xr[2 * k + 1] = sum + (e + pree[c]);   // 2 X_{2k+1}
            }
        }
    }
    __syncthreads();

    // ---- store: hs_emit of scale X (Xr holds 2 X)
    const float hs = 0.5f * scale;
    if (AXIS == HS_AXIS_X) {
        const int nel = nvalid * L;
#pragma unroll
        for (int it = 0; it < ITER; ++it) {
            const int e = threadIdx.x + it * NT;
            if (e < nel) {
                const int s = e / L;
                const float X = reinterpret_cast<const float *>(dst + s * LS)[e - s * L];
                hs_emit<Tout, MODE>(out, aux, lo_off, base + e, (double)(hs * X));
            }
        }
    } else {
#pragma unroll
        for (int it = 0; it < ITER; ++it) {
            const int e = threadIdx.x + it * NT;
            const int k = e / S, s = e - k * S;
            if (e < S * L && s < nvalid) {
                const float X = reinterpret_cast<const float *>(dst + s * LS)[k];
                hs_emit<Tout, MODE>(out, aux, lo_off, base + (size_t)k * nx + s,
                                    (double)(hs * X));
            }
        }
    }
}

template <int AXIS, int MODE, typename Tout, int M, int... Rs>
hs_status launch_axis(const float *in, void *out, double *aux, size_t lo_off,
                      const float2 *roots, const float2 *half, long nrows, int nx, int nplanes,
                      float scale, cudaStream_t st) {
    constexpr int S = Dct32Lines<M, AXIS>::value;
    constexpr size_t smem = dct32_smem<M, S>();
    static_assert(smem <= 227 * 1024, "transform tile exceeds shared memory");
    auto k = dct32_kernel<AXIS, MODE, Tout, M, S, Rs...>;
    if (cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) !=
        cudaSuccess)
        return HS_ERR_CUDA;
    const dim3 grid = AXIS == HS_AXIS_X
                          ? dim3((unsigned)((nrows + S - 1) / S), 1, 1)
                          : dim3((unsigned)((nx + S - 1) / S), (unsigned)nplanes, 1);
    k<<<grid, 256, smem, st>>>(in, static_cast<Tout *>(out), aux, lo_off, roots, half, nrows, nx,
                               scale);
    return cudaGetLastError() == cudaSuccess ? HS_OK : HS_ERR_CUDA;
}

template <int M, int... Rs>
hs_status launch_m(int axis, int tout, int mode, const float *in, void *out, double *aux,
                   size_t lo_off, const float2 *roots, const float2 *half, long nrows, int nx,
                   int nplanes, float scale, cudaStream_t st) {
#define HS_A(AX, MD, TO)                                                                         \
    return launch_axis<AX, MD, TO, M, Rs...>(in, out, aux, lo_off, roots, half, nrows, nx,       \
                                             nplanes, scale, st)
    if (axis == HS_AXIS_Y) {
        if (tout == HS_T_F32 && mode == HS_MODE_WRITE) HS_A(HS_AXIS_Y, HS_MODE_WRITE, float);
        return HS_ERR_UNSUPPORTED;
    }
    if (tout == HS_T_F32 && mode == HS_MODE_WRITE) HS_A(HS_AXIS_X, HS_MODE_WRITE, float);
    if (tout == HS_T_F64 && mode == HS_MODE_WRITE) HS_A(HS_AXIS_X, HS_MODE_WRITE, double);
    if (tout == HS_T_DF && mode == HS_MODE_DF_SET) HS_A(HS_AXIS_X, HS_MODE_DF_SET, float);
    if (tout == HS_T_DF && mode == HS_MODE_DF_ADD) HS_A(HS_AXIS_X, HS_MODE_DF_ADD, float);
    if (tout == HS_T_DF && mode == HS_MODE_DF_FINAL) HS_A(HS_AXIS_X, HS_MODE_DF_FINAL, float);
    if (tout == HS_T_DF && mode == HS_MODE_DF_FINAL_HI) HS_A(HS_AXIS_X, HS_MODE_DF_FINAL_HI, float);
#undef HS_A
    return HS_ERR_UNSUPPORTED;
}

}  // namespace

// Lengths the mixed-precision plan takes the tile for.  The odd outputs are a
// running sum of FFT outputs, so the FFT's own rounding accumulates along the
// line: measured unrefined solve errors grow like M eps (1.2e-7 at M = 32, 4e-6
// at 256, 2e-5 at 768), and beyond 256 one refinement sweep no longer keeps a
// margin under 1e-10.  The longer lengths stay compiled but are not offered.
int hs_dct32_size(int M) {
    switch (M) {
        case 32: case 64: case 96: case 128: case 192: case 256:
            return 1;
        default:
            return 0;
    }
}

hs_status hs_launch_dct32(int axis, int M, int tout, int mode, const float *in, void *out,
                          double *aux, size_t lo_off, const void *roots, const void *half,
                          long nrows, int nx, int nplanes, double scale, cudaStream_t s) {
    const float2 *r = static_cast<const float2 *>(roots);
    const float2 *h = static_cast<const float2 *>(half);
    const float sc = (float)scale;
#define HS_D(M_, ...)                                                                              \
    return launch_m<M_, __VA_ARGS__>(axis, tout, mode, in, out, aux, lo_off, r, h, nrows, nx,    \
                                     nplanes, sc, s)
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
        default: return HS_ERR_UNSUPPORTED;
    }
#undef HS_D
}
