// DST-I passes of the mixed path as sine-matrix GEMMs on the fifth-generation
// tensor cores (tcgen05).  Section 3.6 writes the 2-D transform of a z-plane
// as the matrix product W_l = V^T F_l with the sine basis V; along one axis
// this is, for every line x of length N,
//     X_p = sum_{i=1..N} sin(pi p i / (N + 1)) x_i,   p = 1..N,
// i.e. OUT = IN S^T with S[p, i] = sin(pi p i / (N + 1)) (S is symmetric).
// For N + 1 <= 256 the whole contraction fits one MMA tile in N, and at
// GB300's tensor rate it costs less than moving the lines through HBM.
//
// Precision (the mixed path computes its transforms in FP32): each line is
// scaled by a power of two 2^e so that its largest magnitude lies in
// [2^14, 2^15), then split into two FP16 parts x = x0 + x1 (x0 = fp16(x),
// x1 = fp16(x - x0): 22 significant bits); S is split the same way (s0, s1,
// computed in FP64 on the host).  The MMA accumulates x0 s0 + x0 s1 + x1 s0
// in FP32 in tensor memory (the dropped x1 s1 term is 2^-22 of the product),
// and the epilogue multiplies by 2^-e and the transform's scale.  The result
// matches an FP32 transform to a few units of 2^-22 of the line's largest
// magnitude.
//
// Kernel structure (persistent, one or two CTAs per SM, 416 threads):
//   warps 0-7   producers: per tile, the power-of-two scale of each of the
//               128 lines (one read of the lines), then per K chunk of 64 the
//               FP16 split of the 128 lines written to shared memory in the
//               128-byte-swizzle K-major layout; thread 0 also issues the bulk
//               copy of the chunk's pre-swizzled sine-matrix split tiles;
//   warps 8-11  epilogue: the FP32 accumulator from tensor memory (each warp
//               its 32 lanes = lines), scaled, to global memory;
//   warp 12     tensor memory allocation and, on one thread, the MMAs
//               (3 per K step of 16) and their commits.
// Two shared-memory stages and two tensor-memory accumulators let the loads of
// tile t + 1 and the epilogue of tile t - 1 overlap the MMAs of tile t.
// Every wait is bounded: a wait that runs out sets the launch's error flag and
// the CTA winds down (waiting, bounded, for its own copies and MMAs, then
// freeing its tensor memory).
//
// x axis: a line is a row of the interior array (contiguous); tiles are 128
// consecutive rows.  y axis: a line is a column p of one z-plane (stride Nx);
// tiles are 128 consecutive columns of one plane, so every global access of
// the producers (a warp reads 32 consecutive p) and of the epilogue (a warp
// writes 32 consecutive p) is coalesced.
#include <cuda_fp16.h>
#include <math.h>
#include <string.h>

#include <algorithm>
#include <cmath>

#include "hs_internal.cuh"
#include "hs_tc.cuh"

namespace {

using namespace hs_tc;

constexpr int GM = 128;         // lines per tile (the MMA's M)
constexpr int GKC = 64;         // K elements per stage (one 128-byte swizzle row of FP16)
constexpr int GSTAGES = 2;
constexpr int NPROD = 8;        // producer warps
constexpr int NEPI = 4;         // epilogue warps
constexpr int MMA_WARP = NPROD + NEPI;
constexpr int NTHR = (NPROD + NEPI + 1) * 32;
constexpr uint32_t WAIT_POLLS = 1u << 24;   // per wait: about one second

struct GemmArgs {
    const float *in;
    void *out;
    double *aux;          // FP64 u of the pair-final mode
    size_t lo_off;        // lo plane offset of pair outputs (interior count)
    int Nx, Ny, Nz;
    int N;                // line length of the axis (contraction length and outputs)
    long nlines;          // x: Ny Nz rows; y: Nx columns per plane
    int pblocks;          // y: column blocks per plane
    int ntiles;
    float scale;
    const uint4 *bsplit;  // [chunks][2][NPAD rows][8 x 16 bytes], pre-swizzled
    int *err;             // set to 1 when a wait gave up
    const int *skip;      // refinement converged: the pass returns at once
};

// byte offset of 16-byte chunk c8 (0..7) of row m in a 128-byte-swizzle K-major tile
__device__ __forceinline__ uint32_t swz(int m, int c8) {
    return (uint32_t)((m >> 3) * 1024 + (m & 7) * 128 + ((c8 ^ (m & 7)) << 4));
}

// 2^k as an FP32 number, -126 <= k <= 127
__device__ __forceinline__ float pow2f(int k) { return __int_as_float((k + 127) << 23); }

// power-of-two exponent e with max * 2^e in [2^14, 2^15) (0 for an all-zero line)
__device__ __forceinline__ int line_exponent(float mx) {
    return mx > 0.f ? 14 - ilogbf(mx) : 0;
}

// x 2^e split into FP16 parts: lo16 bits of `h0w` / `h1w` take element 2i, hi16 element 2i+1
__device__ __forceinline__ void split_pair(float a, float b, float s1, float s2, uint32_t &w0,
                                           uint32_t &w1) {
    const float as = (a * s1) * s2, bs = (b * s1) * s2;
    const __half2 h0 = __floats2half2_rn(as, bs);
    const float2 back = __half22float2(h0);
    const __half2 h1 = __floats2half2_rn(as - back.x, bs - back.y);
    w0 = *reinterpret_cast<const uint32_t *>(&h0);
    w1 = *reinterpret_cast<const uint32_t *>(&h1);
}

}  // namespace

namespace {

// Shared memory of one CTA: GSTAGES stages of {A0, A1 (the line splits, 128 x
// 64 FP16 each), B0, B1 (the sine-matrix splits, NPAD x 64 FP16 each)}, then the
// control block (mbarriers, tensor memory address, abort flag, line exponents).
template <int NPAD>
struct GemmLayout {
    static constexpr uint32_t A_BYTES = GM * 128;
    static constexpr uint32_t B_BYTES = NPAD * 128;
    static constexpr uint32_t STAGE = 2 * A_BYTES + 2 * B_BYTES;
    static constexpr uint32_t NACC = NPAD <= 32 ? 32 : (NPAD <= 64 ? 64 : (NPAD <= 128 ? 128 : 256));
    static constexpr uint32_t TMEM_COLS = 2 * NACC;
    static constexpr uint32_t CTRL = 2048;
    // x epilogue: a 32 x 33 FP32 transposition tile per epilogue warp
    static constexpr uint32_t EPI = NEPI * 32 * 33 * 4;
    static constexpr uint32_t BYTES = GSTAGES * STAGE + CTRL + EPI + 1024;   // + alignment slack
};

enum { B_FULL = 0, B_BFULL = 2, B_EMPTY = 4, B_ACCFULL = 6, B_ACCEMPTY = 8, B_EXP = 10,
       B_DRAIN = 12, B_COUNT = 13 };

template <int AXIS, int MODE, typename Tout, int NPAD, int KCH>
__global__ void __launch_bounds__(NTHR, 1) dst_gemm_kernel(GemmArgs g) {
    typedef GemmLayout<NPAD> LY;
    if (g.skip && *g.skip) return;
    extern __shared__ uint8_t smem_raw[];
    uint8_t *base = reinterpret_cast<uint8_t *>(
        (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~static_cast<uintptr_t>(1023));
    uint8_t *ctrl = base + GSTAGES * LY::STAGE;
    uint64_t *bar = reinterpret_cast<uint64_t *>(ctrl);
    uint32_t *s_tmem = reinterpret_cast<uint32_t *>(ctrl + 8 * B_COUNT);
    volatile int *s_abort = reinterpret_cast<volatile int *>(ctrl + 8 * B_COUNT + 4);
    int *sexp = reinterpret_cast<int *>(ctrl + 256);   // [2][GM] line exponents
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;

    if (tid == 0) {
        for (int s = 0; s < GSTAGES; ++s) {
            mbar_init(&bar[B_FULL + s], NPROD * 32);
            mbar_init(&bar[B_BFULL + s], 1);
            mbar_init(&bar[B_EMPTY + s], 1);
        }
        for (int b = 0; b < 2; ++b) {
            mbar_init(&bar[B_ACCFULL + b], 1);
            mbar_init(&bar[B_ACCEMPTY + b], NEPI * 32);
            mbar_init(&bar[B_EXP + b], NPROD * 32);
        }
        mbar_init(&bar[B_DRAIN], 1);
        *s_abort = 0;
        asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
    }
    if (warp == MMA_WARP) tmem_alloc(s_tmem, LY::TMEM_COLS);
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tbase = *s_tmem;

    auto fail = [&]() {
        *s_abort = 1;
        atomicExch(g.err, 1);
    };

    if (warp < NPROD) {
        // ------------------------------------------------------------ producers
        uint32_t c = 0;                       // K chunks started by this CTA
        int last_v[GSTAGES] = {-1, -1};       // thread 0: last bulk copy per stage
        bool ok = true;
        for (int t = blockIdx.x, tt = 0; ok && t < g.ntiles; t += gridDim.x, ++tt) {
            const int buf = tt & 1;
            const uint32_t u = (uint32_t)tt >> 1;
            if (u >= 1 && !mbar_wait(&bar[B_ACCEMPTY + buf], (u - 1) & 1, WAIT_POLLS, s_abort)) {
                fail();
                break;
            }
            // pass 1: power-of-two scale of each of this warp's 16 lines
            int ex[4];   // exponents of the lines whose chunks this lane converts
            const float *lp[4];
            bool lv[4];
            if (AXIS == HS_AXIS_X) {
                // lines m = 16 warp + i; the lane converts lines 16 warp + (lane >> 3) + 4q.
                // Four lines at a time, every load of a group issued before its
                // maxima (a line of N <= 255 is at most 8 loads per lane)
#pragma unroll
                for (int i0 = 0; i0 < 16; i0 += 4) {
                    float v[4][8];
#pragma unroll
                    for (int d = 0; d < 4; ++d) {
                        const long r = (long)t * GM + 16 * warp + i0 + d;
                        const float *row = g.in + (size_t)(r < g.nlines ? r : 0) * g.N;
#pragma unroll
                        for (int u = 0; u < 8; ++u) {
                            const int k = lane + 32 * u;
                            v[d][u] = (r < g.nlines && k < g.N) ? row[k] : 0.f;
                        }
                    }
#pragma unroll
                    for (int d = 0; d < 4; ++d) {
                        float mx = 0.f;
#pragma unroll
                        for (int u = 0; u < 8; ++u) mx = fmaxf(mx, fabsf(v[d][u]));
#pragma unroll
                        for (int o = 16; o > 0; o >>= 1)
                            mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
                        const int i = i0 + d, m = 16 * warp + i;
                        const int e = line_exponent(mx);
                        if (lane == 0) sexp[buf * GM + m] = e;
                        if ((i & 3) == (lane >> 3)) ex[i >> 2] = e;
                    }
                }
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    const int m = 16 * warp + (lane >> 3) + 4 * q;
                    const long r = (long)t * GM + m;
                    lv[q] = r < g.nlines;
                    lp[q] = g.in + (size_t)(lv[q] ? r : 0) * g.N;
                }
            } else {
                // line m = 16 warp + (lane & 15) is column p of plane l; the two
                // half-warps take the two halves of its j range
                const int l = t / g.pblocks, pb = t - l * g.pblocks;
                const int m = 16 * warp + (lane & 15);
                const int p = pb * GM + m;
                const bool valid = p < g.Nx;
                const float *col = g.in + (size_t)l * g.Ny * g.Nx + (valid ? p : 0);
                float mx = 0.f;
                if (valid) {
                    // 16 independent loads per group: the column's latency is paid
                    // once per 16 rows, not once per row
                    const int half = (g.N + 1) / 2;
                    const int j0 = (lane >> 4) * half, j1 = min(g.N, j0 + half);
                    int j = j0;
                    for (; j + 16 <= j1; j += 16) {
                        float v[16];
#pragma unroll
                        for (int u = 0; u < 16; ++u) v[u] = col[(size_t)(j + u) * g.Nx];
#pragma unroll
                        for (int u = 0; u < 16; ++u) mx = fmaxf(mx, fabsf(v[u]));
                    }
                    for (; j < j1; ++j) mx = fmaxf(mx, fabsf(col[(size_t)j * g.Nx]));
                }
                mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, 16));
                const int e = line_exponent(mx);
                if (lane < 16) sexp[buf * GM + m] = e;
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    ex[q] = e;
                    lv[q] = valid;
                    lp[q] = col;
                }
            }
            mbar_arrive(&bar[B_EXP + buf]);   // release: the epilogue reads sexp[buf]
            float s1[4], s2[4];
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                s1[q] = pow2f(ex[q] / 2);
                s2[q] = pow2f(ex[q] - ex[q] / 2);
            }
            // pass 2: the FP16 splits of each K chunk into a free stage
            for (int kc = 0; kc < KCH; ++kc, ++c) {
                const int s = (int)(c & 1);
                const uint32_t v = c >> 1;
                if (v >= 1 && !mbar_wait(&bar[B_EMPTY + s], (v - 1) & 1, WAIT_POLLS, s_abort)) {
                    fail();
                    ok = false;
                    break;
                }
                uint8_t *st = base + s * LY::STAGE;
                if (tid == 0) {
                    mbar_arrive_tx(&bar[B_BFULL + s], 2 * LY::B_BYTES);
                    bulk_g2s(st + 2 * LY::A_BYTES, g.bsplit + (size_t)kc * (2 * LY::B_BYTES / 16),
                             2 * LY::B_BYTES, &bar[B_BFULL + s]);
                    last_v[s] = (int)v;
                }
                // all 32 loads of this lane's chunk pieces first (one memory latency
                // per chunk), then the splits and the swizzled stores
                float x[4][8];
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    const int c8 = AXIS == HS_AXIS_X ? (lane & 7) : (lane >> 4) + 2 * q;
                    const int k0 = kc * GKC + c8 * 8;
#pragma unroll
                    for (int i = 0; i < 8; ++i) {
                        const int k = k0 + i;
                        x[q][i] = 0.f;
                        if (lv[q] && k < g.N)
                            x[q][i] = AXIS == HS_AXIS_X ? lp[q][k] : lp[q][(size_t)k * g.Nx];
                    }
                }
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    int m, c8;
                    if (AXIS == HS_AXIS_X) {
                        m = 16 * warp + (lane >> 3) + 4 * q;
                        c8 = lane & 7;
                    } else {
                        m = 16 * warp + (lane & 15);
                        c8 = (lane >> 4) + 2 * q;
                    }
                    uint4 h0, h1;
                    split_pair(x[q][0], x[q][1], s1[q], s2[q], h0.x, h1.x);
                    split_pair(x[q][2], x[q][3], s1[q], s2[q], h0.y, h1.y);
                    split_pair(x[q][4], x[q][5], s1[q], s2[q], h0.z, h1.z);
                    split_pair(x[q][6], x[q][7], s1[q], s2[q], h0.w, h1.w);
                    const uint32_t off = swz(m, c8);
                    *reinterpret_cast<uint4 *>(st + off) = h0;
                    *reinterpret_cast<uint4 *>(st + LY::A_BYTES + off) = h1;
                }
                fence_async_smem();
                mbar_arrive(&bar[B_FULL + s]);
            }
        }
        // the CTA must not end with its own bulk copies in flight (this wait is not
        // cut short by the abort flag)
        if (tid == 0) {
            volatile int never = 0;
            for (int s = 0; s < GSTAGES; ++s)
                if (last_v[s] >= 0 &&
                    !mbar_wait(&bar[B_BFULL + s], (uint32_t)last_v[s] & 1, WAIT_POLLS, &never))
                    fail();
        }
    } else if (warp < MMA_WARP) {
        // ------------------------------------------------------------- epilogue
        const int w = warp - NPROD;               // == warp % 4: TMEM lanes 32 w .. 32 w + 31
        const int m = 32 * w + lane;              // the line this thread writes
        for (int t = blockIdx.x, tt = 0; t < g.ntiles; t += gridDim.x, ++tt) {
            const int buf = tt & 1;
            const uint32_t u = (uint32_t)tt >> 1;
            if (!mbar_wait(&bar[B_ACCFULL + buf], u & 1, WAIT_POLLS, s_abort) ||
                !mbar_wait(&bar[B_EXP + buf], u & 1, WAIT_POLLS, s_abort)) {
                fail();
                break;
            }
            tc_fence_after();
            const int e = sexp[buf * GM + m];
            const float f1 = pow2f(-(e / 2)), f2 = pow2f(-(e - e / 2));
            size_t o0, ostep;
            bool valid;
            if (AXIS == HS_AXIS_X) {
                const long r = (long)t * GM + m;
                valid = r < g.nlines;
                o0 = (size_t)(valid ? r : 0) * g.N;   // out[r, n] = o0 + n
                ostep = 1;
            } else {
                const int l = t / g.pblocks, pb = t - l * g.pblocks;
                const int p = pb * GM + m;
                valid = p < g.Nx;
                o0 = (size_t)l * g.Ny * g.Nx + (valid ? p : 0);   // out[l, n, p]
                ostep = (size_t)g.Nx;
            }
            const uint32_t tl = tbase + ((uint32_t)(32 * w) << 16) + (uint32_t)buf * LY::NACC;
            if (AXIS == HS_AXIS_X) {
                // lane = line in TMEM; through a transposition tile so that a warp's
                // stores cover 32 consecutive modes of one line (coalesced)
                float *T = reinterpret_cast<float *>(ctrl + LY::CTRL) + w * 32 * 33;
#pragma unroll 1
                for (int c0 = 0; c0 < NPAD; c0 += 32) {
                    float v[32];
                    tmem_ld32(tl + (uint32_t)c0, v);
#pragma unroll
                    for (int k = 0; k < 32; ++k) T[lane * 33 + k] = ((v[k] * f1) * f2) * g.scale;
                    __syncwarp();
                    const int n = c0 + lane;
                    if constexpr (MODE == HS_MODE_DF_ADD || MODE == HS_MODE_DF_FINAL ||
                                  MODE == HS_MODE_DF_FINAL_HI) {
                        // read-modify-write of the pair iterate: 8 lines' (hi, lo) loaded
                        // before any is updated
                        float *o = reinterpret_cast<float *>(g.out);
#pragma unroll 1
                        for (int k0 = 0; k0 < 32; k0 += 8) {
                            float hi[8], lo[8];
#pragma unroll
                            for (int d = 0; d < 8; ++d) {
                                const long r = (long)t * GM + 32 * w + k0 + d;
                                const bool ok = r < g.nlines && n < g.N;
                                const size_t idx = (size_t)(ok ? r : 0) * g.N + (ok ? n : 0);
                                hi[d] = ok ? o[idx] : 0.f;
                                lo[d] = ok && MODE != HS_MODE_DF_FINAL_HI ? o[idx + g.lo_off] : 0.f;
                            }
#pragma unroll
                            for (int d = 0; d < 8; ++d) {
                                const long r = (long)t * GM + 32 * w + k0 + d;
                                if (r < g.nlines && n < g.N) {
                                    const size_t idx = (size_t)r * g.N + n;
                                    dfloat a;
                                    a.hi = hi[d];
                                    a.lo = lo[d];
                                    dfloat b;
                                    b.hi = T[(k0 + d) * 33 + lane];
                                    b.lo = 0.f;
                                    const dfloat sum = df_add(a, b);
                                    if constexpr (MODE == HS_MODE_DF_ADD) {
                                        o[idx] = sum.hi;
                                        o[idx + g.lo_off] = sum.lo;
                                    } else {
                                        g.aux[idx] = (double)sum.hi + (double)sum.lo;
                                    }
                                }
                            }
                        }
                    } else {
#pragma unroll 4
                        for (int kk = 0; kk < 32; ++kk) {
                            const long r = (long)t * GM + 32 * w + kk;
                            if (r < g.nlines && n < g.N)
                                hs_emit<Tout, MODE>(static_cast<Tout *>(g.out), g.aux, g.lo_off,
                                                    (size_t)r * g.N + n, (double)T[kk * 33 + lane]);
                        }
                    }
                    __syncwarp();
                }
                tc_fence_before();
                mbar_arrive(&bar[B_ACCEMPTY + buf]);
                continue;
            }
#pragma unroll 1
            for (int c0 = 0; c0 < NPAD; c0 += 32) {
                float v[32];
                tmem_ld32(tl + (uint32_t)c0, v);
                if (valid) {
#pragma unroll
                    for (int k = 0; k < 32; ++k) {
                        const int n = c0 + k;
                        if (n < g.N)
                            hs_emit<Tout, MODE>(static_cast<Tout *>(g.out), g.aux, g.lo_off,
                                                o0 + (size_t)n * ostep,
                                                (double)(((v[k] * f1) * f2) * g.scale));
                    }
                }
            }
            tc_fence_before();
            mbar_arrive(&bar[B_ACCEMPTY + buf]);
        }
    } else if (lane == 0) {
        // ------------------------------------------------------------------ MMAs
        constexpr uint32_t IDESC = idesc_f16_f32(GM, NPAD);
        uint32_t c = 0;
        bool issued = false;
        bool ok = true;
        for (int t = blockIdx.x, tt = 0; ok && t < g.ntiles; t += gridDim.x, ++tt) {
            const int buf = tt & 1;
            const uint32_t u = (uint32_t)tt >> 1;
            if (u >= 1 && !mbar_wait(&bar[B_ACCEMPTY + buf], (u - 1) & 1, WAIT_POLLS, s_abort)) {
                fail();
                break;
            }
            tc_fence_after();
            const uint32_t dcol = tbase + (uint32_t)buf * LY::NACC;
            for (int kc = 0; kc < KCH; ++kc, ++c) {
                const int s = (int)(c & 1);
                const uint32_t v = c >> 1;
                if (!mbar_wait(&bar[B_FULL + s], v & 1, WAIT_POLLS, s_abort) ||
                    !mbar_wait(&bar[B_BFULL + s], v & 1, WAIT_POLLS, s_abort)) {
                    fail();
                    ok = false;
                    break;
                }
                tc_fence_after();
                const uint32_t st = saddr(base + s * LY::STAGE);
                const uint32_t a0 = st, a1 = st + LY::A_BYTES;
                const uint32_t b0 = st + 2 * LY::A_BYTES, b1 = b0 + LY::B_BYTES;
#pragma unroll
                for (int kk = 0; kk < GKC / 16; ++kk) {
                    const uint32_t ko = (uint32_t)kk * 32;   // 16 FP16 = 32 bytes along K
                    const uint32_t acc = (kc | kk) != 0;
                    mma_f16(dcol, sdesc_sw128(a0 + ko), sdesc_sw128(b0 + ko), IDESC, acc);
                    mma_f16(dcol, sdesc_sw128(a0 + ko), sdesc_sw128(b1 + ko), IDESC, 1);
                    mma_f16(dcol, sdesc_sw128(a1 + ko), sdesc_sw128(b0 + ko), IDESC, 1);
                }
                issued = true;
                mma_commit(&bar[B_EMPTY + s]);   // the stage is free once these MMAs are done
            }
            if (!ok) break;
            mma_commit(&bar[B_ACCFULL + buf]);
        }
        // every MMA of this CTA has completed before the tensor memory is freed
        // (this wait is not cut short by the abort flag)
        if (issued) {
            volatile int never = 0;
            mma_commit(&bar[B_DRAIN]);
            if (!mbar_wait(&bar[B_DRAIN], 0, WAIT_POLLS, &never)) fail();
        }
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (warp == MMA_WARP) tmem_free(tbase, LY::TMEM_COLS);
}

}  // namespace

// =================================================================== host side
namespace {

// Nearest FP16 number (ties to even) of a double, as its bit pattern, from the
// IEEE binary16 definition (normal numbers: 11 significant bits; subnormals:
// spacing 2^-24).  |v| stays far below the FP16 overflow threshold here.
uint16_t half_bits(double v) {
    const uint16_t sign = std::signbit(v) ? 0x8000u : 0u;
    const double a = fabs(v);
    if (a == 0.0) return sign;
    int e2 = 0;
    frexp(a, &e2);
    int E = e2 - 1;   // a in [2^E, 2^(E+1))
    if (E < -14) return (uint16_t)(sign | (uint16_t)nearbyint(ldexp(a, 24)));   // 1024 -> min normal
    double m = nearbyint(ldexp(a, 10 - E));   // [1024, 2048]
    if (m == 2048.0) {
        m = 1024.0;
        ++E;
    }
    return (uint16_t)(sign | (uint16_t)((E + 15) << 10) | (uint16_t)(m - 1024.0));
}

double half_value(uint16_t b) {
    const int E = (b >> 10) & 0x1F, m = b & 0x3FF;
    const double a = E == 0 ? ldexp((double)m, -24) : ldexp((double)(1024 + m), E - 25);
    return (b & 0x8000u) ? -a : a;
}

// sin(pi num / den) with the argument reduced exactly to [0, pi/2] first
double sin_pi_frac(long num, long den) {
    long m = num % (2 * den);
    if (m < 0) m += 2 * den;
    double sign = 1.0;
    if (m >= den) {
        m -= den;
        sign = -1.0;
    }
    if (2 * m > den) m = den - m;
    return sign * sin(M_PI * (double)m / (double)den);
}

int gemm_chunks(int M) { return (M - 1 + GKC - 1) / GKC; }

struct KernelInfo {
    const void *fn;
    int smem;
    int per_sm;
};

template <int AXIS, int MODE, typename Tout, int NPAD>
KernelInfo gemm_kernel_info() {
    constexpr int KCH = (NPAD - 1 + GKC - 1) / GKC;
    static KernelInfo info = [] {
        KernelInfo k;
        k.fn = reinterpret_cast<const void *>(&dst_gemm_kernel<AXIS, MODE, Tout, NPAD, KCH>);
        k.smem = (int)GemmLayout<NPAD>::BYTES;
        k.per_sm = 0;
        if (cudaFuncSetAttribute(&dst_gemm_kernel<AXIS, MODE, Tout, NPAD, KCH>,
                                 cudaFuncAttributeMaxDynamicSharedMemorySize, k.smem) != cudaSuccess ||
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(
                &k.per_sm, &dst_gemm_kernel<AXIS, MODE, Tout, NPAD, KCH>, NTHR, k.smem) !=
                cudaSuccess) {
            cudaGetLastError();
            k.per_sm = 0;
        }
        return k;
    }();
    return info;
}

template <int AXIS, int MODE, typename Tout>
KernelInfo gemm_pick(int M) {
    switch (M) {
        case 32: return gemm_kernel_info<AXIS, MODE, Tout, 32>();
        case 64: return gemm_kernel_info<AXIS, MODE, Tout, 64>();
        case 96: return gemm_kernel_info<AXIS, MODE, Tout, 96>();
        case 128: return gemm_kernel_info<AXIS, MODE, Tout, 128>();
        case 192: return gemm_kernel_info<AXIS, MODE, Tout, 192>();
        case 256: return gemm_kernel_info<AXIS, MODE, Tout, 256>();
        default: return KernelInfo{nullptr, 0, 0};
    }
}

}  // namespace

int hs_dst_gemm_size(int M) {
    return M == 32 || M == 64 || M == 96 || M == 128 || M == 192 || M == 256;
}

size_t hs_dst_gemm_table_bytes(int M) {
    return hs_dst_gemm_size(M) ? (size_t)gemm_chunks(M) * 2 * M * 128 : 0;
}

// The sine matrix S[n, k] = sin(pi (n + 1)(k + 1) / M) (n, k < M - 1; zero
// padding up to M rows and a whole number of 64-wide K chunks), split into
// FP16 parts s0 = fp16(S), s1 = fp16(S - s0), laid out chunk by chunk as the
// kernel's shared-memory B tiles: [chunk][split][row n][128-byte swizzled row].
void hs_dst_gemm_table(int M, uint8_t *host) {
    const int N = M - 1, KCH = gemm_chunks(M);
    memset(host, 0, hs_dst_gemm_table_bytes(M));
    for (int kc = 0; kc < KCH; ++kc)
        for (int n = 0; n < M; ++n)
            for (int kl = 0; kl < GKC; ++kl) {
                const int k = kc * GKC + kl;
                const double v = (n < N && k < N) ? sin_pi_frac((long)(n + 1) * (k + 1), M) : 0.0;
                const uint16_t h0 = half_bits(v);
                const uint16_t h1 = half_bits(v - half_value(h0));
                const size_t off = (size_t)(n >> 3) * 1024 + (n & 7) * 128 +
                                   ((((kl >> 3) ^ (n & 7)) << 4) | ((kl & 7) * 2));
                uint8_t *t0 = host + (size_t)(kc * 2 + 0) * M * 128;
                uint8_t *t1 = host + (size_t)(kc * 2 + 1) * M * 128;
                memcpy(t0 + off, &h0, 2);
                memcpy(t1 + off, &h1, 2);
            }
}

hs_status hs_launch_dst_gemm(const hs_plan_s *P, int axis, int tin, const void *in, int tout,
                             void *out, int mode, double scale, cudaStream_t s, double *aux) {
    const int M = axis == HS_AXIS_X ? P->Nx + 1 : P->Ny + 1;
    if (!P->d_gemm[axis] || !P->d_gemm_err || tin != HS_T_F32 || !hs_dst_gemm_size(M))
        return HS_ERR_UNSUPPORTED;
    KernelInfo k{nullptr, 0, 0};
    if (axis == HS_AXIS_X) {
        if (tout == HS_T_F32 && mode == HS_MODE_WRITE)
            k = gemm_pick<HS_AXIS_X, HS_MODE_WRITE, float>(M);
        else if (tout == HS_T_F64 && mode == HS_MODE_WRITE)
            k = gemm_pick<HS_AXIS_X, HS_MODE_WRITE, double>(M);
        else if (tout == HS_T_DF && mode == HS_MODE_DF_SET)
            k = gemm_pick<HS_AXIS_X, HS_MODE_DF_SET, float>(M);
        else if (tout == HS_T_DF && mode == HS_MODE_DF_ADD)
            k = gemm_pick<HS_AXIS_X, HS_MODE_DF_ADD, float>(M);
        else if (tout == HS_T_DF && mode == HS_MODE_DF_FINAL)
            k = gemm_pick<HS_AXIS_X, HS_MODE_DF_FINAL, float>(M);
        else if (tout == HS_T_DF && mode == HS_MODE_DF_FINAL_HI)
            k = gemm_pick<HS_AXIS_X, HS_MODE_DF_FINAL_HI, float>(M);
    } else if (tout == HS_T_F32 && mode == HS_MODE_WRITE) {
        k = gemm_pick<HS_AXIS_Y, HS_MODE_WRITE, float>(M);
    }
    if (!k.fn || k.per_sm < 1) return HS_ERR_UNSUPPORTED;
    GemmArgs g;
    g.in = static_cast<const float *>(in);
    g.out = out;
    g.aux = aux;
    g.lo_off = (size_t)P->Nx * P->Ny * P->Nz;
    g.Nx = P->Nx;
    g.Ny = P->Ny;
    g.Nz = P->Nz;
    g.N = M - 1;
    if (axis == HS_AXIS_X) {
        g.nlines = (long)P->Ny * P->Nz;
        g.pblocks = 0;
        g.ntiles = (int)((g.nlines + GM - 1) / GM);
    } else {
        g.nlines = P->Nx;
        g.pblocks = (P->Nx + GM - 1) / GM;
        g.ntiles = g.pblocks * P->Nz;
    }
    g.scale = (float)scale;
    g.bsplit = static_cast<const uint4 *>(P->d_gemm[axis]);
    g.err = P->d_gemm_err;
    g.skip = P->cur_skip;
    int sms = 0;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, P->device) != cudaSuccess) {
        cudaGetLastError();
        return HS_ERR_CUDA;
    }
    const int grid = std::min(g.ntiles, sms * k.per_sm);
    void *args[] = {&g};
    if (cudaLaunchKernel(k.fn, dim3(grid), dim3(NTHR), args, (size_t)k.smem, s) != cudaSuccess) {
        cudaGetLastError();
        return HS_ERR_CUDA;
    }
    return HS_OK;
}
