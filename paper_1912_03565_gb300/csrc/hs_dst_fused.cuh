// DST-I tiles with fewer shared-memory passes (FP32).
//
// Same transform as dst_fast_tile (hs_tiles.cuh): the odd extension of a line
// of N = M - 1 values, packed as M complex points z_n = e_{2n} + i e_{2n+1},
// a length-M complex FFT (Stockham, radices R1, middle..., RL), and
// X_k = [(W_{M-k}.y - W_k.y) + cos(pi k/M)(W_k.x - W_{M-k}.x)
//        + sin(pi k/M)(W_k.y + W_{M-k}.y)] / 4  (Section 3.6's DST by FFT).
// Two passes through shared memory are removed:
//   * the first radix stage takes its R1 inputs straight from global memory
//     (each z_n is two elements of the extension, read where they lie in the
//     line, mirrored and negated past the middle), instead of the line being
//     written to shared memory first and read back;
//   * x-lines only: the last stage keeps its outputs W_K, K = j + Ns r, in
//     registers and gets the partner W_{M-K} from lane Ns - j of the same line
//     with a warp shuffle, so the pairing needs no shared-memory pass either.
// A two-stage length (M = R1 RL) then moves each point through shared memory
// once (stage-1 store, last-stage load) instead of four times.  y-lines keep
// the shared-memory pairing: their lanes run across lines for coalescing.
#pragma once

#include "hs_tiles.cuh"

namespace hs_tiles {

// In-place length-32 DFT (forward) as 4 x 8: the length-4 and length-8 DFTs use
// the constant 48th roots, the twiddles W_32^(n2 k1) between them come from the
// line's table of M-th roots (W_32^m = W_M^(m M / 32)).  Natural order in; the
// result X[k1 + 4 k2] is left at x[8 k1 + k2] (see nat()).
__device__ __forceinline__ void dft32_inplace(float2 *x, const float2 *roots, int stride) {
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
                const float2 r = roots[n2 * k1 * stride];
                a = make_float2(a.x * r.x - a.y * r.y, a.x * r.y + a.y * r.x);
            }
            x[8 * k1 + n2] = a;
        }
    }
#pragma unroll
    for (int k1 = 0; k1 < 4; ++k1) Dft<float, 8>::run(x + 8 * k1);
}

// Where output r of dft_regs<R> is stored.
template <int R>
__host__ __device__ constexpr int nat(int r) {
    return R == 32 ? 8 * (r % 4) + r / 4 : r;
}

// In-register DFT of length R: constant roots where R divides 48, else 32.
template <int R, int M>
__device__ __forceinline__ void dft_regs(float2 *v, const float2 *roots) {
    if constexpr (R == 32)
        dft32_inplace(v, roots, M / 32);
    else
        Dft<float, R>::run(v);
}

// Element m of the odd extension of the line at `row` (m in [0, 2M)).
template <bool COH, typename Tin, int M>
__device__ __forceinline__ float ext_x(const Tin *row, int m) {
    if (m == 0 || m == M) return 0.f;
    if (m < M) return (float)ldc<COH>(row + (m - 1));
    return -(float)ldc<COH>(row + (2 * M - m - 1));
}

// One Stockham stage of radix R done in place: every thread loads the inputs of
// all its butterflies (CNT of them) into registers, the block synchronises, and
// the outputs overwrite the same buffer.  One line buffer instead of two: twice
// the CTAs fit in shared memory where that was the limit.
template <int M, int S, int R, int Ns>
__device__ __forceinline__ void fstage_inplace(float2 *buf, const float2 *roots) {
    constexpr int LS = LineStride<M>::value;
    constexpr int MR = M / R;
    constexpr int stride = M / (Ns * R);
    constexpr int NT = 256;
    constexpr int TOT = S * MR;
    constexpr int CNT = (TOT + NT - 1) / NT;
    float2 v[CNT][R];
#pragma unroll
    for (int c = 0; c < CNT; ++c) {
        const int t = threadIdx.x + c * NT;
        if (t < TOT) {
            const int sl = t / MR;
            const int j = t - sl * MR;
            const float2 *x = buf + sl * LS;
#pragma unroll
            for (int r = 0; r < R; ++r) v[c][r] = x[PAD(j + r * MR)];
        }
    }
    __syncthreads();
#pragma unroll
    for (int c = 0; c < CNT; ++c) {
        const int t = threadIdx.x + c * NT;
        if (t < TOT) {
            const int sl = t / MR;
            const int j = t - sl * MR;
            const int k = j % Ns;
            if (Ns > 1 && k > 0) {
#pragma unroll
                for (int r = 1; r < R; ++r) {
                    const float2 w = roots[k * r * stride];
                    const float2 a = v[c][r];
                    v[c][r] = make_float2(a.x * w.x - a.y * w.y, a.x * w.y + a.y * w.x);
                }
            }
            Dft<float, R>::run(v[c]);
            const int idxD = (j / Ns) * Ns * R + k;
            float2 *y = buf + sl * LS;
#pragma unroll
            for (int r = 0; r < R; ++r) y[PAD(idxD + r * Ns)] = v[c][r];
        }
    }
    __syncthreads();
}

template <int M, int S, int Ns>
__device__ __forceinline__ void fstages_inplace(float2 *, const float2 *) {}

template <int M, int S, int Ns, int R, int... Rest>
__device__ __forceinline__ void fstages_inplace(float2 *buf, const float2 *roots) {
    fstage_inplace<M, S, R, Ns>(buf, roots);
    fstages_inplace<M, S, Ns * R, Rest...>(buf, roots);
}

// Registers of the in-place stages: every stage after the first (and the last
// one of y tiles, which goes back through shared memory) holds at most 32
// complex values per thread.
template <int M, int S, int R>
__host__ __device__ constexpr bool stage_fits() {
    return ((S * (M / R) + 255) / 256) * R <= 32;
}
template <int AXIS, int M, int S, int R1, int RL, int... Rmid>
__host__ __device__ constexpr bool fused_inplace() {
    return (stage_fits<M, S, Rmid>() && ... && true) &&
           (AXIS == HS_AXIS_X || stage_fits<M, S, RL>());
}

// Shared memory of a fused tile: the two root tables and one line buffer per
// line (in place) or two.
template <int AXIS, int M, int S, int R1, int RL, int... Rmid>
__host__ __device__ constexpr size_t fused_smem() {
    return sizeof(float2) *
           ((size_t)2 * M + 1 +
            (size_t)(fused_inplace<AXIS, M, S, R1, RL, Rmid...>() ? 1 : 2) * S *
                LineStride<M>::value);
}

// One CTA: S whole lines.  Radices: R1 first, RL last, Rmid... in between.
template <typename Tin, typename Tout, int AXIS, int MODE, int M, int S, bool COH, int R1, int RL,
          int... Rmid>
__device__ __forceinline__ void dst_fused_tile(const Tin *in, Tout *out, double *aux,
                                               const float2 *roots_g, const float2 *half_g,
                                               int Nx, int Ny, int Nz, float scale,
                                               unsigned char *smem_raw, int bx, int by) {
    constexpr int N = M - 1;
    constexpr int LS = LineStride<M>::value;
    constexpr int NT = 256;
    static_assert(R1 != 32, "the first stage runs before the root table is complete");
    constexpr int B1 = M / R1;   // first-stage butterflies per line
    constexpr int NsL = M / RL;  // butterflies (and Ns) of the last stage
    const size_t lo_off = (size_t)Nx * Ny * Nz;
    (void)lo_off;
    float2 *roots = reinterpret_cast<float2 *>(smem_raw);
    float2 *half = roots + M;
    float2 *buf0 = half + (M + 1);
    float2 *buf1 = buf0 + S * LS;
    for (int t = threadIdx.x; t < M; t += NT) roots[t] = roots_g[t];
    for (int t = threadIdx.x; t <= M; t += NT) half[t] = half_g[t];

    // ---- stage 1 from global memory
    long row0 = 0;
    int nvalid;
    size_t base;
    if constexpr (AXIS == HS_AXIS_X) {
        const long nrows = (long)Ny * Nz;
        row0 = (long)bx * S;
        nvalid = (int)min((long)S, nrows - row0);
        base = (size_t)row0 * N;
    } else {
        const int p0 = bx * S;
        nvalid = min(S, Nx - p0);
        base = (size_t)by * N * Nx + p0;
    }
    for (int t = threadIdx.x; t < S * B1; t += NT) {
        // x: lanes run along a line (t = s B1 + j); y: across lines (t = j S + s),
        // so consecutive lanes read consecutive columns of a row
        const int s = AXIS == HS_AXIS_X ? t / B1 : t % S;
        const int j = AXIS == HS_AXIS_X ? t - s * B1 : t / S;
        float2 v[R1];
        if (s < nvalid) {
            if constexpr (AXIS == HS_AXIS_X) {
                const Tin *row = in + base + (size_t)s * N;
#pragma unroll
                for (int r = 0; r < R1; ++r) {
                    const int n = j + r * B1;
                    v[r].x = ext_x<COH, Tin, M>(row, 2 * n);
                    v[r].y = ext_x<COH, Tin, M>(row, 2 * n + 1);
                }
            } else {
                const Tin *col = in + base + s;
#pragma unroll
                for (int r = 0; r < R1; ++r) {
                    const int n = j + r * B1;
                    const int m0 = 2 * n, m1 = 2 * n + 1;
                    v[r].x = (m0 == 0 || m0 == M) ? 0.f
                             : (m0 < M ? (float)ldc<COH>(col + (size_t)(m0 - 1) * Nx)
                                       : -(float)ldc<COH>(col + (size_t)(2 * M - m0 - 1) * Nx));
                    v[r].y = (m1 < M) ? (float)ldc<COH>(col + (size_t)(m1 - 1) * Nx)
                                      : -(float)ldc<COH>(col + (size_t)(2 * M - m1 - 1) * Nx);
                }
            }
        } else {
#pragma unroll
            for (int r = 0; r < R1; ++r) v[r] = make_float2(0.f, 0.f);
        }
        dft_regs<R1, M>(v, roots);
        float2 *y = buf0 + s * LS;
#pragma unroll
        for (int r = 0; r < R1; ++r) y[PAD(j * R1 + r)] = v[r];
    }
    __syncthreads();

    constexpr bool INPL = fused_inplace<AXIS, M, S, R1, RL, Rmid...>();
    float2 *src = buf0, *dst = buf1;
    if constexpr (INPL)
        fstages_inplace<M, S, R1, Rmid...>(buf0, roots);   // middle stages, one buffer
    else
        fstages<float, M, S, R1, Rmid...>(src, dst, roots);  // each ends in a barrier

    const float q = scale * 0.25f;
    if constexpr (AXIS == HS_AXIS_X) {
        // ---- last stage in registers, pairing by shuffles within the line's lanes
        static_assert(NsL <= 32 && (32 % NsL) == 0, "a line's last-stage lanes must share a warp");
        // whole warps take part in every shuffle: the loop runs over a multiple of
        // 32 lanes; lanes past the tile's S lines read nothing and store nothing
        constexpr int NB = ((S * NsL + 31) / 32) * 32;
        const int nel_rows = nvalid;
        for (int t = threadIdx.x; t < NB; t += NT) {
            const int s = t / NsL;
            const int j = t - s * NsL;
            const bool inl = s < S;
            const float2 *x = src + (inl ? s : 0) * LS;
            float2 v[RL];
#pragma unroll
            for (int r = 0; r < RL; ++r) v[r] = inl ? x[PAD(j + r * NsL)] : make_float2(0.f, 0.f);
            if (j > 0) {
#pragma unroll
                for (int r = 1; r < RL; ++r) {
                    const float2 w = roots[j * r];
                    const float2 a = v[r];
                    v[r] = make_float2(a.x * w.x - a.y * w.y, a.x * w.y + a.y * w.x);
                }
            }
            dft_regs<RL, M>(v, roots);   // v[nat(r)] = W_{j + NsL r}
            const int lane = threadIdx.x & 31;
            const int src_lane = (lane & ~(NsL - 1)) | ((NsL - j) & (NsL - 1));
            const bool live = inl && s < nel_rows;
            Tout *orow = out + base + (size_t)s * N;
            double *arow = aux ? aux + base + (size_t)s * N : nullptr;
            constexpr bool RMW = MODE == HS_MODE_DF_ADD || MODE == HS_MODE_DF_FINAL ||
                                 MODE == HS_MODE_DF_FINAL_HI;
            // read-modify-write modes: every (hi, lo) of this lane's outputs is
            // loaded before the first store (the stores could alias the loads as
            // far as the compiler knows, which would serialise them); for a
            // length-32 last stage the registers are not there, so it loads per output
            constexpr bool PRE = RMW && RL <= 24;
            float uh[PRE ? RL : 1], ul[PRE ? RL : 1];
            if constexpr (PRE) {
#pragma unroll
                for (int r = 0; r < RL; ++r) {
                    const int K = j + NsL * r;
                    const bool ok = live && K > 0;
                    uh[r] = ok ? ldc<COH>(orow + (K - 1)) : 0.f;
                    ul[r] = ok && MODE != HS_MODE_DF_FINAL_HI ? ldc<COH>(orow + (K - 1) + lo_off)
                                                              : 0.f;
                }
            }
#pragma unroll
            for (int r = 0; r < RL; ++r) {
                // partner of K = j + NsL r is M - K = (NsL - j) + NsL (RL - 1 - r) (j > 0),
                // or NsL (RL - r) held by this lane (j = 0)
                const float px = __shfl_sync(0xffffffffu, v[nat<RL>(RL - 1 - r)].x, src_lane);
                const float py = __shfl_sync(0xffffffffu, v[nat<RL>(RL - 1 - r)].y, src_lane);
                const float2 Wk = v[nat<RL>(r)];
                const float2 Wm = j > 0 ? make_float2(px, py) : v[nat<RL>((RL - r) % RL)];
                const int K = j + NsL * r;
                if (live && K > 0) {
                    const float2 cs = half[K];
                    const float X =
                        ((Wm.y - Wk.y) + cs.x * (Wk.x - Wm.x) + cs.y * (Wk.y + Wm.y)) * q;
                    if constexpr (PRE) {
                        dfloat a;
                        a.hi = uh[r];
                        a.lo = ul[r];
                        const dfloat sum = df_add(a, df_of(X));
                        if constexpr (MODE == HS_MODE_DF_ADD) {
                            orow[K - 1] = sum.hi;
                            orow[K - 1 + lo_off] = sum.lo;
                        } else {
                            arow[K - 1] = (double)sum.hi + (double)sum.lo;
                        }
                    } else {
                        hs_emit<Tout, MODE>(orow, arow, lo_off, (size_t)(K - 1), (double)X);
                    }
                }
            }
        }
    } else {
        // ---- last stage through shared memory, pairing read back per output
        if constexpr (INPL) {
            fstage_inplace<M, S, RL, NsL>(buf0, roots);
            src = buf0;
        } else {
            fstage<float, M, S, RL, NsL>(src, dst, roots);
            __syncthreads();
            src = dst;
        }
#pragma unroll 4
        for (int e = threadIdx.x; e < S * N; e += NT) {
            const int kk = e / S;
            const int s = e - kk * S;
            if (s < nvalid) {
                const int k = kk + 1;
                const float2 Wk = src[s * LS + PAD(k)];
                const float2 Wm = src[s * LS + PAD(M - k)];
                const float2 cs = half[k];
                const float X = ((Wm.y - Wk.y) + cs.x * (Wk.x - Wm.x) + cs.y * (Wk.y + Wm.y)) * q;
                hs_emit<Tout, MODE>(out, aux, lo_off, base + (size_t)kk * Nx + s, (double)X);
            }
        }
    }
}

}  // namespace hs_tiles
