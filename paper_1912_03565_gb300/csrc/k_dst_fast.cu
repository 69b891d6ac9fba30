// Compile-time-sized DST-I kernels for the line lengths the solver meets most
// (N + 1 = M in {32, 64, 96, 128, 192, 256, 384, 512, 768, 1024}).
//
// Same algorithm as k_dst.cu (odd extension, length-M complex FFT of the
// packed line, X_k from W_k and W_{M-k}; Section 3.6's "2D DST by FFT"), but
// every size, radix and stride is a template constant: the index arithmetic
// of the Stockham stages becomes shifts and multiplies, and each thread does
// one radix-R butterfly (R up to 16) in registers per stage, so a 256-point
// line takes two passes through shared memory instead of four.  In-register
// DFTs of size R = R1 R2 use the Cooley-Tukey split n = R2 n1 + n2,
// k = k1 + R1 k2 with the twiddles W_R^(n2 k1) taken from the 48th roots
// below (every R used divides 48).
#include "hs_internal.cuh"

namespace {

__device__ __forceinline__ double cos48(int k) {
    switch (k) {
        case 0: return 1.0;
        case 1: return 0.9914448613738104;
        case 2: return 0.9659258262890683;
        case 3: return 0.9238795325112867;
        case 4: return 0.8660254037844387;
        case 5: return 0.7933533402912352;
        case 6: return 0.7071067811865476;
        case 7: return 0.6087614290087207;
        case 8: return 0.5000000000000001;
        case 9: return 0.38268343236508984;
        case 10: return 0.25881904510252074;
        case 11: return 0.1305261922200517;
        case 12: return 0.0;
        case 13: return -0.1305261922200516;
        case 14: return -0.25881904510252063;
        case 15: return -0.3826834323650895;
        case 16: return -0.4999999999999998;
        case 17: return -0.6087614290087207;
        case 18: return -0.7071067811865475;
        case 19: return -0.793353340291235;
        case 20: return -0.8660254037844387;
        case 21: return -0.9238795325112867;
        case 22: return -0.9659258262890682;
        case 23: return -0.9914448613738104;
        case 24: return -1.0;
        case 25: return -0.9914448613738104;
        case 26: return -0.9659258262890683;
        case 27: return -0.9238795325112868;
        case 28: return -0.8660254037844388;
        case 29: return -0.7933533402912352;
        case 30: return -0.7071067811865479;
        case 31: return -0.6087614290087209;
        case 32: return -0.5000000000000004;
        case 33: return -0.3826834323650895;
        case 34: return -0.25881904510252063;
        case 35: return -0.13052619222005163;
        case 36: return 0.0;
        case 37: return 0.13052619222005127;
        case 38: return 0.2588190451025203;
        case 39: return 0.38268343236508917;
        case 40: return 0.5000000000000001;
        case 41: return 0.6087614290087199;
        case 42: return 0.7071067811865474;
        case 43: return 0.7933533402912349;
        case 44: return 0.8660254037844384;
        case 45: return 0.9238795325112868;
        case 46: return 0.9659258262890681;
        case 47: return 0.9914448613738104;
        default: return 0.0;
    }
}
__device__ __forceinline__ double sin48(int k) {
    switch (k) {
        case 0: return 0.0;
        case 1: return 0.13052619222005157;
        case 2: return 0.25881904510252074;
        case 3: return 0.3826834323650898;
        case 4: return 0.49999999999999994;
        case 5: return 0.6087614290087207;
        case 6: return 0.7071067811865475;
        case 7: return 0.7933533402912352;
        case 8: return 0.8660254037844386;
        case 9: return 0.9238795325112867;
        case 10: return 0.9659258262890683;
        case 11: return 0.9914448613738104;
        case 12: return 1.0;
        case 13: return 0.9914448613738104;
        case 14: return 0.9659258262890683;
        case 15: return 0.9238795325112868;
        case 16: return 0.8660254037844387;
        case 17: return 0.7933533402912352;
        case 18: return 0.7071067811865476;
        case 19: return 0.6087614290087209;
        case 20: return 0.49999999999999994;
        case 21: return 0.3826834323650899;
        case 22: return 0.258819045102521;
        case 23: return 0.130526192220052;
        case 24: return 0.0;
        case 25: return -0.13052619222005177;
        case 26: return -0.2588190451025208;
        case 27: return -0.38268343236508967;
        case 28: return -0.4999999999999997;
        case 29: return -0.6087614290087207;
        case 30: return -0.7071067811865471;
        case 31: return -0.7933533402912349;
        case 32: return -0.8660254037844384;
        case 33: return -0.9238795325112868;
        case 34: return -0.9659258262890683;
        case 35: return -0.9914448613738104;
        case 36: return -1.0;
        case 37: return -0.9914448613738105;
        case 38: return -0.9659258262890684;
        case 39: return -0.923879532511287;
        case 40: return -0.8660254037844386;
        case 41: return -0.7933533402912357;
        case 42: return -0.7071067811865477;
        case 43: return -0.6087614290087209;
        case 44: return -0.5000000000000004;
        case 45: return -0.38268343236508956;
        case 46: return -0.25881904510252157;
        case 47: return -0.13052619222005168;
        default: return 0.0;
    }
}

template <typename T> struct Cx;
template <> struct Cx<double> { typedef double2 t; };
template <> struct Cx<float> { typedef float2 t; };

template <typename T2, typename T>
__device__ __forceinline__ T2 mk2(T x, T y) {
    T2 r;
    r.x = x;
    r.y = y;
    return r;
}

// y * W_R^m (forward sign): W = cos(2 pi m/R) - i sin(2 pi m/R)
template <typename Tc, int R>
__device__ __forceinline__ typename Cx<Tc>::t twiddle_const(typename Cx<Tc>::t y, int m) {
    const int k = (m % R) * (48 / R);
    if (k == 0) return y;
    if (k == 12) return mk2<typename Cx<Tc>::t>(y.y, -y.x);     // -i
    if (k == 24) return mk2<typename Cx<Tc>::t>(-y.x, -y.y);    // -1
    if (k == 36) return mk2<typename Cx<Tc>::t>(-y.y, y.x);     // +i
    const Tc c = (Tc)cos48(k), s = (Tc)sin48(k);
    return mk2<typename Cx<Tc>::t>(y.x * c + y.y * s, y.y * c - y.x * s);
}

template <typename Tc, int R> struct Dft;

template <typename Tc> struct Dft<Tc, 2> {
    typedef typename Cx<Tc>::t T2;
    static __device__ __forceinline__ void run(T2 *v) {
        const T2 a = v[0], b = v[1];
        v[0] = mk2<T2>(a.x + b.x, a.y + b.y);
        v[1] = mk2<T2>(a.x - b.x, a.y - b.y);
    }
};

template <typename Tc> struct Dft<Tc, 3> {
    typedef typename Cx<Tc>::t T2;
    static __device__ __forceinline__ void run(T2 *v) {
        const Tc k3 = (Tc)0.86602540378443864676;
        const T2 a = v[0];
        const T2 s = mk2<T2>(v[1].x + v[2].x, v[1].y + v[2].y);
        const T2 d = mk2<T2>(v[1].x - v[2].x, v[1].y - v[2].y);
        const T2 t = mk2<T2>(a.x - (Tc)0.5 * s.x, a.y - (Tc)0.5 * s.y);
        v[0] = mk2<T2>(a.x + s.x, a.y + s.y);
        v[1] = mk2<T2>(t.x + k3 * d.y, t.y - k3 * d.x);
        v[2] = mk2<T2>(t.x - k3 * d.y, t.y + k3 * d.x);
    }
};

template <typename Tc> struct Dft<Tc, 4> {
    typedef typename Cx<Tc>::t T2;
    static __device__ __forceinline__ void run(T2 *v) {
        const T2 s02 = mk2<T2>(v[0].x + v[2].x, v[0].y + v[2].y);
        const T2 d02 = mk2<T2>(v[0].x - v[2].x, v[0].y - v[2].y);
        const T2 s13 = mk2<T2>(v[1].x + v[3].x, v[1].y + v[3].y);
        const T2 d13 = mk2<T2>(v[1].y - v[3].y, v[3].x - v[1].x);  // -i (v1 - v3)
        v[0] = mk2<T2>(s02.x + s13.x, s02.y + s13.y);
        v[2] = mk2<T2>(s02.x - s13.x, s02.y - s13.y);
        v[1] = mk2<T2>(d02.x + d13.x, d02.y + d13.y);
        v[3] = mk2<T2>(d02.x - d13.x, d02.y - d13.y);
    }
};

// R = R1 * R2 with R1 = 4 when possible, else 2, else 3.
template <typename Tc, int R> struct Dft {
    typedef typename Cx<Tc>::t T2;
    static constexpr int R1 = (R % 4 == 0) ? 4 : ((R % 2 == 0) ? 2 : 3);
    static constexpr int R2 = R / R1;
    static __device__ __forceinline__ void run(T2 *x) {
        T2 y[R];
#pragma unroll
        for (int n2 = 0; n2 < R2; ++n2) {
            T2 t[R1];
#pragma unroll
            for (int n1 = 0; n1 < R1; ++n1) t[n1] = x[R2 * n1 + n2];
            Dft<Tc, R1>::run(t);
#pragma unroll
            for (int k1 = 0; k1 < R1; ++k1) y[n2 * R1 + k1] = twiddle_const<Tc, R>(t[k1], n2 * k1);
        }
#pragma unroll
        for (int k1 = 0; k1 < R1; ++k1) {
            T2 t[R2];
#pragma unroll
            for (int n2 = 0; n2 < R2; ++n2) t[n2] = y[n2 * R1 + k1];
            Dft<Tc, R2>::run(t);
#pragma unroll
            for (int k2 = 0; k2 < R2; ++k2) x[k1 + R1 * k2] = t[k2];
        }
    }
};

// Shared-memory layout of a line: complex element i lives at PAD(i) = i + i/16,
// so the stride-16 writes of a first radix-16 stage fall in distinct banks.
__device__ __forceinline__ int PAD(int i) { return i + (i >> 4); }
template <int M> struct LineStride { static constexpr int value = M + (M >> 4) + 1; };

// One Stockham stage of radix R on S lines of length M (line stride LS).
template <typename Tc, int M, int S, int R, int Ns>
__device__ __forceinline__ void fstage(const typename Cx<Tc>::t *__restrict__ src,
                                       typename Cx<Tc>::t *__restrict__ dst,
                                       const typename Cx<Tc>::t *__restrict__ roots) {
    typedef typename Cx<Tc>::t T2;
    constexpr int LS = LineStride<M>::value;
    constexpr int MR = M / R;
    constexpr int stride = M / (Ns * R);
    for (int t = threadIdx.x; t < S * MR; t += blockDim.x) {
        const int s = t / MR;
        const int j = t - s * MR;
        const int k = j % Ns;
        const T2 *x = src + s * LS;
        T2 *y = dst + s * LS;
        T2 v[R];
#pragma unroll
        for (int r = 0; r < R; ++r) v[r] = x[PAD(j + r * MR)];
        if (Ns > 1 && k > 0) {
#pragma unroll
            for (int r = 1; r < R; ++r) {
                const T2 w = roots[k * r * stride];
                const T2 a = v[r];
                v[r] = mk2<T2>(a.x * w.x - a.y * w.y, a.x * w.y + a.y * w.x);
            }
        }
        Dft<Tc, R>::run(v);
        const int idxD = (j / Ns) * Ns * R + k;
#pragma unroll
        for (int r = 0; r < R; ++r) y[PAD(idxD + r * Ns)] = v[r];
    }
}

template <typename Tc, int M, int S, int Ns>
__device__ __forceinline__ void fstages(typename Cx<Tc>::t *&src, typename Cx<Tc>::t *&dst,
                                        const typename Cx<Tc>::t *roots) {}

template <typename Tc, int M, int S, int Ns, int R, int... Rest>
__device__ __forceinline__ void fstages(typename Cx<Tc>::t *&src, typename Cx<Tc>::t *&dst,
                                        const typename Cx<Tc>::t *roots) {
    fstage<Tc, M, S, R, Ns>(src, dst, roots);
    __syncthreads();
    typename Cx<Tc>::t *t = src;
    src = dst;
    dst = t;
    fstages<Tc, M, S, Ns * R, Rest...>(src, dst, roots);
}

// Real element m of a line's odd extension, stored inside the padded complex layout.
__device__ __forceinline__ int ZPAD(int m) { return 2 * PAD(m >> 1) + (m & 1); }

// FP32 tiles use up to ~74 KB of shared memory, so three CTAs fit an SM; the
// register cap keeps the third one resident.
template <typename Tc, typename Tin, typename Tout, int AXIS, int MODE, int M, int S, int... Rs>
__global__ void __launch_bounds__(256, (sizeof(Tc) == 4 ? 3 : 1))
dst_fast_kernel(const Tin *in, Tout *out, double *aux, const typename Cx<Tc>::t *roots_g,
                const typename Cx<Tc>::t *half_g, int Nx, int Ny, int Nz, Tc scale,
                const int *skip) {
    if (skip && *skip) return;
    typedef typename Cx<Tc>::t T2;
    constexpr int N = M - 1;
    constexpr int LS = LineStride<M>::value;
    constexpr int twoM = 2 * M;
    constexpr int NT = 256;
    constexpr int ITER = (S * N + NT - 1) / NT;  // elements per thread in load/store phases
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const size_t lo_off = (size_t)Nx * Ny * Nz;  // lo plane of a double-float output
    (void)lo_off;
    T2 *roots = reinterpret_cast<T2 *>(smem_raw);
    T2 *half = roots + M;
    T2 *buf0 = half + (M + 1);
    T2 *buf1 = buf0 + S * LS;
    for (int t = threadIdx.x; t < M; t += NT) roots[t] = roots_g[t];
    for (int t = threadIdx.x; t <= M; t += NT) half[t] = half_g[t];

    Tc *z = reinterpret_cast<Tc *>(buf0);
    for (int s = threadIdx.x; s < S; s += NT) {
        z[s * 2 * LS + ZPAD(0)] = (Tc)0;
        z[s * 2 * LS + ZPAD(M)] = (Tc)0;
    }
    size_t base;
    int nvalid;
    // all global loads of the tile are issued before any shared-memory store
    Tc v[ITER];
    if (AXIS == HS_AXIS_X) {
        const long nrows = (long)Ny * Nz;
        const long row0 = (long)blockIdx.x * S;
        base = (size_t)row0 * N;
        nvalid = (int)min((long)S, nrows - row0);
        const int nel = nvalid * N;
#pragma unroll
        for (int it = 0; it < ITER; ++it) {
            const int e = threadIdx.x + it * NT;
            v[it] = (e < nel) ? (Tc)in[base + e] : (Tc)0;
        }
#pragma unroll
        for (int it = 0; it < ITER; ++it) {
            const int e = threadIdx.x + it * NT;
            if (e < S * N) {
                const int s = e / N;
                const int i = e - s * N;
                z[s * 2 * LS + ZPAD(i + 1)] = v[it];
                z[s * 2 * LS + ZPAD(twoM - 1 - i)] = -v[it];
            }
        }
    } else {
        const int p0 = blockIdx.x * S;
        base = (size_t)blockIdx.y * N * Nx + p0;
        nvalid = min(S, Nx - p0);
#pragma unroll
        for (int it = 0; it < ITER; ++it) {
            const int e = threadIdx.x + it * NT;
            const int j = e / S;
            const int s = e - j * S;
            v[it] = (e < S * N && s < nvalid) ? (Tc)in[base + (size_t)j * Nx + s] : (Tc)0;
        }
#pragma unroll
        for (int it = 0; it < ITER; ++it) {
            const int e = threadIdx.x + it * NT;
            if (e < S * N) {
                const int j = e / S;
                const int s = e - j * S;
                z[s * 2 * LS + ZPAD(j + 1)] = v[it];
                z[s * 2 * LS + ZPAD(twoM - 1 - j)] = -v[it];
            }
        }
    }
    __syncthreads();

    T2 *src = buf0, *dst = buf1;
    fstages<Tc, M, S, 1, Rs...>(src, dst, roots);

    const Tc q = scale * (Tc)0.25;
    if (AXIS == HS_AXIS_X) {
        const int nel = nvalid * N;
        if constexpr (MODE == HS_MODE_DF_ADD || MODE == HS_MODE_DF_FINAL) {
            // read every (hi, lo) of the tile before any store
            float uh[ITER], ul[ITER];
#pragma unroll
            for (int it = 0; it < ITER; ++it) {
                const int e = threadIdx.x + it * NT;
                uh[it] = (e < nel) ? out[base + e] : 0.f;
                ul[it] = (e < nel) ? out[base + e + lo_off] : 0.f;
            }
#pragma unroll
            for (int it = 0; it < ITER; ++it) {
                const int e = threadIdx.x + it * NT;
                if (e < nel) {
                    const int s = e / N;
                    const int k = e - s * N + 1;
                    const T2 Wk = src[s * LS + PAD(k)];
                    const T2 Wm = src[s * LS + PAD(M - k)];
                    const T2 cs = half[k];
                    const Tc X = ((Wm.y - Wk.y) + cs.x * (Wk.x - Wm.x) + cs.y * (Wk.y + Wm.y)) * q;
                    dfloat a;
                    a.hi = uh[it];
                    a.lo = ul[it];
                    const dfloat r = df_add(a, df_of((float)X));
                    if constexpr (MODE == HS_MODE_DF_ADD) {
                        out[base + e] = r.hi;
                        out[base + e + lo_off] = r.lo;
                    } else {
                        aux[base + e] = (double)r.hi + (double)r.lo;
                    }
                }
            }
        } else {
#pragma unroll
            for (int it = 0; it < ITER; ++it) {
                const int e = threadIdx.x + it * NT;
                if (e < nel) {
                    const int s = e / N;
                    const int k = e - s * N + 1;
                    const T2 Wk = src[s * LS + PAD(k)];
                    const T2 Wm = src[s * LS + PAD(M - k)];
                    const T2 cs = half[k];
                    const Tc X = ((Wm.y - Wk.y) + cs.x * (Wk.x - Wm.x) + cs.y * (Wk.y + Wm.y)) * q;
                    hs_emit<Tout, MODE>(out, aux, lo_off, base + e, (double)X);
                }
            }
        }
    } else {
#pragma unroll
        for (int it = 0; it < ITER; ++it) {
            const int e = threadIdx.x + it * NT;
            const int kk = e / S;
            const int s = e - kk * S;
            if (e < S * N && s < nvalid) {
                const int k = kk + 1;
                const T2 Wk = src[s * LS + PAD(k)];
                const T2 Wm = src[s * LS + PAD(M - k)];
                const T2 cs = half[k];
                const Tc X = ((Wm.y - Wk.y) + cs.x * (Wk.x - Wm.x) + cs.y * (Wk.y + Wm.y)) * q;
                hs_emit<Tout, MODE>(out, aux, lo_off, base + (size_t)kk * Nx + s, (double)X);
            }
        }
    }
}

// Lines per CTA: about 4096 (FP32) or 2048 (FP64) complex points per buffer;
// y-lines at least 16 (FP32) / 8 (FP64) so each row segment is 64 bytes; never
// more than fits in 227 KB of shared memory.
template <typename Tc, int M, int AXIS>
struct Lines {
    static constexpr int pts = (sizeof(Tc) == 4) ? 4096 : 2048;
    static constexpr int base = (pts / M) > 0 ? (pts / M) : 1;
    static constexpr int ymin = (sizeof(Tc) == 4) ? 16 : 8;
    static constexpr int want = (AXIS == HS_AXIS_Y && base < ymin) ? ymin : base;
    static constexpr int fit = (int)((227 * 1024 / (2 * sizeof(Tc)) - (2 * M + 1)) /
                                     (2 * (M + (M >> 4) + 1)));
    static constexpr int value = want < fit ? want : fit;
};

template <typename Tc, int M, int S>
constexpr size_t fast_smem() {
    return sizeof(typename Cx<Tc>::t) * ((size_t)2 * M + 1 + (size_t)2 * S * LineStride<M>::value);
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
    if (tc == HS_T_F64) {
        const DstAxis &ax = P->axd[axis];
        if (tin == HS_T_F64 && tout == HS_T_F64 && mode == HS_MODE_WRITE)
            return launch_sized<double, double, double, HS_MODE_WRITE>(P, axis, ax, in, out, scale, s, aux);
        if (tin == HS_T_F64 && tout == HS_T_F64 && mode == HS_MODE_ADD)
            return launch_sized<double, double, double, HS_MODE_ADD>(P, axis, ax, in, out, scale, s, aux);
        return HS_ERR_UNSUPPORTED;
    }
    const DstAxis &ax = P->axf[axis];
    if (tin == HS_T_F64 && tout == HS_T_F32 && mode == HS_MODE_WRITE)
        return launch_sized<float, double, float, HS_MODE_WRITE>(P, axis, ax, in, out, scale, s, aux);
    if (tin == HS_T_F32 && tout == HS_T_F32 && mode == HS_MODE_WRITE)
        return launch_sized<float, float, float, HS_MODE_WRITE>(P, axis, ax, in, out, scale, s, aux);
    if (tin == HS_T_F32 && tout == HS_T_F64 && mode == HS_MODE_WRITE)
        return launch_sized<float, float, double, HS_MODE_WRITE>(P, axis, ax, in, out, scale, s, aux);
    if (tin == HS_T_F32 && tout == HS_T_F64 && mode == HS_MODE_ADD)
        return launch_sized<float, float, double, HS_MODE_ADD>(P, axis, ax, in, out, scale, s, aux);
    if (tin == HS_T_F32 && tout == HS_T_DF && mode == HS_MODE_DF_SET)
        return launch_sized<float, float, float, HS_MODE_DF_SET>(P, axis, ax, in, out, scale, s, aux);
    if (tin == HS_T_F32 && tout == HS_T_DF && mode == HS_MODE_DF_ADD)
        return launch_sized<float, float, float, HS_MODE_DF_ADD>(P, axis, ax, in, out, scale, s, aux);
    if (tin == HS_T_F32 && tout == HS_T_DF && mode == HS_MODE_DF_FINAL)
        return launch_sized<float, float, float, HS_MODE_DF_FINAL>(P, axis, ax, in, out, scale, s, aux);
    return HS_ERR_UNSUPPORTED;
}
