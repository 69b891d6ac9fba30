// DST-I kernels along x (contiguous lines) and y (stride-Nx lines) of an
// interior array [Nz][Ny][Nx] (Section 3.6: the 2-D transform of every
// z-plane, done by FFT).
//
// A line x_1..x_N is odd-extended to z_0..z_{2M-1} (M = N + 1: z_k = x_k,
// z_{2M-k} = -x_k, z_0 = z_M = 0).  Read as M complex numbers
// w_n = z_{2n} + i z_{2n+1}, a length-M complex FFT W gives the length-2M
// transform Z_k = E_k + exp(-i pi k/M) O_k with E_k = (W_k + conj W_{M-k})/2,
// O_k = (W_k - conj W_{M-k})/(2i), and Z_k = -2i X_k, so
//     X_k = [ (d - b) + cos(pi k/M) (a - c) + sin(pi k/M) (b + d) ] / 4,
// with W_k = a + ib and W_{M-k} = c + id.  The FFT is a mixed-radix (4, 2, 3)
// Stockham FFT in shared memory (ping-pong buffers, one barrier per stage).
// Lengths whose M has other prime factors use direct O(N^2) sums.
//
// Each CTA owns S whole lines: for x, S consecutive rows; for y, S
// consecutive columns p of one plane, so every global load and store is a
// run of S contiguous elements across the CTA (coalesced).  The same tile is
// read before it is written, so in-place calls are safe.
#include "hs_internal.cuh"

namespace {

template <typename T> struct Cplx;
template <> struct Cplx<double> { typedef double2 t; };
template <> struct Cplx<float> { typedef float2 t; };

template <typename T2, typename T>
__device__ __forceinline__ T2 mk(T x, T y) {
    T2 r;
    r.x = x;
    r.y = y;
    return r;
}

template <typename T2>
__device__ __forceinline__ T2 cmul(T2 a, T2 b) {
    return mk<T2>(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}

template <typename T2>
__device__ __forceinline__ T2 cadd(T2 a, T2 b) { return mk<T2>(a.x + b.x, a.y + b.y); }
template <typename T2>
__device__ __forceinline__ T2 csub(T2 a, T2 b) { return mk<T2>(a.x - b.x, a.y - b.y); }
// -i * z
template <typename T2>
__device__ __forceinline__ T2 cmi(T2 z) { return mk<T2>(z.y, -z.x); }

template <typename Tc, int R>
__device__ __forceinline__ void dft_small(typename Cplx<Tc>::t *v) {
    typedef typename Cplx<Tc>::t T2;
    if (R == 2) {
        T2 a = v[0], b = v[1];
        v[0] = cadd(a, b);
        v[1] = csub(a, b);
    } else if (R == 4) {
        T2 s02 = cadd(v[0], v[2]), d02 = csub(v[0], v[2]);
        T2 s13 = cadd(v[1], v[3]), d13 = cmi(csub(v[1], v[3]));
        v[0] = cadd(s02, s13);
        v[2] = csub(s02, s13);
        v[1] = cadd(d02, d13);
        v[3] = csub(d02, d13);
    } else {  // R == 3, w = exp(-2 pi i / 3)
        const Tc k3 = (Tc)0.86602540378443864676;
        T2 a = v[0];
        T2 s = cadd(v[1], v[2]), d = csub(v[1], v[2]);
        T2 t = mk<T2>(a.x - (Tc)0.5 * s.x, a.y - (Tc)0.5 * s.y);
        v[0] = cadd(a, s);
        v[1] = mk<T2>(t.x + k3 * d.y, t.y - k3 * d.x);
        v[2] = mk<T2>(t.x - k3 * d.y, t.y + k3 * d.x);
    }
}

template <typename Tc, int R>
__device__ __forceinline__ void stockham_stage(const typename Cplx<Tc>::t *src,
                                               typename Cplx<Tc>::t *dst,
                                               const typename Cplx<Tc>::t *roots, int M, int LS,
                                               int S, int Ns) {
    typedef typename Cplx<Tc>::t T2;
    const int MR = M / R;
    const int stride = M / (Ns * R);
    for (int t = threadIdx.x; t < S * MR; t += blockDim.x) {
        const int s = t / MR;
        const int j = t - s * MR;
        const int k = j % Ns;
        const T2 *x = src + s * LS;
        T2 *y = dst + s * LS;
        T2 v[R];
#pragma unroll
        for (int r = 0; r < R; ++r) {
            v[r] = x[j + r * MR];
            if (r > 0 && k > 0) v[r] = cmul(v[r], roots[k * r * stride]);
        }
        dft_small<Tc, R>(v);
        const int idxD = (j / Ns) * Ns * R + k;
#pragma unroll
        for (int r = 0; r < R; ++r) y[idxD + r * Ns] = v[r];
    }
}

template <typename Tc, typename Tin, typename Tout, int AXIS, int MODE>
__global__ void __launch_bounds__(256)
dst_fft_kernel(DstAxis ax, const Tin *in, Tout *out, double *aux, int Nx, int Ny, int Nz, int S,
               Tc scale, const int *skip) {
    if (skip && *skip) return;
    typedef typename Cplx<Tc>::t T2;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const size_t lo_off = (size_t)Nx * Ny * Nz;  // lo plane of a double-float output
    (void)lo_off;
    const int N = ax.N, M = ax.M;
    const int LS = M + 1;  // padded line stride (complex elements): fewer bank conflicts
    T2 *roots = reinterpret_cast<T2 *>(smem_raw);
    T2 *half = roots + M;
    T2 *buf0 = half + (M + 1);
    T2 *buf1 = buf0 + (size_t)S * LS;

    for (int t = threadIdx.x; t < M; t += blockDim.x)
        roots[t] = reinterpret_cast<const T2 *>(ax.roots)[t];
    for (int t = threadIdx.x; t <= M; t += blockDim.x)
        half[t] = reinterpret_cast<const T2 *>(ax.half)[t];

    // ---- load: odd extension of S lines into buf0 (as 2M reals per line)
    Tc *z = reinterpret_cast<Tc *>(buf0);
    const int twoM = 2 * M;
    const int zs = 2 * LS;  // line stride in reals
    for (int s = threadIdx.x; s < S; s += blockDim.x) {
        z[(size_t)s * zs] = (Tc)0;
        z[(size_t)s * zs + M] = (Tc)0;
    }
    size_t base;
    int nvalid;
    if (AXIS == HS_AXIS_X) {
        const long nrows = (long)Ny * Nz;
        const long row0 = (long)blockIdx.x * S;
        base = (size_t)row0 * Nx;
        nvalid = (int)min((long)S, nrows - row0);
        for (int t = threadIdx.x; t < S * N; t += blockDim.x) {
            const int s = t / N;
            const int i = t - s * N;
            Tc v = (Tc)0;
            if (s < nvalid) v = (Tc)in[base + t];
            z[(size_t)s * zs + i + 1] = v;
            z[(size_t)s * zs + twoM - 1 - i] = -v;
        }
    } else {
        const int p0 = blockIdx.x * S;
        const int l = blockIdx.y;
        base = (size_t)l * Ny * Nx + p0;
        nvalid = min(S, Nx - p0);
        for (int t = threadIdx.x; t < S * N; t += blockDim.x) {
            const int j = t / S;
            const int s = t - j * S;
            Tc v = (Tc)0;
            if (s < nvalid) v = (Tc)in[base + (size_t)j * Nx + s];
            z[(size_t)s * zs + j + 1] = v;
            z[(size_t)s * zs + twoM - 1 - j] = -v;
        }
    }
    __syncthreads();

    // ---- complex FFT of length M on every line
    T2 *src = buf0, *dst = buf1;
    int Ns = 1;
    for (int st = 0; st < ax.nst; ++st) {
        const int R = ax.radix[st];
        if (R == 4)
            stockham_stage<Tc, 4>(src, dst, roots, M, LS, S, Ns);
        else if (R == 2)
            stockham_stage<Tc, 2>(src, dst, roots, M, LS, S, Ns);
        else
            stockham_stage<Tc, 3>(src, dst, roots, M, LS, S, Ns);
        __syncthreads();
        T2 *tmp = src;
        src = dst;
        dst = tmp;
        Ns *= R;
    }

    // ---- post-processing: X_k from W_k and W_{M-k}
    const Tc q = scale * (Tc)0.25;
    if (AXIS == HS_AXIS_X) {
        for (int t = threadIdx.x; t < S * N; t += blockDim.x) {
            const int s = t / N;
            const int k = t - s * N + 1;
            if (s >= nvalid) continue;
            const T2 Wk = src[(size_t)s * LS + k];
            const T2 Wm = src[(size_t)s * LS + (M - k)];
            const T2 cs = half[k];
            const Tc X = ((Wm.y - Wk.y) + cs.x * (Wk.x - Wm.x) + cs.y * (Wk.y + Wm.y)) * q;
            hs_emit<Tout, MODE>(out, aux, lo_off, base + t, (double)X);
        }
    } else {
        for (int t = threadIdx.x; t < S * N; t += blockDim.x) {
            const int kk = t / S;
            const int s = t - kk * S;
            const int k = kk + 1;
            if (s >= nvalid) continue;
            const T2 Wk = src[(size_t)s * LS + k];
            const T2 Wm = src[(size_t)s * LS + (M - k)];
            const T2 cs = half[k];
            const Tc X = ((Wm.y - Wk.y) + cs.x * (Wk.x - Wm.x) + cs.y * (Wk.y + Wm.y)) * q;
            hs_emit<Tout, MODE>(out, aux, lo_off, base + (size_t)kk * Nx + s, (double)X);
        }
    }
}

// Direct sums X_k = sum_i x_i sin(pi k i / M) for lengths without an FFT plan.
template <typename Tc, typename Tin, typename Tout, int AXIS, int MODE>
__global__ void __launch_bounds__(256)
dst_direct_kernel(DstAxis ax, const Tin *in, Tout *out, double *aux, int Nx, int Ny, int Nz, int S,
                  Tc scale, const int *skip) {
    if (skip && *skip) return;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const size_t lo_off = (size_t)Nx * Ny * Nz;  // lo plane of a double-float output
    (void)lo_off;
    const int N = ax.N, M = ax.M, twoM = 2 * M;
    Tc *sint = reinterpret_cast<Tc *>(smem_raw);
    Tc *xs = sint + twoM;
    for (int t = threadIdx.x; t < twoM; t += blockDim.x)
        sint[t] = reinterpret_cast<const Tc *>(ax.sintab)[t];
    size_t base;
    int nvalid;
    if (AXIS == HS_AXIS_X) {
        const long nrows = (long)Ny * Nz;
        const long row0 = (long)blockIdx.x * S;
        base = (size_t)row0 * Nx;
        nvalid = (int)min((long)S, nrows - row0);
        for (int t = threadIdx.x; t < S * N; t += blockDim.x) {
            const int s = t / N;
            xs[t] = (s < nvalid) ? (Tc)in[base + t] : (Tc)0;
        }
    } else {
        const int p0 = blockIdx.x * S;
        base = (size_t)blockIdx.y * Ny * Nx + p0;
        nvalid = min(S, Nx - p0);
        for (int t = threadIdx.x; t < S * N; t += blockDim.x) {
            const int j = t / S;
            const int s = t - j * S;
            xs[s * N + j] = (s < nvalid) ? (Tc)in[base + (size_t)j * Nx + s] : (Tc)0;
        }
    }
    __syncthreads();
    for (int t = threadIdx.x; t < S * N; t += blockDim.x) {
        int s, k;
        if (AXIS == HS_AXIS_X) {
            s = t / N;
            k = t - s * N + 1;
        } else {
            s = t % S;
            k = t / S + 1;
        }
        if (s >= nvalid) continue;
        Tc acc = (Tc)0;
        int m = 0;
        const Tc *x = xs + s * N;
        for (int i = 1; i <= N; ++i) {
            m += k;
            if (m >= twoM) m -= twoM;
            acc += x[i - 1] * sint[m];
        }
        const size_t idx = (AXIS == HS_AXIS_X) ? base + t : base + (size_t)(k - 1) * Nx + s;
        hs_emit<Tout, MODE>(out, aux, lo_off, idx, (double)(acc * scale));
    }
}

// Lines per CTA and dynamic shared memory; 0 when even one line does not fit.
template <typename Tc>
int lines_per_cta(const DstAxis &ax, int axis, size_t *smem) {
    const long cap = 227 * 1024;
    long fixed, per, budget;
    int smin;
    if (ax.fft) {
        const long c2 = 2 * (long)sizeof(Tc);
        fixed = (long)(2 * ax.M + 1) * c2;
        per = 2L * (ax.M + 1) * c2;
        budget = 96 * 1024;
        smin = (axis == HS_AXIS_Y) ? (int)(32 / sizeof(Tc)) : 1;
    } else {
        fixed = 2L * ax.M * (long)sizeof(Tc);
        per = (long)ax.N * (long)sizeof(Tc);
        budget = 48 * 1024;
        smin = 1;
    }
    long S = (budget - fixed) / per;
    if (S < smin) S = smin;
    if (S > 64) S = 64;
    const long fit = (cap - fixed) / per;
    if (S > fit) S = fit;
    if (S < 1) return 0;
    *smem = (size_t)(fixed + S * per);
    return (int)S;
}

template <typename Tc, typename Tin, typename Tout, int MODE>
hs_status launch_typed(const hs_plan_s *P, int axis, const void *in, void *out, double scale,
                       cudaStream_t s, double *aux) {
    const DstAxis &ax = (sizeof(Tc) == 8) ? P->axd[axis] : P->axf[axis];
    size_t smem = 0;
    const int S = lines_per_cta<Tc>(ax, axis, &smem);
    if (S == 0) return HS_ERR_UNSUPPORTED;
    dim3 grid;
    if (axis == HS_AXIS_X) {
        const long nrows = (long)P->Ny * P->Nz;
        grid = dim3((unsigned)((nrows + S - 1) / S), 1, 1);
    } else {
        grid = dim3((unsigned)((P->Nx + S - 1) / S), (unsigned)P->Nz, 1);
    }
    const Tin *pin = static_cast<const Tin *>(in);
    Tout *pout = static_cast<Tout *>(out);
    if (ax.fft) {
        if (axis == HS_AXIS_X) {
            auto k = dst_fft_kernel<Tc, Tin, Tout, HS_AXIS_X, MODE>;
            cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
            k<<<grid, 256, smem, s>>>(ax, pin, pout, aux, P->Nx, P->Ny, P->Nz, S, (Tc)scale,
                                      P->cur_skip);
        } else {
            auto k = dst_fft_kernel<Tc, Tin, Tout, HS_AXIS_Y, MODE>;
            cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
            k<<<grid, 256, smem, s>>>(ax, pin, pout, aux, P->Nx, P->Ny, P->Nz, S, (Tc)scale,
                                      P->cur_skip);
        }
    } else {
        if (axis == HS_AXIS_X) {
            auto k = dst_direct_kernel<Tc, Tin, Tout, HS_AXIS_X, MODE>;
            cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
            k<<<grid, 256, smem, s>>>(ax, pin, pout, aux, P->Nx, P->Ny, P->Nz, S, (Tc)scale,
                                      P->cur_skip);
        } else {
            auto k = dst_direct_kernel<Tc, Tin, Tout, HS_AXIS_Y, MODE>;
            cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
            k<<<grid, 256, smem, s>>>(ax, pin, pout, aux, P->Nx, P->Ny, P->Nz, S, (Tc)scale,
                                      P->cur_skip);
        }
    }
    return cudaGetLastError() == cudaSuccess ? HS_OK : HS_ERR_CUDA;
}

}  // namespace

int hs_dst_fits(const DstAxis &ax, int axis, int tc) {
    size_t smem;
    return tc == HS_T_F64 ? lines_per_cta<double>(ax, axis, &smem) > 0
                          : lines_per_cta<float>(ax, axis, &smem) > 0;
}

hs_status hs_launch_dst(const hs_plan_s *P, int axis, int tc, int tin, const void *in, int tout,
                        void *out, int mode, double scale, cudaStream_t s, double *aux) {
    const int v = P->dst_variant[axis];
    if (v == HS_DST_HALF && tc == HS_T_F64) {
        // one M/2-point FFT per line; modes it does not cover fall through
        const hs_status st = hs_launch_dst_half(P, axis, tin, in, tout, out, mode, scale, s);
        if (st != HS_ERR_UNSUPPORTED) return st;
    }
    if (v == HS_DST_GEMM && tc == HS_T_F32) {
        // tensor-core sine-matrix product; modes it does not cover fall through
        const hs_status st = hs_launch_dst_gemm(P, axis, tin, in, tout, out, mode, scale, s, aux);
        if (st != HS_ERR_UNSUPPORTED) return st;
    }
    if (v == HS_DST_TWOPASS && axis == HS_AXIS_Y && tc == HS_T_F32 && tin == HS_T_F32 &&
        tout == HS_T_F32 && mode == HS_MODE_WRITE && P->d_ytmp &&
        hs_dst_twopass_size(P->axf[HS_AXIS_Y].M))
        return hs_launch_dst_twopass_y(P, static_cast<const float *>(in),
                                       static_cast<float *>(out), scale, s);
    if ((v == HS_DST_FUSED || v == HS_DST_FUSED_WIDE) && tc == HS_T_F32 &&
        hs_dst_fast_size(P->axd[axis].M)) {
        const int wide = v == HS_DST_FUSED_WIDE;
        const hs_status st =
            axis == HS_AXIS_X
                ? hs_launch_dst_fused_x(P, tin, in, tout, out, mode, scale, s, aux, wide)
                : hs_launch_dst_fused_y(P, tin, in, tout, out, mode, scale, s, aux, wide);
        if (st != HS_ERR_UNSUPPORTED) return st;
    }
    if (v != HS_DST_GENERIC && hs_dst_fast_size(P->axd[axis].M))
        return hs_launch_dst_fast(P, axis, tc, tin, in, tout, out, mode, scale, s, aux);
    if (tc == HS_T_F64) {
        if (tin == HS_T_F64 && tout == HS_T_F64 && mode == HS_MODE_WRITE)
            return launch_typed<double, double, double, HS_MODE_WRITE>(P, axis, in, out, scale, s, aux);
        if (tin == HS_T_F64 && tout == HS_T_F64 && mode == HS_MODE_ADD)
            return launch_typed<double, double, double, HS_MODE_ADD>(P, axis, in, out, scale, s, aux);
        return HS_ERR_UNSUPPORTED;
    }
    if (tin == HS_T_F64 && tout == HS_T_F32 && mode == HS_MODE_WRITE)
        return launch_typed<float, double, float, HS_MODE_WRITE>(P, axis, in, out, scale, s, aux);
    if (tin == HS_T_F32 && tout == HS_T_F32 && mode == HS_MODE_WRITE)
        return launch_typed<float, float, float, HS_MODE_WRITE>(P, axis, in, out, scale, s, aux);
    if (tin == HS_T_F32 && tout == HS_T_F64 && mode == HS_MODE_WRITE)
        return launch_typed<float, float, double, HS_MODE_WRITE>(P, axis, in, out, scale, s, aux);
    if (tin == HS_T_F32 && tout == HS_T_F64 && mode == HS_MODE_ADD)
        return launch_typed<float, float, double, HS_MODE_ADD>(P, axis, in, out, scale, s, aux);
    if (tin == HS_T_F32 && tout == HS_T_DF && mode == HS_MODE_DF_SET)
        return launch_typed<float, float, float, HS_MODE_DF_SET>(P, axis, in, out, scale, s, aux);
    if (tin == HS_T_F32 && tout == HS_T_DF && mode == HS_MODE_DF_ADD)
        return launch_typed<float, float, float, HS_MODE_DF_ADD>(P, axis, in, out, scale, s, aux);
    if (tin == HS_T_F32 && tout == HS_T_DF && mode == HS_MODE_DF_FINAL)
        return launch_typed<float, float, float, HS_MODE_DF_FINAL>(P, axis, in, out, scale, s, aux);
    if (tin == HS_T_F32 && tout == HS_T_DF && mode == HS_MODE_DF_FINAL_HI)
        return launch_typed<float, float, float, HS_MODE_DF_FINAL_HI>(P, axis, in, out, scale, s, aux);
    return HS_ERR_UNSUPPORTED;
}
