// Half-length DST-I (FP64 plans): the sine transform of Section 3.6,
//   X_k = sum_{j=1..N} x_j sin(pi j k / M),  M = N + 1,  k = 1..N,
// computed through ONE complex FFT of M/2 points per line instead of the M-point
// FFT of the packed odd extension (hs_tiles.cuh), i.e. about half the FP64
// arithmetic.  The reduction (a standard real-data formulation of the DST-I):
//   y_0 = 0,  y_j = sin(pi j / M) (x_j + x_{M-j}) + (x_j - x_{M-j}) / 2,  j = 1..M-1
//   (the first part is even about M/2, the second odd), and Y = DFT_M(y), so
//   Re Y_k = X_{2k+1} - X_{2k-1},   Im Y_k = -X_{2k}.
// Y of the real sequence y comes from the M/2-point complex FFT Z of
// z_m = y_{2m} + i y_{2m+1}:
//   Y_k = (Z_k + conj Z_{M/2-k}) / 2 - (i/2) W^k (Z_k - conj Z_{M/2-k}),  W = e^{-2 pi i/M}.
// The even outputs are -Im Y_k; the odd outputs are the running sum
// X_{2k+1} = Re Y_0 / 2 + sum_{k'=1..k} Re Y_k' (X_{-1} = -X_1), taken per line by
// one warp with shuffles.  Its rounding grows with the line length (measured: the
// FP64 solve's distance from the oracle 2e-14 at N = 1023 against 1.2e-15 with
// the M-point FFT; 1e-15..5e-15 up to N = 255).
//
// One CTA owns S whole lines (x: rows of one plane-row block, contiguous; y:
// S columns of one plane, read as row segments).  Shared memory: the FFT's
// twiddles (M/2 roots), the post-processing roots W^k, the pairs
// (sin(pi j/M) + 1/2, sin(pi j/M) - 1/2) that make y_j = c+_j x_j + c-_j x_{M-j}
// one multiply and one FMA, and two line buffers of M/2 complex points (padded)
// that also hold the staged input x and the output X as real arrays.  The FP64
// pipe bounds this kernel (GB300: about two FP64 lanes per clock per SM), so the
// post-processing keeps 2 Y_k (four additions and four FMAs per k) and the one
// factor scale / 2 is applied at the store; each lane's four consecutive k run
// a sequential prefix sum before the warp-wide scan of the lane totals.
#include "hs_internal.cuh"
#include "hs_tiles.cuh"

namespace {

using namespace hs_tiles;

template <int M, int AXIS>
struct HalfLines {
    static constexpr int base = 4096 / M > 0 ? 4096 / M : 1;
    static constexpr int value = (AXIS == HS_AXIS_Y && base < 8) ? 8 : base;
};

template <int M, int S>
constexpr size_t half_smem() {
    // rootsH[M/2] + wk[M/2] + cpm[M] (double2), 2 buffers of S lines
    return sizeof(double2) * ((size_t)2 * M + (size_t)2 * S * LineStride<M / 2>::value);
}

template <int AXIS, int MODE, int M, int S, int... Rs>
__global__ void __launch_bounds__(256, 2)
dst_half_kernel(const double *__restrict__ in, double *out, const double2 *__restrict__ roots_g,
                const double2 *__restrict__ half_g, int Nx, int Ny, int Nz, double scale,
                const int *skip) {
    if (skip && *skip) return;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    constexpr int H = M / 2;
    constexpr int N = M - 1;
    constexpr int LS = LineStride<H>::value;   // complex slots per line
    constexpr int NT = 256;
    constexpr int ITER = (S * N + NT - 1) / NT;
    double2 *rootsH = reinterpret_cast<double2 *>(smem_raw);
    double2 *wk = rootsH + H;
    double2 *cpm = wk + H;
    double2 *buf0 = cpm + M;
    double2 *buf1 = buf0 + S * LS;
    for (int t = threadIdx.x; t < H; t += NT) {
        rootsH[t] = roots_g[2 * t];   // e^{-2 pi i t / H}
        wk[t] = roots_g[t];           // e^{-2 pi i t / M}
    }
    for (int t = threadIdx.x; t < M; t += NT) {   // sin(pi t / M) +- 1/2
        const double sn = half_g[t].y;
        cpm[t] = make_double2(sn + 0.5, sn - 0.5);
    }

    // ---- load: every global load of the tile issued before any shared store;
    // x_j (j = 1..N) of line s goes to the real array xr = buf1 + s LS at index j
    size_t base;
    int nvalid;
    double v[ITER];
    if (AXIS == HS_AXIS_X) {
        const long nrows = (long)Ny * Nz;
        const long row0 = (long)blockIdx.x * S;
        base = (size_t)row0 * N;
        nvalid = (int)min((long)S, nrows - row0);
        const int nel = nvalid * N;
#pragma unroll
        for (int it = 0; it < ITER; ++it) {
            const int e = threadIdx.x + it * NT;
            v[it] = (e < nel) ? in[base + e] : 0.0;
        }
#pragma unroll
        for (int it = 0; it < ITER; ++it) {
            const int e = threadIdx.x + it * NT;
            if (e < S * N) {
                const int s = e / N;
                const int i = e - s * N;
                reinterpret_cast<double *>(buf1 + s * LS)[i + 1] = v[it];
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
            v[it] = (e < S * N && s < nvalid) ? in[base + (size_t)j * Nx + s] : 0.0;
        }
#pragma unroll
        for (int it = 0; it < ITER; ++it) {
            const int e = threadIdx.x + it * NT;
            if (e < S * N) {
                const int j = e / S;
                const int s = e - j * S;
                reinterpret_cast<double *>(buf1 + s * LS)[j + 1] = v[it];
            }
        }
    }
    __syncthreads();

    // ---- pre-processing: z_m = y_{2m} + i y_{2m+1} into buf0
    for (int t = threadIdx.x; t < S * H; t += NT) {
        const int s = t / H;
        const int m = t - s * H;
        const double *xr = reinterpret_cast<const double *>(buf1 + s * LS);
        double y0 = 0.0;
        if (m > 0) {
            const double2 c = cpm[2 * m];
            y0 = fma(c.x, xr[2 * m], c.y * xr[M - 2 * m]);
        }
        const double2 c = cpm[2 * m + 1];
        const double y1 = fma(c.x, xr[2 * m + 1], c.y * xr[M - 2 * m - 1]);
        buf0[s * LS + PAD(m)] = make_double2(y0, y1);
    }
    __syncthreads();

    double2 *src = buf0, *dst = buf1;
    fstages<double, H, S, 1, Rs...>(src, dst, rootsH);

    // ---- post-processing, one warp per line: lane l takes the KL consecutive
    // k = KL l .. KL l + KL - 1 (values kept doubled: 2 Y_k); the odd outputs are
    // the running sum of 2 Re Y_k (2 Re Y_0 halved), by a per-lane prefix sum and
    // a warp scan of the lane totals
    constexpr int KL = (H + 31) / 32;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    for (int s = warp; s < S; s += NT / 32) {
        const double2 *Z = src + s * LS;
        double *Xr = reinterpret_cast<double *>(dst + s * LS);   // 2 X_k at index k - 1
        double re[KL];
        double run = 0.0;
#pragma unroll
        for (int c = 0; c < KL; ++c) {
            const int k = lane * KL + c;
            re[c] = 0.0;
            if (k < H) {
                const double2 A = Z[PAD(k)];
                const double2 B = Z[PAD(k == 0 ? 0 : H - k)];   // conj(B) enters
                const double p = A.x + B.x, q = A.y - B.y, r = A.y + B.y, t = A.x - B.x;
                const double2 w = wk[k];   // (cos, -sin)
                double r2 = fma(w.x, r, fma(w.y, t, p));        // 2 Re Y_k
                const double i2 = fma(w.y, r, fma(-w.x, t, q)); // 2 Im Y_k
                if (k > 0) Xr[2 * k - 1] = -i2;                 // 2 X_{2k}
                if (k == 0) r2 *= 0.5;                          // 2 X_1 = Re 2Y_0 / 2
                run += r2;
            }
            re[c] = run;   // inclusive prefix within the lane
        }
        // exclusive scan of the lane totals
        double tot = run;
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            const double o = __shfl_up_sync(0xffffffffu, tot, d);
            if (lane >= d) tot += o;
        }
        double before = __shfl_up_sync(0xffffffffu, tot, 1);   // lanes 0..lane-1
        if (lane == 0) before = 0.0;
#pragma unroll
        for (int c = 0; c < KL; ++c) {
            const int k = lane * KL + c;
            if (k < H) Xr[2 * k] = before + re[c];   // 2 X_{2k+1}
        }
    }
    __syncthreads();

    // ---- store: out = scale X (write) or out += scale X (add); Xr holds 2 X
    const double hs = 0.5 * scale;
    if (AXIS == HS_AXIS_X) {
        const int nel = nvalid * N;
#pragma unroll
        for (int it = 0; it < ITER; ++it) {
            const int e = threadIdx.x + it * NT;
            if (e < nel) {
                const int s = e / N;
                const int i = e - s * N;
                const double X = reinterpret_cast<const double *>(dst + s * LS)[i];
                hs_emit<double, MODE>(out, nullptr, 0, base + e, hs * X);
            }
        }
    } else {
#pragma unroll
        for (int it = 0; it < ITER; ++it) {
            const int e = threadIdx.x + it * NT;
            const int kk = e / S;
            const int s = e - kk * S;
            if (e < S * N && s < nvalid) {
                const double X = reinterpret_cast<const double *>(dst + s * LS)[kk];
                hs_emit<double, MODE>(out, nullptr, 0, base + (size_t)kk * Nx + s, hs * X);
            }
        }
    }
}

template <int MODE, int M, int... Rs>
hs_status launch_half_m(const hs_plan_s *P, int axis, const void *in, void *out, double scale,
                        cudaStream_t st) {
    const DstAxis &ax = P->axd[axis];
    const double2 *roots = static_cast<const double2 *>(ax.roots);
    const double2 *half = static_cast<const double2 *>(ax.half);
    const double *x = static_cast<const double *>(in);
    double *y = static_cast<double *>(out);
    if (axis == HS_AXIS_X) {
        constexpr int S = HalfLines<M, HS_AXIS_X>::value;
        constexpr size_t smem = half_smem<M, S>();
        static_assert(smem <= 227 * 1024, "half-length tile exceeds shared memory");
        auto k = dst_half_kernel<HS_AXIS_X, MODE, M, S, Rs...>;
        if (cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) !=
            cudaSuccess)
            return HS_ERR_CUDA;
        const long nrows = (long)P->Ny * P->Nz;
        k<<<(unsigned)((nrows + S - 1) / S), 256, smem, st>>>(x, y, roots, half, P->Nx, P->Ny,
                                                              P->Nz, scale, P->cur_skip);
    } else {
        constexpr int S = HalfLines<M, HS_AXIS_Y>::value;
        constexpr size_t smem = half_smem<M, S>();
        static_assert(smem <= 227 * 1024, "half-length tile exceeds shared memory");
        auto k = dst_half_kernel<HS_AXIS_Y, MODE, M, S, Rs...>;
        if (cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) !=
            cudaSuccess)
            return HS_ERR_CUDA;
        dim3 grid((unsigned)((P->Nx + S - 1) / S), (unsigned)P->Nz, 1);
        k<<<grid, 256, smem, st>>>(x, y, roots, half, P->Nx, P->Ny, P->Nz, scale, P->cur_skip);
    }
    return cudaGetLastError() == cudaSuccess ? HS_OK : HS_ERR_CUDA;
}

template <int MODE>
hs_status launch_half(const hs_plan_s *P, int axis, const void *in, void *out, double scale,
                      cudaStream_t st) {
    // radices of the M/2-point FFT (each divides 48: the constant twiddles)
    switch (P->axd[axis].M) {
        case 32: return launch_half_m<MODE, 32, 16>(P, axis, in, out, scale, st);
        case 64: return launch_half_m<MODE, 64, 8, 4>(P, axis, in, out, scale, st);
        case 96: return launch_half_m<MODE, 96, 16, 3>(P, axis, in, out, scale, st);
        case 128: return launch_half_m<MODE, 128, 16, 4>(P, axis, in, out, scale, st);
        case 192: return launch_half_m<MODE, 192, 16, 6>(P, axis, in, out, scale, st);
        case 256: return launch_half_m<MODE, 256, 16, 8>(P, axis, in, out, scale, st);
        case 384: return launch_half_m<MODE, 384, 16, 12>(P, axis, in, out, scale, st);
        case 512: return launch_half_m<MODE, 512, 16, 16>(P, axis, in, out, scale, st);
        case 768: return launch_half_m<MODE, 768, 16, 8, 3>(P, axis, in, out, scale, st);
        case 1024: return launch_half_m<MODE, 1024, 16, 16, 2>(P, axis, in, out, scale, st);
        default: return HS_ERR_UNSUPPORTED;
    }
}

}  // namespace

int hs_dst_half_size(int M) {
    switch (M) {
        case 32: case 64: case 96: case 128: case 192: case 256: case 384: case 512: case 768:
        case 1024:
            return 1;
        default:
            return 0;
    }
}

hs_status hs_launch_dst_half(const hs_plan_s *P, int axis, int tin, const void *in, int tout,
                             void *out, int mode, double scale, cudaStream_t s) {
    if (tin != HS_T_F64 || tout != HS_T_F64 || !hs_dst_half_size(P->axd[axis].M))
        return HS_ERR_UNSUPPORTED;
    if (mode == HS_MODE_WRITE) return launch_half<HS_MODE_WRITE>(P, axis, in, out, scale, s);
    if (mode == HS_MODE_ADD) return launch_half<HS_MODE_ADD>(P, axis, in, out, scale, s);
    return HS_ERR_UNSUPPORTED;
}
