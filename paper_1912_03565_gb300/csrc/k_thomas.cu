// z-direction tridiagonal solves, one per sine mode (p, q) (Section 3.6).
//
// Row l of the system of mode (p, q) is
//     lambda_{l-1}(p,q) w_{l-1} + lambda_l(p,q) w_l + lambda_{l+1}(p,q) w_{l+1} = Fhat_l,
//     lambda_nu(p,q) = 4 a_nu cos(th_p) cos(th_q) + 2 b_nu cos(th_p) + 2 c_nu cos(th_q) + d_nu,
// with the coefficients of row l.  It is solved by LU without pivoting (Section
// 3.6 names an LU solve and no pivoting; the systems are indefinite for k^2 above the
// mode's eigenvalue, so small pivots are reported, not avoided).
//
// The elimination factors do not depend on the right-hand side, so they are
// computed once per coefficient set and cached in FP64:
//     c'_l = upper_l / m_l,   alpha_l = 1 / m_l,   beta_l = lower_l / m_l,
//     m_l  = diag_l - lower_l c'_{l-1}.
// A solve is then d'_l = alpha_l F_l - beta_l d'_{l-1} (forward) and
// w_l = d'_l - c'_l w_{l+1} (backward): three FP64 operations per unknown.
// One thread owns one (p, q) column; threads of a warp own consecutive p, so
// every plane access is coalesced.
#include "hs_tiles.cuh"

namespace {

using namespace hs_tiles;

__device__ __forceinline__ void atomic_min_pos(double *addr, double v) {
    atomicMin(reinterpret_cast<unsigned long long *>(addr),
              (unsigned long long)__double_as_longlong(v));
}
__device__ __forceinline__ void atomic_max_pos(double *addr, double v) {
    atomicMax(reinterpret_cast<unsigned long long *>(addr),
              (unsigned long long)__double_as_longlong(v));
}

__global__ void __launch_bounds__(256) factor_kernel(int Nx, int Ny, int Nz,
                                                      const double *__restrict__ coef,
                                                      const double *__restrict__ cx,
                                                      const double *__restrict__ cy,
                                                      double *__restrict__ fac,
                                                      float *__restrict__ fac32,
                                                      double *__restrict__ red) {
    const size_t plane = (size_t)Nx * Ny;
    const size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    double minpiv = __longlong_as_double(0x7ff0000000000000LL);  // +inf
    double maxdiag = 0.0;
    if (idx < plane) {
        const int q = (int)(idx / Nx);
        const int p = (int)(idx - (size_t)q * Nx);
        const double cp = cx[p], cq = cy[q];
        const double P4 = 4.0 * cp * cq, Q2 = 2.0 * cp, R2 = 2.0 * cq;
        double *cpr = fac;
        double *alpha = fac ? fac + (size_t)Nz * plane : nullptr;
        double *beta = fac ? fac + 2 * (size_t)Nz * plane : nullptr;
        double cprev = 0.0;
        for (int l = 0; l < Nz; ++l) {
            const double *cf = coef + (size_t)l * 12;
            const double lo = cf[0] * P4 + cf[1] * Q2 + cf[2] * R2 + cf[3];
            const double di = cf[4] * P4 + cf[5] * Q2 + cf[6] * R2 + cf[7];
            const double up = cf[8] * P4 + cf[9] * Q2 + cf[10] * R2 + cf[11];
            const double m = (l == 0) ? di : di - lo * cprev;
            const double inv = 1.0 / m;
            const double c1 = up * inv;
            const size_t o = (size_t)l * plane + idx;
            const double b1 = (l == 0) ? 0.0 : lo * inv;
            if (fac) {
                cpr[o] = c1;
                alpha[o] = inv;
                beta[o] = b1;
            }
            if (fac32) {
                fac32[o] = (float)c1;
                fac32[(size_t)Nz * plane + o] = (float)inv;
                fac32[2 * (size_t)Nz * plane + o] = (float)b1;
            }
            cprev = c1;
            minpiv = fmin(minpiv, fabs(m));
            maxdiag = fmax(maxdiag, fabs(di));
        }
    }
    for (int o = 16; o > 0; o >>= 1) {
        minpiv = fmin(minpiv, __shfl_down_sync(0xffffffffu, minpiv, o));
        maxdiag = fmax(maxdiag, __shfl_down_sync(0xffffffffu, maxdiag, o));
    }
    if ((threadIdx.x & 31) == 0) {
        atomic_min_pos(red + 0, minpiv);
        atomic_max_pos(red + 1, maxdiag);
    }
}

// FP64 path: data holds Fhat on entry and W on exit (forward sweep in place).
__global__ void __launch_bounds__(256) thomas64_kernel(int Nx, int Ny, int Nz,
                                                        double *__restrict__ data,
                                                        const double *__restrict__ fac,
                                                        const int *skip) {
    if (skip && *skip) return;
    const size_t plane = (size_t)Nx * Ny;
    const size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= plane) return;
    thomas_column<double, double, double, false, false>(Nz, plane, idx, data, (double *)nullptr, fac,
                                          fac + (size_t)Nz * plane, fac + 2 * (size_t)Nz * plane);
}

// Mixed path, FP64 factors (plans with small pivots): FP32 Fhat in, FP32 W
// out; the forward sweep is kept in FP64 scratch.
__global__ void __launch_bounds__(256) thomas32_kernel(int Nx, int Ny, int Nz,
                                                        float *__restrict__ data,
                                                        double *__restrict__ scratch,
                                                        const double *__restrict__ fac,
                                                        const int *skip) {
    if (skip && *skip) return;
    const size_t plane = (size_t)Nx * Ny;
    const size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= plane) return;
    thomas_column<float, double, double, false, false>(Nz, plane, idx, data, scratch, fac,
                                         fac + (size_t)Nz * plane, fac + 2 * (size_t)Nz * plane);
}

// Mixed path, well-conditioned plans: the factors rounded to FP32 and an FP32
// recurrence, in place (Fhat in, W out).  The error this adds to the fast
// solve, ~2^-24 times the condition of the z-system, is removed by the
// refinement sweeps like the FP32 transform error.
template <int CHK, bool PIPE, int NT, bool STREAM>
__global__ void __launch_bounds__(NT) thomas_f32_kernel(int Nx, int Ny, int Nz,
                                                        float *__restrict__ data,
                                                        const float *__restrict__ fac,
                                                        const int *skip) {
    if (skip && *skip) return;
    const size_t plane = (size_t)Nx * Ny;
    const size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= plane) return;
    thomas_column<float, float, float, false, PIPE, CHK, STREAM>(
        Nz, plane, idx, data, (float *)nullptr, fac, fac + (size_t)Nz * plane,
        fac + 2 * (size_t)Nz * plane);
}

// Streaming factor loads where the forward sweep's values (the whole data array,
// FP32) fit in about three quarters of the 129 MB L2.
bool stream_factors(const hs_plan_s *P) {
    return (size_t)P->Nx * P->Ny * P->Nz * sizeof(float) <= ((size_t)96 << 20);
}

template <int CHK, bool PIPE, int NT>
void launch_f32(const hs_plan_s *P, float *data, cudaStream_t s) {
    const size_t plane = (size_t)P->Nx * P->Ny;
    const unsigned blocks = (unsigned)((plane + NT - 1) / NT);
    if (stream_factors(P))
        thomas_f32_kernel<CHK, PIPE, NT, true><<<blocks, NT, 0, s>>>(P->Nx, P->Ny, P->Nz, data,
                                                                    P->d_fac32, P->cur_skip);
    else
        thomas_f32_kernel<CHK, PIPE, NT, false><<<blocks, NT, 0, s>>>(P->Nx, P->Ny, P->Nz, data,
                                                                     P->d_fac32, P->cur_skip);
}

// Balanced mapping: a whole number of blocks per SM and the columns shared
// evenly among them (block size rounded up to a warp, at most NTMAX), so that
// no SM runs a second round of blocks while others idle -- at 255^2 columns the
// fixed 256-thread blocks give 254 blocks for 152 SMs.
template <int CHK, int NTMAX>
void launch_f32_bal(const hs_plan_s *P, float *data, cudaStream_t s) {
    static int sms = 0;
    if (sms == 0 && cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, P->device) !=
                        cudaSuccess) {
        cudaGetLastError();
        sms = 148;
    }
    const size_t plane = (size_t)P->Nx * P->Ny;
    const size_t per_sm = (plane + sms - 1) / sms;
    const size_t k = (per_sm + NTMAX - 1) / NTMAX;               // blocks per SM
    const unsigned blocks = (unsigned)(sms * k);
    const unsigned nt = (unsigned)(((plane + blocks - 1) / blocks + 31) / 32 * 32);
    if (stream_factors(P))
        thomas_f32_kernel<CHK, true, NTMAX, true><<<blocks, nt, 0, s>>>(P->Nx, P->Ny, P->Nz, data,
                                                                       P->d_fac32, P->cur_skip);
    else
        thomas_f32_kernel<CHK, true, NTMAX, false><<<blocks, nt, 0, s>>>(P->Nx, P->Ny, P->Nz, data,
                                                                        P->d_fac32, P->cur_skip);
}

}  // namespace

hs_status hs_launch_factor(const hs_plan_s *P, cudaStream_t s) {
    const size_t plane = (size_t)P->Nx * P->Ny;
    const unsigned blocks = (unsigned)((plane + 255) / 256);
    factor_kernel<<<blocks, 256, 0, s>>>(P->Nx, P->Ny, P->Nz, P->d_coef, P->d_cx, P->d_cy,
                                         P->d_fac, P->d_fac32, P->d_red);
    return cudaGetLastError() == cudaSuccess ? HS_OK : HS_ERR_CUDA;
}

hs_status hs_launch_thomas(const hs_plan_s *P, int tio, void *data, double *scratch,
                           cudaStream_t s) {
    const size_t plane = (size_t)P->Nx * P->Ny;
    const unsigned blocks = (unsigned)((plane + 255) / 256);
    if (tio == HS_T_F64)
        thomas64_kernel<<<blocks, 256, 0, s>>>(P->Nx, P->Ny, P->Nz, static_cast<double *>(data),
                                               P->d_fac, P->cur_skip);
    else if (P->thomas32)
        switch (P->thomas_variant) {
            // thread mapping of the FP32 z-solves: one thread per (p,q) column;
            // chunk depth, software pipelining and block size vary
            case HS_THOMAS_PIPE8_128: launch_f32<8, true, 128>(P, static_cast<float *>(data), s); break;
            case HS_THOMAS_PLAIN16_256: launch_f32<16, false, 256>(P, static_cast<float *>(data), s); break;
            case HS_THOMAS_PIPE16_128: launch_f32<16, true, 128>(P, static_cast<float *>(data), s); break;
            case HS_THOMAS_BAL8_512: launch_f32_bal<8, 512>(P, static_cast<float *>(data), s); break;
            case HS_THOMAS_BAL16_256: launch_f32_bal<16, 256>(P, static_cast<float *>(data), s); break;
            default: launch_f32<16, true, 256>(P, static_cast<float *>(data), s); break;
        }
    else
        thomas32_kernel<<<blocks, 256, 0, s>>>(P->Nx, P->Ny, P->Nz, static_cast<float *>(data),
                                               scratch, P->d_fac, P->cur_skip);
    return cudaGetLastError() == cudaSuccess ? HS_OK : HS_ERR_CUDA;
}
