// Preconditioner mode: the direct solver as the preconditioner of BiCGStab for
// a Helmholtz coefficient k^2 that varies in x, y and z (the use the paper's
// introduction names).  The outer operator is the compact scheme with K = k^2
// given per interior node (zero Dirichlet data), scaled by h_z^2 like the
// per-row coefficients of Section 3.3, so that for K = K(z) it is the 27-point
// operator of eq. (stencil27):
//   4th order: h_z^2 [ Lap_h U + sum_{a<b} (h_a^2 + h_b^2)/12 d_a^2 d_b^2 U
//                      + K_c U_c / 2 + (1/12) sum_{6 face neighbours} K U ]
//   2nd order: h_z^2 [ Lap_h U + K_c U_c ]
// The Krylov vectors are FP64; every vector operation is a kernel here, and
// the solve of the plan (FP64 or mixed path, assembled right-hand side) is the
// preconditioner, applied from the right (van der Vorst's BiCGStab).
#include <string.h>

#include <new>

#include "hs_internal.cuh"

namespace {

constexpr int PC_BLOCKS = 1216;   // 152 SMs x 8
constexpr int PC_THREADS = 256;

struct OpArgs {
    int Nx, Ny, Nz, order;
    double ihx2, ihy2, ihz2, hz2;
    double wxy, wxz, wyz;   // (h_a^2 + h_b^2) / 12 / (h_a^2 h_b^2)
};

// y = A(K) u on the interior (u = 0 outside).  One thread per point.
__global__ void __launch_bounds__(256) general_apply_kernel(OpArgs a, const double *__restrict__ K,
                                                            const double *__restrict__ u,
                                                            double *__restrict__ y) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const int j = blockIdx.y;
    const int l = blockIdx.z;
    if (i >= a.Nx) return;
    const size_t sy = a.Nx, sz = (size_t)a.Nx * a.Ny;
    const size_t c = (size_t)l * sz + (size_t)j * sy + i;
    auto U = [&](int di, int dj, int dl) -> double {
        const int ii = i + di, jj = j + dj, ll = l + dl;
        if (ii < 0 || ii >= a.Nx || jj < 0 || jj >= a.Ny || ll < 0 || ll >= a.Nz) return 0.0;
        return __ldg(u + c + (long)dl * (long)sz + (long)dj * (long)sy + di);
    };
    auto KU = [&](int di, int dj, int dl) -> double {
        const int ii = i + di, jj = j + dj, ll = l + dl;
        if (ii < 0 || ii >= a.Nx || jj < 0 || jj >= a.Ny || ll < 0 || ll >= a.Nz) return 0.0;
        const long o = (long)dl * (long)sz + (long)dj * (long)sy + di;
        return __ldg(K + c + o) * __ldg(u + c + o);
    };
    const double uc = U(0, 0, 0);
    const double xs = U(-1, 0, 0) + U(1, 0, 0), ys = U(0, -1, 0) + U(0, 1, 0),
                 zs = U(0, 0, -1) + U(0, 0, 1);
    double v = (xs - 2.0 * uc) * a.ihx2 + (ys - 2.0 * uc) * a.ihy2 + (zs - 2.0 * uc) * a.ihz2;
    if (a.order == 2) {
        v += __ldg(K + c) * uc;
    } else {
        // d_a^2 d_b^2 u = (4 edge values) - 2 (4 face values of the pair) + 4 u_c, / (h_a^2 h_b^2)
        const double exy = U(1, 1, 0) + U(1, -1, 0) + U(-1, 1, 0) + U(-1, -1, 0);
        const double exz = U(1, 0, 1) + U(1, 0, -1) + U(-1, 0, 1) + U(-1, 0, -1);
        const double eyz = U(0, 1, 1) + U(0, 1, -1) + U(0, -1, 1) + U(0, -1, -1);
        v += a.wxy * (exy - 2.0 * (xs + ys) + 4.0 * uc);
        v += a.wxz * (exz - 2.0 * (xs + zs) + 4.0 * uc);
        v += a.wyz * (eyz - 2.0 * (ys + zs) + 4.0 * uc);
        const double kn = KU(-1, 0, 0) + KU(1, 0, 0) + KU(0, -1, 0) + KU(0, 1, 0) +
                          KU(0, 0, -1) + KU(0, 0, 1);
        v += 0.5 * __ldg(K + c) * uc + kn * (1.0 / 12.0);
    }
    y[c] = a.hz2 * v;
}

// Block sum of v into *out (one atomic per block).
__device__ __forceinline__ void block_add(double v, double *out) {
    __shared__ double part[PC_THREADS / 32];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (lane == 0) part[w] = v;
    __syncthreads();
    if (w == 0) {
        v = lane < PC_THREADS / 32 ? part[lane] : 0.0;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        if (lane == 0) atomicAdd(out, v);
    }
}

// out[0] += (a, b), out[1] += (c, d) (second pair optional)
__global__ void __launch_bounds__(PC_THREADS) dot2_kernel(size_t n, const double *__restrict__ a,
                                                          const double *__restrict__ b,
                                                          const double *__restrict__ c,
                                                          const double *__restrict__ d,
                                                          double *out) {
    double s0 = 0.0, s1 = 0.0;
    for (size_t k = (size_t)blockIdx.x * blockDim.x + threadIdx.x; k < n;
         k += (size_t)gridDim.x * blockDim.x) {
        s0 = fma(a[k], b[k], s0);
        if (c) s1 = fma(c[k], d[k], s1);
    }
    block_add(s0, out);
    if (c) {
        __syncthreads();
        block_add(s1, out + 1);
    }
}

// p = r + beta (p - omega v)
__global__ void __launch_bounds__(PC_THREADS) update_p_kernel(size_t n, const double *__restrict__ r,
                                                              double *__restrict__ p,
                                                              const double *__restrict__ v,
                                                              double beta, double omega) {
    for (size_t k = (size_t)blockIdx.x * blockDim.x + threadIdx.x; k < n;
         k += (size_t)gridDim.x * blockDim.x)
        p[k] = r[k] + beta * (p[k] - omega * v[k]);
}

// s = r - alpha v
__global__ void __launch_bounds__(PC_THREADS) update_s_kernel(size_t n, const double *__restrict__ r,
                                                              const double *__restrict__ v,
                                                              double *__restrict__ s, double alpha) {
    for (size_t k = (size_t)blockIdx.x * blockDim.x + threadIdx.x; k < n;
         k += (size_t)gridDim.x * blockDim.x)
        s[k] = r[k] - alpha * v[k];
}

// x += alpha phat + omega shat; r = s - omega t; out[0] += ||r||^2
__global__ void __launch_bounds__(PC_THREADS) update_xr_kernel(
    size_t n, double *__restrict__ x, const double *__restrict__ phat,
    const double *__restrict__ shat, double *__restrict__ r, const double *__restrict__ s,
    const double *__restrict__ t, double alpha, double omega, double *out) {
    double acc = 0.0;
    for (size_t k = (size_t)blockIdx.x * blockDim.x + threadIdx.x; k < n;
         k += (size_t)gridDim.x * blockDim.x) {
        x[k] += alpha * phat[k] + omega * shat[k];
        const double rk = s[k] - omega * t[k];
        r[k] = rk;
        acc = fma(rk, rk, acc);
    }
    block_add(acc, out);
}

// r = F - r (r holds A x on entry); rhat = r; out[0] += ||F||^2, out[1] += ||r||^2
__global__ void __launch_bounds__(PC_THREADS) init_r_kernel(size_t n, const double *__restrict__ F,
                                                            double *__restrict__ r,
                                                            double *__restrict__ rhat,
                                                            double *out) {
    double f2 = 0.0, r2 = 0.0;
    for (size_t k = (size_t)blockIdx.x * blockDim.x + threadIdx.x; k < n;
         k += (size_t)gridDim.x * blockDim.x) {
        const double rk = F[k] - r[k];
        r[k] = rk;
        rhat[k] = rk;
        f2 = fma(F[k], F[k], f2);
        r2 = fma(rk, rk, r2);
    }
    block_add(f2, out);
    __syncthreads();
    block_add(r2, out + 1);
}

unsigned blocks_for(size_t n) {
    const size_t b = (n + PC_THREADS - 1) / PC_THREADS;
    return (unsigned)(b < PC_BLOCKS ? (b > 0 ? b : 1) : PC_BLOCKS);
}

}  // namespace

struct hs_precond_s {
    hs_plan_t plan;
    const double *K;
    size_t n;
    OpArgs op;
    double *buf;      // r, rhat, p, v, s, t, phat, shat (n each)
    double *d_red;    // 4 reduction slots
};

namespace {

hs_status apply_op(const hs_precond_s *C, const double *u, double *y, cudaStream_t s) {
    dim3 grid((unsigned)((C->op.Nx + 127) / 128), (unsigned)C->op.Ny, (unsigned)C->op.Nz);
    general_apply_kernel<<<grid, 128, 0, s>>>(C->op, C->K, u, y);
    return cudaGetLastError() == cudaSuccess ? HS_OK : HS_ERR_CUDA;
}

hs_status reduce(const hs_precond_s *C, cudaStream_t s, double *host, int count) {
    if (cudaMemcpyAsync(host, C->d_red, count * sizeof(double), cudaMemcpyDeviceToHost, s) !=
            cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess ||
        cudaMemsetAsync(C->d_red, 0, 4 * sizeof(double), s) != cudaSuccess) {
        cudaGetLastError();
        return HS_ERR_CUDA;
    }
    return HS_OK;
}

}  // namespace

extern "C" {

hs_status hs_precond_create(hs_precond_t *out, hs_plan_t P, const double *K) {
    if (!out || !P || !K) return HS_ERR_INVALID_ARG;
    *out = nullptr;
    if (P->equation != HS_HELMHOLTZ || (P->order != 2 && P->order != 4)) return HS_ERR_UNSUPPORTED;
    if (!P->have_coeff) return HS_ERR_NO_COEFF;
    hs_precond_s *C = new (std::nothrow) hs_precond_s;
    if (!C) return HS_ERR_OOM;
    memset(C, 0, sizeof(*C));
    C->plan = P;
    C->K = K;
    C->n = (size_t)P->Nx * P->Ny * P->Nz;
    OpArgs &a = C->op;
    a.Nx = P->Nx;
    a.Ny = P->Ny;
    a.Nz = P->Nz;
    a.order = P->order;
    const double hx2 = P->hx * P->hx, hy2 = P->hy * P->hy, hz2 = P->hz * P->hz;
    a.ihx2 = 1.0 / hx2;
    a.ihy2 = 1.0 / hy2;
    a.ihz2 = 1.0 / hz2;
    a.hz2 = hz2;
    a.wxy = (hx2 + hy2) / 12.0 / (hx2 * hy2);
    a.wxz = (hx2 + hz2) / 12.0 / (hx2 * hz2);
    a.wyz = (hy2 + hz2) / 12.0 / (hy2 * hz2);
    if (cudaMalloc((void **)&C->buf, 8 * C->n * sizeof(double)) != cudaSuccess ||
        cudaMalloc((void **)&C->d_red, 4 * sizeof(double)) != cudaSuccess ||
        cudaMemset(C->d_red, 0, 4 * sizeof(double)) != cudaSuccess) {
        cudaGetLastError();
        if (C->buf) cudaFree(C->buf);
        if (C->d_red) cudaFree(C->d_red);
        delete C;
        return HS_ERR_OOM;
    }
    *out = C;
    return HS_OK;
}

hs_status hs_precond_apply(hs_precond_t C, const double *u, double *y, void *stream) {
    if (!C || !u || !y) return HS_ERR_INVALID_ARG;
    return apply_op(C, u, y, static_cast<cudaStream_t>(stream));
}

hs_status hs_precond_solve(hs_precond_t C, const double *F, double *x, double tol, int maxit,
                           void *stream, hs_precond_info *info) {
    HsRange range("hs_precond_solve");
    if (!C || !F || !x || !(tol >= 0.0) || maxit < 1) return HS_ERR_INVALID_ARG;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const size_t n = C->n;
    double *r = C->buf, *rhat = r + n, *p = rhat + n, *v = p + n, *sv = v + n, *t = sv + n,
           *phat = t + n, *shat = phat + n;
    const unsigned nb = blocks_for(n);
    hs_plan_t P = C->plan;
    auto precond = [&](const double *in, double *outv) {
        return hs_solve(P, in, HS_F64, HS_RHS_ASSEMBLED, nullptr, outv, 1, stream, nullptr);
    };
    if (info) memset(info, 0, sizeof(*info));
    hs_status st;
    double h[2];
    if (cudaMemsetAsync(C->d_red, 0, 4 * sizeof(double), s) != cudaSuccess) return HS_ERR_CUDA;
    if ((st = apply_op(C, x, r, s)) != HS_OK) return st;
    init_r_kernel<<<nb, PC_THREADS, 0, s>>>(n, F, r, rhat, C->d_red);
    if ((st = reduce(C, s, h, 2)) != HS_OK) return st;
    const double nF = sqrt(h[0]);
    double rel = nF > 0 ? sqrt(h[1]) / nF : 0.0;
    if (cudaMemsetAsync(p, 0, n * sizeof(double), s) != cudaSuccess ||
        cudaMemsetAsync(v, 0, n * sizeof(double), s) != cudaSuccess)
        return HS_ERR_CUDA;
    double rho = 1.0, alpha = 1.0, omega = 1.0;
    int it = 0;
    hs_status outcome = HS_WARN_NOT_CONVERGED;
    while (rel > tol && it < maxit) {
        dot2_kernel<<<nb, PC_THREADS, 0, s>>>(n, rhat, r, nullptr, nullptr, C->d_red);
        if ((st = reduce(C, s, h, 1)) != HS_OK) return st;
        const double rho_new = h[0];
        if (rho_new == 0.0 || omega == 0.0) {
            outcome = HS_ERR_NONFINITE;   // breakdown
            break;
        }
        const double beta = (rho_new / rho) * (alpha / omega);
        update_p_kernel<<<nb, PC_THREADS, 0, s>>>(n, r, p, v, beta, omega);
        if ((st = precond(p, phat)) < 0) return st;
        if ((st = apply_op(C, phat, v, s)) != HS_OK) return st;
        dot2_kernel<<<nb, PC_THREADS, 0, s>>>(n, rhat, v, nullptr, nullptr, C->d_red);
        if ((st = reduce(C, s, h, 1)) != HS_OK) return st;
        if (h[0] == 0.0) {
            outcome = HS_ERR_NONFINITE;
            break;
        }
        alpha = rho_new / h[0];
        update_s_kernel<<<nb, PC_THREADS, 0, s>>>(n, r, v, sv, alpha);
        if ((st = precond(sv, shat)) < 0) return st;
        if ((st = apply_op(C, shat, t, s)) != HS_OK) return st;
        dot2_kernel<<<nb, PC_THREADS, 0, s>>>(n, t, sv, t, t, C->d_red);
        if ((st = reduce(C, s, h, 2)) != HS_OK) return st;
        omega = h[1] > 0.0 ? h[0] / h[1] : 0.0;
        update_xr_kernel<<<nb, PC_THREADS, 0, s>>>(n, x, phat, shat, r, sv, t, alpha, omega,
                                                    C->d_red);
        if ((st = reduce(C, s, h, 1)) != HS_OK) return st;
        rho = rho_new;
        rel = nF > 0 ? sqrt(h[0]) / nF : 0.0;
        if (info && it < HS_PRECOND_MAX_HIST) info->history[it] = rel;
        ++it;
        if (!(rel == rel)) {   // NaN
            outcome = HS_ERR_NONFINITE;
            break;
        }
    }
    if (rel <= tol) outcome = HS_OK;
    if (info) {
        info->iterations = it;
        info->rel_residual = rel;
    }
    if (cudaGetLastError() != cudaSuccess) return HS_ERR_CUDA;
    return outcome;
}

hs_status hs_precond_destroy(hs_precond_t C) {
    if (!C) return HS_OK;
    cudaDeviceSynchronize();
    if (C->buf) cudaFree(C->buf);
    if (C->d_red) cudaFree(C->d_red);
    delete C;
    return HS_OK;
}

}  // extern "C"
