// Right-hand-side operator with Dirichlet lifting, FP64 27-point residual and
// a sum-of-squares reduction.
//
// Right-hand sides (F carries the factor h_z^2 of the stencil form, Sections
// 3.2-3.5; D_a is the undivided second difference f_{+1} - 2 f + f_{-1}):
//   2nd order:  F = h_z^2 f
//   4th order:  F = h_z^2 (f + (Dx + Dy + Dz) f / 12)                 eq. (scheme4)
//   CD:         F = h_z^2 (f + (Dx + Dy + Dz) f / 12
//                          + h_z gamma_l (f_{l+1} - f_{l-1}) / 24)     eq. (cd_rhs)
//   6th order:  F = h^2 [ f + (Dx + Dy + Dz) f / 12 - (Dx^2 + Dy^2 + Dz^2) f / 240
//                        + (Dx Dy + Dx Dz + Dy Dz) f / 90 - h^2 K_l f / 20
//                        + h^3 K_{z,l} (f_{l+1} - f_{l-1}) / 120 ]     eq. (scheme6)
// The 6th-order form writes the f-derivatives of eq. (scheme6) as explicit
// differences: the term k_l^2 U of Delta_h(k^2 U) acts as k^2 f, "nabla^4 f"
// is the sum of pure fourth derivatives, and the second neighbour beyond a
// face is the ghost f_{-1} = 2 f_0 - f_1 + h^2 (f_nn)_face (face data 0 when
// absent, the zero derivative data the paper mentions).
// Lifting: every stencil neighbour on a boundary node contributes
// -coef * g to F (the Dirichlet data of eq. (bc) moved to the right side).
#include "hs_internal.cuh"

namespace {

struct RhsArgs {
    int Nx, Ny, Nz;
    double hz;           // h_z (the uniform h for order 6)
    int order, equation, rhs_kind;
    const double *coef;  // [Nz][3][4]
    const double *c0;    // [Nz+2]
    const double *c1;    // [Nz+2]
    DevBoundary b;
};

template <typename T>
__device__ __forceinline__ double ld(const T *p, size_t i) {
    return (double)__ldg(p + i);
}

template <typename T>
__device__ double boundary_value(const RhsArgs &a, int i, int j, int l) {
    const int Nx2 = a.Nx + 2, Ny2 = a.Ny + 2;
    const T *p;
    size_t idx;
    if (l == 0 || l == a.Nz + 1) {
        p = static_cast<const T *>(a.b.face[l == 0 ? 4 : 5]);
        idx = (size_t)j * Nx2 + i;
    } else if (j == 0 || j == a.Ny + 1) {
        p = static_cast<const T *>(a.b.face[j == 0 ? 2 : 3]);
        idx = (size_t)l * Nx2 + i;
    } else {
        p = static_cast<const T *>(a.b.face[i == 0 ? 0 : 1]);
        idx = (size_t)l * Ny2 + j;
    }
    return p ? ld(p, idx) : 0.0;
}

// Subtract the boundary-node terms of row (i, j, l) (node indices, interior).
template <typename T>
__device__ double lift_terms(const RhsArgs &a, int i, int j, int l) {
    double acc = 0.0;
    const double *cf = a.coef + (size_t)(l - 1) * 12;
    for (int dl = -1; dl <= 1; ++dl) {
        const int ll = l + dl;
        for (int dj = -1; dj <= 1; ++dj) {
            const int jj = j + dj;
            for (int di = -1; di <= 1; ++di) {
                const int ii = i + di;
                const bool bnd = (ll == 0 || ll == a.Nz + 1 || jj == 0 || jj == a.Ny + 1 ||
                                  ii == 0 || ii == a.Nx + 1);
                if (!bnd) continue;
                const int m = (di != 0 && dj != 0) ? 0 : (di != 0 ? 1 : (dj != 0 ? 2 : 3));
                const double c = cf[(dl + 1) * 4 + m];
                if (c != 0.0) acc += c * boundary_value<T>(a, ii, jj, ll);
            }
        }
    }
    return acc;
}

template <typename T>
__global__ void __launch_bounds__(256) rhs_kernel(RhsArgs a, const T *__restrict__ f,
                                                   double *__restrict__ F) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x + 1;  // node indices
    const int j = blockIdx.y * blockDim.y + threadIdx.y + 1;
    const int l = blockIdx.z + 1;
    if (i > a.Nx || j > a.Ny) return;
    const size_t out = ((size_t)(l - 1) * a.Ny + (j - 1)) * a.Nx + (i - 1);
    double val;
    if (a.rhs_kind == HS_RHS_ASSEMBLED) {
        val = ld(f, out);
    } else {
        const size_t sx = 1, sy = (size_t)(a.Nx + 2), sz = sy * (a.Ny + 2);
        const size_t c = (size_t)l * sz + (size_t)j * sy + i;
        const double fc = ld(f, c);
        const double fxm = ld(f, c - sx), fxp = ld(f, c + sx);
        const double fym = ld(f, c - sy), fyp = ld(f, c + sy);
        const double fzm = ld(f, c - sz), fzp = ld(f, c + sz);
        const double Dx = fxm - 2.0 * fc + fxp;
        const double Dy = fym - 2.0 * fc + fyp;
        const double Dz = fzm - 2.0 * fc + fzp;
        const double h = a.hz, h2 = h * h;
        if (a.equation == HS_CONVDIFF) {
            const double g = a.c0[l];
            val = h2 * (fc + (Dx + Dy + Dz) * (1.0 / 12.0) + h * g * (fzp - fzm) * (1.0 / 24.0));
        } else if (a.order == 2) {
            val = h2 * fc;
        } else if (a.order == 4) {
            val = h2 * (fc + (Dx + Dy + Dz) * (1.0 / 12.0));
        } else {
            // second neighbours along each axis, ghosts beyond the faces
            const T *fnn;
            double fx2m, fx2p, fy2m, fy2p, fz2m, fz2p;
            if (i >= 2) {
                fx2m = ld(f, c - 2 * sx);
            } else {
                fnn = static_cast<const T *>(a.b.fnn[0]);
                fx2m = 2.0 * fxm - fc + (fnn ? h2 * ld(fnn, (size_t)l * (a.Ny + 2) + j) : 0.0);
            }
            if (i <= a.Nx - 1) {
                fx2p = ld(f, c + 2 * sx);
            } else {
                fnn = static_cast<const T *>(a.b.fnn[1]);
                fx2p = 2.0 * fxp - fc + (fnn ? h2 * ld(fnn, (size_t)l * (a.Ny + 2) + j) : 0.0);
            }
            if (j >= 2) {
                fy2m = ld(f, c - 2 * sy);
            } else {
                fnn = static_cast<const T *>(a.b.fnn[2]);
                fy2m = 2.0 * fym - fc + (fnn ? h2 * ld(fnn, (size_t)l * (a.Nx + 2) + i) : 0.0);
            }
            if (j <= a.Ny - 1) {
                fy2p = ld(f, c + 2 * sy);
            } else {
                fnn = static_cast<const T *>(a.b.fnn[3]);
                fy2p = 2.0 * fyp - fc + (fnn ? h2 * ld(fnn, (size_t)l * (a.Nx + 2) + i) : 0.0);
            }
            if (l >= 2) {
                fz2m = ld(f, c - 2 * sz);
            } else {
                fnn = static_cast<const T *>(a.b.fnn[4]);
                fz2m = 2.0 * fzm - fc + (fnn ? h2 * ld(fnn, (size_t)j * (a.Nx + 2) + i) : 0.0);
            }
            if (l <= a.Nz - 1) {
                fz2p = ld(f, c + 2 * sz);
            } else {
                fnn = static_cast<const T *>(a.b.fnn[5]);
                fz2p = 2.0 * fzp - fc + (fnn ? h2 * ld(fnn, (size_t)j * (a.Nx + 2) + i) : 0.0);
            }
            const double Dx4 = fx2m - 4.0 * fxm + 6.0 * fc - 4.0 * fxp + fx2p;
            const double Dy4 = fy2m - 4.0 * fym + 6.0 * fc - 4.0 * fyp + fy2p;
            const double Dz4 = fz2m - 4.0 * fzm + 6.0 * fc - 4.0 * fzp + fz2p;
            // mixed differences: 4 edge mid-points per plane pair
            const double exy = ld(f, c - sx - sy) + ld(f, c + sx - sy) + ld(f, c - sx + sy) +
                               ld(f, c + sx + sy);
            const double exz = ld(f, c - sx - sz) + ld(f, c + sx - sz) + ld(f, c - sx + sz) +
                               ld(f, c + sx + sz);
            const double eyz = ld(f, c - sy - sz) + ld(f, c + sy - sz) + ld(f, c - sy + sz) +
                               ld(f, c + sy + sz);
            const double sxn = fxm + fxp, syn = fym + fyp, szn = fzm + fzp;
            const double DxDy = exy - 2.0 * (sxn + syn) + 4.0 * fc;
            const double DxDz = exz - 2.0 * (sxn + szn) + 4.0 * fc;
            const double DyDz = eyz - 2.0 * (syn + szn) + 4.0 * fc;
            const double K = a.c0[l], Kz = a.c1[l];
            const double F6 = fc + (Dx + Dy + Dz) * (1.0 / 12.0) -
                              (Dx4 + Dy4 + Dz4) * (1.0 / 240.0) +
                              (DxDy + DxDz + DyDz) * (1.0 / 90.0) - h2 * K * fc * (1.0 / 20.0) +
                              h2 * h * Kz * (fzp - fzm) * (1.0 / 120.0);
            val = h2 * F6;
        }
    }
    const bool near = (i == 1 || i == a.Nx || j == 1 || j == a.Ny || l == 1 || l == a.Nz);
    if (near) val -= lift_terms<T>(a, i, j, l);
    F[out] = val;
}

// r = F - A U with U = 0 outside the interior.
template <typename Tr>
__global__ void __launch_bounds__(256) residual_kernel(int Nx, int Ny, int Nz,
                                                        const double *__restrict__ coef,
                                                        const double *__restrict__ F,
                                                        const double *__restrict__ U,
                                                        Tr *__restrict__ r) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const int j = blockIdx.y * blockDim.y + threadIdx.y;
    const int l = blockIdx.z;
    if (i >= Nx || j >= Ny) return;
    const size_t plane = (size_t)Nx * Ny;
    const double *cf = coef + (size_t)l * 12;
    double acc = 0.0;
    for (int dl = -1; dl <= 1; ++dl) {
        const int ll = l + dl;
        if (ll < 0 || ll >= Nz) continue;
        const double *P = U + (size_t)ll * plane;
        const double ca = cf[(dl + 1) * 4 + 0], cb = cf[(dl + 1) * 4 + 1];
        const double cc = cf[(dl + 1) * 4 + 2], cd = cf[(dl + 1) * 4 + 3];
        const bool im = i > 0, ip = i < Nx - 1, jm = j > 0, jp = j < Ny - 1;
        const size_t c = (size_t)j * Nx + i;
        double corners = 0.0, xn = 0.0, yn = 0.0;
        if (jm) {
            const size_t r0 = c - Nx;
            if (im) corners += __ldg(P + r0 - 1);
            if (ip) corners += __ldg(P + r0 + 1);
            yn += __ldg(P + r0);
        }
        if (jp) {
            const size_t r0 = c + Nx;
            if (im) corners += __ldg(P + r0 - 1);
            if (ip) corners += __ldg(P + r0 + 1);
            yn += __ldg(P + r0);
        }
        if (im) xn += __ldg(P + c - 1);
        if (ip) xn += __ldg(P + c + 1);
        acc += ca * corners + cb * xn + cc * yn + cd * __ldg(P + c);
    }
    const size_t o = (size_t)l * plane + (size_t)j * Nx + i;
    r[o] = (Tr)(F[o] - acc);
}

template <typename T>
__global__ void __launch_bounds__(256) sumsq_kernel(const T *__restrict__ x, size_t n,
                                                     double *out) {
    double acc = 0.0;
    for (size_t k = (size_t)blockIdx.x * blockDim.x + threadIdx.x; k < n;
         k += (size_t)gridDim.x * blockDim.x) {
        const double v = (double)x[k];
        acc += v * v;
    }
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
    __shared__ double part[8];
    if ((threadIdx.x & 31) == 0) part[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        double s = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += part[w];
        atomicAdd(out, s);
    }
}

}  // namespace

hs_status hs_launch_rhs(const hs_plan_s *P, const void *f, int f_dtype, int rhs_kind,
                        const DevBoundary &b, double *F, cudaStream_t s) {
    RhsArgs a;
    a.Nx = P->Nx;
    a.Ny = P->Ny;
    a.Nz = P->Nz;
    a.hz = P->hz;
    a.order = P->order;
    a.equation = P->equation;
    a.rhs_kind = rhs_kind;
    a.coef = P->d_coef;
    a.c0 = P->d_c0;
    a.c1 = P->d_c1;
    a.b = b;
    dim3 block(32, 8, 1);
    dim3 grid((P->Nx + 31) / 32, (P->Ny + 7) / 8, P->Nz);
    if (f_dtype == HS_F64)
        rhs_kernel<double><<<grid, block, 0, s>>>(a, static_cast<const double *>(f), F);
    else
        rhs_kernel<float><<<grid, block, 0, s>>>(a, static_cast<const float *>(f), F);
    return cudaGetLastError() == cudaSuccess ? HS_OK : HS_ERR_CUDA;
}

hs_status hs_launch_residual(const hs_plan_s *P, const double *F, const double *U, float *r32,
                             double *r64, cudaStream_t s) {
    dim3 block(32, 8, 1);
    dim3 grid((P->Nx + 31) / 32, (P->Ny + 7) / 8, P->Nz);
    if (r32)
        residual_kernel<float><<<grid, block, 0, s>>>(P->Nx, P->Ny, P->Nz, P->d_coef, F, U, r32);
    else
        residual_kernel<double><<<grid, block, 0, s>>>(P->Nx, P->Ny, P->Nz, P->d_coef, F, U, r64);
    return cudaGetLastError() == cudaSuccess ? HS_OK : HS_ERR_CUDA;
}

hs_status hs_launch_sumsq(const double *x64, const float *x32, size_t n, double *d_out,
                          cudaStream_t s) {
    const int blocks = (int)((n + 255) / 256 < 1216 ? (n + 255) / 256 : 1216);
    if (x32)
        sumsq_kernel<float><<<blocks > 0 ? blocks : 1, 256, 0, s>>>(x32, n, d_out);
    else
        sumsq_kernel<double><<<blocks > 0 ? blocks : 1, 256, 0, s>>>(x64, n, d_out);
    return cudaGetLastError() == cudaSuccess ? HS_OK : HS_ERR_CUDA;
}
