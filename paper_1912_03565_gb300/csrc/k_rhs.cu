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
#include "hs_resid_sf.cuh"
#include "hs_rhs_sf.cuh"
#include "hs_tiles.cuh"

namespace {

using namespace hs_tiles;

template <typename T, int OUT_DF>
__global__ void __launch_bounds__(256) rhs_kernel(RhsArgs a, const T *__restrict__ f,
                                                   void *__restrict__ Fout) {
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
    if (a.has_faces && near) val -= lift_terms<T>(a, i, j, l);
    if (OUT_DF) {
        const dfloat d = df_from_double(val);
        float *Fo = static_cast<float *>(Fout);
        Fo[out] = d.hi;
        Fo[out + (size_t)a.Nx * a.Ny * a.Nz] = d.lo;
    } else {
        static_cast<double *>(Fout)[out] = val;
    }
}

template <typename T, int OUT_DF>
__global__ void __launch_bounds__(RTX *RTY) rhs_tiled_kernel(RhsArgs a, const T *__restrict__ f,
                                                             void *__restrict__ Fout) {
    __shared__ double pl[5][RHY][RHX];
    const int tx = threadIdx.x, ty = threadIdx.y, tid = ty * RTX + tx;
    const int i0 = 1 + blockIdx.x * RTX, j0 = 1 + blockIdx.y * RTY;
    const int lbeg = 1 + (blockIdx.z + a.bz0) * RZ;
    const int lend = min(lbeg + RZ - 1, a.Nz);
    const size_t n = (size_t)a.Nx * a.Ny * a.Nz;
    const double h = a.hz, h2 = h * h;

    auto load_plane = [&](int l) {
        double(*P)[RHX] = pl[(l + 10) % 5];
        for (int e = tid; e < RHX * RHY; e += RTX * RTY) {
            const int ey = e / RHX, ex = e - ey * RHX;
            P[ey][ex] = node_or_ghost<T>(a, f, i0 - 2 + ex, j0 - 2 + ey, l);
        }
    };
    for (int l = lbeg - 2; l <= lbeg + 1; ++l) load_plane(l);
    const int i = i0 + tx, j = j0 + ty;
    const int cx = tx + 2, cy = ty + 2;
    for (int l = lbeg; l <= lend; ++l) {
        load_plane(l + 2);
        __syncthreads();
        if (i <= a.Nx && j <= a.Ny) {
            const double(*Pm2)[RHX] = pl[(l + 8) % 5];
            const double(*Pm)[RHX] = pl[(l + 9) % 5];
            const double(*P0)[RHX] = pl[(l + 10) % 5];
            const double(*Pp)[RHX] = pl[(l + 11) % 5];
            const double(*Pp2)[RHX] = pl[(l + 12) % 5];
            const double fc = P0[cy][cx];
            const double fzm = Pm[cy][cx], fzp = Pp[cy][cx];
            const double S1 = (P0[cy][cx - 1] + P0[cy][cx + 1]) + (P0[cy - 1][cx] + P0[cy + 1][cx]) +
                              (fzm + fzp);
            double val;
            if (a.equation == HS_CONVDIFF) {
                const double g = a.c0[l];
                val = h2 * (0.5 * fc + S1 * (1.0 / 12.0) + h * g * (fzp - fzm) * (1.0 / 24.0));
            } else if (a.order == 2) {
                val = h2 * fc;
            } else if (a.order == 4) {
                val = h2 * (0.5 * fc + S1 * (1.0 / 12.0));
            } else {
                const double S2 = (P0[cy][cx - 2] + P0[cy][cx + 2]) +
                                  (P0[cy - 2][cx] + P0[cy + 2][cx]) + (Pm2[cy][cx] + Pp2[cy][cx]);
                const double E = ((P0[cy - 1][cx - 1] + P0[cy - 1][cx + 1]) +
                                  (P0[cy + 1][cx - 1] + P0[cy + 1][cx + 1])) +
                                 ((Pm[cy][cx - 1] + Pm[cy][cx + 1]) + (Pm[cy - 1][cx] + Pm[cy + 1][cx])) +
                                 ((Pp[cy][cx - 1] + Pp[cy][cx + 1]) + (Pp[cy - 1][cx] + Pp[cy + 1][cx]));
                const double K = a.c0[l], Kz = a.c1[l];
                const double F6 = (67.0 / 120.0 - h2 * K * (1.0 / 20.0)) * fc + S1 * (1.0 / 18.0) -
                                  S2 * (1.0 / 240.0) + E * (1.0 / 90.0) +
                                  h2 * h * Kz * (1.0 / 120.0) * (fzp - fzm);
                val = h2 * F6;
            }
            const bool near = (i == 1 || i == a.Nx || j == 1 || j == a.Ny || l == 1 || l == a.Nz);
            if (a.has_faces && near) val -= lift_terms<T>(a, i, j, l);
            const size_t out = ((size_t)(l - 1) * a.Ny + (j - 1)) * a.Nx + (i - 1);
            if (OUT_DF) {
                const dfloat d = df_from_double(val);
                float *Fo = static_cast<float *>(Fout);
                Fo[out] = d.hi;
                Fo[out + n] = d.lo;
            } else {
                static_cast<double *>(Fout)[out] = val;
            }
        }
        __syncthreads();
    }
}

// Ghost nodes of the 6th-order right-hand side (one node beyond a face along
// its normal, 2 f_0 - f_1 + h^2 (f_nn)_face: node_or_ghost), into the layout
// of hs_plan_s::d_ghost: x faces for node planes pl0 .. pl1, y faces likewise,
// and the z-lo / z-hi ghost planes when zlo / zhi.
template <typename T>
__global__ void __launch_bounds__(256) ghost_kernel(RhsArgs a, const T *__restrict__ f,
                                                    double *__restrict__ g, int pl0, int pl1,
                                                    int zlo, int zhi) {
    // 32-bit index arithmetic: at most 2 (Nz + 2)(Nx + Ny + 4) + 2 (Nx + 2)(Ny + 2)
    // items, far below 2^31 for any grid that fits in memory
    const int np = pl1 - pl0 + 1;
    const int nyx = a.Ny + 2, nxx = a.Nx + 2;
    const int cx = 2 * np * nyx, cy = 2 * np * nxx, cz = nyx * nxx;
    double *gx = g;
    double *gy = gx + 2 * (size_t)(a.Nz + 2) * nyx;
    double *gz = gy + 2 * (size_t)(a.Nz + 2) * nxx;
    const int nzs = (zlo != 0) + (zhi != 0);   // z faces to form
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < cx + cy + nzs * cz;
         t += gridDim.x * blockDim.x) {
        if (t < cx) {
            const int side = t >= np * nyx;
            const int r = t - side * np * nyx;
            const int q = r / nyx;
            const int pl = pl0 + q, j = r - q * nyx;
            gx[((size_t)side * (a.Nz + 2) + pl) * nyx + j] =
                node_or_ghost<T>(a, f, side ? a.Nx + 2 : -1, j, pl);
        } else if (t < cx + cy) {
            const int u = t - cx;
            const int side = u >= np * nxx;
            const int r = u - side * np * nxx;
            const int q = r / nxx;
            const int pl = pl0 + q, i = r - q * nxx;
            gy[((size_t)side * (a.Nz + 2) + pl) * nxx + i] =
                node_or_ghost<T>(a, f, i, side ? a.Ny + 2 : -1, pl);
        } else {
            const int u = t - cx - cy;
            const int side = (zlo && u < cz) ? 0 : 1;
            const int r = u - (u < cz ? 0 : cz);
            const int j = r / nxx, i = r - j * nxx;
            gz[(size_t)side * cz + r] = node_or_ghost<T>(a, f, i, j, side ? a.Nz + 2 : -1);
        }
    }
}

// Mixed path, nodal f: the sum-factorised double-float tile (hs_rhs_sf.cuh).
// CTAs per SM the register allocation of the sum-factorised kernel is sized for
#ifndef HS_RHS_SF_MINB
#define HS_RHS_SF_MINB 3
#endif

template <int KIND, typename T>
__global__ void __launch_bounds__(SFX *SFY, HS_RHS_SF_MINB) rhs_sf_kernel(RhsArgs a, const T *__restrict__ f,
                                                          float *__restrict__ Fo, double *f2out,
                                                          const float4 *__restrict__ rw,
                                                          float2 W) {
    constexpr int H = KIND == SF_O6 ? 2 : 1;
    __shared__ __align__(16) unsigned char smem[sf_smem_bytes<H, T>()];
    rhs_sf_tile<KIND, T>(a, f, Fo, f2out, rw, W, smem, blockIdx.x, blockIdx.y,
                         blockIdx.z + a.bz0);
}

template <typename T>
void launch_rhs_sf(const hs_plan_s *P, const RhsArgs &a, const T *f, float *Fo, double *f2,
                   int cnt, cudaStream_t s) {
    dim3 tg((P->Nx + SFX - 1) / SFX, (P->Ny + SFY - 1) / SFY, (unsigned)cnt);
    const float4 *rw = P->d_rhs_df + (P->Nz + 2);
    const float2 W = P->rhs_sf_W;
    if (P->equation == HS_CONVDIFF)
        rhs_sf_kernel<SF_CD, T><<<tg, SFX * SFY, 0, s>>>(a, f, Fo, f2, rw, W);
    else if (P->order == 6)
        rhs_sf_kernel<SF_O6, T><<<tg, SFX * SFY, 0, s>>>(a, f, Fo, f2, rw, W);
    else if (P->order == 4)
        rhs_sf_kernel<SF_O4, T><<<tg, SFX * SFY, 0, s>>>(a, f, Fo, f2, rw, W);
    else
        rhs_sf_kernel<SF_O2, T><<<tg, SFX * SFY, 0, s>>>(a, f, Fo, f2, rw, W);
}

// The lean pair residual (hs_resid_sf.cuh); XY: x- and y-neighbour sums merged
// (b_nu = c_nu on every row); ULO: U has a lo plane (else only its hi plane
// is read, the lo parts being zero).
template <bool XY, bool ULO = true>
__global__ void __launch_bounds__(RSX *RSY) residual_sf_kernel(int Nx, int Ny, int Nz,
                                                                const float2 *__restrict__ coef,
                                                                const float *__restrict__ F,
                                                                const float *__restrict__ U,
                                                                float *__restrict__ r,
                                                                const int *skip, double *r2out,
                                                                const double *norms, int m,
                                                                int sel, int zt) {
    if (skip && *skip) return;
    if (sel == HS_RESID_SEL_DF && residual_use_f64(norms, m)) return;
    __shared__ __align__(16) float2 ring[resid_async_smem() / sizeof(float2)];
    residual_sf_tile_async<XY, ULO>(Nx, Ny, Nz, coef, F, U, r, r2out, ring, blockIdx.x,
                                    blockIdx.y, blockIdx.z, zt);
}

__global__ void __launch_bounds__(QTX *QTY) residual64_zmarch_kernel(
    int Nx, int Ny, int Nz, const double *__restrict__ coef, const float *__restrict__ F,
    const float *__restrict__ U, float *__restrict__ r, const int *skip, double *r2out,
    const double *norms, int m, int sel) {
    if (skip && *skip) return;
    if (sel == HS_RESID_SEL_F64 && !residual_use_f64(norms, m)) return;
    __shared__ __align__(16) unsigned char smem[2 * QHY * QHX * sizeof(double)];
    residual64_tile<false>(Nx, Ny, Nz, coef, F, U, r, r2out, smem, blockIdx.x, blockIdx.y,
                           blockIdx.z);
}

__global__ void refine_gate_kernel(const double *r2, const double *f2, double tol2, int *skip) {
    if (*skip == 0 && *r2 <= tol2 * *f2) *skip = 1;
}

// u (FP64) = hi + lo of a double-float array.
__global__ void __launch_bounds__(256) df_to_f64_kernel(const float *__restrict__ x, size_t n,
                                                         double *__restrict__ u) {
    for (size_t k = (size_t)blockIdx.x * blockDim.x + threadIdx.x; k < n;
         k += (size_t)gridDim.x * blockDim.x)
        u[k] = (double)x[k] + (double)x[k + n];
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

hs_status hs_upload_rhs(hs_plan_s *P, const void *fh, void *fd, int chunks, int f_dtype,
                        const DevBoundary &b, void *F, int out_df, cudaStream_t s, double *f2) {
    const int K = chunks < 1 ? 1 : (chunks > HS_UP_CHUNKS ? HS_UP_CHUNKS : chunks);
    const size_t esz = f_dtype == HS_F64 ? 8 : 4;
    const size_t pb = (size_t)(P->Nx + 2) * (P->Ny + 2) * esz;   // bytes per node plane
    const int TZ = hs_rhs_tile_planes(P, out_df);
    const int tz = (P->Nz + TZ - 1) / TZ;
    const unsigned char *src = static_cast<const unsigned char *>(fh);
    unsigned char *dst = static_cast<unsigned char *>(fd);
    int copied = 0;   // node planes [0, copied) are on their way
    for (int k = 0; k < K; ++k) {
        const int t0 = (k * tz) / K, t1 = ((k + 1) * tz) / K;
        // the slab's last tile reads node planes up to min(t1 RZ, Nz) + 2 (<= Nz + 1)
        const int need = k == K - 1 ? P->Nz + 2 : (t1 * TZ + 3 < P->Nz + 2 ? t1 * TZ + 3 : P->Nz + 2);
        if (need > copied) {
            if (cudaMemcpyAsync(dst + copied * pb, src + copied * pb, (size_t)(need - copied) * pb,
                                cudaMemcpyHostToDevice, P->up_stream) != cudaSuccess)
                return HS_ERR_CUDA;
            copied = need;
        }
        if (cudaEventRecord(P->up_ev[k], P->up_stream) != cudaSuccess ||
            cudaStreamWaitEvent(s, P->up_ev[k], 0) != cudaSuccess)
            return HS_ERR_CUDA;
        if (t1 > t0) {
            const hs_status st = hs_launch_rhs(P, fd, f_dtype, HS_RHS_NODAL, b, F, out_df, s, f2,
                                               t0, t1 - t0);
            if (st != HS_OK) return st;
        }
    }
    return HS_OK;
}

namespace {

// Planes per z-slab of a z-marching kernel launched as (xy tiles) x (slabs)
// CTAs: the depth whose CTAs fill whole waves best.  A CTA's time is taken as
// its slab's planes plus `halo` planes on each side and about two planes of
// prologue, and a launch as (waves of CTAs) x (one CTA's time), waves =
// ceil(CTAs / (resident CTAs per SM x SMs)).  Slabs hold 4 to 64 planes: short
// CTAs let the block scheduler even out tiles that cost more (those touching a
// face form ghost nodes in FP64), so of two depths within 2 % of each other the
// shorter is taken.  At 255^3 this gives 7 slabs of 37 planes (4 waves of the
// right-hand side, 3 of the residual) instead of 8 of 32 (4.5 and 3.4 waves).
int zmarch_depth(long tiles, int Nz, int halo, int resident, int sms) {
    const long slots = (long)(resident > 0 ? resident : 1) * (sms > 0 ? sms : 1);
    const int zmin = Nz < 4 ? Nz : 4;
    int best = Nz < 64 ? Nz : 64;
    long best_cost = -1;
    for (int ns = 1; ns <= Nz; ++ns) {
        const int zt = (Nz + ns - 1) / ns;
        if (zt > 64) continue;
        if (zt < zmin) break;
        const long ctas = tiles * ((Nz + zt - 1) / zt);
        const long cost = ((ctas + slots - 1) / slots) * (zt + 2 * halo + 2);
        if (best_cost < 0 || cost * 50 <= best_cost * 51) {
            if (best_cost < 0 || cost < best_cost) best_cost = cost;
            best = zt;
        }
    }
    return best;
}

int sm_count(const hs_plan_s *P) {
    static int sms = 0;
    if (sms == 0 && cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, P->device) !=
                        cudaSuccess) {
        cudaGetLastError();
        sms = 148;
    }
    return sms;
}

template <typename K>
int resident_ctas(K kernel, int threads) {
    int nb = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, kernel, threads, 0) != cudaSuccess) {
        cudaGetLastError();
        return 2;
    }
    return nb > 0 ? nb : 1;
}

// depth of the mixed right-hand side (rhs_sf_kernel; the FP64-f instance)
int sf_rhs_depth(const hs_plan_s *P) {
    static int res[4] = {0, 0, 0, 0};
    const int kind = P->equation == HS_CONVDIFF ? SF_CD
                                                : (P->order == 6 ? SF_O6 : (P->order == 4 ? SF_O4 : SF_O2));
    if (res[kind] == 0)
        res[kind] = kind == SF_CD   ? resident_ctas(rhs_sf_kernel<SF_CD, double>, SFX * SFY)
                    : kind == SF_O6 ? resident_ctas(rhs_sf_kernel<SF_O6, double>, SFX * SFY)
                    : kind == SF_O4 ? resident_ctas(rhs_sf_kernel<SF_O4, double>, SFX * SFY)
                                    : resident_ctas(rhs_sf_kernel<SF_O2, double>, SFX * SFY);
    const long tiles = (long)((P->Nx + SFX - 1) / SFX) * ((P->Ny + SFY - 1) / SFY);
    return zmarch_depth(tiles, P->Nz, kind == SF_O6 ? 2 : 1, res[kind], sm_count(P));
}

// depth of the pair residual (residual_sf_kernel)
int sf_resid_depth(const hs_plan_s *P) {
    static int res = 0;
    if (res == 0) res = resident_ctas(residual_sf_kernel<true>, RSX * RSY);
    const long tiles = (long)((P->Nx + RSX - 1) / RSX) * ((P->Ny + RSY - 1) / RSY);
    return zmarch_depth(tiles, P->Nz, 1, res, sm_count(P));
}

}  // namespace

int hs_sf_zdepth(const hs_plan_s *P) { return sf_resid_depth(P); }

int hs_rhs_tile_planes(const hs_plan_s *P, int out_df) { return out_df ? sf_rhs_depth(P) : RZ; }

hs_status hs_launch_rhs(const hs_plan_s *P, const void *f, int f_dtype, int rhs_kind,
                        const DevBoundary &b, void *F, int out_df, cudaStream_t s, double *f2,
                        int bz0, int nbz) {
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
    a.rc = P->d_rhs_df;
    a.b = b;
    a.ghost = nullptr;
    a.has_faces = 0;
    for (int k = 0; k < 6; ++k)
        if (b.face[k]) a.has_faces = 1;
    if (rhs_kind == HS_RHS_NODAL) {
        const int TZ = hs_rhs_tile_planes(P, out_df);
        const int tz = (P->Nz + TZ - 1) / TZ;
        a.zt = TZ;
        a.bz0 = bz0 < 0 ? 0 : bz0;
        const int cnt = nbz < 0 ? tz - a.bz0 : nbz;
        if (cnt <= 0) return HS_OK;
        if (out_df) {
            a.ghost = nullptr;
            if (f_dtype == HS_F64 && P->d_ghost && P->order == 6 &&
                P->equation == HS_HELMHOLTZ) {
                // the ghost nodes of the node planes these z-tiles read
                const int lo = 1 + a.bz0 * TZ - 2;
                const int hi = (a.bz0 + cnt) * TZ + 2;
                const int pl0 = lo < 0 ? 0 : lo, pl1 = hi > P->Nz + 1 ? P->Nz + 1 : hi;
                const long work = 2L * (pl1 - pl0 + 1) * (P->Nx + P->Ny + 4) +
                                  (long)((lo < 0) + (hi > P->Nz + 1)) * (P->Nx + 2) * (P->Ny + 2);
                const unsigned gb = (unsigned)((work + 255) / 256 < 4096 ? (work + 255) / 256 : 4096);
                ghost_kernel<double><<<gb, 256, 0, s>>>(a, static_cast<const double *>(f),
                                                        P->d_ghost, pl0, pl1, lo < 0,
                                                        hi > P->Nz + 1);
                a.ghost = P->d_ghost;
            }
            if (f_dtype == HS_F64)
                launch_rhs_sf<double>(P, a, static_cast<const double *>(f), static_cast<float *>(F),
                                      f2, cnt, s);
            else
                launch_rhs_sf<float>(P, a, static_cast<const float *>(f), static_cast<float *>(F),
                                     f2, cnt, s);
            return cudaGetLastError() == cudaSuccess ? HS_OK : HS_ERR_CUDA;
        }
        dim3 tb(RTX, RTY, 1);
        dim3 tg((P->Nx + RTX - 1) / RTX, (P->Ny + RTY - 1) / RTY, (unsigned)cnt);
        if (f_dtype == HS_F64)
            rhs_tiled_kernel<double, 0><<<tg, tb, 0, s>>>(a, static_cast<const double *>(f), F);
        else
            rhs_tiled_kernel<float, 0><<<tg, tb, 0, s>>>(a, static_cast<const float *>(f), F);
        return cudaGetLastError() == cudaSuccess ? HS_OK : HS_ERR_CUDA;
    }
    a.bz0 = 0;
    dim3 block(32, 8, 1);
    dim3 grid((P->Nx + 31) / 32, (P->Ny + 7) / 8, P->Nz);
    if (f_dtype == HS_F64) {
        if (out_df)
            rhs_kernel<double, 1><<<grid, block, 0, s>>>(a, static_cast<const double *>(f), F);
        else
            rhs_kernel<double, 0><<<grid, block, 0, s>>>(a, static_cast<const double *>(f), F);
    } else {
        if (out_df)
            rhs_kernel<float, 1><<<grid, block, 0, s>>>(a, static_cast<const float *>(f), F);
        else
            rhs_kernel<float, 0><<<grid, block, 0, s>>>(a, static_cast<const float *>(f), F);
    }
    return cudaGetLastError() == cudaSuccess ? HS_OK : HS_ERR_CUDA;
}

hs_status hs_launch_residual_df(const hs_plan_s *P, const float *F, const float *U, float *r,
                                cudaStream_t s, double *r2, int prec, const double *norms,
                                int m, bool u_lo_zero) {
    dim3 qb(QTX, QTY, 1);
    dim3 qg((P->Nx + QTX - 1) / QTX, (P->Ny + QTY - 1) / QTY, (P->Nz + QZ - 1) / QZ);
    if (u_lo_zero && prec != HS_RESID_DF) return HS_ERR_UNSUPPORTED;
    if (prec == HS_RESID_DF || prec == HS_RESID_SEL_DF) {
        const int zt = hs_sf_zdepth(P);
        dim3 sg((P->Nx + RSX - 1) / RSX, (P->Ny + RSY - 1) / RSY, (P->Nz + zt - 1) / zt);
        if (u_lo_zero && P->resid_xy)
            residual_sf_kernel<true, false><<<sg, RSX * RSY, 0, s>>>(
                P->Nx, P->Ny, P->Nz, P->d_coef_df, F, U, r, P->cur_skip, r2, norms, m, prec, zt);
        else if (u_lo_zero)
            residual_sf_kernel<false, false><<<sg, RSX * RSY, 0, s>>>(
                P->Nx, P->Ny, P->Nz, P->d_coef_df, F, U, r, P->cur_skip, r2, norms, m, prec, zt);
        else if (P->resid_xy)
            residual_sf_kernel<true><<<sg, RSX * RSY, 0, s>>>(P->Nx, P->Ny, P->Nz, P->d_coef_df, F,
                                                              U, r, P->cur_skip, r2, norms, m, prec,
                                                              zt);
        else
            residual_sf_kernel<false><<<sg, RSX * RSY, 0, s>>>(P->Nx, P->Ny, P->Nz, P->d_coef_df,
                                                               F, U, r, P->cur_skip, r2, norms, m,
                                                               prec, zt);
    }
    if (prec == HS_RESID_F64 || prec == HS_RESID_SEL_F64)
        residual64_zmarch_kernel<<<qg, qb, 0, s>>>(P->Nx, P->Ny, P->Nz, P->d_coef, F, U, r,
                                                   P->cur_skip, r2, norms, m, prec);
    return cudaGetLastError() == cudaSuccess ? HS_OK : HS_ERR_CUDA;
}

hs_status hs_launch_gate(const double *r2, const double *f2, double tol, int *skip,
                         cudaStream_t s) {
    refine_gate_kernel<<<1, 1, 0, s>>>(r2, f2, tol * tol, skip);
    return cudaGetLastError() == cudaSuccess ? HS_OK : HS_ERR_CUDA;
}

hs_status hs_launch_df_to_f64(const float *x, size_t n, double *u, cudaStream_t s) {
    const unsigned blocks = (unsigned)((n + 255) / 256 < 4864 ? (n + 255) / 256 : 4864);
    df_to_f64_kernel<<<blocks > 0 ? blocks : 1, 256, 0, s>>>(x, n, u);
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
