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
#include "hs_df.cuh"
#include "hs_internal.cuh"

namespace {

struct RhsArgs {
    int Nx, Ny, Nz;
    double hz;           // h_z (the uniform h for order 6)
    int order, equation, rhs_kind;
    const double *coef;  // [Nz][3][4]
    const double *c0;    // [Nz+2]
    const double *c1;    // [Nz+2]
    const float4 *rc;    // [Nz+2]: per-row double-float RHS weights (see rhs_tiled_df_kernel)
    int has_faces;       // 0: every Dirichlet face is zero, so the lifting vanishes
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

// Adds a per-thread value over the CTA and atomically to *out (thread 0).
__device__ __forceinline__ void block_sum_to(double v, double *out) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    __shared__ double part[32];
    const int tid = threadIdx.x + threadIdx.y * blockDim.x;
    const int nw = (blockDim.x * blockDim.y + 31) >> 5;
    __syncthreads();
    if ((tid & 31) == 0) part[tid >> 5] = v;
    __syncthreads();
    if (tid == 0) {
        double s = 0.0;
        for (int w = 0; w < nw; ++w) s += part[w];
        atomicAdd(out, s);
    }
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

// OUT_DF = 0: F is FP64; OUT_DF = 1: F is stored as a double-float pair (hi, lo).
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

// ---------------------------------------------------------------------------
// Tiled right-hand side for nodal f: a CTA owns a TX x TY patch of interior
// points and marches over RZ planes in z with a ring of five f-planes in
// shared memory (halo 2 in x and y; the second neighbours beyond a face are
// the ghosts 2 f_0 - f_1 + h^2 (f_nn)_face, filled in at load time).  The
// 6th-order operator is evaluated in the summed form
//   F6 / h^2 = (67/120 - h^2 K_l / 20) f + S1 / 18 - S2 / 240 + E / 90
//              + (h^3 K_{z,l} / 120) (f_{l+1} - f_{l-1}),
// where S1 sums the 6 face neighbours, S2 the 6 second neighbours and E the 12
// edge mid-points (the same operator as the expanded form above:
// Dx+Dy+Dz = S1 - 6 f, Dx^2+Dy^2+Dz^2 = S2 - 4 S1 + 18 f,
// DxDy+DxDz+DyDz = E - 4 S1 + 12 f).
constexpr int RTX = 32, RTY = 8, RZ = 16;
constexpr int RHX = RTX + 4, RHY = RTY + 4;

template <typename T>
__device__ double node_or_ghost(const RhsArgs &a, const T *f, int i, int j, int l) {
    const int Nx = a.Nx, Ny = a.Ny, Nz = a.Nz;
    const size_t sy = (size_t)(Nx + 2), sz = sy * (Ny + 2);
    const double h2 = a.hz * a.hz;
    const bool xin = i >= 0 && i <= Nx + 1, yin = j >= 0 && j <= Ny + 1, zin = l >= 0 && l <= Nz + 1;
    if (xin && yin && zin) return ld(f, (size_t)l * sz + (size_t)j * sy + i);
    // ghosts exist one node beyond a face, along that face's normal only
    if (!xin && yin && zin && (i == -1 || i == Nx + 2)) {
        const int i0 = (i == -1) ? 0 : Nx + 1, i1 = (i == -1) ? 1 : Nx;
        const T *fnn = static_cast<const T *>(a.b.fnn[i == -1 ? 0 : 1]);
        const size_t r = (size_t)l * sz + (size_t)j * sy;
        return 2.0 * ld(f, r + i0) - ld(f, r + i1) +
               (fnn ? h2 * ld(fnn, (size_t)l * (Ny + 2) + j) : 0.0);
    }
    if (xin && !yin && zin && (j == -1 || j == Ny + 2)) {
        const int j0 = (j == -1) ? 0 : Ny + 1, j1 = (j == -1) ? 1 : Ny;
        const T *fnn = static_cast<const T *>(a.b.fnn[j == -1 ? 2 : 3]);
        const size_t r = (size_t)l * sz + i;
        return 2.0 * ld(f, r + (size_t)j0 * sy) - ld(f, r + (size_t)j1 * sy) +
               (fnn ? h2 * ld(fnn, (size_t)l * (Nx + 2) + i) : 0.0);
    }
    if (xin && yin && !zin && (l == -1 || l == Nz + 2)) {
        const int l0 = (l == -1) ? 0 : Nz + 1, l1 = (l == -1) ? 1 : Nz;
        const T *fnn = static_cast<const T *>(a.b.fnn[l == -1 ? 4 : 5]);
        const size_t r = (size_t)j * sy + i;
        return 2.0 * ld(f, (size_t)l0 * sz + r) - ld(f, (size_t)l1 * sz + r) +
               (fnn ? h2 * ld(fnn, (size_t)j * (Nx + 2) + i) : 0.0);
    }
    return 0.0;  // never read by an interior point
}

template <typename T, int OUT_DF>
__global__ void __launch_bounds__(RTX *RTY) rhs_tiled_kernel(RhsArgs a, const T *__restrict__ f,
                                                             void *__restrict__ Fout) {
    __shared__ double pl[5][RHY][RHX];
    const int tx = threadIdx.x, ty = threadIdx.y, tid = ty * RTX + tx;
    const int i0 = 1 + blockIdx.x * RTX, j0 = 1 + blockIdx.y * RTY;
    const int lbeg = 1 + blockIdx.z * RZ;
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

// The same tiled operator in double-float arithmetic (mixed path): f enters
// shared memory as (hi, lo) pairs (FP64 f split with integer operations,
// FP32 f exact), the sums and products use two_sum / two_prod, and F is
// written as its two FP32 planes.  Ghost values and the Dirichlet lifting
// (points next to a face only) are formed in FP64 and then split.
template <typename T>
__device__ __forceinline__ dfloat node_df(const RhsArgs &a, const T *f, int i, int j, int l) {
    const bool in = i >= 0 && i <= a.Nx + 1 && j >= 0 && j <= a.Ny + 1 && l >= 0 && l <= a.Nz + 1;
    if (in) {
        const size_t sy = (size_t)(a.Nx + 2), sz = sy * (a.Ny + 2);
        return df_of(__ldg(f + (size_t)l * sz + (size_t)j * sy + i));
    }
    return df_split_bits(node_or_ghost<T>(a, f, i, j, l));
}

__device__ __forceinline__ dfloat dsum(dfloat a, dfloat b) { return df_add(a, b); }

// Sum of double-float terms without renormalising after each one: the hi parts
// go through two_sum (exact), their errors and the lo parts are added in FP32.
struct LeanSum {
    float s, e;
    __device__ __forceinline__ LeanSum(dfloat a) : s(a.hi), e(a.lo) {}
    __device__ __forceinline__ void add(dfloat a) {
        float t, err;
        df_two_sum(s, a.hi, t, err);
        s = t;
        e += err + a.lo;
    }
    __device__ __forceinline__ dfloat get() const {
        dfloat r;
        df_fast_two_sum(s, e, r.hi, r.lo);
        return r;
    }
};

template <typename T>
__global__ void __launch_bounds__(RTX *RTY) rhs_tiled_df_kernel(RhsArgs a, const T *__restrict__ f,
                                                                float *__restrict__ Fo,
                                                                double *f2out) {
    __shared__ float ph[5][RHY][RHX];
    __shared__ float pq[5][RHY][RHX];
    constexpr int NT = RTX * RTY;
    constexpr int PER = (RHX * RHY + NT - 1) / NT;
    const int tx = threadIdx.x, ty = threadIdx.y, tid = ty * RTX + tx;
    const int i0 = 1 + blockIdx.x * RTX, j0 = 1 + blockIdx.y * RTY;
    const int lbeg = 1 + blockIdx.z * RZ;
    const int lend = min(lbeg + RZ - 1, a.Nz);
    const size_t n = (size_t)a.Nx * a.Ny * a.Nz;
    const dfloat H2 = df_from_double(a.hz * a.hz);
    const dfloat C18 = df_from_double(1.0 / 18.0), C240 = df_from_double(-1.0 / 240.0);
    const dfloat C90 = df_from_double(1.0 / 90.0), C12 = df_from_double(1.0 / 12.0);
    const dfloat HALF = df_of(0.5f);

    dfloat reg[PER];
    auto fetch = [&](int l) {
#pragma unroll
        for (int k = 0; k < PER; ++k) {
            const int e = tid + k * NT;
            const int ey = e / RHX, ex = e - ey * RHX;
            reg[k] = (e < RHX * RHY) ? node_df<T>(a, f, i0 - 2 + ex, j0 - 2 + ey, l)
                                     : df_of(0.f);
        }
    };
    auto store = [&](int l) {
        const int slot = (l + 10) % 5;
#pragma unroll
        for (int k = 0; k < PER; ++k) {
            const int e = tid + k * NT;
            if (e < RHX * RHY) {
                const int ey = e / RHX, ex = e - ey * RHX;
                ph[slot][ey][ex] = reg[k].hi;
                pq[slot][ey][ex] = reg[k].lo;
            }
        }
    };
    for (int l = lbeg - 2; l <= lbeg + 1; ++l) {
        fetch(l);
        store(l);
    }
    fetch(lbeg + 2);
    float fsq = 0.f;
    const int i = i0 + tx, j = j0 + ty;
    const int cx = tx + 2, cy = ty + 2;
    for (int l = lbeg; l <= lend; ++l) {
        store(l + 2);               // slot of plane l - 3, last read in the previous step
        __syncthreads();
        if (l + 3 <= lend + 2) fetch(l + 3);   // in flight during this plane's arithmetic
        if (i <= a.Nx && j <= a.Ny) {
            const int sm2 = (l + 8) % 5, sm = (l + 9) % 5, s0 = (l + 10) % 5, sp = (l + 11) % 5,
                      sp2 = (l + 12) % 5;
#define HS_G(S, Y, X) dfloat{ph[S][Y][X], pq[S][Y][X]}
            const dfloat fc = HS_G(s0, cy, cx);
            const dfloat fzm = HS_G(sm, cy, cx), fzp = HS_G(sp, cy, cx);
            LeanSum a1(HS_G(s0, cy, cx - 1));
            a1.add(HS_G(s0, cy, cx + 1));
            a1.add(HS_G(s0, cy - 1, cx));
            a1.add(HS_G(s0, cy + 1, cx));
            a1.add(fzm);
            a1.add(fzp);
            const dfloat S1 = a1.get();
            dfloat val;
            const float4 w = a.rc[l];
            if (a.equation == HS_CONVDIFF) {
                const dfloat g = dfloat{w.z, w.w};
                const dfloat dz = df_add_accurate(fzp, df_neg(fzm));
                val = df_mul(H2, dsum(dsum(df_mul(HALF, fc), df_mul(C12, S1)), df_mul(g, dz)));
            } else if (a.order == 2) {
                val = df_mul(H2, fc);
            } else if (a.order == 4) {
                val = df_mul(H2, dsum(df_mul(HALF, fc), df_mul(C12, S1)));
            } else {
                LeanSum a2(HS_G(s0, cy, cx - 2));
                a2.add(HS_G(s0, cy, cx + 2));
                a2.add(HS_G(s0, cy - 2, cx));
                a2.add(HS_G(s0, cy + 2, cx));
                a2.add(HS_G(sm2, cy, cx));
                a2.add(HS_G(sp2, cy, cx));
                const dfloat S2 = a2.get();
                LeanSum a3(HS_G(s0, cy - 1, cx - 1));
                a3.add(HS_G(s0, cy - 1, cx + 1));
                a3.add(HS_G(s0, cy + 1, cx - 1));
                a3.add(HS_G(s0, cy + 1, cx + 1));
                a3.add(HS_G(sm, cy, cx - 1));
                a3.add(HS_G(sm, cy, cx + 1));
                a3.add(HS_G(sm, cy - 1, cx));
                a3.add(HS_G(sm, cy + 1, cx));
                a3.add(HS_G(sp, cy, cx - 1));
                a3.add(HS_G(sp, cy, cx + 1));
                a3.add(HS_G(sp, cy - 1, cx));
                a3.add(HS_G(sp, cy + 1, cx));
                const dfloat E = a3.get();
                const dfloat alpha = dfloat{w.x, w.y};
                const dfloat eps = dfloat{w.z, w.w};
                const dfloat dz = df_add_accurate(fzp, df_neg(fzm));
                dfloat F6 = df_mul(alpha, fc);
                F6 = dsum(F6, df_mul(C18, S1));
                F6 = dsum(F6, df_mul(C240, S2));
                F6 = dsum(F6, df_mul(C90, E));
                F6 = dsum(F6, df_mul(eps, dz));
                val = df_mul(H2, F6);
            }
#undef HS_G
            const bool near = (i == 1 || i == a.Nx || j == 1 || j == a.Ny || l == 1 || l == a.Nz);
            if (a.has_faces && near)
                val = df_add_accurate(val, df_neg(df_split_bits(lift_terms<T>(a, i, j, l))));
            const size_t out = ((size_t)(l - 1) * a.Ny + (j - 1)) * a.Nx + (i - 1);
            Fo[out] = val.hi;
            Fo[out + n] = val.lo;
            fsq = fmaf(val.hi, val.hi, fsq);
        }
        __syncthreads();
    }
    if (f2out) block_sum_to((double)fsq, f2out);
}

// r = F - A U in double-float arithmetic: F and U are (hi, lo) pairs, the
// per-row coefficients are split into FP32 pairs, U = 0 outside the interior.
// A U_hi is accumulated exactly enough (two_sum / two_prod); A U_lo, which is
// ~2^-24 of it, in plain FP32.  r is rounded to FP32.
__global__ void __launch_bounds__(256) residual_df_kernel(int Nx, int Ny, int Nz,
                                                           const float2 *__restrict__ coef,
                                                           const float *__restrict__ F,
                                                           const float *__restrict__ U,
                                                           float *__restrict__ r) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const int j = blockIdx.y * blockDim.y + threadIdx.y;
    const int l = blockIdx.z;
    if (i >= Nx || j >= Ny) return;
    const size_t plane = (size_t)Nx * Ny;
    const size_t n = plane * Nz;
    const float2 *cf = coef + (size_t)l * 12;
    const bool im = i > 0, ip = i < Nx - 1, jm = j > 0, jp = j < Ny - 1;
    const size_t c = (size_t)j * Nx + i;
    dfloat acc;
    acc.hi = 0.f;
    acc.lo = 0.f;
    float acc_lo = 0.f;
#pragma unroll
    for (int dl = -1; dl <= 1; ++dl) {
        const int ll = l + dl;
        if (ll < 0 || ll >= Nz) continue;
        const float *P = U + (size_t)ll * plane;
        const float *Q = P + n;  // lo plane
        float h[9], q[9];
        // 0: (i-1,j-1) 1: (i+1,j-1) 2: (i,j-1) 3: (i-1,j+1) 4: (i+1,j+1) 5: (i,j+1)
        // 6: (i-1,j) 7: (i+1,j) 8: (i,j)
        const bool ok[9] = {jm && im, jm && ip, jm, jp && im, jp && ip, jp, im, ip, true};
        const long off[9] = {-(long)Nx - 1, -(long)Nx + 1, -(long)Nx, (long)Nx - 1, (long)Nx + 1,
                             (long)Nx, -1, 1, 0};
#pragma unroll
        for (int k = 0; k < 9; ++k) {
            h[k] = ok[k] ? __ldg(P + (long)c + off[k]) : 0.f;
            q[k] = ok[k] ? __ldg(Q + (long)c + off[k]) : 0.f;
        }
        const dfloat C = df_add(df_make(h[0], h[1]), df_make(h[3], h[4]));
        const dfloat X = df_make(h[6], h[7]);
        const dfloat Y = df_make(h[2], h[5]);
        dfloat ce;
        ce.hi = h[8];
        ce.lo = 0.f;
        const float2 ka = cf[(dl + 1) * 4 + 0], kb = cf[(dl + 1) * 4 + 1];
        const float2 kc = cf[(dl + 1) * 4 + 2], kd = cf[(dl + 1) * 4 + 3];
        dfloat t = df_mul(dfloat{ka.x, ka.y}, C);
        t = df_add(t, df_mul(dfloat{kb.x, kb.y}, X));
        t = df_add(t, df_mul(dfloat{kc.x, kc.y}, Y));
        t = df_add(t, df_mul(dfloat{kd.x, kd.y}, ce));
        acc = df_add(acc, t);
        acc_lo += ka.x * ((q[0] + q[1]) + (q[3] + q[4])) + kb.x * (q[6] + q[7]) +
                  kc.x * (q[2] + q[5]) + kd.x * q[8];
    }
    const size_t o = (size_t)l * plane + c;
    const dfloat res = df_add_accurate(dfloat{F[o], F[o + n]}, df_neg(acc));
    r[o] = res.hi + (res.lo - acc_lo);
}

// z-marching double-float residual.  A CTA owns a RTX x RTY patch and RZ
// planes; a ring of three U-planes (hi and lo, halo 1) sits in shared memory.
// For every plane each thread forms the in-plane sums of its column once --
// corners C, x-neighbours X, y-neighbours Y (exact pair sums of the FP32 hi
// parts, plain FP32 sums of the lo parts) -- and keeps the last three planes'
// sums in registers, so output row l costs 12 products
//     A U_l = sum_nu a_nu C_nu + b_nu X_nu + c_nu Y_nu + d_nu U_nu,
// accumulated as an unnormalised pair (two_prod into two_sum; cross terms and
// lo parts in FP32), and one accurate pair subtraction F - A U.
struct PlaneSums {
    float C, Ce, X, Xe, Y, Ye, U;   // hi sums with their two_sum errors; U = centre hi
    float L;                        // lo parts: C_lo etc. folded per coefficient below
    float Clo, Xlo, Ylo, Ulo;
};

__device__ __forceinline__ void acc_term(float &S, float &E, float2 k, float v, float ve,
                                         float vlo) {
    // S + E += (k.x + k.y) * (v + ve + vlo)
    const float p = k.x * v;
    const float pe = fmaf(k.x, v, -p);
    float s, t;
    df_two_sum(S, p, s, t);
    S = s;
    E += t + pe + fmaf(k.x, ve + vlo, k.y * v);
}

constexpr int QTX = 32, QTY = 8, QZ = 16;
constexpr int QHX = QTX + 2, QHY = QTY + 2;

__global__ void __launch_bounds__(QTX *QTY) residual_zmarch_kernel(int Nx, int Ny, int Nz,
                                                                    const float2 *__restrict__ coef,
                                                                    const float *__restrict__ F,
                                                                    const float *__restrict__ U,
                                                                    float *__restrict__ r,
                                                                    const int *skip, double *r2out) {
    if (skip && *skip) return;
    // two plane slots: the plane whose sums are being formed and the next one,
    // whose global loads are issued into registers before the current plane's
    // arithmetic (so their latency overlaps it)
    __shared__ float uh[2][QHY][QHX];
    __shared__ float ul[2][QHY][QHX];
    constexpr int NT = QTX * QTY;
    constexpr int PER = (QHX * QHY + NT - 1) / NT;
    const int tx = threadIdx.x, ty = threadIdx.y, tid = ty * QTX + tx;
    const int i0 = blockIdx.x * QTX, j0 = blockIdx.y * QTY;  // 0-based interior indices
    const int lbeg = blockIdx.z * QZ;
    const int lend = min(lbeg + QZ, Nz);                      // exclusive
    const size_t plane = (size_t)Nx * Ny;
    const size_t n = plane * Nz;
    const int i = i0 + tx, j = j0 + ty;
    const bool active = i < Nx && j < Ny;

    float rh[PER], rl[PER];
    auto fetch = [&](int l) {
#pragma unroll
        for (int k = 0; k < PER; ++k) {
            const int e = tid + k * NT;
            const int ey = e / QHX, ex = e - ey * QHX;
            const int ii = i0 - 1 + ex, jj = j0 - 1 + ey;
            rh[k] = 0.f;
            rl[k] = 0.f;
            if (e < QHX * QHY && l >= 0 && l < Nz && ii >= 0 && ii < Nx && jj >= 0 && jj < Ny) {
                const size_t o = (size_t)l * plane + (size_t)jj * Nx + ii;
                rh[k] = __ldg(U + o);
                rl[k] = __ldg(U + n + o);
            }
        }
    };
    auto store = [&](int l) {
        const int slot = (l + 2) & 1;
#pragma unroll
        for (int k = 0; k < PER; ++k) {
            const int e = tid + k * NT;
            if (e < QHX * QHY) {
                const int ey = e / QHX, ex = e - ey * QHX;
                uh[slot][ey][ex] = rh[k];
                ul[slot][ey][ex] = rl[k];
            }
        }
    };
    auto sums = [&](int l, PlaneSums &ps) {
        const int sl = (l + 2) & 1;
        const int cx = tx + 1, cy = ty + 1;
        float s, e, s2, e2;
        df_two_sum(uh[sl][cy - 1][cx - 1], uh[sl][cy - 1][cx + 1], s, e);
        df_two_sum(uh[sl][cy + 1][cx - 1], uh[sl][cy + 1][cx + 1], s2, e2);
        float s3, e3;
        df_two_sum(s, s2, s3, e3);
        ps.C = s3;
        ps.Ce = e3 + (e + e2);
        df_two_sum(uh[sl][cy][cx - 1], uh[sl][cy][cx + 1], ps.X, ps.Xe);
        df_two_sum(uh[sl][cy - 1][cx], uh[sl][cy + 1][cx], ps.Y, ps.Ye);
        ps.U = uh[sl][cy][cx];
        ps.Clo = (ul[sl][cy - 1][cx - 1] + ul[sl][cy - 1][cx + 1]) +
                 (ul[sl][cy + 1][cx - 1] + ul[sl][cy + 1][cx + 1]);
        ps.Xlo = ul[sl][cy][cx - 1] + ul[sl][cy][cx + 1];
        ps.Ylo = ul[sl][cy - 1][cx] + ul[sl][cy + 1][cx];
        ps.Ulo = ul[sl][cy][cx];
    };

    PlaneSums pm, p0, pp;
    float rsq = 0.f;
    fetch(lbeg - 1);
    store(lbeg - 1);
    __syncthreads();
    sums(lbeg - 1, pm);
    fetch(lbeg);
    __syncthreads();
    store(lbeg);
    __syncthreads();
    sums(lbeg, p0);
    fetch(lbeg + 1);
    for (int l = lbeg; l < lend; ++l) {
        __syncthreads();          // slot of plane l + 1 (= that of l - 1) is free
        store(l + 1);
        __syncthreads();
        fetch(l + 2);             // in flight during the arithmetic below
        sums(l + 1, pp);
        if (active) {
            const float2 *cf = coef + (size_t)l * 12;
            float S = 0.f, E = 0.f;
            const PlaneSums *q[3] = {&pm, &p0, &pp};
#pragma unroll
            for (int nu = 0; nu < 3; ++nu) {
                const int ll = l + nu - 1;
                if (ll < 0 || ll >= Nz) continue;
                const PlaneSums &ps = *q[nu];
                acc_term(S, E, cf[nu * 4 + 0], ps.C, ps.Ce, ps.Clo);
                acc_term(S, E, cf[nu * 4 + 1], ps.X, ps.Xe, ps.Xlo);
                acc_term(S, E, cf[nu * 4 + 2], ps.Y, ps.Ye, ps.Ylo);
                acc_term(S, E, cf[nu * 4 + 3], ps.U, 0.f, ps.Ulo);
            }
            const size_t o = (size_t)l * plane + (size_t)j * Nx + i;
            dfloat au;
            df_fast_two_sum(S, E, au.hi, au.lo);
            const dfloat res = df_add_accurate(dfloat{F[o], F[o + n]}, df_neg(au));
            const float rv = res.hi + res.lo;
            r[o] = rv;
            rsq = fmaf(rv, rv, rsq);
        }
        pm = p0;
        p0 = pp;
    }
    if (r2out) block_sum_to((double)rsq, r2out);
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

hs_status hs_launch_rhs(const hs_plan_s *P, const void *f, int f_dtype, int rhs_kind,
                        const DevBoundary &b, void *F, int out_df, cudaStream_t s, double *f2) {
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
    a.has_faces = 0;
    for (int k = 0; k < 6; ++k)
        if (b.face[k]) a.has_faces = 1;
    if (rhs_kind == HS_RHS_NODAL) {
        dim3 tb(RTX, RTY, 1);
        dim3 tg((P->Nx + RTX - 1) / RTX, (P->Ny + RTY - 1) / RTY, (P->Nz + RZ - 1) / RZ);
        if (f_dtype == HS_F64) {
            if (out_df)
                rhs_tiled_df_kernel<double><<<tg, tb, 0, s>>>(a, static_cast<const double *>(f),
                                                              static_cast<float *>(F), f2);
            else
                rhs_tiled_kernel<double, 0><<<tg, tb, 0, s>>>(a, static_cast<const double *>(f), F);
        } else {
            if (out_df)
                rhs_tiled_df_kernel<float><<<tg, tb, 0, s>>>(a, static_cast<const float *>(f),
                                                             static_cast<float *>(F), f2);
            else
                rhs_tiled_kernel<float, 0><<<tg, tb, 0, s>>>(a, static_cast<const float *>(f), F);
        }
        return cudaGetLastError() == cudaSuccess ? HS_OK : HS_ERR_CUDA;
    }
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
                                cudaStream_t s, double *r2) {
    dim3 block(32, 8, 1);
    dim3 grid((P->Nx + 31) / 32, (P->Ny + 7) / 8, P->Nz);
    if (P->residual_simple) {
        residual_df_kernel<<<grid, block, 0, s>>>(P->Nx, P->Ny, P->Nz, P->d_coef_df, F, U, r);
    } else {
        dim3 qb(QTX, QTY, 1);
        dim3 qg((P->Nx + QTX - 1) / QTX, (P->Ny + QTY - 1) / QTY, (P->Nz + QZ - 1) / QZ);
        residual_zmarch_kernel<<<qg, qb, 0, s>>>(P->Nx, P->Ny, P->Nz, P->d_coef_df, F, U, r,
                                                 P->cur_skip, r2);
    }
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
