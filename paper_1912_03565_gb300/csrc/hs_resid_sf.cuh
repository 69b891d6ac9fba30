// Lean double-float residual r = F - A U of the refinement (mixed path; the
// 27-point operator of eq. (stencil27) with per-row coefficients).
//
// A CTA owns a RSX x RSY patch of columns and marches over RSZ planes in z.
// For every plane, each thread forms the in-plane sums of its column once --
// corners C, x-neighbours X, y-neighbours Y (or their sum X + Y when the plane
// coefficients satisfy b_nu = c_nu on every row, as at 6th order and whenever
// h_x = h_y) -- and keeps the last three planes' sums in registers, so output
// row l costs 12 (or 9) products
//     A U_l = sum_nu a_nu C_nu + b_nu X_nu + c_nu Y_nu + d_nu U_nu.
// The hi parts of the sums and products are accumulated exactly (two_sum,
// two_prod), their errors and the lo parts in FP32, then F - A U is formed
// with an accurate pair subtraction (rounding about 2^-47 of the largest
// term).  U is held in shared memory as interleaved (hi, lo) pairs.
//
// Two loaders feed the same arithmetic: residual_sf_tile (register prefetch of
// one plane, loads through L2 when COH: the persistent batch kernel reads data
// written earlier in its own launch) and residual_sf_tile_async (stand-alone
// kernel: a ring of RQ_SLOTS planes filled by cp.async, RQ_SLOTS - 1 planes of U
// and the matching F pairs in flight, no registers held for them).
#pragma once

#include "hs_async.cuh"
#include "hs_tiles.cuh"

namespace hs_tiles {

// tile: x, y columns; z planes at most (a launch may use fewer: zt)
constexpr int RSX = 32, RSY = 8, RSZ = 32;
constexpr int RSHX = RSX + 2, RSHY = RSY + 2;

struct PSum {
    float C, X, Y, U;   // hi sums (X: X + Y when merged) and the centre hi
    float Cl, Xl, Yl, Ul;   // the rest: two_sum errors plus the sums of the lo parts
};

// In-plane sums of the column at tile position (tx, ty) of one plane slot.
template <bool XY>
__device__ __forceinline__ void resid_plane_sums(const float2 *sl, int tx, int ty, PSum &ps) {
    const int c = (ty + 1) * RSHX + tx + 1;
    const float2 a = sl[c - RSHX - 1], b = sl[c - RSHX + 1];
    const float2 g = sl[c + RSHX - 1], d = sl[c + RSHX + 1];
    const float2 xm = sl[c - 1], xp = sl[c + 1], ym = sl[c - RSHX], yp = sl[c + RSHX];
    const float2 u = sl[c];
    float s, e, s2, e2, s3, e3;
    df_two_sum(a.x, b.x, s, e);
    df_two_sum(g.x, d.x, s2, e2);
    df_two_sum(s, s2, s3, e3);
    ps.C = s3;
    ps.Cl = (e3 + (e + e2)) + ((a.y + b.y) + (g.y + d.y));
    if (XY) {
        df_two_sum(xm.x, xp.x, s, e);
        df_two_sum(ym.x, yp.x, s2, e2);
        df_two_sum(s, s2, s3, e3);
        ps.X = s3;
        ps.Xl = (e3 + (e + e2)) + ((xm.y + xp.y) + (ym.y + yp.y));
    } else {
        float xe, ye;
        df_two_sum(xm.x, xp.x, ps.X, xe);
        df_two_sum(ym.x, yp.x, ps.Y, ye);
        ps.Xl = xe + (xm.y + xp.y);
        ps.Yl = ye + (ym.y + yp.y);
    }
    ps.U = u.x;
    ps.Ul = u.y;
}

// The same sums for an iterate whose lo parts are all zero (the first residual
// after the FP32 solve), from a plane of hi values: the sums of the lo parts
// vanish, Ul = 0.
template <bool XY>
__device__ __forceinline__ void resid_plane_sums_hi(const float *sl, int tx, int ty, PSum &ps) {
    const int c = (ty + 1) * RSHX + tx + 1;
    const float a = sl[c - RSHX - 1], b = sl[c - RSHX + 1];
    const float g = sl[c + RSHX - 1], d = sl[c + RSHX + 1];
    const float xm = sl[c - 1], xp = sl[c + 1], ym = sl[c - RSHX], yp = sl[c + RSHX];
    float s, e, s2, e2, s3, e3;
    df_two_sum(a, b, s, e);
    df_two_sum(g, d, s2, e2);
    df_two_sum(s, s2, s3, e3);
    ps.C = s3;
    ps.Cl = e3 + (e + e2);
    if (XY) {
        df_two_sum(xm, xp, s, e);
        df_two_sum(ym, yp, s2, e2);
        df_two_sum(s, s2, s3, e3);
        ps.X = s3;
        ps.Xl = e3 + (e + e2);
    } else {
        df_two_sum(xm, xp, ps.X, ps.Xl);
        df_two_sum(ym, yp, ps.Y, ps.Yl);
    }
    ps.U = sl[c];
    ps.Ul = 0.f;
}

// r_l = F_l - A U_l at one point from the plane sums of rows l - 1, l, l + 1.
// The row's coefficient pairs are read two at a time (16-byte loads).  r only
// feeds the FP32 correction solve: it is formed as the exact difference of the
// hi parts (two_sum) plus the low-order terms, rounded once to FP32 -- the same
// error bound (about 2^-47 |F| + 2^-24 |r|) as a full pair subtraction.
template <bool XY, bool ULO = true>
__device__ __forceinline__ float resid_point(const float2 *__restrict__ cf, int l, int Nz,
                                             const PSum &pm, const PSum &p0, const PSum &pp,
                                             float2 Fl) {
    float S = 0.f, E = 0.f;
    const PSum *q[3] = {&pm, &p0, &pp};
    const float4 *cf4 = reinterpret_cast<const float4 *>(cf);
#pragma unroll
    for (int nu = 0; nu < 3; ++nu) {
        const int ll = l + nu - 1;
        if (ll < 0 || ll >= Nz) continue;
        const PSum &ps = *q[nu];
        const float4 ab = cf4[2 * nu], cd = cf4[2 * nu + 1];
        acc_term(S, E, make_float2(ab.x, ab.y), ps.C, ps.Cl);
        acc_term(S, E, make_float2(ab.z, ab.w), ps.X, ps.Xl);
        if (!XY) acc_term(S, E, make_float2(cd.x, cd.y), ps.Y, ps.Yl);
        if (ULO) acc_term(S, E, make_float2(cd.z, cd.w), ps.U, ps.Ul);
        else acc_term_hi(S, E, make_float2(cd.z, cd.w), ps.U);
    }
    float d, de;
    df_two_sum(Fl.x, -S, d, de);   // F_hi - S exactly
    return d + (de + (Fl.y - E));
}

// Register-prefetch loader.  COH: F and U were written earlier in the same
// launch (persistent batch kernel): read them through L2.
template <bool XY, bool COH>
__device__ __forceinline__ void residual_sf_tile(int Nx, int Ny, int Nz,
                                                 const float2 *__restrict__ coef,
                                                 const float *__restrict__ F,
                                                 const float *__restrict__ U,
                                                 float *__restrict__ r, double *r2out,
                                                 float2 *ring, int bx, int by, int bz,
                                                 int zt = RSZ) {
    // ring: 2 plane slots of RSHY x RSHX pairs (the plane being summed, the next)
    constexpr int NT = RSX * RSY;
    constexpr int PER = (RSHX * RSHY + NT - 1) / NT;
    const int tid = threadIdx.x;
    const int tx = tid & (RSX - 1), ty = tid / RSX;
    const int i0 = bx * RSX, j0 = by * RSY;   // 0-based interior indices
    const int lbeg = bz * zt;
    const int lend = min(lbeg + zt, Nz);     // exclusive
    const size_t plane = (size_t)Nx * Ny;
    const size_t n = plane * Nz;
    const int i = i0 + tx, j = j0 + ty;
    const bool active = i < Nx && j < Ny;
    const bool xy_in = i0 >= 1 && i0 + RSX < Nx && j0 >= 1 && j0 + RSY < Ny;

    int goff[PER], soff[PER];
#pragma unroll
    for (int k = 0; k < PER; ++k) {
        const int e = tid + k * NT;
        const int ey = e / RSHX, ex = e - ey * RSHX;
        const int ii = i0 - 1 + ex, jj = j0 - 1 + ey;
        const bool ok = e < RSHX * RSHY && ii >= 0 && ii < Nx && jj >= 0 && jj < Ny;
        goff[k] = ok ? jj * Nx + ii : -1;
        soff[k] = e < RSHX * RSHY ? e : -1;
    }
    float2 reg[PER];
    auto fetch = [&](int l) {
        const bool zin = l >= 0 && l < Nz;
        const float *ph = U + (size_t)(zin ? l : 0) * plane;
#pragma unroll
        for (int k = 0; k < PER; ++k) {
            if (soff[k] < 0) continue;
            if (xy_in && zin) {
                reg[k] = make_float2(ldc<COH>(ph + goff[k]), ldc<COH>(ph + n + goff[k]));
            } else {
                reg[k] = make_float2(0.f, 0.f);
                if (zin && goff[k] >= 0)
                    reg[k] = make_float2(ldc<COH>(ph + goff[k]), ldc<COH>(ph + n + goff[k]));
            }
        }
    };
    auto store = [&](int l) {
        float2 *slot = ring + ((l + 2) & 1) * (RSHX * RSHY);
#pragma unroll
        for (int k = 0; k < PER; ++k)
            if (soff[k] >= 0) slot[soff[k]] = reg[k];
    };
    auto sums = [&](int l, PSum &ps) {
        resid_plane_sums<XY>(ring + ((l + 2) & 1) * (RSHX * RSHY), tx, ty, ps);
    };

    PSum pm, p0, pp;
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
            const size_t o = (size_t)l * plane + (size_t)j * Nx + i;
            const float rv = resid_point<XY>(coef + (size_t)l * 12, l, Nz, pm, p0, pp,
                                             make_float2(ldc<COH>(F + o), ldc<COH>(F + o + n)));
            r[o] = rv;
            rsq = fmaf(rv, rv, rsq);
        }
        pm = p0;
        p0 = pp;
    }
    if (r2out) block_sum_to((double)rsq, r2out);
}

// The same tile fed by cp.async: RQ_SLOTS ring slots, each holding one U plane
// with its halo (RSHX x RSHY pairs) and the F pairs of the output plane below
// it.  Stream index k carries U plane lbeg - 1 + k and F of plane lbeg - 2 + k;
// step k waits for its slot, takes the plane sums, and refills the slot read at
// step k - 1 with stream index k + RQ_SLOTS - 1.
constexpr int RQ_SLOTS = 4;
constexpr size_t resid_async_smem() {
    return (size_t)RQ_SLOTS * (RSHX * RSHY + RSX * RSY) * sizeof(float2);
}

template <bool XY, bool ULO = true>
__device__ __forceinline__ void residual_sf_tile_async(int Nx, int Ny, int Nz,
                                                       const float2 *__restrict__ coef,
                                                       const float *__restrict__ F,
                                                       const float *__restrict__ U,
                                                       float *__restrict__ r, double *r2out,
                                                       float2 *smem, int bx, int by, int bz,
                                                       int zt) {
    constexpr int NT = RSX * RSY;
    constexpr int PER = (RSHX * RSHY + NT - 1) / NT;
    constexpr int HALO = RSHX * RSHY;
    constexpr int D = RQ_SLOTS - 1;          // stream indices in flight ahead
    float2 *uring = smem;                    // [RQ_SLOTS][HALO]
    float2 *fring = smem + RQ_SLOTS * HALO;  // [RQ_SLOTS][NT]
    // !ULO: the lo plane of U is zero and is not read; the U slots hold hi values
    float *uring_hi = reinterpret_cast<float *>(smem);
    const int tid = threadIdx.x;
    const int tx = tid & (RSX - 1), ty = tid / RSX;
    const int i0 = bx * RSX, j0 = by * RSY;
    const int lbeg = bz * zt;
    const int lend = min(lbeg + zt, Nz);    // exclusive
    const size_t plane = (size_t)Nx * Ny;
    const size_t n = plane * Nz;
    const int i = i0 + tx, j = j0 + ty;
    const bool active = i < Nx && j < Ny;
    const size_t col = (size_t)j * Nx + i;

    int goff[PER], soff[PER];
#pragma unroll
    for (int k = 0; k < PER; ++k) {
        const int e = tid + k * NT;
        const int ey = e / RSHX, ex = e - ey * RSHX;
        const int ii = i0 - 1 + ex, jj = j0 - 1 + ey;
        const bool ok = e < HALO && ii >= 0 && ii < Nx && jj >= 0 && jj < Ny;
        goff[k] = ok ? jj * Nx + ii : -1;
        soff[k] = e < HALO ? e : -1;
    }
    auto issue = [&](int k) {
        const int p = lbeg - 1 + k;          // U plane
        const int slot = k & (RQ_SLOTS - 1);
        if (p <= lend) {
            float2 *us = uring + slot * HALO;
            float *uh = uring_hi + slot * HALO;
            const bool zin = p >= 0 && p < Nz;
#pragma unroll
            for (int q = 0; q < PER; ++q) {
                if (soff[q] < 0) continue;
                const bool v = zin && goff[q] >= 0;
                const float *src = v ? U + (size_t)p * plane + goff[q] : U;
                if (ULO) {
                    cp_async<4>(&us[soff[q]].x, src, v);
                    cp_async<4>(&us[soff[q]].y, v ? src + n : U, v);
                } else {
                    cp_async<4>(&uh[soff[q]], src, v);
                }
            }
        }
        const int lf = p - 1;                // output plane whose F rides with U plane p
        if (active && lf >= lbeg && lf < lend) {
            const float *src = F + (size_t)lf * plane + col;
            cp_async<4>(&fring[slot * NT + tid].x, src, true);
            cp_async<4>(&fring[slot * NT + tid].y, src + n, true);
        }
        cp_async_commit();
    };
    // wait for stream index k and take the plane sums of its U plane
    auto take = [&](int k, PSum &ps) {
        cp_async_wait<D - 1>();
        __syncthreads();
        const int slot = k & (RQ_SLOTS - 1);
        if (ULO) resid_plane_sums<XY>(uring + slot * HALO, tx, ty, ps);
        else resid_plane_sums_hi<XY>(uring_hi + slot * HALO, tx, ty, ps);
    };

#pragma unroll
    for (int k = 0; k < D; ++k) issue(k);
    PSum pm, p0, pp;
    take(0, pm);
    issue(D);
    take(1, p0);
    issue(D + 1);
    float rsq = 0.f;
    for (int l = lbeg; l < lend; ++l) {
        const int k = l - lbeg + 2;
        take(k, pp);
        issue(k + D);
        if (active) {
            const float rv = resid_point<XY, ULO>(coef + (size_t)l * 12, l, Nz, pm, p0, pp,
                                                  fring[(k & (RQ_SLOTS - 1)) * NT + tid]);
            r[(size_t)l * plane + col] = rv;
            rsq = fmaf(rv, rv, rsq);
        }
        pm = p0;
        p0 = pp;
    }
    cp_async_wait<0>();
    if (r2out) block_sum_to((double)rsq, r2out);
}

}  // namespace hs_tiles
