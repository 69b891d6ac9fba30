// Sum-factorised double-float right-hand side of the mixed path (eqs. scheme4,
// scheme6, cd_rhs with the readings of the 6th-order form documented in
// k_rhs.cu).
//
// The 6th-order operator written with integer weights,
//     F6 = A_l f + W G + Eps_l (f_{l+1} - f_{l-1}),
//     G  = 40 S1 - 3 S2 + 8 E,      W = h^2 / 720,
//     A_l = h^2 (67/120 - h^2 K_l / 20),   Eps_l = h^2 h^3 K_{z,l} / 120,
// (S1: the 6 face neighbours, S2: the 6 second neighbours, E: the 12 edge
// mid-points; 40/720 = 1/18, 3/720 = 1/240, 8/720 = 1/90), is evaluated from
// three in-plane sums per node plane and column,
//     N4 = 4 in-plane face neighbours, D4 = 4 in-plane diagonals,
//     Q4 = 4 in-plane second neighbours,
// as S1(l) = N4(l) + f_{l-1} + f_{l+1}, S2(l) = Q4(l) + f_{l-2} + f_{l+2},
// E(l) = D4(l) + N4(l-1) + N4(l+1): N4 of a plane serves three output planes
// and the column values f_{l-2..l+2} stay in registers while the tile marches
// in z.  4th order: F4 = W (6 f + S1) with W = h^2 / 12; CD adds
// G_l (f_{l+1} - f_{l-1}) with G_l = h^2 h gamma_l / 24.
//
// Arithmetic: values are FP32 pairs (hi, lo).  Sums of hi parts go through
// two_sum (exact), their errors and the lo parts are added in FP32; the
// integer weights 40 and 3 multiply through two_prod (exact), 8 and 6 are
// exact scalings; pair x pair products keep the three leading partial
// products.  The result is rounded to a normalised pair once, at the end.
// Rounding: about 2^-46 of the largest intermediate (the same level as the
// per-term pair arithmetic it replaces, with a third of the instructions).
#pragma once

#include <type_traits>

#include "hs_async.cuh"
#include "hs_tiles.cuh"

namespace hs_tiles {

// unnormalised pair: value s + e, |e| small against |s|
struct LPair {
    float s, e;
};

__device__ __forceinline__ LPair lp_of(float hi, float lo) { return LPair{hi, lo}; }

// x + (hi, lo): the hi parts exactly (two_sum), the rest in FP32
__device__ __forceinline__ void lp_add(LPair &x, float hi, float lo) {
    float s, t;
    df_two_sum(x.s, hi, s, t);
    x.s = s;
    x.e += t + lo;
}
__device__ __forceinline__ void lp_add(LPair &x, LPair y) { lp_add(x, y.s, y.e); }

// k * x for a small integer k held exactly in FP32 (the product's rounding
// error is recovered by an FMA)
__device__ __forceinline__ LPair lp_scale(float k, LPair x) {
    const float p = k * x.s;
    return LPair{p, fmaf(k, x.s, -p) + k * x.e};
}

// (c.hi + c.lo) * x, the three leading partial products
__device__ __forceinline__ LPair lp_mul(float2 c, LPair x) {
    const float p = c.x * x.s;
    float e = fmaf(c.x, x.s, -p);
    e = fmaf(c.x, x.e, e);
    e = fmaf(c.y, x.s, e);
    return LPair{p, e};
}

// x - y
__device__ __forceinline__ LPair lp_sub(LPair x, LPair y) {
    LPair r = x;
    lp_add(r, -y.s, -y.e);
    return r;
}

enum { SF_O2 = 0, SF_O4 = 1, SF_CD = 2, SF_O6 = 3 };

// tile: x, y columns; z planes at most (the depth of a launch, RhsArgs::zt, is
// SFZ or a smaller power of two when the problem is too small to fill the GPU)
constexpr int SFX = 32, SFY = 8, SFZ = 32;

template <int H>
struct SfGeom {
    static constexpr int HX = SFX + 2 * H, HY = SFY + 2 * H;  // halo tile
    static constexpr int NPL = 2 * H + 1;                    // ring of node planes
    static constexpr int NT = SFX * SFY;
    static constexpr int PER = (HX * HY + NT - 1) / NT;      // halo elements per thread
};

// Raw node planes (type T) in flight ahead of the pair ring: SF_RAW - 1.
constexpr int SF_RAW = 4;

// pair ring (NPL planes of pairs, or of FP32 values for FP32 f) + raw ring
// The pair ring holds (hi, lo) pairs for FP64 f and wherever ghost nodes exist
// (halo 2, 6th order: a ghost 2 f_0 - f_1 + h^2 f_nn is not an FP32 number even
// for FP32 f), else FP32 values.
template <int H, typename T>
constexpr bool sf_pair_ring() {
    return sizeof(T) == 8 || H == 2;
}
template <int H, typename T>
constexpr size_t sf_smem_bytes() {
    return (size_t)SfGeom<H>::NPL * SfGeom<H>::HX * SfGeom<H>::HY *
               (sf_pair_ring<H, T>() ? sizeof(float2) : sizeof(float)) +
           (size_t)SF_RAW * SfGeom<H>::HX * SfGeom<H>::HY * sizeof(T);
}

enum { SF_K_SKIP = 0, SF_K_NODE, SF_K_XLO, SF_K_XHI, SF_K_YLO, SF_K_YHI, SF_K_ZERO };

// Conversion of one raw node plane into the pair ring for a tile that touches
// an x or y face or for a ghost plane beyond a z face (kept out of line: it is
// rare, and inlined it would raise the register count of the whole march).
// E: float2 (pairs) or float.  Each thread converts its own elements.
template <typename T, typename E, int H, int PER, int HX>
__device__ __noinline__ void sf_convert_edge(const RhsArgs &a, const T *f, const T *rs, E *dst,
                                             const int *soff, const int *kind, int pl, int i0,
                                             int j0) {
    const bool zghost = pl < 0 || pl > a.Nz + 1;
#pragma unroll
    for (int q = 0; q < PER; ++q) {
        const int kq = kind[q];
        if (kq == SF_K_SKIP) continue;
        const int e = soff[q];
        const int ey = e / HX, ex = e - ey * HX;
        double v;
        if (zghost) {
            v = node_or_ghost<T>(a, f, i0 - H + ex, j0 - H + ey, pl);
        } else if (kq == SF_K_NODE) {
            v = (double)rs[e];
        } else if (kq == SF_K_ZERO) {
            v = 0.0;
        } else {
            // ghost: 2 f_0 - f_1 + h^2 (f_nn)_face, f_0 and f_1 the two nodes inward
            const int step = kq == SF_K_XLO ? 1 : (kq == SF_K_XHI ? -1 : (kq == SF_K_YLO ? HX : -HX));
            const int face = kq - SF_K_XLO;   // 0..3: x-lo, x-hi, y-lo, y-hi
            const T *fnn = static_cast<const T *>(a.b.fnn[face]);
            const size_t fi = face < 2 ? (size_t)pl * (a.Ny + 2) + (j0 - H + ey)
                                       : (size_t)pl * (a.Nx + 2) + (i0 - H + ex);
            // (h^2 formed here: FP64 issues at a small fraction of the FP32 rate,
            // and every thread of a face tile converts a plane at every step)
            v = 2.0 * (double)rs[e + step] - (double)rs[e + 2 * step] +
                (fnn ? (a.hz * a.hz) * (double)__ldg(fnn + fi) : 0.0);
        }
        const dfloat d = df_split_bits(v);
        if constexpr (sizeof(E) == 8) dst[e] = make_float2(d.hi, d.lo);
        else dst[e] = d.hi;
    }
}

// Raw-plane loads of one node plane for a tile that touches an x or y face, or
// of a ghost plane beyond a z face, when the ghost nodes were precomputed
// (RhsArgs::ghost, FP64 f): nodes from f, ghost nodes from the ghost arrays,
// zeros where the stencil never reads (corners).  The raw plane then holds
// every value the march reads, so it takes the plain conversion.
template <typename T, int H, int PER, int HX>
__device__ __noinline__ void sf_issue_ghost(const RhsArgs &a, const T *f, T *dst,
                                            const int *soff, const int *goff, const int *kind,
                                            int pl, int i0, int j0) {
    const size_t sy = (size_t)(a.Nx + 2), sz = sy * (a.Ny + 2);
    const double *gx = a.ghost;
    const double *gy = gx + 2 * (size_t)(a.Nz + 2) * (a.Ny + 2);
    const double *gz = gy + 2 * (size_t)(a.Nz + 2) * (a.Nx + 2);
    const bool zghost = pl < 0 || pl > a.Nz + 1;
#pragma unroll
    for (int q = 0; q < PER; ++q) {
        const int kq = kind[q];
        if (kq == SF_K_SKIP) continue;
        const int e = soff[q];
        const int ey = e / HX, ex = e - ey * HX;
        const void *src = nullptr;
        if (zghost) {
            if (kq == SF_K_NODE) src = gz + (pl < 0 ? 0 : sz) + goff[q];
        } else if (kq == SF_K_NODE) {
            src = f + (size_t)pl * sz + goff[q];
        } else if (kq == SF_K_XLO || kq == SF_K_XHI) {
            src = gx + ((size_t)(kq == SF_K_XHI ? a.Nz + 2 : 0) + pl) * (a.Ny + 2) + (j0 - H + ey);
        } else if (kq == SF_K_YLO || kq == SF_K_YHI) {
            src = gy + ((size_t)(kq == SF_K_YHI ? a.Nz + 2 : 0) + pl) * (a.Nx + 2) + (i0 - H + ex);
        }
        cp_async<sizeof(T)>(dst + e, src ? src : static_cast<const void *>(f), src != nullptr);
    }
}

// One CTA: columns (i0 .. i0+SFX-1) x (j0 .. j0+SFY-1), planes lbeg .. lend.
// KIND: SF_O2 / SF_O4 / SF_CD (halo 1) or SF_O6 (halo 2).  T: type of f (FP64
// f is split into pairs with integer operations; FP32 f has lo = 0 and the
// ring holds hi only).  rw: per-row weights (order 6: A_l, Eps_l; CD: G_l in
// .z/.w); W: the constant pair weight.
//
// Loading: node planes stream through a raw ring of SF_RAW slots filled by
// cp.async, SF_RAW - 1 planes ahead of use; each step converts one raw plane
// into the pair ring (FP64 values split into pairs with integer operations).
// Ghost nodes beyond an x or y face, 2 f_0 - f_1 + h^2 (f_nn)_face, are formed
// during that conversion from the raw plane; the ghost planes beyond a z face
// are formed node by node (node_or_ghost).  When RhsArgs::ghost holds them
// precomputed (6th order, FP64 f; stand-alone solves) they are loaded like
// nodes instead, and every plane takes the plain conversion: face tiles then
// cost about what interior tiles do (the in-tile formation is FP64 work on the
// critical path of every plane step).  f is never written during a launch, so
// the L1-cached copy is safe in the persistent batch kernel too.
template <int KIND, typename T>
__device__ __forceinline__ void rhs_sf_tile(const RhsArgs &a, const T *__restrict__ f,
                                            float *__restrict__ Fo, double *f2out,
                                            const float4 *__restrict__ rw, float2 W,
                                            unsigned char *smem, int bx, int by, int bz) {
    constexpr int H = KIND == SF_O6 ? 2 : 1;
    constexpr bool GHOSTS = H == 2 && sizeof(T) == 8;
    typedef SfGeom<H> G;
    constexpr bool PAIR = sf_pair_ring<H, T>();
    typedef typename std::conditional<PAIR, float2, float>::type E;
    E(*ring)[G::HY][G::HX] = reinterpret_cast<E(*)[G::HY][G::HX]>(smem);

    const int tid = threadIdx.x;
    const int tx = tid & (SFX - 1), ty = tid / SFX;
    const int i0 = 1 + bx * SFX, j0 = 1 + by * SFY;    // node indices of the first column
    const int lbeg = 1 + bz * a.zt;
    const int lend = min(lbeg + a.zt - 1, a.Nz);
    const size_t n = (size_t)a.Nx * a.Ny * a.Nz;
    const size_t sy = (size_t)(a.Nx + 2), sz = sy * (a.Ny + 2);
    // every halo node of the tile is a node of the grid (no ghost in x, y)
    const bool xy_in = i0 - H >= 0 && i0 + SFX - 1 + H <= a.Nx + 1 && j0 - H >= 0 &&
                       j0 + SFY - 1 + H <= a.Ny + 1;

    // per-thread halo elements: in-plane offset and kind, fixed for the whole march
    int goff[G::PER], soff[G::PER], kind[G::PER];
#pragma unroll
    for (int k = 0; k < G::PER; ++k) {
        const int e = tid + k * G::NT;
        const int ey = e / G::HX, ex = e - ey * G::HX;
        const int ii = i0 - H + ex, jj = j0 - H + ey;
        const bool xin = ii >= 0 && ii <= a.Nx + 1, yin = jj >= 0 && jj <= a.Ny + 1;
        goff[k] = jj * (int)sy + ii;
        soff[k] = e < G::HX * G::HY ? e : -1;
        kind[k] = soff[k] < 0                        ? SF_K_SKIP
                  : (xin && yin)                     ? SF_K_NODE
                  : (yin && ii == -1)                ? SF_K_XLO
                  : (yin && ii == a.Nx + 2)          ? SF_K_XHI
                  : (xin && jj == -1)                ? SF_K_YLO
                  : (xin && jj == a.Ny + 2)          ? SF_K_YHI
                                                     : SF_K_ZERO;
    }
    T *raw = reinterpret_cast<T *>(smem + (size_t)G::NPL * G::HX * G::HY * sizeof(E));
    constexpr int HALO = G::HX * G::HY;
    // stream index k: node plane lbeg - H + k; kend: last index
    const int kend = lend - lbeg + 2 * H;
    // precomputed ghost nodes (6th order, FP64 f): every plane takes the plain
    // conversion, face tiles and z-ghost planes load through sf_issue_ghost
    const bool ghosts = GHOSTS && a.ghost != nullptr;
    auto issue = [&](int k) {
        const int pl = lbeg - H + k;
        const bool zin = pl >= 0 && pl <= a.Nz + 1;
        if (k <= kend && (zin || ghosts)) {
            T *dst = raw + (k & (SF_RAW - 1)) * HALO;
            if (ghosts && (!xy_in || !zin)) {
                sf_issue_ghost<T, H, G::PER, G::HX>(a, f, dst, soff, goff, kind, pl, i0, j0);
            } else {
                const T *src = f + (size_t)pl * sz;
#pragma unroll
                for (int q = 0; q < G::PER; ++q) {
                    if (kind[q] == SF_K_SKIP) continue;
                    const bool v = kind[q] == SF_K_NODE;
                    cp_async<sizeof(T)>(dst + soff[q], v ? src + goff[q] : f, v);
                }
            }
        }
        cp_async_commit();
    };
    // raw plane k -> pair ring slot `slot` (every thread its own elements)
    auto convert = [&](int k, int slot) {
        const int pl = lbeg - H + k;
        E *dst = &ring[slot][0][0];
        const T *rs = raw + (k & (SF_RAW - 1)) * HALO;
        if (!ghosts && (!xy_in || pl < 0 || pl > a.Nz + 1)) {
            sf_convert_edge<T, E, H, G::PER, G::HX>(a, f, rs, dst, soff, kind, pl, i0, j0);
            return;
        }
#pragma unroll
        for (int q = 0; q < G::PER; ++q) {
            if (kind[q] == SF_K_SKIP) continue;
            const int e = soff[q];
            if constexpr (sizeof(T) == 8) {
                const dfloat d = df_split_bits(rs[e]);
                dst[e] = make_float2(d.hi, d.lo);
            } else if constexpr (PAIR) {
                dst[e] = make_float2((float)rs[e], 0.f);
            } else {
                dst[e] = (float)rs[e];
            }
        }
    };
    constexpr int D = SF_RAW - 1;
    auto take = [&](int k, int slot) {
        cp_async_wait<D - 1>();
        __syncthreads();
        convert(k, slot);
        issue(k + D);
    };

    // Ring slots are counted from the tile's first plane: node plane p sits in
    // slot (p - lbeg + H) mod NPL, and the march below is unrolled NPL-fold so
    // every slot index is a compile-time constant.
    auto get = [&](int slot, int dy, int dx) -> LPair {
        const E v = ring[slot][ty + H + dy][tx + H + dx];
        if constexpr (PAIR) return LPair{v.x, v.y};
        else return LPair{v, 0.f};
    };
    // sum of the 4 in-plane points at distance d along the axes or the diagonals
    auto ring4 = [&](int slot, int d, bool diag) -> LPair {
        LPair s = diag ? get(slot, -d, -d) : get(slot, 0, -d);
        if (diag) {
            lp_add(s, get(slot, -d, d));
            lp_add(s, get(slot, d, -d));
            lp_add(s, get(slot, d, d));
        } else {
            lp_add(s, get(slot, 0, d));
            lp_add(s, get(slot, -d, 0));
            lp_add(s, get(slot, d, 0));
        }
        return s;
    };

    // prologue: node planes lbeg - H .. lbeg + H - 1 into pair slots 0 .. 2H - 1
#pragma unroll
    for (int k = 0; k < D; ++k) issue(k);
#pragma unroll
    for (int k = 0; k < 2 * H; ++k) take(k, k);
    __syncthreads();

    const int i = i0 + tx, j = j0 + ty;
    const bool active = i <= a.Nx && j <= a.Ny;
    // column window c[k] = f(l - H + k) and the in-plane face-neighbour sums
    LPair c[2 * H + 1];
    LPair n4m = LPair{0.f, 0.f}, n40 = LPair{0.f, 0.f};
#pragma unroll
    for (int k = 0; k < 2 * H; ++k) c[k] = get(k, 0, 0);
    if constexpr (KIND == SF_O6) {
        n4m = ring4(H - 1, 1, false);
        n40 = ring4(H, 1, false);
    }
    float fsq = 0.f;
    for (int lb = lbeg; lb <= lend; lb += G::NPL) {
#pragma unroll
        for (int u = 0; u < G::NPL; ++u) {
            const int l = lb + u;
            if (l > lend) break;
            // slot of node plane l + d: (u + H + d) mod NPL
            constexpr int NP = G::NPL;
            // plane l + H (stream index l - lbeg + 2H) into the slot of plane l - H - 1
            take(l - lbeg + 2 * H, (u + 2 * H) % NP);
            __syncthreads();
            c[2 * H] = get((u + 2 * H) % NP, 0, 0);
            LPair val;
            const LPair fc = c[H];
            if constexpr (KIND == SF_O2) {
                val = lp_mul(W, fc);
            } else if constexpr (KIND == SF_O4 || KIND == SF_CD) {
                LPair s1 = ring4((u + H) % NP, 1, false);
                lp_add(s1, c[0]);
                lp_add(s1, c[2]);
                LPair g = lp_scale(6.f, fc);
                lp_add(g, s1);
                val = lp_mul(W, g);
                if constexpr (KIND == SF_CD) {
                    const float4 w = rw[l];
                    lp_add(val, lp_mul(make_float2(w.z, w.w), lp_sub(c[2], c[0])));
                }
            } else {
                const LPair n4p = ring4((u + H + 1) % NP, 1, false);
                LPair s1 = n40;
                lp_add(s1, c[1]);
                lp_add(s1, c[3]);
                LPair s2 = ring4((u + H) % NP, 2, false);
                lp_add(s2, c[0]);
                lp_add(s2, c[4]);
                LPair e = ring4((u + H) % NP, 1, true);
                lp_add(e, n4m);
                lp_add(e, n4p);
                // G = 40 S1 - 3 S2 + 8 E
                LPair g = lp_scale(40.f, s1);
                lp_add(g, lp_scale(-3.f, s2));
                lp_add(g, LPair{8.f * e.s, 8.f * e.e});
                const float4 w = rw[l];
                val = lp_mul(make_float2(w.x, w.y), fc);
                lp_add(val, lp_mul(W, g));
                lp_add(val, lp_mul(make_float2(w.z, w.w), lp_sub(c[3], c[1])));
                n4m = n40;
                n40 = n4p;
            }
#pragma unroll
            for (int k = 0; k < 2 * H; ++k) c[k] = c[k + 1];
            if (active) {
                dfloat out;
                df_two_sum(val.s, val.e, out.hi, out.lo);
                const bool near =
                    i == 1 || i == a.Nx || j == 1 || j == a.Ny || l == 1 || l == a.Nz;
                if (a.has_faces && near)
                    out = df_add_accurate(out, df_neg(df_split_bits(lift_terms<T>(a, i, j, l))));
                const size_t o = ((size_t)(l - 1) * a.Ny + (j - 1)) * a.Nx + (i - 1);
                Fo[o] = out.hi;
                Fo[o + n] = out.lo;
                fsq = fmaf(out.hi, out.hi, fsq);
            }
        }
    }
    cp_async_wait<0>();
    if (f2out) block_sum_to((double)fsq, f2out);
}

}  // namespace hs_tiles
