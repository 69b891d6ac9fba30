// Device side of the batched persistent solve (Section 3.6 per problem) (shared by the kernel variants,
// one translation unit each, and the host code in k_batch.cu).
//
// Many independent problems (uneven sizes, their own k(z), 1..4 right-hand
// sides each) are solved by the mixed path in ONE kernel launch: a grid of
// persistent CTAs (as many as can be resident) takes work items from a queue
// (an atomic counter over an item list).  An item is one tile of one stage of
// one (problem, right-hand side): the right-hand side, a transform pass, the
// z-solves, the residual, ... -- the same tile code as the stand-alone
// kernels (hs_tiles.cuh), reading data produced earlier in the launch through
// L2 only.  Items are listed stage by stage, so every item depends only on
// items earlier in the list; a CTA waits (bounded) until all tiles of the
// previous stage of its own (problem, RHS) are done, counted per stage with
// atomics.  Since CTAs take items in list order and all CTAs are resident,
// the items a CTA waits for are already running or claimed by a CTA that runs
// them next: no deadlock.  A wait that exceeds its limit sets an error flag
// that the host reads (HS_ERR_TIMEOUT); later waits then give up at once, so
// the launch always ends.
#pragma once

#include "hs_dst_fused.cuh"
#include "hs_resid_sf.cuh"
#include "hs_rhs_sf.cuh"
#include "hs_tiles.cuh"

namespace hs_batch {

using namespace hs_tiles;

enum StageType : int {
    ST_RHS = 0,
    ST_DSTX_F = 1,       // forward x: F_hi (pass 0) or r -> w
    ST_DSTY = 2,         // forward or inverse y, in place, with a scale
    ST_THOMAS = 3,
    ST_IDSTX_SET = 4,    // inverse x into U (double-float), first pass
    ST_IDSTX_ADD = 5,    // inverse x, U += correction
    ST_IDSTX_FINAL = 6,  // inverse x, u = U + correction (FP64)
    ST_IDSTX_W64 = 7,    // inverse x straight into u (no refinement)
    ST_RESIDUAL = 8
};

constexpr int BMAX_STAGES = 6 + 6 * HS_INFO_MAX_ITERS;

struct BatchWork {
    int Nx, Ny, Nz, Mx, My;
    int thomas32;
    const float2 *coef_df;
    const float *fac32;
    const double *fac64;
    double *scr64;
    const float2 *rx, *hx, *ry, *hy;   // FP32 transform tables of x and y
    RhsArgs rhs;
    const void *f;
    double *u;
    float *F, *U, *w;
    float sx, sy;
    int gx, gy, gz;                    // RHS / residual tile grid
    int dxg, dyg;                      // x-transform groups, y-transform groups per plane
    int lx;                            // x lines per x-transform tile
    const double *coef64;              // FP64 stencil rows (FP64 residual)
    double *norms;                     // [0] ||F||^2, [m] ||r_m||^2 (when norms_on)
    const float4 *rw;                  // per-row weights of the sum-factorised right-hand side
    float2 rhsW;                       // its constant pair weight
    int resid_xy;                      // b_nu = c_nu on every row (merged residual sums)
    int need[BMAX_STAGES];
};

struct StageList {
    int n;
    int type[BMAX_STAGES];
};

struct BatchArgs {
    const BatchWork *works;
    const int2 *items;  // x: work index + 65536 * stage, y: tile
    int nitems;
    int *next;
    int *done;          // [nworks][BMAX_STAGES]
    int *err;
    long long spin_limit;
    int f_is_f64;
    double tol2;        // > 0: a (problem, RHS) stops refining once ||r||^2 <= tol2 ||F||^2
    int norms_on;       // accumulate the squared norms (tolerance or automatic residual)
    int resid_mode;     // HS_RESID_DF / HS_RESID_F64 / HS_RESID_AUTO
    StageList stages;
    int sweep_of[BMAX_STAGES];   // refinement sweep a stage belongs to (0: first solve)
};

namespace {

__device__ __forceinline__ int ld_volatile(const int *p) {
    return *reinterpret_cast<const volatile int *>(p);
}

template <int AXIS, int MODE, int M, int... Rs>
__device__ __forceinline__ void dst_tile_m(const BatchWork &W, const float *in, void *out,
                                           float scale, unsigned char *smem, int tile) {
    constexpr int S = Lines<float, M, AXIS>::value;
    const float2 *roots = AXIS == HS_AXIS_X ? W.rx : W.ry;
    const float2 *half = AXIS == HS_AXIS_X ? W.hx : W.hy;
    const int bx = AXIS == HS_AXIS_X ? tile : tile % W.dyg;
    const int by = AXIS == HS_AXIS_X ? 0 : tile / W.dyg;
    double *aux =
        (MODE == HS_MODE_DF_SET || MODE == HS_MODE_DF_ADD || MODE == HS_MODE_DF_FINAL) ? W.u
                                                                                      : nullptr;
    dst_fast_tile<float, float, float, AXIS, MODE, M, S, true, Rs...>(
        in, static_cast<float *>(out), aux, roots, half, W.Nx, W.Ny, W.Nz, scale, smem, bx, by);
}

// The fused tiles (hs_dst_fused.cuh): radices R1 (first), RL (last), Rmid.
template <int AXIS, int MODE, int M, int R1, int RL, int... Rmid>
__device__ __forceinline__ void dst_fused_m(const BatchWork &W, const float *in, void *out,
                                            float scale, unsigned char *smem, int tile) {
    constexpr int S = Lines<float, M, AXIS>::value;
    const float2 *roots = AXIS == HS_AXIS_X ? W.rx : W.ry;
    const float2 *half = AXIS == HS_AXIS_X ? W.hx : W.hy;
    const int bx = AXIS == HS_AXIS_X ? tile : tile % W.dyg;
    const int by = AXIS == HS_AXIS_X ? 0 : tile / W.dyg;
    double *aux =
        (MODE == HS_MODE_DF_SET || MODE == HS_MODE_DF_ADD || MODE == HS_MODE_DF_FINAL) ? W.u
                                                                                      : nullptr;
    dst_fused_tile<float, float, AXIS, MODE, M, S, true, R1, RL, Rmid...>(
        in, static_cast<float *>(out), aux, roots, half, W.Nx, W.Ny, W.Nz, scale, smem, bx, by);
}

template <int M, int... Rs>
__device__ __forceinline__ void dst_w64_m(const BatchWork &W, const float *in, float scale,
                                          unsigned char *smem, int tile) {
    constexpr int S = Lines<float, M, HS_AXIS_X>::value;
    dst_fast_tile<float, float, double, HS_AXIS_X, HS_MODE_WRITE, M, S, true, Rs...>(
        in, W.u, nullptr, W.rx, W.hx, W.Nx, W.Ny, W.Nz, scale, smem, tile, 0);
}

template <int M, int R1, int RL, int... Rmid>
__device__ __forceinline__ void dst_w64_fused_m(const BatchWork &W, const float *in, float scale,
                                                unsigned char *smem, int tile) {
    constexpr int S = Lines<float, M, HS_AXIS_X>::value;
    dst_fused_tile<float, double, HS_AXIS_X, HS_MODE_WRITE, M, S, true, R1, RL, Rmid...>(
        in, W.u, nullptr, W.rx, W.hx, W.Nx, W.Ny, W.Nz, scale, smem, tile, 0);
}

// Dispatch a transform tile on the line length (staged or fused tiles).
template <bool FUSED, int AXIS, int MODE>
__device__ void dst_tile(const BatchWork &W, const float *in, void *out, float scale,
                         unsigned char *smem, int tile) {
    const int M = AXIS == HS_AXIS_X ? W.Mx : W.My;
    if constexpr (FUSED) {
        switch (M) {
            case 32: dst_fused_m<AXIS, MODE, 32, 8, 4>(W, in, out, scale, smem, tile); break;
            case 64: dst_fused_m<AXIS, MODE, 64, 16, 4>(W, in, out, scale, smem, tile); break;
            case 96: dst_fused_m<AXIS, MODE, 96, 16, 6>(W, in, out, scale, smem, tile); break;
            case 128: dst_fused_m<AXIS, MODE, 128, 16, 8>(W, in, out, scale, smem, tile); break;
            case 192: dst_fused_m<AXIS, MODE, 192, 16, 12>(W, in, out, scale, smem, tile); break;
            case 256: dst_fused_m<AXIS, MODE, 256, 16, 16>(W, in, out, scale, smem, tile); break;
            case 384: dst_fused_m<AXIS, MODE, 384, 16, 12, 2>(W, in, out, scale, smem, tile); break;
            default: break;
        }
    } else {
        switch (M) {
            case 32: dst_tile_m<AXIS, MODE, 32, 8, 4>(W, in, out, scale, smem, tile); break;
            case 64: dst_tile_m<AXIS, MODE, 64, 16, 4>(W, in, out, scale, smem, tile); break;
            case 96: dst_tile_m<AXIS, MODE, 96, 16, 6>(W, in, out, scale, smem, tile); break;
            case 128: dst_tile_m<AXIS, MODE, 128, 16, 8>(W, in, out, scale, smem, tile); break;
            case 192: dst_tile_m<AXIS, MODE, 192, 16, 12>(W, in, out, scale, smem, tile); break;
            case 256: dst_tile_m<AXIS, MODE, 256, 16, 16>(W, in, out, scale, smem, tile); break;
            case 384: dst_tile_m<AXIS, MODE, 384, 16, 8, 3>(W, in, out, scale, smem, tile); break;
            default: break;
        }
    }
}

template <bool FUSED>
__device__ void dst_w64_tile(const BatchWork &W, const float *in, float scale,
                             unsigned char *smem, int tile) {
    if constexpr (FUSED) {
        switch (W.Mx) {
            case 32: dst_w64_fused_m<32, 8, 4>(W, in, scale, smem, tile); break;
            case 64: dst_w64_fused_m<64, 16, 4>(W, in, scale, smem, tile); break;
            case 96: dst_w64_fused_m<96, 16, 6>(W, in, scale, smem, tile); break;
            case 128: dst_w64_fused_m<128, 16, 8>(W, in, scale, smem, tile); break;
            case 192: dst_w64_fused_m<192, 16, 12>(W, in, scale, smem, tile); break;
            case 256: dst_w64_fused_m<256, 16, 16>(W, in, scale, smem, tile); break;
            case 384: dst_w64_fused_m<384, 16, 12, 2>(W, in, scale, smem, tile); break;
            default: break;
        }
    } else {
        switch (W.Mx) {
            case 32: dst_w64_m<32, 8, 4>(W, in, scale, smem, tile); break;
            case 64: dst_w64_m<64, 16, 4>(W, in, scale, smem, tile); break;
            case 96: dst_w64_m<96, 16, 6>(W, in, scale, smem, tile); break;
            case 128: dst_w64_m<128, 16, 8>(W, in, scale, smem, tile); break;
            case 192: dst_w64_m<192, 16, 12>(W, in, scale, smem, tile); break;
            case 256: dst_w64_m<256, 16, 16>(W, in, scale, smem, tile); break;
            case 384: dst_w64_m<384, 16, 8, 3>(W, in, scale, smem, tile); break;
            default: break;
        }
    }
}

// Tolerance mode: has this (problem, RHS) converged at or before sweep m?  The
// residual of sweep j (j >= 1) is complete before any later stage runs, so every
// tile of a stage takes the same decision.
__device__ __forceinline__ bool converged(const BatchArgs &A, const BatchWork &W, int m) {
    if (A.tol2 <= 0.0 || m < 1) return false;
    const double f2 = __ldcg(W.norms);
    for (int j = 1; j <= m; ++j)
        if (__ldcg(W.norms + j) <= A.tol2 * f2) return true;
    return false;
}

template <bool FUSED>
__device__ void run_tile(const BatchArgs &A, const BatchWork &W, int stage, int type, int tile,
                         unsigned char *smem) {
    const size_t plane = (size_t)W.Nx * W.Ny;
    if (A.tol2 > 0.0) {
        const int m = A.sweep_of[stage];
        // a residual runs unless an earlier sweep converged; the rest of a sweep
        // runs unless its own residual says converged
        const bool skip = type == ST_RESIDUAL ? converged(A, W, m - 1) : converged(A, W, m);
        if (skip) {
            if (type == ST_IDSTX_FINAL) {
                // the converged iterate is the answer: u = U_hi + U_lo on this tile
                const size_t n = plane * W.Nz;
                const size_t r0 = (size_t)tile * W.lx * W.Nx;
                const size_t r1 = min(n, r0 + (size_t)W.lx * W.Nx);
                for (size_t k = r0 + threadIdx.x; k < r1; k += blockDim.x)
                    W.u[k] = (double)__ldcg(W.U + k) + (double)__ldcg(W.U + n + k);
            }
            return;
        }
    }
    switch (type) {
        case ST_RHS: {
            const int bx = tile % W.gx, by = (tile / W.gx) % W.gy, bz = tile / (W.gx * W.gy);
            double *f2 = A.norms_on ? W.norms : nullptr;
            // the stand-alone solve's tile (same rounding, so batch and stand-alone
            // results agree to the last bit of the transforms)
            const int kind = W.rhs.equation == HS_CONVDIFF ? SF_CD
                             : (W.rhs.order == 6 ? SF_O6 : (W.rhs.order == 4 ? SF_O4 : SF_O2));
            if (A.f_is_f64) {
                const double *f = static_cast<const double *>(W.f);
                switch (kind) {
                    case SF_O6: rhs_sf_tile<SF_O6, double>(W.rhs, f, W.F, f2, W.rw, W.rhsW, smem, bx, by, bz); break;
                    case SF_O4: rhs_sf_tile<SF_O4, double>(W.rhs, f, W.F, f2, W.rw, W.rhsW, smem, bx, by, bz); break;
                    case SF_CD: rhs_sf_tile<SF_CD, double>(W.rhs, f, W.F, f2, W.rw, W.rhsW, smem, bx, by, bz); break;
                    default: rhs_sf_tile<SF_O2, double>(W.rhs, f, W.F, f2, W.rw, W.rhsW, smem, bx, by, bz); break;
                }
            } else {
                const float *f = static_cast<const float *>(W.f);
                switch (kind) {
                    case SF_O6: rhs_sf_tile<SF_O6, float>(W.rhs, f, W.F, f2, W.rw, W.rhsW, smem, bx, by, bz); break;
                    case SF_O4: rhs_sf_tile<SF_O4, float>(W.rhs, f, W.F, f2, W.rw, W.rhsW, smem, bx, by, bz); break;
                    case SF_CD: rhs_sf_tile<SF_CD, float>(W.rhs, f, W.F, f2, W.rw, W.rhsW, smem, bx, by, bz); break;
                    default: rhs_sf_tile<SF_O2, float>(W.rhs, f, W.F, f2, W.rw, W.rhsW, smem, bx, by, bz); break;
                }
            }
            break;
        }
        case ST_RESIDUAL: {
            const int bx = tile % W.gx, by = (tile / W.gx) % W.gy, bz = tile / (W.gx * W.gy);
            const int m = A.sweep_of[stage];
            double *r2 = A.norms_on ? W.norms + m : nullptr;
            const bool f64 = A.resid_mode == HS_RESID_F64 ||
                             (A.resid_mode == HS_RESID_AUTO &&
                              residual_use_f64(W.norms, m));
            // tiles are RSZ = 2 QZ planes deep: the FP64 tile runs on both halves
            if (f64) {
                residual64_tile<true>(W.Nx, W.Ny, W.Nz, W.coef64, W.F, W.U, W.w, r2, smem, bx, by,
                                      2 * bz);
                __syncthreads();
                residual64_tile<true>(W.Nx, W.Ny, W.Nz, W.coef64, W.F, W.U, W.w, r2, smem, bx, by,
                                      2 * bz + 1);
            } else if (W.resid_xy) {
                residual_sf_tile<true, true>(W.Nx, W.Ny, W.Nz, W.coef_df, W.F, W.U, W.w, r2,
                                             reinterpret_cast<float2 *>(smem), bx, by, bz);
            } else {
                residual_sf_tile<false, true>(W.Nx, W.Ny, W.Nz, W.coef_df, W.F, W.U, W.w, r2,
                                              reinterpret_cast<float2 *>(smem), bx, by, bz);
            }
            break;
        }
        case ST_DSTX_F:
            // the first pass transforms F_hi (the first plane of F); later ones the residual
            dst_tile<FUSED, HS_AXIS_X, HS_MODE_WRITE>(W, stage == 1 ? W.F : W.w, W.w, 1.f, smem, tile);
            break;
        case ST_DSTY: {
            // forward y follows a forward x (stage type of the previous stage)
            const bool inverse = A.stages.type[stage - 1] == ST_THOMAS;
            dst_tile<FUSED, HS_AXIS_Y, HS_MODE_WRITE>(W, W.w, W.w, inverse ? W.sy : 1.f, smem, tile);
            break;
        }
        case ST_THOMAS: {
            const size_t idx = (size_t)tile * blockDim.x + threadIdx.x;
            if (idx < plane) {
                const size_t nz = (size_t)W.Nz * plane;
                if (W.thomas32)
                    thomas_column<float, float, float, true, false>(W.Nz, plane, idx, W.w, (float *)nullptr,
                                                             W.fac32, W.fac32 + nz,
                                                             W.fac32 + 2 * nz);
                else
                    thomas_column<float, double, double, true, false>(W.Nz, plane, idx, W.w, W.scr64,
                                                               W.fac64, W.fac64 + nz,
                                                               W.fac64 + 2 * nz);
            }
            break;
        }
        case ST_IDSTX_SET: dst_tile<FUSED, HS_AXIS_X, HS_MODE_DF_SET>(W, W.w, W.U, W.sx, smem, tile); break;
        case ST_IDSTX_ADD: dst_tile<FUSED, HS_AXIS_X, HS_MODE_DF_ADD>(W, W.w, W.U, W.sx, smem, tile); break;
        case ST_IDSTX_FINAL:
            dst_tile<FUSED, HS_AXIS_X, HS_MODE_DF_FINAL>(W, W.w, W.U, W.sx, smem, tile);
            break;
        case ST_IDSTX_W64: dst_w64_tile<FUSED>(W, W.w, W.sx, smem, tile); break;
        default: break;
    }
}

// The scheduler loop of every persistent CTA.  Thread 0 claims items from the
// queue one ahead (the atomic's latency overlaps the current tile), publishes
// the previous item's completion, and waits for the current item's
// dependency unless this CTA has already seen it met (counters only grow);
// the tile index and flags reach the other threads through shared memory, so
// an item costs two barriers.
template <bool FUSED>
__device__ __forceinline__ void batch_body(const BatchArgs &A) {
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ int s_it, s_wi, s_stage, s_tile, s_bail;
    __shared__ int s_pend_w, s_pend_s, s_ok_w, s_ok_s;  // thread 0's bookkeeping
    int next_it = 0;  // thread 0: the item claimed for the next loop trip (kept in a register
                      // so the atomic's latency overlaps the current tile)
    if (threadIdx.x == 0) {
        next_it = atomicAdd(A.next, 1);
        s_pend_w = -1;
        s_ok_w = -1;
        s_ok_s = -1;
    }
    for (;;) {
        if (threadIdx.x == 0) {
            if (s_pend_w >= 0) {
                __threadfence();
                atomicAdd(A.done + (size_t)s_pend_w * BMAX_STAGES + s_pend_s, 1);
                s_pend_w = -1;
            }
            const int it = next_it;
            int bail = 0;
            if (it < A.nitems) {
                next_it = atomicAdd(A.next, 1);
                const int2 item = A.items[it];
                const int wi = item.x & 0xFFFF, stage = item.x >> 16;
                if (stage > 0 && !(wi == s_ok_w && stage - 1 == s_ok_s)) {
                    const int *cnt = A.done + (size_t)wi * BMAX_STAGES + (stage - 1);
                    const int need = A.works[wi].need[stage - 1];
                    long long spins = 0;
                    while (ld_volatile(cnt) < need) {
                        if (ld_volatile(A.err) || ++spins > A.spin_limit) {
                            atomicExch(A.err, 1);
                            bail = 1;
                            break;
                        }
                        __nanosleep(100);
                    }
                    __threadfence();
                    if (!bail) {
                        s_ok_w = wi;
                        s_ok_s = stage - 1;
                    }
                }
                s_wi = wi;
                s_stage = stage;
                s_tile = item.y;
                s_pend_w = wi;
                s_pend_s = stage;
            }
            s_it = it;
            s_bail = bail;
        }
        __syncthreads();
        if (s_it >= A.nitems) break;
        const int stage = s_stage;
        if (!s_bail) run_tile<FUSED>(A, A.works[s_wi], stage, A.stages.type[stage], s_tile, smem);
        __syncthreads();
    }
}

}  // namespace

// Kernel variants (registers capped for 2 or 3 resident CTAs per SM; staged or
// fused transform tiles), each in its own translation unit; the host picks one
// per batch.
const void *batch_kernel_v2();
const void *batch_kernel_v3();
const void *batch_kernel_v2f();
const void *batch_kernel_v3f();

}  // namespace hs_batch
