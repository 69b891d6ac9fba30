// Batched solves in one persistent launch.
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
// the items a CTA waits for are already running: no deadlock.  A wait that
// exceeds its limit sets an error flag that the host reads (HS_ERR_TIMEOUT);
// later waits then give up at once, so the launch always ends.
// The launch (counter resets + kernel) is captured in a CUDA graph per stream.
#include <string.h>

#include <new>
#include <vector>

#include "hs_tiles.cuh"

using namespace hs_tiles;

namespace {

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
    if constexpr (MODE == HS_MODE_DF_SET || MODE == HS_MODE_DF_ADD || MODE == HS_MODE_DF_FINAL) {
        dst_fast_tile<float, float, float, AXIS, MODE, M, S, true, Rs...>(
            in, static_cast<float *>(out), W.u, roots, half, W.Nx, W.Ny, W.Nz, scale, smem, bx, by);
    } else {
        dst_fast_tile<float, float, float, AXIS, MODE, M, S, true, Rs...>(
            in, static_cast<float *>(out), nullptr, roots, half, W.Nx, W.Ny, W.Nz, scale, smem,
            bx, by);
    }
}

template <int M, int... Rs>
__device__ __forceinline__ void dst_w64_m(const BatchWork &W, const float *in, float scale,
                                          unsigned char *smem, int tile) {
    constexpr int S = Lines<float, M, HS_AXIS_X>::value;
    dst_fast_tile<float, float, double, HS_AXIS_X, HS_MODE_WRITE, M, S, true, Rs...>(
        in, W.u, nullptr, W.rx, W.hx, W.Nx, W.Ny, W.Nz, scale, smem, tile, 0);
}

// Dispatch a transform tile on the line length.
template <int AXIS, int MODE>
__device__ void dst_tile(const BatchWork &W, const float *in, void *out, float scale,
                         unsigned char *smem, int tile) {
    const int M = AXIS == HS_AXIS_X ? W.Mx : W.My;
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

__device__ void dst_w64_tile(const BatchWork &W, const float *in, float scale,
                             unsigned char *smem, int tile) {
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
            if (A.f_is_f64)
                rhs_df_tile<double>(W.rhs, static_cast<const double *>(W.f), W.F, f2, smem, bx,
                                    by, bz);
            else
                rhs_df_tile<float>(W.rhs, static_cast<const float *>(W.f), W.F, f2, smem, bx, by,
                                   bz);
            break;
        }
        case ST_RESIDUAL: {
            const int bx = tile % W.gx, by = (tile / W.gx) % W.gy, bz = tile / (W.gx * W.gy);
            const int m = A.sweep_of[stage];
            double *r2 = A.norms_on ? W.norms + m : nullptr;
            const bool f64 = A.resid_mode == HS_RESID_F64 ||
                             (A.resid_mode == HS_RESID_AUTO && residual_use_f64(W.norms, m));
            if (f64)
                residual64_tile<true>(W.Nx, W.Ny, W.Nz, W.coef64, W.F, W.U, W.w, r2, smem, bx, by,
                                      bz);
            else
                residual_tile<true>(W.Nx, W.Ny, W.Nz, W.coef_df, W.F, W.U, W.w, r2, smem, bx, by,
                                    bz);
            break;
        }
        case ST_DSTX_F:
            // the first pass transforms F_hi (the first plane of F); later ones the residual
            dst_tile<HS_AXIS_X, HS_MODE_WRITE>(W, stage == 1 ? W.F : W.w, W.w, 1.f, smem, tile);
            break;
        case ST_DSTY: {
            // forward y follows a forward x (stage type of the previous stage)
            const bool inverse = A.stages.type[stage - 1] == ST_THOMAS;
            dst_tile<HS_AXIS_Y, HS_MODE_WRITE>(W, W.w, W.w, inverse ? W.sy : 1.f, smem, tile);
            break;
        }
        case ST_THOMAS: {
            const size_t idx = (size_t)tile * blockDim.x + threadIdx.x;
            if (idx < plane) {
                const size_t nz = (size_t)W.Nz * plane;
                if (W.thomas32)
                    thomas_column<float, float, float, true>(W.Nz, plane, idx, W.w, (float *)nullptr,
                                                             W.fac32, W.fac32 + nz,
                                                             W.fac32 + 2 * nz);
                else
                    thomas_column<float, double, double, true>(W.Nz, plane, idx, W.w, W.scr64,
                                                               W.fac64, W.fac64 + nz,
                                                               W.fac64 + 2 * nz);
            }
            break;
        }
        case ST_IDSTX_SET: dst_tile<HS_AXIS_X, HS_MODE_DF_SET>(W, W.w, W.U, W.sx, smem, tile); break;
        case ST_IDSTX_ADD: dst_tile<HS_AXIS_X, HS_MODE_DF_ADD>(W, W.w, W.U, W.sx, smem, tile); break;
        case ST_IDSTX_FINAL:
            dst_tile<HS_AXIS_X, HS_MODE_DF_FINAL>(W, W.w, W.U, W.sx, smem, tile);
            break;
        case ST_IDSTX_W64: dst_w64_tile(W, W.w, W.sx, smem, tile); break;
        default: break;
    }
}

__global__ void __launch_bounds__(256, 2) batch_kernel(BatchArgs A) {
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ int cur;
    __shared__ int bail;
    for (;;) {
        if (threadIdx.x == 0) cur = atomicAdd(A.next, 1);
        __syncthreads();
        const int it = cur;
        if (it >= A.nitems) break;
        const int2 item = A.items[it];
        const int wi = item.x & 0xFFFF, stage = item.x >> 16, tile = item.y;
        const BatchWork &W = A.works[wi];
        if (threadIdx.x == 0) {
            bail = 0;
            if (stage > 0) {
                const int *cnt = A.done + (size_t)wi * BMAX_STAGES + (stage - 1);
                const int need = W.need[stage - 1];
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
            }
            if (ld_volatile(A.err)) bail = 1;
        }
        __syncthreads();
        if (!bail) run_tile(A, W, stage, A.stages.type[stage], tile, smem);
        __syncthreads();
        if (threadIdx.x == 0) {
            __threadfence();
            atomicAdd(A.done + (size_t)wi * BMAX_STAGES + stage, 1);
        }
    }
}

}  // namespace

// ------------------------------------------------------------------- host side

struct hs_batch_s {
    int n;                            // problems
    int f_dtype, sweeps;
    std::vector<hs_plan_t> plans;     // one per problem: tables, factors, first-RHS buffers
    std::vector<void *> extra;        // buffers of the further right-hand sides
    std::vector<BatchWork> works;     // one per (problem, RHS)
    std::vector<int> work_of;         // first work index of each problem
    std::vector<int> nrhs;
    BatchWork *d_works;
    int2 *d_items;
    int *d_ctr;                       // [0] next, [1] err, then done counters
    int nitems, nworks, grid;
    size_t smem;
    long long spin_limit;
    double tol;
    int resid_mode;
    double *d_norms;                  // [nworks][HS_INFO_MAX_ITERS + 1]
    StageList stages;
    int sweep_of[BMAX_STAGES];
    cudaGraphExec_t graph;
    cudaStream_t graph_stream;
    int have_graph;
    size_t bytes;
};

namespace {

size_t dst_smem_for(int M, int axis) {
    switch (M) {
#define HS_CASE(MM)                                                                          \
    case MM:                                                                                 \
        return axis == HS_AXIS_X ? fast_smem<float, MM, Lines<float, MM, HS_AXIS_X>::value>() \
                                 : fast_smem<float, MM, Lines<float, MM, HS_AXIS_Y>::value>();
        HS_CASE(32) HS_CASE(64) HS_CASE(96) HS_CASE(128) HS_CASE(192) HS_CASE(256) HS_CASE(384)
#undef HS_CASE
        default: return 0;
    }
}

int lines_for(int M, int axis) {
    switch (M) {
#define HS_CASE(MM)                                                                   \
    case MM:                                                                          \
        return axis == HS_AXIS_X ? Lines<float, MM, HS_AXIS_X>::value                 \
                                 : Lines<float, MM, HS_AXIS_Y>::value;
        HS_CASE(32) HS_CASE(64) HS_CASE(96) HS_CASE(128) HS_CASE(192) HS_CASE(256) HS_CASE(384)
#undef HS_CASE
        default: return 0;
    }
}

void free_batch(hs_batch_s *B) {
    if (!B) return;
    if (B->have_graph) cudaGraphExecDestroy(B->graph);
    for (hs_plan_t p : B->plans)
        if (p) hs_destroy(p);
    for (void *q : B->extra)
        if (q) cudaFree(q);
    if (B->d_works) cudaFree(B->d_works);
    if (B->d_items) cudaFree(B->d_items);
    if (B->d_ctr) cudaFree(B->d_ctr);
    if (B->d_norms) cudaFree(B->d_norms);
    delete B;
}

}  // namespace

extern "C" {

hs_status hs_batch_create(hs_batch_t *out, const hs_problem_desc *probs, int nprob, int f_dtype,
                          int sweeps) {
    if (!out || !probs || nprob < 1 || nprob > 65535) return HS_ERR_INVALID_ARG;
    *out = nullptr;
    if (f_dtype != HS_F64 && f_dtype != HS_F32) return HS_ERR_INVALID_ARG;
    if (sweeps < 0 || sweeps >= HS_INFO_MAX_ITERS) return HS_ERR_INVALID_ARG;
    for (int k = 0; k < nprob; ++k) {
        const hs_problem_desc &d = probs[k];
        if (d.nrhs < 1 || d.nrhs > 16 || !d.f || !d.u || !d.c0) return HS_ERR_INVALID_ARG;
        if (!dst_smem_for(d.Nx + 1, HS_AXIS_X) || !dst_smem_for(d.Ny + 1, HS_AXIS_Y))
            return HS_ERR_UNSUPPORTED;  // batched transforms: N + 1 in {32,..,384} of 2^a 3^b
    }
    hs_batch_s *B = new (std::nothrow) hs_batch_s;
    if (!B) return HS_ERR_OOM;
    B->n = nprob;
    B->f_dtype = f_dtype;
    B->sweeps = sweeps;
    B->d_works = nullptr;
    B->d_items = nullptr;
    B->d_ctr = nullptr;
    B->d_norms = nullptr;
    B->tol = 0.0;
    B->resid_mode = HS_RESID_AUTO;
    B->have_graph = 0;
    B->graph_stream = nullptr;
    B->bytes = 0;
    B->spin_limit = 20000000;  // ~2 s of 100 ns naps before a wait gives up

    // stage list: RHS, then (transform x, y, z-solves, inverse y, inverse x) per pass,
    // with the residual before every refinement pass
    StageList &L = B->stages;
    L.n = 0;
    B->sweep_of[L.n] = 0;
    L.type[L.n++] = ST_RHS;
    for (int p = 0; p <= sweeps; ++p) {
        const int first = L.n;
        if (p > 0) L.type[L.n++] = ST_RESIDUAL;
        L.type[L.n++] = ST_DSTX_F;
        L.type[L.n++] = ST_DSTY;
        L.type[L.n++] = ST_THOMAS;
        L.type[L.n++] = ST_DSTY;
        L.type[L.n++] = sweeps == 0 ? ST_IDSTX_W64
                                    : (p == 0 ? ST_IDSTX_SET
                                              : (p == sweeps ? ST_IDSTX_FINAL : ST_IDSTX_ADD));
        for (int k = first; k < L.n; ++k) B->sweep_of[k] = p;
    }

    hs_status st = HS_OK;
    size_t smem = 2 * 5 * RHY * RHX * sizeof(float);
    const size_t res_smem = 2 * 2 * QHY * QHX * sizeof(float);
    if (res_smem > smem) smem = res_smem;
    for (int k = 0; k < nprob && st >= 0; ++k) {
        const hs_problem_desc &d = probs[k];
        hs_plan_t P = nullptr;
        st = hs_plan(&P, d.Nx, d.Ny, d.Nz, d.Lx, d.Ly, d.Lz, d.order, d.equation, HS_BC_DIRICHLET,
                     HS_MIXED, 1);
        if (st < 0) break;
        B->plans.push_back(P);
        st = hs_set_coeff(P, d.c0, d.c1, d.c2, d.cd_variant);
        if (st < 0) break;
        const size_t a = dst_smem_for(d.Nx + 1, HS_AXIS_X), b = dst_smem_for(d.Ny + 1, HS_AXIS_Y);
        if (a > smem) smem = a;
        if (b > smem) smem = b;
        const size_t n = (size_t)d.Nx * d.Ny * d.Nz;
        const size_t fcount = (size_t)(d.Nx + 2) * (d.Ny + 2) * (d.Nz + 2);
        const size_t esz = f_dtype == HS_F64 ? 8 : 4;
        B->work_of.push_back((int)B->works.size());
        B->nrhs.push_back(d.nrhs);
        for (int r = 0; r < d.nrhs; ++r) {
            BatchWork W;
            memset(&W, 0, sizeof(W));
            W.Nx = d.Nx;
            W.Ny = d.Ny;
            W.Nz = d.Nz;
            W.Mx = d.Nx + 1;
            W.My = d.Ny + 1;
            W.thomas32 = P->thomas32;
            W.coef_df = P->d_coef_df;
            W.coef64 = P->d_coef;
            W.fac32 = P->d_fac32;
            W.fac64 = P->d_fac;
            W.rx = static_cast<const float2 *>(P->axf[0].roots);
            W.hx = static_cast<const float2 *>(P->axf[0].half);
            W.ry = static_cast<const float2 *>(P->axf[1].roots);
            W.hy = static_cast<const float2 *>(P->axf[1].half);
            RhsArgs &ra = W.rhs;
            ra.Nx = d.Nx;
            ra.Ny = d.Ny;
            ra.Nz = d.Nz;
            ra.hz = P->hz;
            ra.order = d.order;
            ra.equation = d.equation;
            ra.rhs_kind = HS_RHS_NODAL;
            ra.coef = P->d_coef;
            ra.c0 = P->d_c0;
            ra.c1 = P->d_c1;
            ra.rc = P->d_rhs_df;
            ra.has_faces = 0;
            W.f = static_cast<const unsigned char *>(d.f) + (size_t)r * fcount * esz;
            W.u = d.u + (size_t)r * n;
            if (r == 0) {
                W.F = P->d_Fdf;
                W.U = P->d_Udf;
                W.w = P->d_w32;
                W.scr64 = P->d_dscr;
            } else {
                // F (2n floats), U (2n floats), w (n floats) and, with FP64 factors,
                // the FP64 forward-sweep scratch (n doubles), each 256-byte aligned
                auto up = [](size_t b) { return (b + 255) & ~(size_t)255; };
                const size_t oF = 0, oU = up(oF + 2 * n * sizeof(float));
                const size_t ow = up(oU + 2 * n * sizeof(float));
                const size_t os = up(ow + n * sizeof(float));
                const size_t bytes = os + (W.thomas32 ? 0 : n * sizeof(double));
                void *buf = nullptr;
                if (cudaMalloc(&buf, bytes) != cudaSuccess) {
                    cudaGetLastError();
                    st = HS_ERR_OOM;
                    break;
                }
                B->extra.push_back(buf);
                B->bytes += bytes;
                unsigned char *base = static_cast<unsigned char *>(buf);
                W.F = reinterpret_cast<float *>(base + oF);
                W.U = reinterpret_cast<float *>(base + oU);
                W.w = reinterpret_cast<float *>(base + ow);
                W.scr64 = W.thomas32 ? nullptr : reinterpret_cast<double *>(base + os);
            }
            W.sx = (float)(2.0 / (d.Nx + 1));
            W.sy = (float)(2.0 / (d.Ny + 1));
            W.gx = (d.Nx + RTX - 1) / RTX;
            W.gy = (d.Ny + RTY - 1) / RTY;
            W.gz = (d.Nz + RZ - 1) / RZ;
            const int Sx = lines_for(W.Mx, HS_AXIS_X), Sy = lines_for(W.My, HS_AXIS_Y);
            W.dxg = (int)(((long)d.Ny * d.Nz + Sx - 1) / Sx);
            W.lx = Sx;
            W.dyg = (d.Nx + Sy - 1) / Sy;
            for (int s = 0; s < L.n; ++s) {
                int t = 0;
                switch (L.type[s]) {
                    case ST_RHS:
                    case ST_RESIDUAL: t = W.gx * W.gy * W.gz; break;
                    case ST_DSTY: t = W.dyg * d.Nz; break;
                    case ST_THOMAS: t = (int)(((size_t)d.Nx * d.Ny + 255) / 256); break;
                    default: t = W.dxg; break;
                }
                W.need[s] = t;
            }
            B->works.push_back(W);
        }
    }
    if (st < 0) {
        free_batch(B);
        return st;
    }
    // items: stage by stage over every (problem, RHS)
    std::vector<int2> items;
    for (int s = 0; s < L.n; ++s)
        for (size_t w = 0; w < B->works.size(); ++w)
            for (int t = 0; t < B->works[w].need[s]; ++t)
                items.push_back(make_int2((int)w + 65536 * s, t));
    B->nitems = (int)items.size();
    B->nworks = (int)B->works.size();
    if (B->nworks > 65535) {
        free_batch(B);
        return HS_ERR_UNSUPPORTED;
    }
    B->smem = smem;
    const size_t nslots = (size_t)B->nworks * (HS_INFO_MAX_ITERS + 1);
    if (cudaMalloc((void **)&B->d_norms, nslots * sizeof(double)) != cudaSuccess) {
        cudaGetLastError();
        free_batch(B);
        return HS_ERR_OOM;
    }
    for (int w = 0; w < B->nworks; ++w) B->works[w].norms = B->d_norms + (size_t)w * (HS_INFO_MAX_ITERS + 1);
    if (cudaMalloc((void **)&B->d_works, B->works.size() * sizeof(BatchWork)) != cudaSuccess ||
        cudaMalloc((void **)&B->d_items, items.size() * sizeof(int2)) != cudaSuccess ||
        cudaMalloc((void **)&B->d_ctr, (2 + (size_t)B->nworks * BMAX_STAGES) * sizeof(int)) !=
            cudaSuccess) {
        cudaGetLastError();
        free_batch(B);
        return HS_ERR_OOM;
    }
    B->bytes += B->works.size() * sizeof(BatchWork) + items.size() * sizeof(int2) +
                (2 + (size_t)B->nworks * BMAX_STAGES) * sizeof(int);
    if (cudaMemcpy(B->d_works, B->works.data(), B->works.size() * sizeof(BatchWork),
                   cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(B->d_items, items.data(), items.size() * sizeof(int2),
                   cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaFuncSetAttribute(batch_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)smem) != cudaSuccess) {
        cudaGetLastError();
        free_batch(B);
        return HS_ERR_CUDA;
    }
    int dev = 0, sms = 0, per = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, batch_kernel, 256, smem) !=
            cudaSuccess ||
        per < 1) {
        cudaGetLastError();
        free_batch(B);
        return HS_ERR_UNSUPPORTED;
    }
    B->grid = sms * per;  // every CTA resident: waits only on items already taken
    *out = B;
    return HS_OK;
}

hs_status hs_batch_set_io(hs_batch_t B, int k, const void *f, double *u) {
    if (!B || k < 0 || k >= B->n || !f || !u) return HS_ERR_INVALID_ARG;
    hs_plan_t P = B->plans[k];
    const size_t n = (size_t)P->Nx * P->Ny * P->Nz;
    const size_t fcount = (size_t)(P->Nx + 2) * (P->Ny + 2) * (P->Nz + 2);
    const size_t esz = B->f_dtype == HS_F64 ? 8 : 4;
    const int w0 = B->work_of[k];
    for (int r = 0; r < B->nrhs[k]; ++r) {
        BatchWork &W = B->works[w0 + r];
        W.f = static_cast<const unsigned char *>(f) + (size_t)r * fcount * esz;
        W.u = u + (size_t)r * n;
    }
    if (cudaMemcpy(B->d_works + w0, &B->works[w0], B->nrhs[k] * sizeof(BatchWork),
                   cudaMemcpyHostToDevice) != cudaSuccess) {
        cudaGetLastError();
        return HS_ERR_CUDA;
    }
    return HS_OK;
}

hs_status hs_batch_set_wait_limit(hs_batch_t B, long long spins) {
    if (!B || spins < 1) return HS_ERR_INVALID_ARG;
    B->spin_limit = spins;
    if (B->have_graph) {
        cudaGraphExecDestroy(B->graph);
        B->have_graph = 0;
    }
    return HS_OK;
}

hs_status hs_batch_set_tol(hs_batch_t B, double tol) {
    if (!B || !(tol >= 0.0)) return HS_ERR_INVALID_ARG;
    B->tol = tol;
    if (B->have_graph) {
        cudaGraphExecDestroy(B->graph);
        B->have_graph = 0;
    }
    return HS_OK;
}

hs_status hs_batch_set_residual_precision(hs_batch_t B, int mode) {
    if (!B || (mode != HS_RESID_DF && mode != HS_RESID_F64 && mode != HS_RESID_AUTO))
        return HS_ERR_INVALID_ARG;
    B->resid_mode = mode;
    if (B->have_graph) {
        cudaGraphExecDestroy(B->graph);
        B->have_graph = 0;
    }
    return HS_OK;
}

hs_status hs_batch_debug_stall(hs_batch_t B, int on) {
    // test hook: one dependency of the first (problem, RHS) asks for one tile
    // more than its stage has, so the wait for it can only end by timing out
    if (!B || B->stages.n < 2) return HS_ERR_INVALID_ARG;
    BatchWork &W = B->works[0];
    const int real = W.need[1];
    BatchWork tmp = W;
    tmp.need[1] = real + (on ? 1 : 0);
    if (cudaMemcpy(B->d_works, &tmp, sizeof(BatchWork), cudaMemcpyHostToDevice) != cudaSuccess) {
        cudaGetLastError();
        return HS_ERR_CUDA;
    }
    return HS_OK;
}

hs_status hs_batch_solve(hs_batch_t B, void *stream, int sync) {
    if (!B) return HS_ERR_INVALID_ARG;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    if (!B->have_graph || B->graph_stream != s) {
        if (B->have_graph) cudaGraphExecDestroy(B->graph);
        B->have_graph = 0;
        BatchArgs A;
        A.works = B->d_works;
        A.items = B->d_items;
        A.nitems = B->nitems;
        A.next = B->d_ctr;
        A.err = B->d_ctr + 1;
        A.done = B->d_ctr + 2;
        A.spin_limit = B->spin_limit;
        A.f_is_f64 = B->f_dtype == HS_F64;
        A.tol2 = B->tol * B->tol;
        A.resid_mode = B->resid_mode;
        A.norms_on = B->sweeps >= 1 && (B->tol > 0.0 ||
                                         (B->resid_mode == HS_RESID_AUTO && B->sweeps >= 2));
        A.stages = B->stages;
        for (int k = 0; k < BMAX_STAGES; ++k) A.sweep_of[k] = B->sweep_of[k];
        cudaStream_t cs;
        if (cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking) != cudaSuccess) {
            cudaGetLastError();
            return HS_ERR_CUDA;
        }
        cudaGraph_t g = nullptr;
        bool ok = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal) == cudaSuccess;
        if (ok) {
            cudaMemsetAsync(B->d_ctr, 0, (2 + (size_t)B->nworks * BMAX_STAGES) * sizeof(int), cs);
            cudaMemsetAsync(B->d_norms, 0,
                            (size_t)B->nworks * (HS_INFO_MAX_ITERS + 1) * sizeof(double), cs);
            batch_kernel<<<B->grid, 256, B->smem, cs>>>(A);
            ok = cudaStreamEndCapture(cs, &g) == cudaSuccess && g;
        }
        ok = ok && cudaGraphInstantiate(&B->graph, g, 0) == cudaSuccess;
        if (g) cudaGraphDestroy(g);
        cudaStreamDestroy(cs);
        if (!ok) {
            cudaGetLastError();
            return HS_ERR_CUDA;
        }
        B->have_graph = 1;
        B->graph_stream = s;
    }
    if (cudaGraphLaunch(B->graph, s) != cudaSuccess) {
        cudaGetLastError();
        return HS_ERR_CUDA;
    }
    if (!sync) return HS_OK;
    int err = 0;
    if (cudaMemcpyAsync(&err, B->d_ctr + 1, sizeof(int), cudaMemcpyDeviceToHost, s) !=
            cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess) {
        cudaGetLastError();
        return HS_ERR_CUDA;
    }
    return err ? HS_ERR_TIMEOUT : HS_OK;
}

size_t hs_batch_workspace_bytes(hs_batch_t B) {
    if (!B) return 0;
    size_t t = B->bytes;
    for (hs_plan_t p : B->plans) t += hs_workspace_bytes(p);
    return t;
}

hs_status hs_batch_destroy(hs_batch_t B) {
    if (!B) return HS_OK;
    cudaDeviceSynchronize();
    free_batch(B);
    return HS_OK;
}

}  // extern "C"
