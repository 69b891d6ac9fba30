// Internal declarations shared by the solver's translation units.
#pragma once

#include <cuda_runtime.h>
#include <stddef.h>
#include <stdint.h>

#include "hs.h"

#define HS_MAX_STAGES 16
// Min pivot ratio below which a plan's z-systems count as close to singular: the
// mixed path then keeps FP64 factors (FP64 forward sweep).
#define HS_ILL_PIVOT 1e-4
#define HS_EVENT_PAIRS 128

// One transform axis: DST-I of length N computed through a complex FFT of
// length M = N + 1 on the odd extension of each line (Section 3.6 says the
// 2-D transform is done "by FFT"; this is the packed real-odd formulation).
struct DstAxis {
    int N;              // line length (interior points)
    int M;              // N + 1
    int fft;            // 1: M = 2^a 3^b, mixed-radix FFT; 0: direct O(N^2) sums
    int nst;            // number of FFT stages
    int radix[HS_MAX_STAGES];
    const void *roots;  // M complex: exp(-2 pi i k / M), compute type
    const void *half;   // M + 1 complex: (cos(pi k / M), sin(pi k / M))
    const void *sintab; // 2M reals: sin(pi m / M) (direct path)
};

// HS_AXIS_X / HS_AXIS_Y come from hs.h
enum { HS_T_F64 = 0, HS_T_F32 = 1, HS_T_DF = 2 };
// Output modes of the inverse x-transform: write, accumulate, and the
// double-float iterate updates of the mixed path (set hi = X, lo = 0; add X
// to (hi, lo); add X and write hi + lo as FP64 to the auxiliary array u; the
// same final step for an iterate whose lo plane is zero and was never written:
// only hi is read).
enum { HS_MODE_WRITE = 0, HS_MODE_ADD = 1, HS_MODE_DF_SET = 2, HS_MODE_DF_ADD = 3,
       HS_MODE_DF_FINAL = 4, HS_MODE_DF_FINAL_HI = 5 };

// Device views of the boundary data of one solve (pointers already on device).
struct DevBoundary {
    const void *face[6];
    const void *fnn[6];
};

// Chunks of the pipelined upload of a staged host right-hand side.
#define HS_UP_CHUNKS 4

struct hs_plan_s {
    int Nx, Ny, Nz;
    double Lx, Ly, Lz, hx, hy, hz;
    int order, equation, precision, max_rhs;
    int refine_sweeps;
    double refine_tol;  // > 0: stop refining once ||F - A U|| / ||F|| <= refine_tol
    int *d_skip;        // device flag: 1 once refinement has converged (later kernels return)
    const int *cur_skip;  // the flag the launchers pass on (NULL outside tolerance mode)
    int stage_timing;
    int dst_variant[2];   // per axis: one of HS_DST_* (hs.h)
    int thomas_variant;   // FP32 z-solve mapping: HS_THOMAS_*
    void *d_ytmp;         // complex scratch of the two-pass y transform (Nz x M x Nx float2)
    void *d_gemm[2];      // per axis: FP16 sine-matrix splits of the tensor-core transform
    int *d_gemm_err;      // set by a tensor-core transform whose bounded wait gave up
    int resid_mode;       // HS_RESID_DF / HS_RESID_F64 / HS_RESID_AUTO
    int factor_mode;      // HS_FACTOR_AUTO / F32 / F64 (mixed path z-solves)
    int host_io_mapped;
    cudaStream_t up_stream;   // upload stream of the chunked host-f copy (lazily created)
    // [0, K): chunks of the first right-hand side; [K]: call start; [K + 1 + b]:
    // f staging buffer b free (its last right-hand-side kernel is queued)
    cudaEvent_t up_ev[HS_UP_CHUNKS + 3];
    cudaEvent_t *up_rhs;      // [max_rhs]: copy of right-hand side r done
    int f_buf;                // f staging buffer of the next HS_HOST_F_EARLY solve
    int have_up;   // up_stream and up_ev exist
    // HS_HOST_U_LATE: the copy of a staged u to the host runs on dn_stream, out of
    // one of two staging buffers (d_stage_u, d_stage_u1) used in turn
    cudaStream_t dn_stream;
    cudaEvent_t dn_ev[3];   // [b]: copy out of staging buffer b done; [2]: solve queued
    int dn_pending[2];      // a copy out of buffer b has been queued
    int dn_last;            // buffer of the latest queued copy (-1: none)
    int u_buf;              // staging buffer of the next HS_HOST_U_LATE solve
    int have_dn;
    int have_coeff;
    int cd_variant;
    double min_pivot_ratio;
    int device;

    // coefficient tables (device)
    double *d_coef;     // [Nz][3][4]: C[l][nu][a,b,c,d]
    double *d_c0;       // [Nz+2]: k^2 or gamma at nodes
    double *d_c1;       // [Nz+2]: (k^2)_z (6th-order RHS)
    double *d_cx;       // [Nx]: cos(p pi / (Nx+1))
    double *d_cy;       // [Ny]
    double *d_fac;      // [3][Nz][Ny][Nx]: c'_l, 1/m_l, lower_l/m_l
    float *d_fac32;     // the same rounded to FP32 (mixed path, well-conditioned plans)
    float2 *d_coef_df;  // [Nz][12] coefficients as FP32 pairs (double-float residual)
    int resid_xy;       // b_nu = c_nu on every row: the residual merges x- and y-neighbour sums
    double *d_ghost;    // ghost nodes of the 6th-order mixed right-hand side (FP64 f):
                        // [2][Nz+2][Ny+2] (x faces), [2][Nz+2][Nx+2] (y), [2][Ny+2][Nx+2] (z)
    float4 *d_rhs_df;   // [2][Nz+2] double-float RHS weights.  [0]: 6th order (67/120 - h^2 K/20,
                        // h^3 K_z/120); CD (0, h gamma/24).  [1] (sum-factorised kernel):
                        // 6th order (h^2 (67/120 - h^2 K/20), h^5 K_z/120); CD (0, h^3 gamma/24)
    float2 rhs_sf_W;    // constant pair weight of the sum-factorised kernel (h^2/720, h^2/12, h^2)
    int thomas32;       // mixed path: 1 = FP32 z-solves (min pivot ratio >= 1e-4)
    double *d_red;      // reduction scratch (64 doubles)

    // transform tables
    DstAxis axd[2];     // FP64 compute, x and y
    DstAxis axf[2];     // FP32 compute
    void *d_tables;     // one allocation behind every axis table

    // workspace
    double *d_w64;      // [Nz][Ny][Nx]: FP64 path data, or mixed-path lifted F
    float *d_w32;       // [Nz][Ny][Nx]: mixed-path FP32 work array
    float *d_Fdf;       // [2][Nz][Ny][Nx]: mixed-path lifted F as double-float (hi, lo planes)
    float *d_Udf;       // [2][Nz][Ny][Nx]: mixed-path iterate U as double-float
    double *d_dscr;     // [Nz][Ny][Nx]: mixed-path forward-sweep scratch

    // host staging (allocated on first use with host pointers)
    void *d_stage_f;
    size_t stage_f_bytes;
    void *d_stage_f1;         // second f staging buffer (HS_HOST_F_EARLY)
    size_t stage_f1_bytes;
    double *d_stage_u;
    size_t stage_u_bytes;
    double *d_stage_u1;
    size_t stage_u1_bytes;
    void *d_stage_bnd;
    size_t stage_bnd_bytes;
    void *d_stage_bnd1;       // second boundary staging buffer (HS_HOST_F_EARLY)
    size_t stage_bnd1_bytes;

    cudaEvent_t ev[2 * HS_EVENT_PAIRS];   // stage timing: begin/end pairs
    cudaEvent_t ev_total[2];
    int have_events;
    int timer_used;                       // recorded pairs not yet read
    int timer_stage[HS_EVENT_PAIRS];      // stage index of each pair
    int timer_total_pending;
    float timer_acc[HS_INFO_STAGES];      // per-stage sums of the last solve

    size_t bytes;
    char last_error[256];
};

// ---------------------------------------------------------------- launchers
// Each returns HS_OK or HS_ERR_CUDA (launch error), never synchronises.

// Forward/inverse DST-I along one axis of an interior array [Nz][Ny][Nx].
// out = scale * DST(in) (MODE_WRITE) or out += scale * DST(in) (MODE_ADD,
// FP64 out only), or a double-float mode (tout = HS_T_DF, out = float2 pairs,
// aux = FP64 u for MODE_DF_FINAL).  `in` and `out` may alias (each block owns
// its tile).
hs_status hs_launch_dst(const hs_plan_s *P, int axis, int tc, int tin, const void *in, int tout,
                        void *out, int mode, double scale, cudaStream_t s, double *aux = nullptr);

// Compile-time-sized transform kernels (k_dst_fast.cu): 1 when M = N + 1 has one.
int hs_dst_fast_size(int M);
// NVTX range for the lifetime of a scope (a no-op unless a profiler is attached):
// one per public entry point that launches work.
#include <nvtx3/nvToolsExt.h>
struct HsRange {
    explicit HsRange(const char *name) { nvtxRangePushA(name); }
    ~HsRange() { nvtxRangePop(); }
    HsRange(const HsRange &) = delete;
    HsRange &operator=(const HsRange &) = delete;
};
// Autotune cache (hs_tune_cache.cu): choices of an earlier hs_autotune for a plan
// of the same class (device, shape, order, equation, precision, factor type).
bool hs_tune_lookup(const hs_plan_s *P, int *vx, int *vy, int *thomas, float *msx, float *msy);
void hs_tune_store(const hs_plan_s *P, int vx, int vy, int thomas, float msx, float msy);
// cudaPointerGetAttributes says device or managed memory (NULL counts as device).
bool hs_is_device_ptr(const void *p);
// Enqueue the count of NaN / infinite values of x[0..n) into *dcount (k_finite.cu).
hs_status hs_launch_nonfinite(const void *x, int dtype, size_t n, unsigned long long *dcount,
                              cudaStream_t s);
// Half-length FP64 DST-I (k_dst_half.cu): lengths with a compiled M/2-point FFT.
int hs_dst_half_size(int M);
hs_status hs_launch_dst_half(const hs_plan_s *P, int axis, int tin, const void *in, int tout,
                             void *out, int mode, double scale, cudaStream_t s);
hs_status hs_launch_dst_fast(const hs_plan_s *P, int axis, int tc, int tin, const void *in,
                             int tout, void *out, int mode, double scale, cudaStream_t s,
                             double *aux);
// Its three groups of kernel instances (k_dst_fast_f64.cu, k_dst_fast_f32.cu,
// k_dst_fast_df.cu); HS_ERR_UNSUPPORTED for other type / mode combinations.
hs_status hs_dst_fast_f64(const hs_plan_s *P, int axis, int tin, const void *in, int tout,
                          void *out, int mode, double scale, cudaStream_t s, double *aux);
hs_status hs_dst_fast_f32(const hs_plan_s *P, int axis, int tin, const void *in, int tout,
                          void *out, int mode, double scale, cudaStream_t s, double *aux);
hs_status hs_dst_fast_df(const hs_plan_s *P, int axis, int tin, const void *in, int tout,
                         void *out, int mode, double scale, cudaStream_t s, double *aux);

// Fused FP32 transform tiles (k_dst_fused_x.cu, k_dst_fused_y.cu); HS_ERR_UNSUPPORTED
// for a length or type combination they do not cover.  wide = 1: twice the
// staged tile's lines per CTA (lengths whose in-place tile allows it).
hs_status hs_launch_dst_fused_x(const hs_plan_s *P, int tin, const void *in, int tout, void *out,
                                int mode, double scale, cudaStream_t s, double *aux, int wide);
hs_status hs_launch_dst_fused_y(const hs_plan_s *P, int tin, const void *in, int tout, void *out,
                                int mode, double scale, cudaStream_t s, double *aux, int wide);
// hs_plan with lean = 1: an FP64 plan without the cached z-factorization, used
// as the transform engine and work arrays of other solvers (d_w64, d_dscr).
extern "C" hs_status hs_plan_ex(hs_plan_t *out, int Nx, int Ny, int Nz, double Lx, double Ly,
                                double Lz, int order, int equation, int bc, int precision,
                                int max_rhs, int lean);

// FP64 DCT-I of lines of M + 1 nodes (k_dct.cu), in place allowed; roots: M
// complex exp(-2 pi i k / M), half: M + 1 complex (cos, sin)(pi k / M).  axis X:
// nrows contiguous rows; axis Y: the nx columns of nplanes planes [M + 1][nx].
// HS_ERR_UNSUPPORTED unless M has a compiled FFT (hs_dst_fast_size).
hs_status hs_launch_dct_generic(int axis, int M, const double *in, double *out, const void *half,
                                long nrows, int nx, int nplanes, double scale, cudaStream_t s);
hs_status hs_launch_dct(int axis, int M, const double *in, double *out, const void *roots,
                        const void *half, long nrows, int nx, int nplanes, double scale,
                        cudaStream_t s);
// FP32 DCT-I of the same lines (k_dct32.cu): roots / half as above in FP32;
// tout / mode as hs_launch_dst's (axis Y: FP32 write only); lo_off and aux as
// hs_emit's.  hs_dct32_size: M has a compiled FFT; else HS_ERR_UNSUPPORTED.
int hs_dct32_size(int M);
hs_status hs_launch_dct32(int axis, int M, int tout, int mode, const float *in, void *out,
                          double *aux, size_t lo_off, const void *roots, const void *half,
                          long nrows, int nx, int nplanes, double scale, cudaStream_t s);

// Tensor-core (tcgen05) sine-matrix GEMM transform (k_dst_gemm.cu), mixed path:
// line lengths M = N + 1 in {32, 64, 96, 128, 192, 256}.  The table holds the FP16
// splits of the sine matrix in the kernel's shared-memory layout.
int hs_dst_gemm_size(int M);
size_t hs_dst_gemm_table_bytes(int M);
void hs_dst_gemm_table(int M, uint8_t *host);
hs_status hs_launch_dst_gemm(const hs_plan_s *P, int axis, int tin, const void *in, int tout,
                             void *out, int mode, double scale, cudaStream_t s, double *aux);

// Lines per CTA of the fused tile of length M (0: not built for that length).
int hs_dst_fused_lines_x(int M, int wide);
int hs_dst_fused_lines_y(int M, int wide);

// Two-pass y transform for long lines (k_dst_twopass.cu): 1 for M in {512, 768, 1024};
// needs P->d_ytmp.
int hs_dst_twopass_size(int M);
hs_status hs_launch_dst_twopass_y(const hs_plan_s *P, const float *in, float *out, double scale,
                                  cudaStream_t s);

// 1 when a line of this axis fits the transform kernel's shared memory.
int hs_dst_fits(const DstAxis &ax, int axis, int tc);

// Lifted right-hand side F (interior) from f: FP64 (out_df = 0) or a
// double-float pair in two FP32 planes [2][Nz][Ny][Nx] (out_df = 1).
// Uploads one node-grid right-hand side from host memory fh into the device
// staging buffer fd in `chunks` (1..HS_UP_CHUNKS) chunks of z-planes on
// P->up_stream, behind whatever the caller queued there before, and runs the
// tiled right-hand-side kernel on stream s slab by slab, each slab waiting only
// for the chunk that holds its last plane: the copy overlaps the kernel.
// Needs P->have_up.
hs_status hs_upload_rhs(hs_plan_s *P, const void *fh, void *fd, int chunks, int f_dtype,
                        const DevBoundary &b, void *F, int out_df, cudaStream_t s, double *f2);

// For a nodal f the tiled kernels can run on a slab of z-tiles [bz0, bz0 + nbz)
// (nbz < 0: to the last tile; tiles are RZ output planes).
// z-planes per tile of the nodal right-hand-side kernel (out_df: the mixed path's
// sum-factorised kernel); slab launches count tiles of this height.
int hs_rhs_tile_planes(const hs_plan_s *P, int out_df);
// planes per z-tile of the mixed path's right-hand-side and residual kernels
int hs_sf_zdepth(const hs_plan_s *P);
hs_status hs_launch_rhs(const hs_plan_s *P, const void *f, int f_dtype, int rhs_kind,
                        const DevBoundary &b, void *F, int out_df, cudaStream_t s,
                        double *f2 = nullptr, int bz0 = 0, int nbz = -1);

// Kernel selectors of the automatic residual precision: launch both kernels;
// each returns at once unless the rule (residual_use_f64 on norms, sweep m)
// picks it.
enum { HS_RESID_SEL_DF = 3, HS_RESID_SEL_F64 = 4 };

// r = F - A U (F, U double-float pairs; r FP32) in the arithmetic `prec`
// (HS_RESID_DF, HS_RESID_F64, or both selectors in one call for the automatic
// rule with the squared norms `norms` [||F||^2, ||r_1||^2, ...] and sweep m);
// adds ||r||^2 to *r2 when r2 is not NULL.  u_lo_zero: the lo plane of U is
// zero and was never written (the first residual after the FP32 solve wrote
// U's hi plane only); only HS_RESID_DF takes it.
hs_status hs_launch_residual_df(const hs_plan_s *P, const float *F, const float *U, float *r,
                                cudaStream_t s, double *r2 = nullptr, int prec = HS_RESID_DF,
                                const double *norms = nullptr, int m = 0, bool u_lo_zero = false);

// Sets *skip = 1 when *r2 <= tol^2 * *f2 (refinement converged).
hs_status hs_launch_gate(const double *r2, const double *f2, double tol, int *skip, cudaStream_t s);

// u = hi + lo in FP64 for a double-float array of n pairs (two planes).
hs_status hs_launch_df_to_f64(const float *x, size_t n, double *u, cudaStream_t s);

// r = F - A U on the interior (zero Dirichlet data: F is already lifted).
// r is FP32 (r32 != NULL) or FP64 (r64 != NULL).
hs_status hs_launch_residual(const hs_plan_s *P, const double *F, const double *U, float *r32,
                             double *r64, cudaStream_t s);

// d_out[0] += sum(x^2) over n elements (FP64, or FP32 when x32 != NULL).
hs_status hs_launch_sumsq(const double *x64, const float *x32, size_t n, double *d_out,
                          cudaStream_t s);

// Cached factorization of every z-system; writes the min |pivot| and max
// |diag| reductions to d_red[0..1] (as bit patterns of non-negative doubles).
hs_status hs_launch_factor(const hs_plan_s *P, cudaStream_t s);

// z-solves with the cached factorization.  FP64 path: data is FP64, in place
// (scratch unused).  Mixed path: data is FP32 in place; with FP64 factors the
// forward sweep is kept in the FP64 scratch, with FP32 factors (P->thomas32)
// everything is FP32 and in place.
hs_status hs_launch_thomas(const hs_plan_s *P, int tio, void *data, double *scratch,
                           cudaStream_t s);

// Per-row stencil coefficients C[l][nu][a,b,c,d] for rows l = 1..P->Nz
// (Sections 3.2-3.5).  Reads P's Nz, h, order and equation only; c0..c2 are
// host arrays indexed l = 0..Nz+1.
void hs_stencil_table(const hs_plan_s *P, const double *c0, const double *c1, const double *c2,
                      int cd_variant, double *C);

// Shared output step of the transform kernels (see HS_MODE_*).  For the
// double-float modes Tout is float: the hi plane is out[0, lo_off) and the lo
// plane out[lo_off, 2 lo_off); aux is the FP64 u of HS_MODE_DF_FINAL.
#include "hs_df.cuh"
template <typename Tout, int MODE>
__device__ __forceinline__ void hs_emit(Tout *out, double *aux, size_t lo_off, size_t idx,
                                        double v) {
    if constexpr (MODE == HS_MODE_WRITE) {
        out[idx] = (Tout)v;
    } else if constexpr (MODE == HS_MODE_ADD) {
        out[idx] += (Tout)v;
    } else if constexpr (MODE == HS_MODE_DF_SET) {
        out[idx] = (float)v;
        out[idx + lo_off] = 0.f;
    } else {
        dfloat a;
        a.hi = out[idx];
        a.lo = MODE == HS_MODE_DF_FINAL_HI ? 0.f : out[idx + lo_off];
        dfloat b;
        b.hi = (float)v;
        b.lo = 0.f;
        const dfloat s = df_add(a, b);
        if constexpr (MODE == HS_MODE_DF_ADD) {
            out[idx] = s.hi;
            out[idx + lo_off] = s.lo;
        } else {
            aux[idx] = (double)s.hi + (double)s.lo;
        }
    }
}
