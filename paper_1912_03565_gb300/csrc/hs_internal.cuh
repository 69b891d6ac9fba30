// Internal declarations shared by the solver's translation units.
#pragma once

#include <cuda_runtime.h>
#include <stddef.h>
#include <stdint.h>

#include "hs.h"

#define HS_MAX_STAGES 16
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

enum { HS_AXIS_X = 0, HS_AXIS_Y = 1 };
enum { HS_T_F64 = 0, HS_T_F32 = 1 };
enum { HS_MODE_WRITE = 0, HS_MODE_ADD = 1 };

// Device views of the boundary data of one solve (pointers already on device).
struct DevBoundary {
    const void *face[6];
    const void *fnn[6];
};

struct hs_plan_s {
    int Nx, Ny, Nz;
    double Lx, Ly, Lz, hx, hy, hz;
    int order, equation, precision, max_rhs;
    int refine_sweeps;
    int stage_timing;
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
    double *d_red;      // reduction scratch (64 doubles)

    // transform tables
    DstAxis axd[2];     // FP64 compute, x and y
    DstAxis axf[2];     // FP32 compute
    void *d_tables;     // one allocation behind every axis table

    // workspace
    double *d_w64;      // [Nz][Ny][Nx]: FP64 path data, or mixed-path lifted F
    float *d_w32;       // [Nz][Ny][Nx]: mixed-path FP32 work array
    double *d_dscr;     // [Nz][Ny][Nx]: mixed-path forward-sweep scratch

    // host staging (allocated on first use with host pointers)
    void *d_stage_f;
    size_t stage_f_bytes;
    double *d_stage_u;
    size_t stage_u_bytes;
    void *d_stage_bnd;
    size_t stage_bnd_bytes;

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
// FP64 out only).  `in` and `out` may alias (each block owns its tile).
hs_status hs_launch_dst(const hs_plan_s *P, int axis, int tc, int tin, const void *in, int tout,
                        void *out, int mode, double scale, cudaStream_t s);

// 1 when a line of this axis fits the transform kernel's shared memory.
int hs_dst_fits(const DstAxis &ax, int axis, int tc);

// Lifted right-hand side F (FP64, interior) from f.
hs_status hs_launch_rhs(const hs_plan_s *P, const void *f, int f_dtype, int rhs_kind,
                        const DevBoundary &b, double *F, cudaStream_t s);

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
// (scratch unused).  Mixed path: data is FP32 in place, forward sweep kept in
// the FP64 scratch.
hs_status hs_launch_thomas(const hs_plan_s *P, int tio, void *data, double *scratch,
                           cudaStream_t s);

// Per-row stencil coefficients C[l][nu][a,b,c,d] for rows l = 1..P->Nz
// (Sections 3.2-3.5).  Reads P's Nz, h, order and equation only; c0..c2 are
// host arrays indexed l = 0..Nz+1.
void hs_stencil_table(const hs_plan_s *P, const double *c0, const double *c1, const double *c2,
                      int cd_variant, double *C);
