/*
 * hs.h -- C ABI of the GB300 (sm_103a) separation-of-variables direct solver
 * for 27-point compact schemes of
 *
 *     Laplacian(u) + k(z)^2 u = f            (Helmholtz, 2nd/4th/6th order)
 *     Laplacian(u) + gamma(z) u_z = f        (convection-diffusion, 4th order)
 *
 * on a box with Dirichlet data on all six faces (arXiv 1912.03565: problem
 * statement eqs. (problem), (bc); schemes Sections 2 and 3.2-3.5; solver
 * Section 3.6).  A solve applies the compact right-hand-side operator, a 2-D
 * discrete sine transform (DST-I) along x then y, one tridiagonal system in z
 * per sine mode (p, q), and the inverse transform.
 *
 * Entry points: the single-problem plan (hs_plan ... hs_solve; FP64 and mixed
 * paths, refinement, autotuning, host-buffer staging), an allocation-free
 * residual (hs_residual_static), batches of uneven problems in one graph launch
 * (hs_batch_*), the solver as the preconditioner of BiCGStab for k^2(x, y, z)
 * (hs_precond_*), and the complex plan (hs_zplan_*, hs_zsolve*) for complex
 * k(z), Robin z-faces and Neumann side faces (the general problem of Section 1).
 *
 * Conventions shared by every entry point
 *  - Grids.  N_a interior points per axis, h_a = L_a / (N_a + 1) (Section 2).
 *    Interior arrays are C-ordered [l][j][i] (x fastest), the paper's row
 *    order i + Nx j + Nx Ny l (Section 3.1).  Node-grid arrays include the
 *    boundary nodes: [Nz+2][Ny+2][Nx+2].
 *  - Faces are numbered x-lo, x-hi, y-lo, y-hi, z-lo, z-hi.  Face arrays are
 *    full faces including edges: x-faces [Nz+2][Ny+2], y-faces [Nz+2][Nx+2],
 *    z-faces [Ny+2][Nx+2].  Where faces share an edge or corner node, the
 *    z-face value is used, then the y-face, then the x-face.
 *  - Pointers to bulk data (f, u, faces) may be device pointers or host
 *    pointers; host data are staged through plan-owned device buffers and
 *    copied on the given stream.  The caller keeps every buffer valid until
 *    the stream has passed the solve.
 *  - Errors are returned, never raised: no entry point aborts, traps or
 *    prints.  Negative codes are errors (the outputs are unspecified),
 *    positive codes are warnings (the outputs are valid).
 *  - Distinct plans may be used from distinct host threads concurrently; one
 *    plan must not be used by two threads at once.  The only global state
 *    is the fixed scratch of hs_residual_static and its per-device address.
 */
#ifndef HS_H
#define HS_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef int hs_status;

enum {
    HS_OK = 0,
    HS_WARN_NEAR_SINGULAR = 1,   /* min |pivot| / max |diag| < 1e-13 in some z-system */
    HS_WARN_NOT_CONVERGED = 2,   /* refinement ended above its tolerance (result valid) */
    HS_ERR_INVALID_ARG = -1,
    HS_ERR_UNSUPPORTED = -2,
    HS_ERR_OOM = -3,
    HS_ERR_CUDA = -4,
    HS_ERR_NO_COEFF = -5,        /* hs_solve before hs_set_coeff */
    HS_ERR_TIMEOUT = -6,         /* a bounded device-side wait gave up */
    HS_ERR_NONFINITE = -7
};

enum { HS_HELMHOLTZ = 0, HS_CONVDIFF = 1 };                 /* equation */
enum { HS_BC_DIRICHLET = 0 };                               /* boundary conditions */
enum { HS_FP64 = 0, HS_MIXED = 1 };                          /* precision path */
enum { HS_CD_PAPER = 0, HS_CD_CORRECTED = 1 };               /* CD coefficient variant */
enum { HS_F64 = 0, HS_F32 = 1 };                             /* element type of f / faces */
enum { HS_RHS_NODAL = 0, HS_RHS_ASSEMBLED = 1 };             /* meaning of f */
enum { HS_RESID_DF = 0, HS_RESID_F64 = 1, HS_RESID_AUTO = 2 }; /* refinement residual */
enum { HS_DST_STAGED = 0, HS_DST_FUSED = 1, HS_DST_GENERIC = 2,   /* transform kernels */
       HS_DST_TWOPASS = 3, HS_DST_FUSED_WIDE = 4, HS_DST_GEMM = 5, HS_DST_HALF = 6 };
enum { HS_AXIS_X = 0, HS_AXIS_Y = 1 };                       /* transform axis */
enum { HS_FACTOR_AUTO = 0, HS_FACTOR_F32 = 1, HS_FACTOR_F64 = 2 }; /* mixed z-solve factors */
enum { HS_HOST_F_MAPPED = 1, HS_HOST_U_MAPPED = 2, HS_HOST_F_EARLY = 4,     /* hs_set_host_io */
       HS_HOST_U_LATE = 8 };
enum { HS_THOMAS_PIPE16_256 = 0, HS_THOMAS_PIPE8_128 = 1,    /* FP32 z-solve mapping */
       HS_THOMAS_PLAIN16_256 = 2, HS_THOMAS_PIPE16_128 = 3, HS_THOMAS_BAL8_512 = 4,
       HS_THOMAS_BAL16_256 = 5 };

typedef struct hs_plan_s *hs_plan_t;

/* Dirichlet face values and, for the 6th-order right-hand side only, the
 * normal second derivative of f on each face (d2f/dx2 on the x-faces, ...).
 * Element type: the f_dtype of the solve.  NULL entries mean zero.  For a
 * multi-RHS solve the same boundary data apply to every right-hand side. */
typedef struct {
    const void *face[6];
    const void *fnn[6];
} hs_boundary;

#define HS_INFO_MAX_ITERS 8
#define HS_INFO_STAGES 8

/* Diagnostics of the last right-hand side of a solve.  Filling it makes the
 * solve synchronise the stream. */
typedef struct {
    int iterations;                          /* inverse applications (1 + refinements) */
    double rel_residual[HS_INFO_MAX_ITERS];  /* ||F - A U||_2 / ||F||_2 after each */
    double min_pivot_ratio;                  /* min |pivot| / max |diag| of the z-systems */
    float stage_ms[HS_INFO_STAGES];          /* device time per stage (stage timing on) */
} hs_info;

/* Stage indices of hs_info.stage_ms. */
enum {
    HS_STAGE_RHS = 0,        /* right-hand-side operator + Dirichlet lifting */
    HS_STAGE_DST_X = 1,      /* forward DST along x (all iterations) */
    HS_STAGE_DST_Y = 2,      /* forward DST along y */
    HS_STAGE_THOMAS = 3,     /* z-direction tridiagonal solves */
    HS_STAGE_IDST_Y = 4,     /* inverse DST along y */
    HS_STAGE_IDST_X = 5,     /* inverse DST along x (+ write / update of u) */
    HS_STAGE_RESIDUAL = 6,   /* refinement residual F - A U (mixed path) */
    HS_STAGE_TOTAL = 7
};

/*
 * hs_plan -- create a solver plan for one grid and scheme (Section 2 grid,
 * Sections 3.2-3.5 schemes).
 *   out         receives the plan handle (caller frees it with hs_destroy).
 *   Nx, Ny, Nz  interior points per axis, each >= 1.
 *   Lx, Ly, Lz  box lengths (> 0); h_a = L_a / (N_a + 1).
 *   order       2, 4 or 6 for HS_HELMHOLTZ; 4 for HS_CONVDIFF.  Order 6
 *               needs hx = hy = hz (relative difference <= 1e-12).
 *   equation    HS_HELMHOLTZ or HS_CONVDIFF.
 *   bc          HS_BC_DIRICHLET (the only one).
 *   precision   HS_FP64: every step in FP64.  HS_MIXED: FP32 transforms and
 *               z-solves (FP64 factors where the pivots call for them, see
 *               hs_set_factor_precision), the right-hand side and the iterate
 *               as FP32 pairs, and iterative refinement with an FP32-pair or
 *               FP64 residual (hs_set_residual_precision).
 *   max_rhs     largest nrhs a solve will pass (>= 1).
 * Allocates the plan's device tables and workspace on the current device.
 * Errors: HS_ERR_INVALID_ARG, HS_ERR_UNSUPPORTED, HS_ERR_OOM, HS_ERR_CUDA.
 */
hs_status hs_plan(hs_plan_t *out, int Nx, int Ny, int Nz, double Lx, double Ly, double Lz,
                  int order, int equation, int bc, int precision, int max_rhs);

/*
 * hs_set_coeff -- set the z-dependent coefficient and build the per-row
 * stencil coefficients {a,b,c,d} x {l-1,l,l+1} (Sections 3.2-3.5) and the
 * cached factorization of every z-system (Section 3.6: eigenvalues
 * lambda_nu(p,q) = 4 a_nu cos(th_p) cos(th_q) + 2 b_nu cos(th_p)
 * + 2 c_nu cos(th_q) + d_nu, LU without pivoting).
 *   c0, c1, c2  HOST arrays of length Nz+2 sampled at z_l = l hz, l = 0..Nz+1;
 *               copied.  Helmholtz: c0 = k^2, c1 = (k^2)', c2 = (k^2)''
 *               (c1, c2 may be NULL below order 6; for order 6 they are
 *               required and should be the exact derivatives).  CD: c0 =
 *               gamma, c1 = gamma', c2 = gamma'' (NULL = 0).
 *   cd_variant  HS_CD_CORRECTED (variable-gamma corrections, 4th order for
 *               gamma = gamma(z)) or HS_CD_PAPER (the printed coefficients
 *               with gamma frozen at row l); ignored for Helmholtz.
 * Synchronous.  Returns HS_WARN_NEAR_SINGULAR when some pivot ratio is
 * below 1e-13.  Errors: HS_ERR_INVALID_ARG, HS_ERR_NONFINITE (a sample is
 * NaN or infinite), both leaving the plan as it was; HS_ERR_CUDA, after which
 * the plan has no coefficients (hs_solve returns HS_ERR_NO_COEFF) until a
 * call succeeds.
 */
hs_status hs_set_coeff(hs_plan_t plan, const double *c0, const double *c1, const double *c2,
                       int cd_variant);

/*
 * hs_set_coeff_fn -- hs_set_coeff (Sections 3.2-3.5) from a function: c0, c1,
 * c2 are sampled as fn(z_l, 0, user), fn(z_l, 1, user), fn(z_l, 2, user) at z_l = l hz,
 * l = 0..Nz+1 (the coefficient and its first two z-derivatives: k^2 for
 * Helmholtz, gamma for convection-diffusion), on the calling thread, before
 * the call returns.  Same results and errors as hs_set_coeff.
 */
typedef double (*hs_coeff_fn)(double z, int deriv, void *user);
hs_status hs_set_coeff_fn(hs_plan_t plan, hs_coeff_fn fn, void *user, int cd_variant);

/*
 * hs_set_refinement -- number of refinement sweeps of the HS_MIXED path
 * after its first solve (default 2; 0..HS_INFO_MAX_ITERS-1).  Each sweep
 * computes the residual r = F - A U (precision: hs_set_residual_precision)
 * and adds the fast solve of r to U.  Ignored by the HS_FP64 path.  No paper
 * counterpart (the paper solves in FP64); each sweep reuses Section 3.6's solve.
 * Errors: HS_ERR_INVALID_ARG (sweeps outside that range).
 */
hs_status hs_set_refinement(hs_plan_t plan, int sweeps);

/*
 * hs_set_residual_precision -- arithmetic of the refinement residual (the
 * 27-point operator of eq. stencil27) of the HS_MIXED path (the iterate U and
 * F are kept as FP32 pairs either way):
 *   HS_RESID_DF   FP32-pair arithmetic, rounding ~2^-47 of the largest term;
 *   HS_RESID_F64  FP64 arithmetic (2^-53), about 2x the time of HS_RESID_DF;
 *   HS_RESID_AUTO (default) FP32-pair residuals while each shrinks the previous
 *                 one by at least 16x (||r_0|| = ||F||), FP64 from the sweep
 *                 after one that did not: the pair residual has reached its
 *                 floor (an FP32 correction solve contracts far more).
 *                 Decided on the device from the accumulated norms.
 * Errors: HS_ERR_INVALID_ARG.
 */
hs_status hs_set_residual_precision(hs_plan_t plan, int mode);

/*
 * hs_set_refinement_tol -- tolerance-controlled refinement of the HS_MIXED
 * path (no paper counterpart; the measure is Section 5.1's L2-res): iterative
 * refinement U_{m+1} = U_m + M (F - A U_m), stopped once
 * ||F - A U_m||_2 / ||F||_2 <= tol or after the hs_set_refinement count.
 * tol = 0 (default) runs the fixed count.  The decision is taken on the device
 * (no host synchronisation): the kernels of sweeps after convergence return
 * at once.  With hs_info the same test is made on the host.
 * Errors: HS_ERR_INVALID_ARG (tol < 0 or NaN).
 */
hs_status hs_set_refinement_tol(hs_plan_t plan, double tol);

/*
 * hs_set_transform_variant / hs_get_transform_variant -- the DST-I kernels of
 * one axis (HS_AXIS_X = 0, HS_AXIS_Y = 1; Section 3.6's transforms):
 *   HS_DST_STAGED  compile-time-sized FFT, every radix stage through shared
 *                  memory (line lengths N + 1 in {32,..,1024} of 2^a 3^b);
 *   HS_DST_FUSED   the same lengths, first stage loaded straight from global
 *                  memory and (x) the last stage paired by warp shuffles
 *                  (HS_MIXED plans only);
 *   HS_DST_GENERIC runtime-sized kernels (any length; the only choice for
 *                  lengths without compiled kernels);
 *   HS_DST_TWOPASS y only, HS_MIXED plans, N + 1 in {512, 768, 1024}: the FFT
 *                  split M = 32 M2 over two kernels, every access a whole
 *                  128-byte row segment of 32 columns; allocates a complex
 *                  scratch of 8 bytes per unknown while selected;
 *   HS_DST_FUSED_WIDE  HS_DST_FUSED with twice the lines per CTA (for y,
 *                  longer row segments per access), for the lengths whose
 *                  tile then still runs its stages in one shared buffer
 *                  (HS_ERR_UNSUPPORTED for the others);
 *   HS_DST_GEMM    HS_MIXED plans, N + 1 in {32, 64, 96, 128, 192, 256}: the
 *                  transform as a product with the sine matrix on the tensor
 *                  cores (Section 3.6's V^T F_l; tcgen05 MMA, FP16 x 2 split
 *                  operands, FP32 accumulation in tensor memory, each line
 *                  scaled by a power of two first), accurate to about 2^-22 of
 *                  each line's largest value like an FP32 FFT; allocates the
 *                  split sine matrix (at most 256 KB per axis).  A kernel whose
 *                  bounded internal wait gave up makes the next synchronous
 *                  call (hs_solve with info, hs_autotune) return HS_ERR_TIMEOUT.
 *   HS_DST_HALF    HS_FP64 plans, N + 1 in {32, 64, 96, 128, 192, 256, 384,
 *                  512, 768, 1024}: the transform through one complex FFT of
 *                  (N + 1) / 2 points per line (the real sequence
 *                  sin(pi j/M)(x_j + x_{M-j}) + (x_j - x_{M-j})/2, M = N + 1,
 *                  whose DFT gives the even outputs directly and the odd ones
 *                  by a running sum): about half the FP64 arithmetic of
 *                  HS_DST_STAGED, error growing like the running sum's.
 * Results agree to rounding.  Default: HS_DST_STAGED where compiled.
 * Errors: HS_ERR_INVALID_ARG; HS_ERR_UNSUPPORTED (variant not built for this
 * length, axis or precision); HS_ERR_OOM.
 */
hs_status hs_set_transform_variant(hs_plan_t plan, int axis, int variant);
hs_status hs_get_transform_variant(hs_plan_t plan, int axis, int *variant);

/*
 * hs_set_thomas_variant / hs_get_thomas_variant -- thread mapping of the FP32
 * z-solves of an HS_MIXED plan (Section 3.6's per-mode LU; one thread per
 * (p,q) column, z walked in chunks): HS_THOMAS_PIPE16_256 (default: 16-plane
 * chunks, the next chunk's loads issued before the current chunk's chain,
 * 256-thread blocks), HS_THOMAS_PIPE8_128, HS_THOMAS_PLAIN16_256 (no
 * pipelining, fewer registers), HS_THOMAS_PIPE16_128, and the balanced
 * mappings HS_THOMAS_BAL8_512 / HS_THOMAS_BAL16_256 (8- or 16-plane chunks; a
 * whole number of blocks per SM with the columns shared evenly among them,
 * blocks of at most 512 / 256 threads).  Identical results.
 * Errors: HS_ERR_INVALID_ARG.
 */
hs_status hs_set_thomas_variant(hs_plan_t plan, int variant);
hs_status hs_get_thomas_variant(hs_plan_t plan, int *variant);

/*
 * hs_autotune -- times one forward transform pass per supported variant and
 * axis (`reps` rounds after one untimed; for x of an HS_MIXED plan a round is a
 * forward pass plus the two inverse passes of a refined solve, pair set and
 * final u) on the plan's own work buffers (overwritten) on `stream`, and keeps
 * the fastest
 * variant of each axis; *ms_x, *ms_y (may be NULL) receive the kept variants'
 * times per round.  For an
 * HS_MIXED plan whose coefficients are set and whose factors are FP32, the
 * z-solve mappings are timed the same way and the fastest kept.
 * Synchronous.  Call after hs_set_coeff, before solves (not during capture).
 * The choices are kept in the process-wide autotune cache, keyed by device
 * (name, SM count), Nx, Ny, Nz, order, equation, precision and factor type;
 * a later hs_autotune of a plan with the same key takes them (and the stored
 * times) without timing.  hs_autotune_cache_clear forces fresh timing.
 * Errors: HS_ERR_INVALID_ARG (reps < 1), HS_ERR_CUDA.
 */
hs_status hs_autotune(hs_plan_t plan, void *stream, int reps, float *ms_x, float *ms_y);

/*
 * Autotune cache (no paper counterpart; host only, thread-safe):
 *   hs_autotune_cache_save(path)  writes every entry to a text file, one line
 *       per key: "<device> <sms> <Nx> <Ny> <Nz> <order> <equation> <precision>
 *       <f32_factors> <variant_x> <variant_y> <thomas_variant> <ms_x> <ms_y>"
 *       after a '#' header line (-1 where a field does not apply);
 *   hs_autotune_cache_load(path)  merges a file written that way (later
 *       entries win); a malformed or out-of-range line merges nothing;
 *   hs_autotune_cache_clear()     empties the cache;
 *   hs_autotune_cache_count(&n)   number of entries.
 * Errors: HS_ERR_INVALID_ARG (NULL argument, unreadable / unwritable file,
 * malformed content).
 */
hs_status hs_autotune_cache_save(const char *path);
hs_status hs_autotune_cache_load(const char *path);
hs_status hs_autotune_cache_clear(void);
hs_status hs_autotune_cache_count(int *count);

/*
 * hs_set_factor_precision -- the factors of the mixed path's z-solves
 * (Section 3.6's LU of each mode's tridiagonal system): HS_FACTOR_F32 (FP32
 * factors and sweep, 20 bytes moved per unknown), HS_FACTOR_F64 (FP64 factors,
 * FP64 forward sweep kept in an FP64 scratch: a more accurate correction solve,
 * which can save a refinement sweep, for 32 more bytes of plan memory per
 * unknown), HS_FACTOR_AUTO (default: FP32 unless some z-system has min pivot
 * ratio < 1e-4).  On GB300 at 1023^3 FP64 factors lowered the unrefined error
 * (9.2e-6 -> 4.2e-7) but not the refined one, which the residual's rounding
 * bounds.  May be called before or after hs_set_coeff (refactors).
 * Ignored by the HS_FP64 path.  Errors: HS_ERR_INVALID_ARG, HS_ERR_OOM.
 */
hs_status hs_set_factor_precision(hs_plan_t plan, int mode);

/*
 * hs_set_host_io -- how hs_solve moves host buffers f and u (flags, default 0).
 * Pageable host buffers are staged: f is copied into a plan-owned device buffer
 * -- a nodal f in z-chunks on a second stream, each slab of the right-hand-side
 * kernel starting as soon as its planes have arrived, so copy and kernel
 * overlap -- and u is copied back.  Flags:
 *   HS_HOST_F_MAPPED  a pinned f is read in place by the right-hand-side kernel
 *                     through its device alias (no staging);
 *   HS_HOST_U_MAPPED  a pinned u is written in place by the last transform pass;
 *   HS_HOST_F_EARLY   the copies of a staged f and of host boundary arrays do
 *                     not wait for the work queued before the call on the
 *                     stream, only until the solve before the previous one has
 *                     read the plan's staging buffers (two sets, used in turn),
 *                     so they overlap the previous solve; the right-hand-side
 *                     kernel then runs as one launch after the whole copy.  Use
 *                     only when no work queued on the stream writes those host
 *                     arrays (for example arrays filled by the CPU).
 *   HS_HOST_U_LATE    the copy of a staged u back to the host runs on a
 *                     plan-owned stream after the solve, so it overlaps the work
 *                     queued after the call (the next solve); two device staging
 *                     buffers of u are used in turn.  The host u is complete only
 *                     once a stream made to wait by hs_host_io_wait has reached
 *                     that point (or after cudaDeviceSynchronize).  Solves called
 *                     with an hs_info copy back on the caller's stream as usual.
 * On GB300, 255^3, 6th order, pinned host buffers, back-to-back solves: 2.51 ms
 * per solve staged (2.66 ms copying f whole), 2.22 ms with HS_HOST_F_EARLY; in
 * place: 2.94 (u), 3.19 (f), 3.47 ms (both) -- the kernels' access pattern over
 * the host link costs more than one bulk copy.  Errors: HS_ERR_INVALID_ARG.
 */
hs_status hs_set_host_io(hs_plan_t plan, int mapped);

/*
 * hs_host_io_wait -- makes `stream` wait (without blocking the host) until
 * every copy of u to the host queued by HS_HOST_U_LATE solves of this plan is
 * done.  A no-op when none was queued.  Errors: HS_ERR_INVALID_ARG, HS_ERR_CUDA.
 */
hs_status hs_host_io_wait(hs_plan_t plan, void *stream);

/*
 * hs_set_stage_timing -- when on (1), solves record CUDA events around each
 * stage launch (no synchronisation is added); hs_stage_times and
 * hs_info.stage_ms report them.  Off (0) by default.
 * Errors: HS_ERR_INVALID_ARG (NULL plan).
 */
hs_status hs_set_stage_timing(hs_plan_t plan, int on);

/*
 * hs_solve -- solve A U = F for nrhs right-hand sides on `stream`.
 *   f          rhs_kind HS_RHS_NODAL: f on the node grid, [nrhs][Nz+2][Ny+2][Nx+2];
 *              the library applies the scheme's right-hand-side operator
 *              (2nd: hz^2 f; 4th: hz^2 f^(IV), eq. (scheme4); 6th: hz^2 f^(VI),
 *              eq. (scheme6) with explicit differences; CD: eq. (cd_rhs)).
 *              HS_RHS_ASSEMBLED: F on the interior, [nrhs][Nz][Ny][Nx]
 *              (the operator already applied).  Element type f_dtype.
 *   bnd        Dirichlet and 6th-order face data (NULL = all zero).
 *   u          output, FP64, interior [nrhs][Nz][Ny][Nx].
 *   stream     a cudaStream_t (NULL = the legacy default stream).
 *   info       NULL: the call is asynchronous.  Non-NULL: the call
 *              synchronises and fills the diagnostics of the last RHS; it
 *              first counts the NaN or infinite values of f (hs_check_finite
 *              for device f, a host scan for host f) and returns
 *              HS_ERR_NONFINITE, u untouched, if there are any.
 * nrhs must be between 1 and max_rhs.  Errors: HS_ERR_INVALID_ARG,
 * HS_ERR_NO_COEFF, HS_ERR_NONFINITE (info mode), HS_ERR_CUDA, HS_ERR_OOM
 * (host staging).
 */
hs_status hs_solve(hs_plan_t plan, const void *f, int f_dtype, int rhs_kind,
                   const hs_boundary *bnd, double *u, int nrhs, void *stream, hs_info *info);

/*
 * hs_check_finite -- *count = the number of NaN or infinite values among the n
 * elements (dtype HS_F64 or HS_F32) of the DEVICE array data: a right-hand
 * side, face data or a result (input validation; the paper's data are finite).
 * One pass with a device reduction on `stream`, then a synchronisation.  The
 * count is kept in the plan's scratch, so checks are ordered with the plan's
 * other work on the same stream.  Errors: HS_ERR_INVALID_ARG (NULL plan or
 * count, host pointer, other dtype), HS_ERR_CUDA.
 */
hs_status hs_check_finite(hs_plan_t plan, const void *data, int dtype, size_t n, void *stream,
                          unsigned long long *count);

/*
 * hs_residual -- ||F - A U||_2 and ||F||_2 of a computed solution, in FP64,
 * for one right-hand side given as in hs_solve (L2-res of Section 5.1).
 * Synchronous.  Device or host pointers.  Errors: HS_ERR_INVALID_ARG,
 * HS_ERR_NO_COEFF, HS_ERR_OOM (host staging), HS_ERR_CUDA.
 */
hs_status hs_residual(hs_plan_t plan, const void *f, int f_dtype, int rhs_kind,
                      const hs_boundary *bnd, const double *u, void *stream,
                      double *res_norm, double *rhs_norm);

/*
 * hs_rhs_apply -- the lifted right-hand side F of one right-hand side exactly
 * as a solve forms it: the scheme's operator R_h applied to f (eqs. scheme4,
 * scheme6, cd_rhs; hz^2 f at 2nd order) minus the Dirichlet lifting (problem
 * statement eq. (bc)), or an assembled F copied (HS_RHS_ASSEMBLED, lifting
 * still applied).  f, F: DEVICE pointers (host pointers return
 * HS_ERR_INVALID_ARG); bnd as for hs_solve.  F: FP64 plan -> FP64
 * [Nz][Ny][Nx]; HS_MIXED plan -> the FP32 pair the mixed path works with, two
 * planes [2][Nz][Ny][Nx] (hi, then lo; F = hi + lo).  Asynchronous on
 * `stream`.  Errors: HS_ERR_INVALID_ARG, HS_ERR_NO_COEFF, HS_ERR_OOM (host
 * boundary staging), HS_ERR_CUDA.
 */
hs_status hs_rhs_apply(hs_plan_t plan, const void *f, int f_dtype, int rhs_kind,
                       const hs_boundary *bnd, void *F, void *stream);

/*
 * hs_fp64_fma_rate -- the current device's FP64 fused multiply-add throughput
 * in TFLOP/s (2 flops per FMA), measured with independent DFMA chains on every
 * SM and timed with CUDA events on `stream` (synchronous; about 10 ms).  No
 * paper counterpart: the peak against which the FP64 transforms are reported.
 * Errors: HS_ERR_INVALID_ARG, HS_ERR_CUDA.
 */
hs_status hs_fp64_fma_rate(void *stream, double *tflops);

/*
 * hs_stage_times -- device time per stage (ms[HS_INFO_STAGES], indexed by
 * HS_STAGE_*) summed over the last hs_solve on this plan, when stage timing
 * was on; HS_STAGE_TOTAL is the whole call.  Waits for that solve's events.
 * Errors: HS_ERR_INVALID_ARG (NULL, or timing never on), HS_ERR_CUDA.
 */
hs_status hs_stage_times(hs_plan_t plan, float *ms);

/*
 * hs_residual_static -- ||F - A U||_2 and ||F||_2 for an assembled, lifted
 * right-hand side F (zero Dirichlet data), WITHOUT allocating anything.
 * The paper has no counterpart: this is a library convenience.  It exists for
 * callers that cannot call cudaMalloc -- code whose device memory belongs to
 * its own pool allocator or framework, plugins limited to the buffers they
 * are handed, loops that must not allocate -- and that want to check an
 * iterate without creating a plan (hs_plan allocates its workspace).
 *   Nx..Lz, order, equation, cd_variant, c0..c2  as for hs_plan/hs_set_coeff
 *               (c0..c2 HOST arrays of length Nz+2; order 6 uses h = Lz/(Nz+1)).
 *   F, u       DEVICE arrays [Nz][Ny][Nx] (FP64); host pointers are rejected.
 *   stream     cudaStream_t (NULL = legacy default stream).
 *   res_norm, rhs_norm  host outputs.
 * Scratch: one file-scope device array of fixed size (the coefficient table
 * of up to HS_STATIC_MAX_NZ rows plus partial sums, about 0.8 MB) that every
 * GPU loading the library holds until exit.  Nz > HS_STATIC_MAX_NZ returns
 * HS_ERR_UNSUPPORTED.  The first call on each device looks up the array's
 * device address (cudaGetSymbolAddress) with that device current.  Every call
 * copies the coefficient table from host memory and synchronises the stream,
 * so it must not be made on a stream that is being captured (a capturing
 * stream returns HS_ERR_INVALID_ARG).  Calls share the array: calls that
 * overlap on the GPU (other streams, other host threads) race and must be
 * serialised by the caller.  Synchronous: returns after the norms are read.
 * F and u must be memory of the current device (or managed memory).  Order 6
 * needs hx = hy = hz (as hs_plan).  Errors: HS_ERR_INVALID_ARG,
 * HS_ERR_UNSUPPORTED, HS_ERR_NONFINITE (c0..c2), HS_ERR_CUDA.
 */
#define HS_STATIC_MAX_NZ 8192
hs_status hs_residual_static(int Nx, int Ny, int Nz, double Lx, double Ly, double Lz, int order,
                             int equation, int cd_variant, const double *c0, const double *c1,
                             const double *c2, const double *F, const double *u, void *stream,
                             double *res_norm, double *rhs_norm);

/* ---------------------------------------------------------------- batches
 * Many independent problems solved by the HS_MIXED path in ONE persistent
 * kernel launch (captured in a CUDA graph): uneven sizes, their own
 * coefficient profiles and 1..16 right-hand sides each.  Persistent CTAs take
 * (problem, RHS, stage, tile) work items from a queue and wait -- bounded --
 * for the previous stage of the same problem and RHS.  No paper counterpart
 * (the paper solves one problem at a time); Section 3.6 is the per-problem
 * solve.  Transform lengths N_x + 1 and N_y + 1 must be in
 * {32, 64, 96, 128, 192, 256, 384}. */
typedef struct hs_batch_s *hs_batch_t;

typedef struct {
    int Nx, Ny, Nz;          /* as hs_plan */
    double Lx, Ly, Lz;
    int order, equation, cd_variant;
    const double *c0, *c1, *c2;   /* HOST profiles (as hs_set_coeff), copied */
    int nrhs;                /* 1..16 */
    const void *f;           /* DEVICE, [nrhs][Nz+2][Ny+2][Nx+2] nodal f of the batch's f_dtype */
    double *u;               /* DEVICE, [nrhs][Nz][Ny][Nx] FP64 output */
} hs_problem_desc;

/*
 * hs_batch_create -- plan every problem (tables, cached factorization,
 * workspace per RHS) and the work-item list.  sweeps: refinement sweeps of
 * every solve (0..HS_INFO_MAX_ITERS-1).  Synchronous; allocates.
 * Errors: HS_ERR_INVALID_ARG, HS_ERR_UNSUPPORTED (a transform length outside
 * the set above), HS_ERR_OOM, HS_ERR_CUDA.
 */
hs_status hs_batch_create(hs_batch_t *out, const hs_problem_desc *probs, int nprob, int f_dtype,
                          int sweeps);

/* hs_batch_set_io -- new f and u device pointers of problem k (same layout).
 * Errors: HS_ERR_INVALID_ARG (k out of range, NULL), HS_ERR_CUDA. */
hs_status hs_batch_set_io(hs_batch_t batch, int k, const void *f, double *u);

/*
 * hs_batch_solve -- one graph launch solving every problem of the batch on
 * `stream` (the graph is built on the first call for a stream).  sync = 0:
 * asynchronous; sync = 1: waits and returns HS_ERR_TIMEOUT if a bounded wait
 * inside the launch gave up (the results are then incomplete).
 * Errors: HS_ERR_INVALID_ARG, HS_ERR_TIMEOUT, HS_ERR_OOM and HS_ERR_CUDA
 * (building or launching the graph).
 */
hs_status hs_batch_solve(hs_batch_t batch, void *stream, int sync);

/* hs_batch_set_wait_limit -- spin iterations (about 100 ns each) before a wait
 * inside the launch gives up (default 2e7).  Errors: HS_ERR_INVALID_ARG
 * (spins < 1). */
hs_status hs_batch_set_wait_limit(hs_batch_t batch, long long spins);

/*
 * Preconditioner mode (the use the paper's introduction names): solve
 * A(K) x = F for a Helmholtz coefficient K = k^2 that varies in x, y and z,
 * by BiCGStab (van der Vorst) preconditioned from the right with the solve of
 * a plan whose separable coefficient K_ref(z) approximates K (for instance the
 * plane means).  A(K) is the compact scheme of the plan's order (2 or 4) for a
 * general coefficient, zero Dirichlet data, scaled by h_z^2 like the Section
 * 3.3 coefficients (for K = K(z) it is the plan's own 27-point operator):
 *   4th order: h_z^2 [ Lap_h x + sum_{a<b} (h_a^2 + h_b^2)/12 d_a^2 d_b^2 x
 *                      + K_c x_c / 2 + (1/12) sum_{6 face neighbours} K x ]
 *   2nd order: h_z^2 [ Lap_h x + K_c x_c ]
 * All vectors are FP64 device arrays of Nx Ny Nz interior values [z][y][x].
 */
typedef struct hs_precond_s *hs_precond_t;

#define HS_PRECOND_MAX_HIST 64
typedef struct {
    int iterations;                          /* BiCGStab iterations done */
    double rel_residual;                     /* ||F - A x|| / ||F|| (recurrence) at exit */
    double history[HS_PRECOND_MAX_HIST];     /* the same after each iteration */
} hs_precond_info;

/* hs_precond_create -- workspace (8 FP64 vectors) for `plan` (HELMHOLTZ, order
 * 2 or 4, coefficients set: they are K_ref) and the device coefficient field K
 * (Nx Ny Nz FP64, not copied: it must outlive the object).
 * Errors: HS_ERR_INVALID_ARG, HS_ERR_UNSUPPORTED (order 6, CD), HS_ERR_NO_COEFF,
 * HS_ERR_OOM. */
hs_status hs_precond_create(hs_precond_t *out, hs_plan_t plan, const double *K);

/* hs_precond_apply -- y = A(K) u, the operator above (device FP64 arrays,
 * asynchronous on stream).
 * Errors: HS_ERR_INVALID_ARG, HS_ERR_CUDA. */
hs_status hs_precond_apply(hs_precond_t pc, const double *u, double *y, void *stream);

/* hs_precond_solve -- BiCGStab with the Section 3.6 solve as preconditioner
 * (Section 1's use): x (device FP64, in: initial guess, out: solution) for the
 * assembled right-hand side F; stops at ||F - A x|| / ||F|| <= tol or after maxit
 * iterations (HS_WARN_NOT_CONVERGED, x valid).  Each iteration applies A twice
 * and the plan's solve twice (hs_solve with HS_RHS_ASSEMBLED on `stream`) and
 * synchronises the stream for its four reductions.  HS_ERR_NONFINITE on a
 * BiCGStab breakdown or a NaN.  info may be NULL.  Errors: HS_ERR_INVALID_ARG
 * (NULL, tol < 0 or NaN, maxit < 1), HS_ERR_NONFINITE, HS_ERR_CUDA, and those
 * of hs_solve. */
hs_status hs_precond_solve(hs_precond_t pc, const double *F, double *x, double tol, int maxit,
                           void *stream, hs_precond_info *info);

/* hs_precond_destroy -- free the workspace (K stays the caller's; NULL is
 * accepted).  Returns HS_OK. */
hs_status hs_precond_destroy(hs_precond_t pc);

/* hs_batch_set_tol -- tolerance-controlled refinement per problem and RHS:
 * each stops once ||F - A U||_2 / ||F||_2 <= tol (decided on the device) or
 * after the batch's sweep count; 0 (default) runs every sweep.  Errors:
 * HS_ERR_INVALID_ARG (tol < 0 or NaN). */
hs_status hs_batch_set_tol(hs_batch_t batch, double tol);

/* hs_batch_set_residual_precision -- as hs_set_residual_precision, for every
 * (problem, RHS) of the batch, each deciding on its own (default AUTO).
 * Errors: HS_ERR_INVALID_ARG. */
hs_status hs_batch_set_residual_precision(hs_batch_t batch, int mode);

/* hs_batch_set_variant / hs_batch_get_variant -- the persistent kernel
 * variant: 0 = staged transform tiles, registers capped for 2 resident CTAs
 * (256 threads) per SM; 1 = staged, capped for 3; 2 = fused transform tiles
 * (first stage from global memory, x pairing by shuffles), 2 CTAs; 3 = fused,
 * 3 CTAs; 4 = no persistent kernel: every problem's stand-alone mixed solve
 * (one per RHS) captured into one graph on up to 8 parallel branches, each
 * stage at its own kernel's occupancy (grid reported as 1).  For 0-3 the grid
 * is every CTA the variant can keep resident.  Default: the first persistent
 * variant that fits.  Errors: HS_ERR_INVALID_ARG; HS_ERR_UNSUPPORTED (variant
 * cannot be resident with this batch's shared memory). */
hs_status hs_batch_set_variant(hs_batch_t batch, int variant);
hs_status hs_batch_get_variant(hs_batch_t batch, int *variant, int *grid);

/* hs_batch_graph_kernels -- kernel launches per hs_batch_solve: the kernel
 * nodes of the captured graph (0 before the first solve of the variant).
 * Errors: HS_ERR_INVALID_ARG. */
hs_status hs_batch_graph_kernels(hs_batch_t batch, int *kernels);

/* hs_batch_autotune -- times `reps` solves of the batch (after one warm-up)
 * with each kernel variant on `stream` and keeps the fastest; *ms (may be
 * NULL) receives its mean time per solve.  The solves write the outputs u.
 * Synchronous.  Errors: HS_ERR_INVALID_ARG (reps < 1), HS_ERR_UNSUPPORTED (no
 * variant fits), HS_ERR_TIMEOUT, HS_ERR_OOM, HS_ERR_CUDA. */
hs_status hs_batch_autotune(hs_batch_t batch, void *stream, int reps, float *ms);

/* hs_batch_debug_stall -- test hook: on = 1 makes one dependency of the first
 * problem unsatisfiable, so the next solve must end with HS_ERR_TIMEOUT; on =
 * 0 restores it.  Errors: HS_ERR_INVALID_ARG, HS_ERR_CUDA. */
hs_status hs_batch_debug_stall(hs_batch_t batch, int on);

/* hs_batch_workspace_bytes -- device bytes owned by the batch. */
size_t hs_batch_workspace_bytes(hs_batch_t batch);

/* hs_batch_destroy -- free a batch (NULL accepted).  Synchronises the device. */
hs_status hs_batch_destroy(hs_batch_t batch);

/* hs_workspace_bytes -- device bytes owned by the plan (tables, cached
 * factorization, workspace). */
size_t hs_workspace_bytes(hs_plan_t plan);

/* hs_destroy -- free a plan (NULL is accepted).  Synchronises the device. */
hs_status hs_destroy(hs_plan_t plan);

/* hs_status_str -- static text for a status code. */
const char *hs_status_str(hs_status s);

/* hs_last_error -- text of the last error seen on this plan (never NULL). */
const char *hs_last_error(hs_plan_t plan);

/* ---------------------------------------------------------------------------
 * Complex k(z) and Robin z-faces (FP64; Helmholtz, orders 2 and 4).
 *
 * The general problem of Section 1 (eqs. (problem), (bc)): K = k^2 complex and
 * depending on z only, u = 0 on the four side faces, and on each z-face either
 * u = g (Dirichlet) or alpha u_z + beta u = g (Robin) with complex alpha, beta
 * and complex face data g(x, y).  Interior rows l = 1..Nz are the compact rows
 * of Sections 3.2 (order 2) and 3.3 (order 4) with complex K.  The paper gives
 * no compact closure of a Robin face: a Robin face's plane (l = 0 or Nz + 1)
 * is unknown and its row is the second-order 7-point scheme
 * h_z^2 (dxx + dyy + dzz + K) u = h_z^2 f with the plane outside eliminated by
 * the central difference of the face condition, alpha (u_+1 - u_-1) / (2 h_z) +
 * beta u_0 = g.  The side faces stay Dirichlet, so Section 3.6 applies: the
 * real DSTs act on Re and Im, and each sine mode (p, q) is one complex
 * tridiagonal system in z, solved without pivoting; its LU factors are cached
 * (48 bytes per complex unknown), rebuilt by the first solve after a change of
 * coefficient, faces or side axes.
 *
 * A side axis (x or y) may instead carry u_n = g on both of its faces (the
 * extension Section 1 names; g = 0, or per-face data through hs_zsolve_ex):
 * its boundary nodes become unknowns, the ghost beyond a face is the even
 * reflection plus 2 h g (the central difference of u_n = g), f and the z-face
 * data are reflected evenly, and the cosine transform DCT-I over nodes 0..N+1
 * replaces the sine transform (modes cos(p pi i/(N+1)), p = 0..N+1, same
 * eigenvalue formula).
 *
 * The unknown grid of a plane is [ny][nx]: nx = Nx + 2 (nodes 0..Nx+1) for a
 * Neumann x-axis, else Nx (nodes 1..Nx); likewise ny.  Complex arrays are
 * planar: all real parts, then all imaginary parts.
 *   f:  [2][Nz+2][Ny+2][Nx+2]  on the node grid (device memory);
 *   g_lo, g_hi: [2][ny][nx]    on the unknown grid of the z-face (device
 *                              memory; NULL = 0); Dirichlet side faces are 0;
 *   u:  [2][Nz+2][ny][nx]      every plane (device memory): Dirichlet planes
 *                              receive g, the others the solution.
 * Scalars alpha, beta and the coefficient K are host (re, im) pairs.
 */
typedef struct hs_zplan_s *hs_zplan_t;
enum { HS_ZFACE_DIRICHLET = 0, HS_ZFACE_ROBIN = 1 };
enum { HS_SIDE_DIRICHLET = 0, HS_SIDE_NEUMANN = 1, HS_SIDE_DN = 2, HS_SIDE_ND = 3 };

/* hs_zplan -- plan for an Nx x Ny x Nz interior grid on [0,Lx]x[0,Ly]x[0,Lz]
 * (h_a = L_a / (N_a + 1)), order 2, 4 or 6 (6: Section 3.4's rows, uniform h,
 * |h_x - h_z| and |h_y - h_z| <= 1e-12 h_z, Dirichlet side faces, coefficients
 * through hs_zplan_set_coeff6).  Faces start Dirichlet.  Errors:
 * HS_ERR_INVALID_ARG, HS_ERR_UNSUPPORTED (transform length), HS_ERR_OOM,
 * HS_ERR_CUDA. */
hs_status hs_zplan(hs_zplan_t *out, int Nx, int Ny, int Nz, double Lx, double Ly, double Lz,
                   int order);

/* hs_zplan_set_coeff -- K = k^2 (Sections 3.2, 3.3 with complex K) at the
 * nodes l = 0..Nz+1: host array of Nz + 2
 * (re, im) pairs, copied.  Errors: HS_ERR_INVALID_ARG (NULL, non-finite, or an
 * order-6 plan, which needs hs_zplan_set_coeff6). */
hs_status hs_zplan_set_coeff(hs_zplan_t plan, const double *K);

/* hs_zplan_set_coeff6 -- K, K_z and K_zz at the nodes l = 0..Nz+1 (host arrays
 * of Nz + 2 (re, im) pairs each, copied).  Order 6: the rows of Section 3.4
 * evaluated in complex arithmetic (their coefficients are polynomials in K:
 * K^2 and K_z K terms), and the right-hand side's K terms
 * h^2 (-h^2 K_l f / 20 + h^3 K_z,l (f_{l+1} - f_{l-1}) / 120) (eq. scheme6 with
 * complex K).  Orders 2 and 4 read K only (K_z, K_zz may be NULL).
 * Errors: HS_ERR_INVALID_ARG (NULL where needed, non-finite). */
hs_status hs_zplan_set_coeff6(hs_zplan_t plan, const double *K, const double *Kz,
                              const double *Kzz);

/* hs_zplan_set_precision -- HS_FP64 (default: every step in FP64) or HS_MIXED:
 * the solve of Section 3.6 run in FP32 (FP32 transforms of the planar real
 * and imaginary parts, FP32 z-solves on the cached LU factors rounded to FP32)
 * as the approximate inverse M of an iterative refinement
 * U_0 = M F, U_{m+1} = U_m + M (F - A U_m), m < sweeps, with F, U and the
 * complex 27-point residual in FP32-pair arithmetic (the refined result is as
 * accurate as the FP64 path's to about 1e-10 after one sweep on well-conditioned
 * problems).  Side axes: Dirichlet (FP32 sine tiles), or Neumann on both faces
 * when N + 1 is 32, 64, 96, 128, 192 or 256 (FP32 half-length cosine tile, whose
 * unrefined error grows like (N + 1) eps, 4e-6 at 256); longer Neumann axes and
 * one face of each kind have no FP32 tile (HS_ERR_UNSUPPORTED, and set_sides
 * then refuses such kinds); sweeps 0..8.  The mixed solve allocates, on first use,
 * 20 bytes per complex unknown (FP32 work, FP64 iterate) and 24 for the FP32
 * factors.  Stage timing reports the refinement loop as the transform stage.
 * Errors: HS_ERR_INVALID_ARG, HS_ERR_UNSUPPORTED. */
hs_status hs_zplan_set_precision(hs_zplan_t plan, int precision, int sweeps);

/* hs_zplan_set_faces -- kind (HS_ZFACE_DIRICHLET / HS_ZFACE_ROBIN, eq. bc) of
 * the z-lo and z-hi faces; alpha, beta: host (re, im) pairs, read for Robin faces only
 * (alpha != 0 there).  Errors: HS_ERR_INVALID_ARG, HS_ERR_OOM. */
hs_status hs_zplan_set_faces(hs_zplan_t plan, int lo_kind, const double *alpha_lo,
                             const double *beta_lo, int hi_kind, const double *alpha_hi,
                             const double *beta_hi);

/* hs_zsolve_ex -- hs_zsolve with data on Neumann side faces (Section 1):
 * side[0..3] are the outward normal derivative u_n = g on the x-lo, x-hi
 * faces ([2][Nz+2][Ny+2], planar complex, on the face node grid: planes l,
 * nodes j = 0..Ny+1) and the y-lo, y-hi faces ([2][Nz+2][Nx+2]); NULL entries
 * (or side = NULL) are 0.  The
 * ghost beyond such a face is the mirror value plus 2 h g (second-order
 * central difference), a face's data reflected evenly beyond its own edges.
 * Data on a Dirichlet face (either face of a Dirichlet axis, the low face of an
 * HS_SIDE_DN axis, the high face of an HS_SIDE_ND axis) are rejected
 * (HS_ERR_INVALID_ARG).
 * Other errors as hs_zsolve. */
hs_status hs_zsolve_ex(hs_zplan_t plan, const double *f, const double *g_lo, const double *g_hi,
                       const double *const *side, double *u, void *stream);

/* hs_zsolve_full -- hs_zsolve_ex with the face data of the 6th-order
 * right-hand side: fnn[0..5] are the normal second derivatives f_nn on the
 * x-lo, x-hi ([2][Nz+2][Ny+2]), y-lo, y-hi ([2][Nz+2][Nx+2]) and z-lo, z-hi
 * ([2][Ny+2][Nx+2]) faces, planar complex device arrays on the face node grids
 * (NULL entries, or fnn = NULL, are 0).  They enter the ghost nodes one step
 * beyond a face, f_{-1} = 2 f_0 - f_1 + h^2 (f_nn)_face, that the R6 operator's
 * second neighbours reach (eq. scheme6; the paper's cited compact closure is
 * replaced by this explicit one).  Orders 2 and 4 ignore fnn.
 * Errors: as hs_zsolve_ex. */
hs_status hs_zsolve_full(hs_zplan_t plan, const double *f, const double *g_lo,
                         const double *g_hi, const double *const *side,
                         const double *const *fnn, double *u, void *stream);

/* hs_zplan_set_sides -- kind of the x and y side axes (Section 1; default
 * Dirichlet): HS_SIDE_DIRICHLET (u = 0 on both faces, nodes 1..N unknown),
 * HS_SIDE_NEUMANN (u_n = g on both faces, nodes 0..N+1, cosine transform DCT-I),
 * HS_SIDE_DN (u = 0 on the low face, u_n = g on the high face, nodes 1..N+1) or
 * HS_SIDE_ND (u_n = g on the low face, u = 0 on the high face, nodes 0..N);
 * the last two take the quarter-wave transforms (modes of angle
 * (2p - 1) pi / (2 (N + 1)), p = 1..N+1), computed as the sine transform of the
 * line extended evenly about its Neumann node to 2N + 1 points (an internal
 * plan: about twice the x or y work array).  N + 1 (Neumann) or 2 (N + 1)
 * (mixed) in {32, 64, 96, 128, 192, 256, 384, 512, 768, 1024} run the compiled
 * FFT tiles; other lengths run runtime-sized transforms (the cosine transform
 * by direct sums, O(N^2) per line, lines of at most about 3000 nodes).  The
 * unknown grid is nx = Nx, Nx + 2 or Nx + 1 nodes by the kind, and likewise ny.
 * Errors: HS_ERR_INVALID_ARG (kind), HS_ERR_UNSUPPORTED (no transform for the
 * length; an order-6 plan with other than Dirichlet sides; an HS_MIXED plan with
 * kinds hs_zplan_set_precision refuses), HS_ERR_OOM; on error the previous kinds
 * stay in effect. */
hs_status hs_zplan_set_sides(hs_zplan_t plan, int x_kind, int y_kind);

/* hs_zsolve -- one solve (Section 3.6 with complex rows) on `stream`
 * (asynchronous; the caller keeps f, g and u valid until the stream has
 * passed it).  Errors: HS_ERR_INVALID_ARG (NULL
 * f or u, host pointers), HS_ERR_NO_COEFF (no coefficients yet, or an earlier
 * hs_zplan_set_faces / hs_zplan_set_sides failed part-way: repeat it),
 * HS_ERR_CUDA. */
hs_status hs_zsolve(hs_zplan_t plan, const double *f, const double *g_lo, const double *g_hi,
                    double *u, void *stream);

/* hs_zplan_set_stage_timing -- when on (1), each hs_zsolve records CUDA events
 * on its stream around its stages; hs_zplan_stage_times then waits for the
 * last solve's events and writes the milliseconds of its 5 stages to ms[0..4]:
 * right-hand side, forward transforms (x and y), z-solves, inverse transforms,
 * output copies.  Errors: HS_ERR_INVALID_ARG (timing never switched on),
 * HS_ERR_CUDA. */
hs_status hs_zplan_set_stage_timing(hs_zplan_t plan, int on);
hs_status hs_zplan_stage_times(hs_zplan_t plan, float *ms);

/* Device workspace of the plan in bytes, its last error text, and its release. */
size_t hs_zplan_workspace_bytes(hs_zplan_t plan);
const char *hs_zplan_last_error(hs_zplan_t plan);
void hs_zplan_destroy(hs_zplan_t plan);

#ifdef __cplusplus
}
#endif

#endif /* HS_H */
