// Complex k(z) and Robin z-faces on the FP64 path (orders 2, 4 and 6, Helmholtz).
//
// Section 1's general problem: K = k^2 complex and depending on z only, u = 0
// on the side faces, each z-face Dirichlet (u = g) or Robin (alpha u_z + beta u
// = g, complex alpha, beta).  Interior rows l = 1..Nz are the compact rows of
// Sections 3.2 / 3.3 with complex K; every coefficient is affine in K, so the
// complex table is the real table at Re K plus i times its K-part at Im K.  The
// 6th-order rows (Section 3.4, uniform h, Dirichlet side faces) are polynomials
// in K, K_z and K_zz and are evaluated in complex arithmetic; their right-hand
// side is R6 of eq. scheme6 (K-free part on Re f and Im f, with ghosts
// 2 f_0 - f_1 + h^2 (f_nn)_face one step beyond a face) plus the complex
// h^2 (-h^2 K f / 20 + h^3 K_z (f_{l+1} - f_{l-1}) / 120).  A
// Robin face's plane is unknown and its row is the second-order 7-point scheme
// with the outside plane eliminated by the central difference of the face
// condition (the paper leaves the compact closure to a cited work):
//   lo face (l = 0):      u_-1    = u_1  - 2 h_z (g - beta u_0) / alpha,
//   hi face (l = Nz + 1): u_Nz+2  = u_Nz + 2 h_z (g - beta u_Nz+1) / alpha,
// which gives the row  Rzx dxx + Rzy dyy + 2 u_(inner) + (-2 - 2Rzx - 2Rzy +
// h_z^2 K -+ 2 h_z beta / alpha) u_face = h_z^2 f +- 2 h_z g / alpha.
//
// A side axis may instead carry u_n = g on both faces (g = 0, or per-face data
// through hs_zsolve_ex): its boundary nodes are unknowns, the ghost beyond a
// face is the even reflection plus 2 h g, f and the z-face data are reflected
// evenly, and the cosine transform DCT-I over nodes 0..N+1 (k_dct.cu) replaces
// the sine transform; the modes cos(p pi i/(N+1)), p = 0..N+1, enter the same
// eigenvalue formula, and the per-row coefficients are unchanged.  An axis
// with one face of each kind (HS_SIDE_DN: Dirichlet low face, u_n = g on the
// high face; HS_SIDE_ND the reverse) has N + 1 unknowns (nodes 1..N+1, or
// 0..N) and takes the quarter-wave modes of angle (2p - 1) pi / (2 (N + 1)),
// p = 1..N+1: sines of the nodes 1..N+1 (weight 1/2 at the Neumann node), or
// for HS_SIDE_ND the cosines of the nodes 0..N, which are those sines of the
// reversed line times (-1)^(p+1).  Each such pass runs as the sine transform
// of length 2N + 1 of the line extended evenly about its Neumann node (an
// internal FP64 plan): the forward modes are half its odd outputs, and the
// inverse is that transform of the modes placed at the odd points.
//
// The solve (Section 3.6 with complex rows): the right-hand side kernel writes
// the unknown rows l0..l1 as planar complex data [2][Nu][ny][nx]; the real FP64
// transforms (sine: an internal plan over 2 Nu planes; cosine: k_dct.cu) act on
// Re and Im; one thread per mode (p, q) solves the complex tridiagonal system in
// z by the textbook recurrence (no pivoting); the inverse transforms follow.
#include <math.h>
#include <stdarg.h>
#include <stdio.h>
#include <string.h>

#include <new>
#include <vector>

#include "hs_internal.cuh"
#include "hs_rhs_sf.cuh"   // LPair: unnormalised FP32-pair arithmetic

struct hs_zplan_s {
    int Nx, Ny, Nz, order;
    double Lx, Ly, Lz, hx, hy, hz;
    int kind[2];               // HS_ZFACE_* of the lo and hi faces
    double2 alpha[2], beta[2];
    std::vector<double2> K;    // Nz + 2 nodes
    std::vector<double2> Kz, Kzz;   // order 6: K_z, K_zz at the nodes
    double2 *d_kk;             // order 6: [2][Nz + 2] K and K_z for the right-hand side
    int have_coeff;
    int Nu, l0;                // unknown planes l0 .. l0 + Nu - 1
    int side[2];               // HS_SIDE_* of the x and y axes
    int nx, ny, i0x, i0y;      // unknown grid of a plane; node index of its first point
    int layout_ok;             // transform plan, tables and buffers complete
    hs_plan_s *T;              // FP64 transform plan [2 Nu][ny][nx] (work: d_w64, d_dscr)
    hs_plan_s *TQ[2];          // quarter-wave axis: plan of its lines extended to 2N + 1
    double *d_cos;             // [nx] then [ny]: cos(theta) of each axis' modes
    double2 *d_dct[2];         // Neumann axis: M roots then M + 1 half-angle pairs
    float2 *d_dct32[2];        // the same in FP32 (mixed precision)
    double2 *d_rows;           // [Nu][3][4] complex coefficients of the unknown rows
    float4 *d_rows32;          // the same as FP32 pairs (re hi, re lo, im hi, im lo)
    int resid_xy;              // d_rows32's x and y coefficients agree on every row
    int rows_ok;
    double *d_fac;             // cached LU factors: 3 planar complex arrays [2][Nu][ny][nx]
    int fac_ok;                // the factors match the rows and side tables
    // HS_MIXED: FP32 solves of the correction equation, FP64 residuals, refinement
    int precision, sweeps;
    float *d_w32;              // [2][Nu][ny][nx] FP32 work of the correction solves
    float *d_fac32;            // the LU factors rounded to FP32 (layout of d_fac)
    float *d_Fp, *d_Up;        // F and the iterate as FP32 pairs: [hi: 2][Nu][ny][nx], then lo
    double *d_U;               // [2][Nu][ny][nx] FP64 result
    int fac32_ok;
    int timing;                // record events around the stages of each solve
    int have_ev;
    cudaEvent_t ev[6];         // rhs | forward transforms | z-solves | inverse | output
    char last_error[256];
};

namespace {

void zerr(hs_zplan_s *Z, const char *fmt, ...) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(Z->last_error, sizeof(Z->last_error), fmt, ap);
    va_end(ap);
}

#define ZCK(Z, call)                                                                     \
    do {                                                                                 \
        cudaError_t e_ = (call);                                                         \
        if (e_ != cudaSuccess) {                                                         \
            zerr(Z, "%s failed: %s", #call, cudaGetErrorString(e_));                     \
            return (e_ == cudaErrorMemoryAllocation) ? HS_ERR_OOM : HS_ERR_CUDA;         \
        }                                                                                \
    } while (0)

enum { ZA = 0, ZB = 1, ZC = 2, ZD = 3 };          // corner, x-, y-neighbour, centre
enum { ZLOW = 0, ZMID = 1, ZUPP = 2 };            // planes l - 1, l, l + 1

__host__ __device__ inline double2 cmul(double2 a, double2 b) {
    return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__host__ __device__ inline double2 cadd(double2 a, double2 b) {
    return make_double2(a.x + b.x, a.y + b.y);
}
__host__ __device__ inline double2 csub(double2 a, double2 b) {
    return make_double2(a.x - b.x, a.y - b.y);
}
__host__ __device__ inline double2 cscale(double s, double2 a) {
    return make_double2(s * a.x, s * a.y);
}
__host__ inline double2 cdiv_host(double2 a, double2 b) {
    const double d = b.x * b.x + b.y * b.y;
    return make_double2((a.x * b.x + a.y * b.y) / d, (a.y * b.x - a.x * b.y) / d);
}

// Real coefficients of an interior row (Sections 3.2, 3.3) for a real K at the
// three nodes (Km, K, Kp) = K(z_{l-1}), K(z_l), K(z_{l+1}); blk[nu][m].
void real_row(int order, double Rzx, double Rzy, double hz2, double Km, double K, double Kp,
              double blk[3][4]) {
    memset(blk, 0, sizeof(double) * 12);
    if (order == 2) {
        blk[ZMID][ZB] = Rzx;
        blk[ZMID][ZC] = Rzy;
        blk[ZLOW][ZD] = 1.0;
        blk[ZUPP][ZD] = 1.0;
        blk[ZMID][ZD] = -2.0 * (Rzx + Rzy + 1.0) + hz2 * K;
    } else {
        blk[ZLOW][ZB] = blk[ZUPP][ZB] = (1.0 + Rzx) / 12.0;
        blk[ZLOW][ZC] = blk[ZUPP][ZC] = (1.0 + Rzy) / 12.0;
        blk[ZLOW][ZD] = 2.0 / 3.0 - (Rzx + Rzy) / 6.0 + hz2 * Km / 12.0;
        blk[ZUPP][ZD] = 2.0 / 3.0 - (Rzx + Rzy) / 6.0 + hz2 * Kp / 12.0;
        blk[ZMID][ZA] = (Rzx + Rzy) / 12.0;
        blk[ZMID][ZB] = (4.0 * Rzx - Rzy - 1.0 + hz2 * K / 2.0) / 6.0;
        blk[ZMID][ZC] = (4.0 * Rzy - Rzx - 1.0 + hz2 * K / 2.0) / 6.0;
        blk[ZMID][ZD] = -4.0 * (1.0 + Rzx + Rzy) / 3.0 + hz2 * K / 2.0;
    }
}

// Complex coefficients of a 6th-order interior row (Section 3.4, uniform h): the
// printed coefficients are polynomials in K (K_{l-1}, K_l, K_{l+1}), K_z and K_zz,
// so they are evaluated in complex arithmetic as printed; blk[nu * 4 + m].
void six_row(double h, double2 Km, double2 K, double2 Kp, double2 Kz, double2 Kzz,
             double2 *blk) {
    const double h2 = h * h, h3 = h2 * h, h4 = h2 * h2;
    auto lin = [](double c, double s, double2 x) {   // c + s x
        return make_double2(c + s * x.x, s * x.y);
    };
    for (int k = 0; k < 12; ++k) blk[k] = make_double2(0.0, 0.0);
    blk[ZLOW * 4 + ZA] = blk[ZUPP * 4 + ZA] = make_double2(1.0 / 30.0, 0.0);
    // 1/10 + h^2 K_{l-+1} / 90 -+ h^3 K_z / 120
    const double2 bl = csub(lin(0.1, h2 / 90.0, Km), cscale(h3 / 120.0, Kz));
    const double2 bu = cadd(lin(0.1, h2 / 90.0, Kp), cscale(h3 / 120.0, Kz));
    blk[ZLOW * 4 + ZB] = blk[ZLOW * 4 + ZC] = bl;
    blk[ZUPP * 4 + ZB] = blk[ZUPP * 4 + ZC] = bu;
    // 7/15 - h^2 K_{l-+1} / 90 -+ (h^3 K_z / 20) (1/3 + h^2 K_{l-+1} / 6)
    const double2 tz = cscale(h3 / 20.0, Kz);
    blk[ZLOW * 4 + ZD] = csub(lin(7.0 / 15.0, -h2 / 90.0, Km), cmul(tz, lin(1.0 / 3.0, h2 / 6.0, Km)));
    blk[ZUPP * 4 + ZD] = cadd(lin(7.0 / 15.0, -h2 / 90.0, Kp), cmul(tz, lin(1.0 / 3.0, h2 / 6.0, Kp)));
    blk[ZMID * 4 + ZA] = lin(0.1, h2 / 90.0, K);
    blk[ZMID * 4 + ZB] = blk[ZMID * 4 + ZC] = lin(7.0 / 15.0, -h2 / 90.0, K);
    // -64/15 + 14 h^2 K / 15 - h^4 K^2 / 20 + h^4 K_zz / 20
    blk[ZMID * 4 + ZD] = cadd(csub(lin(-64.0 / 15.0, 14.0 * h2 / 15.0, K), cscale(h4 / 20.0, cmul(K, K))),
                              cscale(h4 / 20.0, Kzz));
}

// Builds the complex rows of the unknown planes and uploads them.
hs_status build_rows(hs_zplan_s *Z) {
    if (!Z->layout_ok) return HS_OK;   // built once a set-up call completes the layout
    const double Rzx = Z->hz * Z->hz / (Z->hx * Z->hx), Rzy = Z->hz * Z->hz / (Z->hy * Z->hy);
    const double hz2 = Z->hz * Z->hz;
    std::vector<double2> rows((size_t)Z->Nu * 12);
    for (int r = 0; r < Z->Nu; ++r) {
        const int l = Z->l0 + r;
        double2 *blk = &rows[(size_t)r * 12];
        if (l == 0 || l == Z->Nz + 1) {   // a Robin face's row
            const int side = l == 0 ? -1 : 1;
            const double2 a = Z->alpha[l == 0 ? 0 : 1], b = Z->beta[l == 0 ? 0 : 1];
            for (int k = 0; k < 12; ++k) blk[k] = make_double2(0.0, 0.0);
            const double2 ba = cdiv_host(b, a);
            blk[ZMID * 4 + ZB] = make_double2(Rzx, 0.0);
            blk[ZMID * 4 + ZC] = make_double2(Rzy, 0.0);
            blk[ZMID * 4 + ZD] = make_double2(-2.0 * (Rzx + Rzy + 1.0) + hz2 * Z->K[l].x -
                                                  side * 2.0 * Z->hz * ba.x,
                                              hz2 * Z->K[l].y - side * 2.0 * Z->hz * ba.y);
            blk[(side < 0 ? ZUPP : ZLOW) * 4 + ZD] = make_double2(2.0, 0.0);
            continue;
        }
        if (Z->order == 6) {
            six_row(Z->hz, Z->K[l - 1], Z->K[l], Z->K[l + 1], Z->Kz[l], Z->Kzz[l], blk);
            continue;
        }
        double re[3][4], im[3][4], z0[3][4];
        const double2 Km = Z->K[l - 1], K = Z->K[l], Kp = Z->K[l + 1];
        real_row(Z->order, Rzx, Rzy, hz2, Km.x, K.x, Kp.x, re);
        real_row(Z->order, Rzx, Rzy, hz2, Km.y, K.y, Kp.y, im);
        real_row(Z->order, Rzx, Rzy, hz2, 0.0, 0.0, 0.0, z0);
        for (int nu = 0; nu < 3; ++nu)
            for (int m = 0; m < 4; ++m)
                blk[nu * 4 + m] = make_double2(re[nu][m], im[nu][m] - z0[nu][m]);
    }
    ZCK(Z, cudaMemcpy(Z->d_rows, rows.data(), rows.size() * sizeof(double2),
                      cudaMemcpyHostToDevice));
    if (Z->d_rows32) {   // the pair copy of the mixed-precision residual
        std::vector<float4> r32(rows.size());
        for (size_t k = 0; k < rows.size(); ++k) {
            const float rh = (float)rows[k].x, ih = (float)rows[k].y;
            r32[k] = make_float4(rh, (float)(rows[k].x - (double)rh), ih, (float)(rows[k].y - (double)ih));
        }
        Z->resid_xy = 1;
        for (size_t k = 0; k < rows.size(); k += 4) {   // (A, B, C, D) of one (row, nu)
            const float4 b = r32[k + 1], c = r32[k + 2];
            if (b.x != c.x || b.y != c.y || b.z != c.z || b.w != c.w) Z->resid_xy = 0;
        }
        ZCK(Z, cudaMemcpy(Z->d_rows32, r32.data(), r32.size() * sizeof(float4),
                          cudaMemcpyHostToDevice));
    }
    Z->rows_ok = 1;
    Z->fac_ok = 0;
    return HS_OK;
}

// cos(pi a / b) with the argument reduced exactly (integers) to [0, pi/2] first.
double cos_pi_frac(long a, long b) {
    a %= 2 * b;
    if (a < 0) a += 2 * b;
    if (a > b) a = 2 * b - a;           // cos is even about pi
    if (2 * a > b) return -cos(M_PI * (double)(b - a) / (double)b);
    return cos(M_PI * (double)a / (double)b);
}
double sin_pi_frac(long a, long b) { return cos_pi_frac(2 * a - b, 2 * b); }

// Mode cosines of both axes and the DCT tables of Neumann axes.
hs_status side_tables(hs_zplan_s *Z) {
    Z->fac_ok = 0;
    std::vector<double> c;
    const int N[2] = {Z->Nx, Z->Ny};
    for (int a = 0; a < 2; ++a) {
        if (Z->side[a] == HS_SIDE_NEUMANN)
            for (int p = 0; p <= N[a] + 1; ++p) c.push_back(cos_pi_frac(p, N[a] + 1));
        else if (Z->side[a] == HS_SIDE_DN || Z->side[a] == HS_SIDE_ND)   // quarter-wave modes
            for (int p = 1; p <= N[a] + 1; ++p) c.push_back(cos_pi_frac(2 * p - 1, 2 * (N[a] + 1)));
        else
            for (int p = 1; p <= N[a]; ++p) c.push_back(cos_pi_frac(p, N[a] + 1));
    }
    if (Z->d_cos) cudaFree(Z->d_cos);
    Z->d_cos = nullptr;
    ZCK(Z, cudaMalloc(&Z->d_cos, c.size() * sizeof(double)));
    ZCK(Z, cudaMemcpy(Z->d_cos, c.data(), c.size() * sizeof(double), cudaMemcpyHostToDevice));
    for (int a = 0; a < 2; ++a) {
        if (Z->d_dct[a]) cudaFree(Z->d_dct[a]);
        Z->d_dct[a] = nullptr;
        if (Z->d_dct32[a]) cudaFree(Z->d_dct32[a]);
        Z->d_dct32[a] = nullptr;
        if (Z->side[a] != HS_SIDE_NEUMANN) continue;
        const int M = N[a] + 1;
        std::vector<double2> t(2 * (size_t)M + 1);
        for (int k = 0; k < M; ++k)   // exp(-2 pi i k / M)
            t[k] = make_double2(cos_pi_frac(2L * k, M), -sin_pi_frac(2L * k, M));
        for (int k = 0; k <= M; ++k) t[M + k] = make_double2(cos_pi_frac(k, M), sin_pi_frac(k, M));
        ZCK(Z, cudaMalloc(&Z->d_dct[a], t.size() * sizeof(double2)));
        ZCK(Z, cudaMemcpy(Z->d_dct[a], t.data(), t.size() * sizeof(double2),
                          cudaMemcpyHostToDevice));
        std::vector<float2> t32(t.size());
        for (size_t k = 0; k < t.size(); ++k) t32[k] = make_float2((float)t[k].x, (float)t[k].y);
        ZCK(Z, cudaMalloc(&Z->d_dct32[a], t32.size() * sizeof(float2)));
        ZCK(Z, cudaMemcpy(Z->d_dct32[a], t32.data(), t32.size() * sizeof(float2),
                          cudaMemcpyHostToDevice));
    }
    return HS_OK;
}

// Buffers of the mixed-precision solve (allocated by the first mixed solve).
void free_mixed(hs_zplan_s *Z) {
    if (Z->d_w32) cudaFree(Z->d_w32);
    if (Z->d_fac32) cudaFree(Z->d_fac32);
    if (Z->d_U) cudaFree(Z->d_U);
    if (Z->d_Fp) cudaFree(Z->d_Fp);
    if (Z->d_Up) cudaFree(Z->d_Up);
    if (Z->d_rows32) cudaFree(Z->d_rows32);
    Z->d_w32 = nullptr;
    Z->d_fac32 = nullptr;
    Z->d_U = nullptr;
    Z->d_Fp = nullptr;
    Z->d_Up = nullptr;
    Z->d_rows32 = nullptr;
    Z->fac32_ok = 0;
}

// (Re)creates the transform plan, row table and side tables for the current
// faces and side axes.
hs_status layout(hs_zplan_s *Z) {
    Z->layout_ok = 0;
    const int l0 = Z->kind[0] == HS_ZFACE_ROBIN ? 0 : 1;
    const int l1 = Z->kind[1] == HS_ZFACE_ROBIN ? Z->Nz + 1 : Z->Nz;
    const int Nu = l1 - l0 + 1;
    // unknowns of a side axis: N (Dirichlet faces), N + 2 (Neumann faces), N + 1
    // (one of each); the first is node 0 when the low face is a Neumann face
    auto count = [](int kind, int N) {
        return kind == HS_SIDE_NEUMANN ? N + 2 : (kind == HS_SIDE_DIRICHLET ? N : N + 1);
    };
    const int nx = count(Z->side[0], Z->Nx), ny = count(Z->side[1], Z->Ny);
    Z->i0x = (Z->side[0] == HS_SIDE_NEUMANN || Z->side[0] == HS_SIDE_ND) ? 0 : 1;
    Z->i0y = (Z->side[1] == HS_SIDE_NEUMANN || Z->side[1] == HS_SIDE_ND) ? 0 : 1;
    Z->l0 = l0;
    // rebuilt after a change of shape, or when an earlier rebuild stopped part-way
    if (!(Z->T && Z->d_rows && Z->d_fac && Nu == Z->Nu && nx == Z->nx && ny == Z->ny)) {
        if (Z->T) hs_destroy(Z->T);
        Z->T = nullptr;
        if (Z->d_rows) cudaFree(Z->d_rows);
        Z->d_rows = nullptr;
        if (Z->d_fac) cudaFree(Z->d_fac);
        Z->d_fac = nullptr;
        free_mixed(Z);   // sized for the previous shape
        Z->Nu = Nu;
        Z->nx = nx;
        Z->ny = ny;
        Z->rows_ok = 0;
        // the sine transforms of Dirichlet axes, and the work arrays; a Neumann
        // axis' own table in this plan is never used
        hs_plan_t T = nullptr;
        const hs_status st = hs_plan_ex(&T, nx, ny, 2 * Nu, Z->Lx, Z->Ly, 1.0, 2, HS_HELMHOLTZ,
                                        HS_BC_DIRICHLET, HS_FP64, 1, 1);
        if (st != HS_OK) {
            zerr(Z, "transform plan: status %d", st);
            return st;
        }
        Z->T = T;
        // the half-length FP64 sine transform where its FFT is compiled (the
        // others keep the plan's default)
        for (int a = 0; a < 2; ++a) (void)hs_set_transform_variant(T, a, HS_DST_HALF);
        ZCK(Z, cudaMalloc(&Z->d_rows, (size_t)Nu * 12 * sizeof(double2)));
        ZCK(Z, cudaMalloc(&Z->d_fac, (size_t)6 * Nu * nx * ny * sizeof(double)));
    }
    // the extended-line plans of quarter-wave axes (their work array holds the
    // lines of length 2N + 1)
    for (int a = 0; a < 2; ++a) {
        const bool q = Z->side[a] == HS_SIDE_DN || Z->side[a] == HS_SIDE_ND;
        const int ex = a == 0 ? 2 * Z->Nx + 1 : nx, ey = a == 1 ? 2 * Z->Ny + 1 : ny;
        hs_plan_s *Q = Z->TQ[a];
        if (Q && (!q || Q->Nx != ex || Q->Ny != ey || Q->Nz != 2 * Nu)) {
            hs_destroy(Q);
            Z->TQ[a] = nullptr;
        }
        if (q && !Z->TQ[a]) {
            hs_plan_t Tq = nullptr;
            const hs_status sq = hs_plan_ex(&Tq, ex, ey, 2 * Nu, 1.0, 1.0, 1.0, 2, HS_HELMHOLTZ,
                                            HS_BC_DIRICHLET, HS_FP64, 1, 1);
            if (sq != HS_OK) {
                zerr(Z, "quarter-wave transform plan: status %d", sq);
                return sq;
            }
            (void)hs_set_transform_variant(Tq, a, HS_DST_HALF);
            Z->TQ[a] = Tq;
        }
    }
    const hs_status st = side_tables(Z);
    if (st == HS_OK) Z->layout_ok = 1;
    return st;
}

bool device_ptr(const void *p) {
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

struct ZRhsArgs {
    int Nx, Ny, Nz, Nu, l0, order;
    int nx, ny, i0x, i0y;   // unknown grid of a plane and its first node
    int neu_x, neu_y;       // side axes with a Neumann face (even reflection there)
    int nlo_x, nhi_x, nlo_y, nhi_y;   // which faces of each axis are Neumann faces
    int kind_lo, kind_hi;
    double hz;
    double2 ga_lo, ga_hi;   // 2 h_z / alpha of each face (Robin)
    const double *f;        // [2][Nz+2][Ny+2][Nx+2]
    const double *g_lo, *g_hi;   // [2][ny][nx] or NULL
    const double *side[4];  // u_n on the x-lo, x-hi ([2][Nz+2][Ny+2]), y-lo, y-hi
                            // ([2][Nz+2][Nx+2]) faces of Neumann axes, or NULL
    double hx, hy;
    const double2 *rows;    // [Nu][3][4]
    double *W;              // [2][Nu][ny][nx]
    const double *fnn[6];   // order 6: f_nn on the x-lo, x-hi ([2][Nz+2][Ny+2]), y-lo, y-hi
                            // ([2][Nz+2][Nx+2]), z-lo, z-hi ([2][Ny+2][Nx+2]) faces, or NULL
    const double2 *kk;      // order 6: [2][Nz+2] K and K_z at the nodes
    double k20, k120;       // order 6: -h_z^4 / 20 and h_z^5 / 120 (the K-term weights)
    int rbase;              // first unknown row of the launch (row rbase + blockIdx.y)
};

// Order 6: f (component comp) at node (i, j, l) of the node grid, or one step
// beyond a face the ghost 2 f_0 - f_1 + h^2 (f_nn)_face (the R6 operator's
// second neighbours; one coordinate at a time leaves the grid).
__device__ inline double f6_node(const ZRhsArgs &a, int comp, int i, int j, int l) {
    const size_t sy = (size_t)a.Nx + 2, sz = sy * (a.Ny + 2);
    const double *fc = a.f + (size_t)comp * sz * (a.Nz + 2);
    int face = -1, i0 = i, j0 = j, l0 = l, di = 0, dj = 0, dl = 0;
    if (i < 0) { face = 0; i0 = 0; di = 1; }
    else if (i > a.Nx + 1) { face = 1; i0 = a.Nx + 1; di = -1; }
    else if (j < 0) { face = 2; j0 = 0; dj = 1; }
    else if (j > a.Ny + 1) { face = 3; j0 = a.Ny + 1; dj = -1; }
    else if (l < 0) { face = 4; l0 = 0; dl = 1; }
    else if (l > a.Nz + 1) { face = 5; l0 = a.Nz + 1; dl = -1; }
    if (face < 0) return fc[(size_t)l * sz + (size_t)j * sy + i];
    double g = 2.0 * fc[(size_t)l0 * sz + (size_t)j0 * sy + i0] -
               fc[(size_t)(l0 + dl) * sz + (size_t)(j0 + dj) * sy + (i0 + di)];
    const double *d = a.fnn[face];
    if (d) {
        size_t k;
        if (face < 2) k = (size_t)comp * (a.Nz + 2) * (a.Ny + 2) + (size_t)l0 * (a.Ny + 2) + j0;
        else if (face < 4) k = (size_t)comp * (a.Nz + 2) * (a.Nx + 2) + (size_t)l0 * (a.Nx + 2) + i0;
        else k = (size_t)comp * (a.Ny + 2) * (a.Nx + 2) + (size_t)j0 * (a.Nx + 2) + i0;
        g += a.hz * a.hz * d[k];
    }
    return g;
}

// Index one node beyond [0, n - 1] of a Neumann axis: the even reflection.
__device__ inline int reflect(int i, int n) { return i < 0 ? -i : (i >= n ? 2 * (n - 1) - i : i); }

// Face data on the unknown grid: beyond a Dirichlet axis 0, beyond a Neumann one reflected.
__device__ inline double2 face_val(const ZRhsArgs &a, const double *g, int j, int i) {
    if (!g) return make_double2(0.0, 0.0);
    if ((j < 0 && a.nlo_y) || (j >= a.ny && a.nhi_y)) j = reflect(j, a.ny);
    if ((i < 0 && a.nlo_x) || (i >= a.nx && a.nhi_x)) i = reflect(i, a.nx);
    if (j < 0 || j >= a.ny || i < 0 || i >= a.nx) return make_double2(0.0, 0.0);
    const size_t k = (size_t)j * a.nx + i, n = (size_t)a.ny * a.nx;
    return make_double2(g[k], g[n + k]);
}

// Data part (2 h g) of the value at node (i, j) of plane l when it is a ghost
// beyond a Neumann face (u_n = g, outward normal): the x-ghost first, then the
// y-ghost, each face's data read along the face with even reflection.
__device__ inline double2 ghost_data(const ZRhsArgs &a, int i, int j, int l) {
    double2 d = make_double2(0.0, 0.0);
    const size_t nzp = (size_t)a.Nz + 2;
    if (a.neu_x && (i < 0 || i > a.Nx + 1)) {
        const double *g = a.side[i < 0 ? 0 : 1];
        if (g) {
            const int jr = reflect(j, a.Ny + 2);
            const size_t k = (size_t)l * (a.Ny + 2) + jr, n = nzp * (a.Ny + 2);
            d.x += 2.0 * a.hx * g[k];
            d.y += 2.0 * a.hx * g[n + k];
        }
    }
    if (a.neu_y && (j < 0 || j > a.Ny + 1)) {
        const double *g = a.side[j < 0 ? 2 : 3];
        if (g) {
            const int ir = reflect(i, a.Nx + 2);
            const size_t k = (size_t)l * (a.Nx + 2) + ir, n = nzp * (a.Nx + 2);
            d.x += 2.0 * a.hy * g[k];
            d.y += 2.0 * a.hy * g[n + k];
        }
    }
    return d;
}

// One thread per unknown (row r = blockIdx.y, (j, i) along x): the compact
// right-hand side of the row, minus the known Dirichlet plane next to it, or the
// Robin row's h_z^2 f plus its face-data term.  FP64 divisions by constants are
// multiplications by the folded reciprocals (an FP64 division costs about ten
// FP64-pipe operations on this GPU).
__global__ void zrhs_kernel(ZRhsArgs a) {
    const size_t plane = (size_t)a.ny * a.nx, n = plane * a.Nu;
    const size_t sy = (size_t)(a.Nx + 2), sz = sy * (a.Ny + 2), nodes = sz * (a.Nz + 2);
    {
        const int r = a.rbase + blockIdx.y;
        const int rem = blockIdx.x * blockDim.x + threadIdx.x;
        if (rem >= (int)plane) return;
        const size_t t = (size_t)r * plane + rem;
        const int j = rem / a.nx, i = rem - j * a.nx;
        const int l = a.l0 + r;
        const int jj = j + a.i0y, ii = i + a.i0x;   // node indices
        // neighbours on the node grid, reflected beyond a Neumann side's faces
        const int im = reflect(ii - 1, a.Nx + 2), ip = reflect(ii + 1, a.Nx + 2);
        const int jm = reflect(jj - 1, a.Ny + 2), jp = reflect(jj + 1, a.Ny + 2);
        const size_t rowc = (size_t)l * sz + (size_t)jj * sy;
        const size_t c = rowc + ii;
        const double hz2 = a.hz * a.hz;
        double2 F;
        for (int comp = 0; comp < 2; ++comp) {
            const double *f = a.f + comp * nodes;
            double v = f[c];
            if (a.order == 4 && l >= 1 && l <= a.Nz) {
                const size_t pl = (size_t)l * sz;
                const double D = (f[rowc + im] + f[rowc + ip] + f[pl + (size_t)jm * sy + ii] +
                                  f[pl + (size_t)jp * sy + ii] + f[c - sz] + f[c + sz]) -
                                 6.0 * f[c];
                v = fma(D, 1.0 / 12.0, v);
            } else if (a.order == 6 && l >= 1 && l <= a.Nz) {
                // K-free part of R6 / h^2: 67/120 f + (40 S1 - 3 S2 + 8 E) / 720 with
                // S1 the 6 face neighbours, S2 the 6 second neighbours (ghosts beyond
                // a face), E the 12 edge mid-points
                const size_t pl = (size_t)l * sz;
                const double S1 = f[rowc + ii - 1] + f[rowc + ii + 1] + f[c - sy] + f[c + sy] +
                                  f[c - sz] + f[c + sz];
                const double S2 = f6_node(a, comp, ii - 2, jj, l) + f6_node(a, comp, ii + 2, jj, l) +
                                  f6_node(a, comp, ii, jj - 2, l) + f6_node(a, comp, ii, jj + 2, l) +
                                  f6_node(a, comp, ii, jj, l - 2) + f6_node(a, comp, ii, jj, l + 2);
                double E = 0.0;
                for (int s1 = -1; s1 <= 1; s1 += 2)
                    for (int s2 = -1; s2 <= 1; s2 += 2) {
                        E += f[pl + (size_t)(jj + s1) * sy + (ii + s2)];   // x-y edges
                        E += f[c + s1 * (long)sz + s2];                     // x-z edges
                        E += f[c + s1 * (long)sz + s2 * (long)sy];          // y-z edges
                    }
                v = fma(40.0 * S1 - 3.0 * S2 + 8.0 * E, 1.0 / 720.0, (67.0 / 120.0) * f[c]);
            }
            if (comp == 0) F.x = hz2 * v; else F.y = hz2 * v;
        }
        if (a.order == 6 && l >= 1 && l <= a.Nz) {
            // the complex K terms h^2 (-h^2 K_l f / 20 + h^3 K_z,l (f_{l+1} - f_{l-1}) / 120)
            const size_t nn = nodes;
            const double2 fcv = make_double2(a.f[c], a.f[nn + c]);
            const double2 dz = make_double2(a.f[c + sz] - a.f[c - sz], a.f[nn + c + sz] - a.f[nn + c - sz]);
            const double2 Kc = a.kk[l], Kzc = a.kk[a.Nz + 2 + l];
            F = cadd(F, cscale(a.k20, cmul(Kc, fcv)));
            F = cadd(F, cscale(a.k120, cmul(Kzc, dz)));
        }
        if (l == 0) {
            F = cadd(F, cmul(a.ga_lo, face_val(a, a.g_lo, j, i)));
        } else if (l == a.Nz + 1) {
            F = csub(F, cmul(a.ga_hi, face_val(a, a.g_hi, j, i)));
        } else {
            // a Dirichlet face's plane next to this row: its values leave through the stencil
            const bool lo = l == 1 && a.kind_lo == HS_ZFACE_DIRICHLET && a.g_lo;
            const bool hi = l == a.Nz && a.kind_hi == HS_ZFACE_DIRICHLET && a.g_hi;
            for (int side = 0; side < 2; ++side) {
                if (!(side == 0 ? lo : hi)) continue;
                const double *g = side == 0 ? a.g_lo : a.g_hi;
                const double2 *w = a.rows + (size_t)r * 12 + (side == 0 ? ZLOW : ZUPP) * 4;
                for (int dj = -1; dj <= 1; ++dj)
                    for (int di = -1; di <= 1; ++di) {
                        const int m = (di != 0 && dj != 0) ? ZA : (di != 0 ? ZB : (dj != 0 ? ZC : ZD));
                        F = csub(F, cmul(w[m], face_val(a, g, j + dj, i + di)));
                    }
            }
        }
        a.W[t] = F.x;
        a.W[n + t] = F.y;
    }
}

// Rows next to a Neumann face with data: the stencil weight of every ghost
// neighbour times its data part leaves for the right-hand side (planes
// 0..Nz+1), added to W after zrhs_kernel.  One thread per face row: x-face rows
// first (all their ghost neighbours, corners included), then y-face rows not
// already on a Neumann x-face with data, so each row is written once.
__global__ void zside_kernel(ZRhsArgs a) {
    const size_t plane = (size_t)a.ny * a.nx, n = plane * a.Nu;
    const bool dx = a.neu_x && (a.side[0] || a.side[1]);
    const bool dy = a.neu_y && (a.side[2] || a.side[3]);
    const size_t cx = dx ? 2 * (size_t)a.Nu * a.ny : 0;
    const size_t cy = dy ? 2 * (size_t)a.Nu * a.nx : 0;
    for (size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x; t < cx + cy;
         t += (size_t)gridDim.x * blockDim.x) {
        int r, i, j;
        if (t < cx) {
            const size_t per = (size_t)a.Nu * a.ny;
            const int face = (int)(t / per);
            const size_t rem = t - face * per;
            r = (int)(rem / a.ny);
            j = (int)(rem - (size_t)r * a.ny);
            i = face ? a.nx - 1 : 0;
        } else {
            const size_t u = t - cx, per = (size_t)a.Nu * a.nx;
            const int face = (int)(u / per);
            const size_t rem = u - face * per;
            r = (int)(rem / a.nx);
            i = (int)(rem - (size_t)r * a.nx);
            j = face ? a.ny - 1 : 0;
            if (dx && (i == 0 || i == a.nx - 1)) continue;   // written by its x-face thread
        }
        const int l = a.l0 + r, ii = i + a.i0x, jj = j + a.i0y;
        double2 F = make_double2(0.0, 0.0);
#pragma unroll 1
        for (int dl = -1; dl <= 1; ++dl) {
            const int ll = l + dl;
            if (ll < 0 || ll > a.Nz + 1) continue;
            const double2 *w = a.rows + (size_t)r * 12 + (dl + 1) * 4;
#pragma unroll 1
            for (int dj = -1; dj <= 1; ++dj)
                for (int di = -1; di <= 1; ++di) {
                    const int i2 = ii + di, j2 = jj + dj;
                    if (i2 >= 0 && i2 <= a.Nx + 1 && j2 >= 0 && j2 <= a.Ny + 1) continue;
                    const int m = (di != 0 && dj != 0) ? ZA : (di != 0 ? ZB : (dj != 0 ? ZC : ZD));
                    F = csub(F, cmul(w[m], ghost_data(a, i2, j2, ll)));
                }
        }
        const size_t k = (size_t)r * plane + (size_t)j * a.nx + i;
        a.W[k] += F.x;
        a.W[n + k] += F.y;
    }
}

// Mixed precision, orders 2 and 4, rows whose right-hand side is the plain
// interior formula (no z-face term, no u_n data on the side faces; neighbours
// beyond a Neumann side face reflected evenly): F = h_z^2 f at order 2,
// F = (h_z^2 / 2) f + (h_z^2 / 12) S1 at order 4 (S1 the six face neighbours;
// the same operator as f + (S1 - 6 f) / 12), for the real and the imaginary
// part alike, in FP32-pair arithmetic (FP64 f split into pairs with integer
// operations, hi parts summed exactly) and written straight into the pair
// planes the refinement works on.  wc, w12: the pair weights h_z^2 / 2 (order 4)
// or h_z^2 (order 2), and h_z^2 / 12.
__global__ void __launch_bounds__(256) zrhs_pair_kernel(ZRhsArgs a, float *__restrict__ Fp,
                                                        float2 wc, float2 w12) {
    using namespace hs_tiles;
    const int plane = a.ny * a.nx;
    const size_t nu = (size_t)plane * a.Nu, n2 = 2 * nu;
    const size_t sy = (size_t)(a.Nx + 2), sz = sy * (a.Ny + 2), nodes = sz * (a.Nz + 2);
    const int r = a.rbase + blockIdx.y;
    const int rem = blockIdx.x * blockDim.x + threadIdx.x;
    if (rem >= plane) return;
    const int j = rem / a.nx, i = rem - j * a.nx;
    const int jj = j + a.i0y, ii = i + a.i0x;   // node indices
    const size_t rowc = (size_t)(a.l0 + r) * sz + (size_t)jj * sy;
    const size_t c = rowc + ii;
    // in-plane neighbours, reflected beyond a Neumann side's faces
    const size_t xm = rowc + reflect(ii - 1, a.Nx + 2), xp = rowc + reflect(ii + 1, a.Nx + 2);
    const size_t ym = (size_t)(a.l0 + r) * sz + (size_t)reflect(jj - 1, a.Ny + 2) * sy + ii;
    const size_t yp = (size_t)(a.l0 + r) * sz + (size_t)reflect(jj + 1, a.Ny + 2) * sy + ii;
    const size_t k = (size_t)r * plane + rem;
    auto pr = [](double x) {
        const dfloat d = df_split_bits(x);
        return LPair{d.hi, d.lo};
    };
#pragma unroll
    for (int comp = 0; comp < 2; ++comp) {
        const double *f = a.f + comp * nodes;
        LPair v = lp_mul(wc, pr(f[c]));
        if (a.order == 4) {
            LPair s1 = pr(f[xm]);
            lp_add(s1, pr(f[xp]));
            lp_add(s1, pr(f[ym]));
            lp_add(s1, pr(f[yp]));
            lp_add(s1, pr(f[c - sz]));
            lp_add(s1, pr(f[c + sz]));
            lp_add(v, lp_mul(w12, s1));
        }
        float hi, lo;
        df_two_sum(v.s, v.e, hi, lo);
        Fp[comp * nu + k] = hi;
        Fp[n2 + comp * nu + k] = lo;
    }
}

// Cached LU of every mode's complex tridiagonal system (one thread per mode
// (p, q); lambda_nu = 4 a cp cq + 2 b cp + 2 c cq + d, Section 3.6; no
// pivoting): per row r the planar complex factors 1/m_r, lower_r/m_r and
// c'_r = upper_r/m_r with m_r = diag_r - lower_r c'_{r-1}, each [2][Nu][ny][nx].
// Quarter-wave pass of one side axis (HS_SIDE_DN / HS_SIDE_ND) through the
// sine transform of length 2n - 1 (n = N + 1 unknowns per line).  W holds the
// 2 Nu planes [ny][nx]; E the extended lines ([2 Nu][ny][2n - 1] along x,
// [2 Nu][2n - 1][nx] along y).  rev: HS_SIDE_ND, whose nodes 0..N are the
// reversed nodes 1..N+1 of the DN form and whose modes carry (-1)^(p+1).
struct QArgs {
    int axis, n, nx, ny, rev;
    long lines;          // 2 Nu ny (x) or 2 Nu nx (y)
    double scale;        // inverse: 2 / n
};

__device__ inline void q_line(const QArgs &q, long line, size_t &wb, size_t &eb, size_t &st) {
    if (q.axis == HS_AXIS_X) {
        wb = (size_t)line * q.n;
        eb = (size_t)line * (2 * q.n - 1);
        st = 1;
    } else {
        const long c = line / q.nx, i = line - c * q.nx;
        wb = (size_t)c * q.n * q.nx + i;
        eb = (size_t)c * (2 * q.n - 1) * q.nx + i;
        st = q.nx;
    }
}

// forward: the line extended evenly about its Neumann node (DN form, nodes 1..2n-1)
__global__ void zq_gather_fwd(QArgs q, const double *__restrict__ W, double *__restrict__ E) {
    const long m = 2 * q.n - 1;
    for (long t = blockIdx.x * (long)blockDim.x + threadIdx.x; t < q.lines * m;
         t += (long)gridDim.x * blockDim.x) {
        const long line = t / m;
        const int k = (int)(t - line * m) + 1;   // node of the extended line
        const int kk = k <= q.n ? k : 2 * q.n - k;   // folded onto 1..n
        const int a = q.rev ? q.n - kk : kk - 1;      // index in W's line
        size_t wb, eb, st;
        q_line(q, line, wb, eb, st);
        E[eb + (size_t)(k - 1) * st] = W[wb + (size_t)a * st];
    }
}

// forward: mode p = half the odd output 2p - 1 (times (-1)^(p+1) for ND)
__global__ void zq_scatter_fwd(QArgs q, const double *__restrict__ E, double *__restrict__ W) {
    for (long t = blockIdx.x * (long)blockDim.x + threadIdx.x; t < q.lines * q.n;
         t += (long)gridDim.x * blockDim.x) {
        const long line = t / q.n;
        const int p = (int)(t - line * q.n) + 1;
        size_t wb, eb, st;
        q_line(q, line, wb, eb, st);
        const double sg = (q.rev && !(p & 1)) ? -0.5 : 0.5;
        W[wb + (size_t)(p - 1) * st] = sg * E[eb + (size_t)(2 * p - 2) * st];
    }
}

// inverse: the modes at the odd points 2p - 1 of the extended line, zeros between
__global__ void zq_gather_inv(QArgs q, const double *__restrict__ W, double *__restrict__ E) {
    const long m = 2 * q.n - 1;
    for (long t = blockIdx.x * (long)blockDim.x + threadIdx.x; t < q.lines * m;
         t += (long)gridDim.x * blockDim.x) {
        const long line = t / m;
        const int k = (int)(t - line * m) + 1;
        size_t wb, eb, st;
        q_line(q, line, wb, eb, st);
        double v = 0.0;
        if (k & 1) {
            const int p = (k + 1) / 2;
            v = W[wb + (size_t)(p - 1) * st];
            if (q.rev && !(p & 1)) v = -v;
        }
        E[eb + (size_t)(k - 1) * st] = v;
    }
}

// inverse: node i of the DN form is output i of the transform, times 2 / n
__global__ void zq_scatter_inv(QArgs q, const double *__restrict__ E, double *__restrict__ W) {
    for (long t = blockIdx.x * (long)blockDim.x + threadIdx.x; t < q.lines * q.n;
         t += (long)gridDim.x * blockDim.x) {
        const long line = t / q.n;
        const int a = (int)(t - line * q.n);
        size_t wb, eb, st;
        q_line(q, line, wb, eb, st);
        const int e = q.rev ? q.n - 1 - a : a;
        W[wb + (size_t)a * st] = q.scale * E[eb + (size_t)e * st];
    }
}

__global__ void zfactor_kernel(double *fac, const double2 *rows, const double *cx,
                               const double *cy, int Nx, int Ny, int Nu) {
    const size_t plane = (size_t)Nx * Ny, n = plane * Nu;
    const size_t col = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
    if (col >= plane) return;
    const int q = (int)(col / Nx), p = (int)(col - (size_t)q * Nx);
    const double cp = cx[p], cq = cy[q];
    const double w4 = 4.0 * cp * cq, wb = 2.0 * cp, wc = 2.0 * cq;
    auto lam = [&](const double2 *b) {
        return make_double2(w4 * b[ZA].x + wb * b[ZB].x + wc * b[ZC].x + b[ZD].x,
                            w4 * b[ZA].y + wb * b[ZB].y + wc * b[ZC].y + b[ZD].y);
    };
    double *F0 = fac, *F1 = fac + 2 * n, *F2 = fac + 4 * n;
    double2 cprev = make_double2(0.0, 0.0);
    for (int r = 0; r < Nu; ++r) {
        const double2 *blk = rows + (size_t)r * 12;
        const double2 lo = lam(blk + ZLOW * 4), di = lam(blk + ZMID * 4), up = lam(blk + ZUPP * 4);
        const double2 piv = r ? csub(di, cmul(lo, cprev)) : di;
        const double inv = 1.0 / (piv.x * piv.x + piv.y * piv.y);
        const double2 ip = make_double2(piv.x * inv, -piv.y * inv);   // 1 / m_r
        const double2 li = r ? cmul(lo, ip) : make_double2(0.0, 0.0);
        const double2 c = cmul(up, ip);
        const size_t k = (size_t)r * plane + col;
        F0[k] = ip.x;
        F0[n + k] = ip.y;
        F1[k] = li.x;
        F1[n + k] = li.y;
        F2[k] = c.x;
        F2[n + k] = c.y;
        cprev = c;
    }
}

// The z-solves with the cached factors, in place on W [2][Nu][ny][nx]:
// d_r = rhs_r / m_r - (lower_r / m_r) d_{r-1}, then w_r = d_r - c'_r w_{r+1}.
// The sweeps walk each column ZCH rows at a time: a chunk's loads are all
// issued before its dependent chain and its in-place stores (which would
// otherwise keep the next row's loads from starting early).
constexpr int ZCH = 8;

__global__ void zthomas_kernel(double *__restrict__ W, const double *__restrict__ fac, int Nx,
                               int Ny, int Nu) {
    const size_t plane = (size_t)Nx * Ny, n = plane * Nu;
    const size_t col = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
    if (col >= plane) return;
    const double *F0 = fac, *F1 = fac + 2 * n, *F2 = fac + 4 * n;
    double2 d = make_double2(0.0, 0.0);
    int r = 0;
    for (; r + ZCH <= Nu; r += ZCH) {
        double2 rhs[ZCH], a[ZCH], b[ZCH];
#pragma unroll
        for (int c = 0; c < ZCH; ++c) {
            const size_t k = (size_t)(r + c) * plane + col;
            rhs[c] = make_double2(W[k], W[n + k]);
            a[c] = make_double2(F0[k], F0[n + k]);
            b[c] = make_double2(F1[k], F1[n + k]);
        }
#pragma unroll
        for (int c = 0; c < ZCH; ++c) {
            d = csub(cmul(rhs[c], a[c]), cmul(b[c], d));
            rhs[c] = d;
        }
#pragma unroll
        for (int c = 0; c < ZCH; ++c) {
            const size_t k = (size_t)(r + c) * plane + col;
            W[k] = rhs[c].x;
            W[n + k] = rhs[c].y;
        }
    }
    for (; r < Nu; ++r) {
        const size_t k = (size_t)r * plane + col;
        const double2 rhs = make_double2(W[k], W[n + k]);
        d = csub(cmul(rhs, make_double2(F0[k], F0[n + k])), cmul(make_double2(F1[k], F1[n + k]), d));
        W[k] = d.x;
        W[n + k] = d.y;
    }
    double2 w = d;
    r = Nu - 2;
    for (; r - ZCH + 1 >= 0; r -= ZCH) {
        double2 dv[ZCH], cc[ZCH];
#pragma unroll
        for (int c = 0; c < ZCH; ++c) {
            const size_t k = (size_t)(r - c) * plane + col;
            dv[c] = make_double2(W[k], W[n + k]);
            cc[c] = make_double2(F2[k], F2[n + k]);
        }
#pragma unroll
        for (int c = 0; c < ZCH; ++c) {
            w = csub(dv[c], cmul(cc[c], w));
            dv[c] = w;
        }
#pragma unroll
        for (int c = 0; c < ZCH; ++c) {
            const size_t k = (size_t)(r - c) * plane + col;
            W[k] = dv[c].x;
            W[n + k] = dv[c].y;
        }
    }
    for (; r >= 0; --r) {
        const size_t k = (size_t)r * plane + col;
        w = csub(make_double2(W[k], W[n + k]), cmul(make_double2(F2[k], F2[n + k]), w));
        W[k] = w.x;
        W[n + k] = w.y;
    }
}

// ------------------------------------------------------------ mixed precision
// FP64 -> FP32 copy of n values (the LU factors).
template <typename Tin>
__global__ void zround_kernel(const Tin *__restrict__ in, float *__restrict__ out, size_t n) {
    for (size_t k = blockIdx.x * (size_t)blockDim.x + threadIdx.x; k < n;
         k += (size_t)gridDim.x * blockDim.x)
        out[k] = (float)in[k];
}

// The z-solves of one correction in FP32 with the FP32-rounded cached factors
// (zthomas_kernel's recurrence).
__global__ void zthomas32_kernel(float *__restrict__ W, const float *__restrict__ fac, int Nx,
                                 int Ny, int Nu) {
    const size_t plane = (size_t)Nx * Ny, n = plane * Nu;
    const size_t col = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
    if (col >= plane) return;
    const float *F0 = fac, *F1 = fac + 2 * n, *F2 = fac + 4 * n;
    float dx = 0.f, dy = 0.f;
    auto fwd = [&](float rx, float ry, float ax, float ay, float bx, float by) {
        const float nx_ = (rx * ax - ry * ay) - (bx * dx - by * dy);
        const float ny_ = (rx * ay + ry * ax) - (bx * dy + by * dx);
        dx = nx_;
        dy = ny_;
    };
    int r = 0;
    for (; r + ZCH <= Nu; r += ZCH) {
        float rx[ZCH], ry[ZCH], ax[ZCH], ay[ZCH], bx[ZCH], by[ZCH];
#pragma unroll
        for (int c = 0; c < ZCH; ++c) {
            const size_t k = (size_t)(r + c) * plane + col;
            rx[c] = W[k];
            ry[c] = W[n + k];
            ax[c] = F0[k];
            ay[c] = F0[n + k];
            bx[c] = F1[k];
            by[c] = F1[n + k];
        }
#pragma unroll
        for (int c = 0; c < ZCH; ++c) {
            fwd(rx[c], ry[c], ax[c], ay[c], bx[c], by[c]);
            rx[c] = dx;
            ry[c] = dy;
        }
#pragma unroll
        for (int c = 0; c < ZCH; ++c) {
            const size_t k = (size_t)(r + c) * plane + col;
            W[k] = rx[c];
            W[n + k] = ry[c];
        }
    }
    for (; r < Nu; ++r) {
        const size_t k = (size_t)r * plane + col;
        fwd(W[k], W[n + k], F0[k], F0[n + k], F1[k], F1[n + k]);
        W[k] = dx;
        W[n + k] = dy;
    }
    float wx = dx, wy = dy;
    auto bwd = [&](float vx, float vy, float cx, float cy) {
        const float nx_ = vx - (cx * wx - cy * wy);
        const float ny_ = vy - (cx * wy + cy * wx);
        wx = nx_;
        wy = ny_;
    };
    r = Nu - 2;
    for (; r - ZCH + 1 >= 0; r -= ZCH) {
        float vx[ZCH], vy[ZCH], cx[ZCH], cy[ZCH];
#pragma unroll
        for (int c = 0; c < ZCH; ++c) {
            const size_t k = (size_t)(r - c) * plane + col;
            vx[c] = W[k];
            vy[c] = W[n + k];
            cx[c] = F2[k];
            cy[c] = F2[n + k];
        }
#pragma unroll
        for (int c = 0; c < ZCH; ++c) {
            bwd(vx[c], vy[c], cx[c], cy[c]);
            vx[c] = wx;
            vy[c] = wy;
        }
#pragma unroll
        for (int c = 0; c < ZCH; ++c) {
            const size_t k = (size_t)(r - c) * plane + col;
            W[k] = vx[c];
            W[n + k] = vy[c];
        }
    }
    for (; r >= 0; --r) {
        const size_t k = (size_t)r * plane + col;
        bwd(W[k], W[n + k], F2[k], F2[n + k]);
        W[k] = wx;
        W[n + k] = wy;
    }
}

// F (FP64 planar complex, n2 values) as FP32 pairs: hi parts at [0, n2), lo at
// [n2, 2 n2) -- the hi half is the FP32 input of the first solve.
__global__ void zsplit_kernel(const double *__restrict__ W, float *__restrict__ P, size_t n2) {
    for (size_t k = blockIdx.x * (size_t)blockDim.x + threadIdx.x; k < n2;
         k += (size_t)gridDim.x * blockDim.x) {
        const dfloat d = df_split_bits(W[k]);
        P[k] = d.hi;
        P[n2 + k] = d.lo;
    }
}

// zsplit_kernel for the unknown rows r0 .. r0 + nr - 1 only (real and imaginary
// planes; nu values per component).
__global__ void zsplit_rows_kernel(const double *__restrict__ W, float *__restrict__ P, size_t nu,
                                   int plane, int r0, int nr) {
    const int per = nr * plane;
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < 2 * per; t += gridDim.x * blockDim.x) {
        const int comp = t >= per;
        const size_t k = comp * nu + (size_t)r0 * plane + (t - comp * per);
        const dfloat d = df_split_bits(W[k]);
        P[k] = d.hi;
        P[2 * nu + k] = d.lo;
    }
}

// r = F - A U in FP32-pair arithmetic (rounding about 2^-46 of the largest term;
// the mixed path's residual): a CTA owns 32 x 8 columns and marches over the Nu
// unknown rows; each U plane (pairs, halo 1, zero beyond the Dirichlet side
// faces) is staged in shared memory once, every thread forms its plane sums
// (corners, x and y neighbours, centre; real and imaginary) once, and each row
// combines the sums of its three planes with its 3 x 4 complex pair
// coefficients.  r is written in FP32 (the input of the next FP32 solve).
constexpr int ZRX = 32, ZRY = 8;

struct ZSums {
    hs_tiles::LPair r[4], i[4];   // A (corners), B (x), C (y; with XY: x + y in B), D (centre)
};

// XY: the x and y coefficient pairs agree on every row (equal steps in x and y),
// so the x- and y-neighbour sums are added first and multiplied once (nine
// complex pair products per row instead of twelve).  Loading: the U plane two
// ahead and the F of the next row are fetched into registers before the
// current row's arithmetic, so their latency overlaps it; one barrier per plane
// (the slot a plane is stored into was last read two planes earlier).
// ULO: U has lo planes; else only its hi planes are read (the first residual of
// a one-sweep solve: the lo parts are zero and were never written).
template <bool XY, bool ULO = true>
__global__ void __launch_bounds__(ZRX * ZRY)
zresid_df_kernel(const float *__restrict__ Fp, const float *__restrict__ Up,
                 const float4 *__restrict__ rows4, float *__restrict__ r32, int nx, int ny, int Nu,
                 int rx, int ry) {
    using namespace hs_tiles;
    constexpr int HX = ZRX + 2, HY = ZRY + 2, NT = ZRX * ZRY;
    constexpr int PER = (HX * HY + NT - 1) / NT;
    __shared__ float4 ring[2][HY][HX];   // (re hi, re lo, im hi, im lo)
    const size_t plane = (size_t)nx * ny, nu = plane * Nu, n2 = 2 * nu;
    const int tid = threadIdx.x;
    const int tx = tid % ZRX, ty = tid / ZRX;
    const int i0 = blockIdx.x * ZRX, j0 = blockIdx.y * ZRY;
    const int i = i0 + tx, j = j0 + ty;
    const bool active = i < nx && j < ny;
    // this thread's halo elements: in-plane offset, -1 outside the unknown grid
    // (zero there: Dirichlet side faces), -2 past the halo tile.  rx / ry: the x / y
    // sides are Neumann faces, whose unknown grid includes the face nodes and
    // whose ghost beyond a face is the even reflection (the face data sit in F)
    int goff[PER];
#pragma unroll
    for (int q = 0; q < PER; ++q) {
        const int e = tid + q * NT;
        const int ey = e / HX, ex = e - ey * HX;
        int jj = j0 - 1 + ey, ii = i0 - 1 + ex;
        if (rx && ii == -1) ii = 1;
        if (rx && ii == nx) ii = nx - 2;
        if (ry && jj == -1) jj = 1;
        if (ry && jj == ny) jj = ny - 2;
        goff[q] = e >= HX * HY ? -2 : ((jj >= 0 && jj < ny && ii >= 0 && ii < nx) ? jj * nx + ii : -1);
    }
    float4 reg[PER];
    float4 fnext = make_float4(0.f, 0.f, 0.f, 0.f);
    auto fetch = [&](int rr) {   // U plane rr (zeros past the last plane)
#pragma unroll
        for (int q = 0; q < PER; ++q) {
            reg[q] = make_float4(0.f, 0.f, 0.f, 0.f);
            if (rr < Nu && goff[q] >= 0) {
                const size_t k = (size_t)rr * plane + goff[q];
                reg[q] = make_float4(Up[k], ULO ? Up[n2 + k] : 0.f, Up[nu + k],
                                     ULO ? Up[n2 + nu + k] : 0.f);
            }
        }
    };
    auto fetchF = [&](int rr) {
        if (active && rr < Nu) {
            const size_t k = (size_t)rr * plane + (size_t)j * nx + i;
            fnext = make_float4(Fp[k], Fp[n2 + k], Fp[nu + k], Fp[n2 + nu + k]);
        }
    };
    auto store = [&](int slot) {
        float4 *dst = &ring[slot][0][0];
#pragma unroll
        for (int q = 0; q < PER; ++q)
            if (goff[q] != -2) dst[tid + q * NT] = reg[q];
    };
    auto sums = [&](int slot, ZSums &S) {
        auto at = [&](int dy, int dx) { return ring[slot][ty + 1 + dy][tx + 1 + dx]; };
        const float4 a = at(-1, -1), b = at(-1, 1), c = at(1, -1), d = at(1, 1);
        S.r[0] = LPair{a.x, a.y};
        lp_add(S.r[0], b.x, b.y);
        lp_add(S.r[0], c.x, c.y);
        lp_add(S.r[0], d.x, d.y);
        S.i[0] = LPair{a.z, a.w};
        lp_add(S.i[0], b.z, b.w);
        lp_add(S.i[0], c.z, c.w);
        lp_add(S.i[0], d.z, d.w);
        const float4 xl = at(0, -1), xr = at(0, 1), yl = at(-1, 0), yr = at(1, 0), o = at(0, 0);
        S.r[1] = LPair{xl.x, xl.y};
        lp_add(S.r[1], xr.x, xr.y);
        S.i[1] = LPair{xl.z, xl.w};
        lp_add(S.i[1], xr.z, xr.w);
        if constexpr (XY) {
            lp_add(S.r[1], yl.x, yl.y);
            lp_add(S.r[1], yr.x, yr.y);
            lp_add(S.i[1], yl.z, yl.w);
            lp_add(S.i[1], yr.z, yr.w);
        } else {
            S.r[2] = LPair{yl.x, yl.y};
            lp_add(S.r[2], yr.x, yr.y);
            S.i[2] = LPair{yl.z, yl.w};
            lp_add(S.i[2], yr.z, yr.w);
        }
        S.r[3] = LPair{o.x, o.y};
        S.i[3] = LPair{o.z, o.w};
    };
    auto zero = [](ZSums &S) {
        for (int m = 0; m < 4; ++m) S.r[m] = S.i[m] = LPair{0.f, 0.f};
    };
    ZSums sm, s0, sp;
    zero(sm);
    zero(s0);
    zero(sp);
    fetch(0);
    store(0);
    __syncthreads();
    sums(0, s0);
    fetch(1);
    fetchF(0);
    for (int r = 0; r < Nu; ++r) {
        const float4 Fr = fnext;
        store((r + 1) & 1);   // plane r + 1 (zeros past the last)
        __syncthreads();
        fetch(r + 2);         // in flight during the arithmetic below
        fetchF(r + 1);
        sums((r + 1) & 1, sp);
        if (active) {
            const size_t k = (size_t)r * plane + (size_t)j * nx + i;
            LPair ar{Fr.x, Fr.y}, ai{Fr.z, Fr.w};
            const float4 *cf = rows4 + (size_t)r * 12;
            const ZSums *S3[3] = {&sm, &s0, &sp};
#pragma unroll
            for (int nuv = 0; nuv < 3; ++nuv) {
#pragma unroll
                for (int m = 0; m < 4; ++m) {
                    if (XY && m == 2) continue;
                    const float4 c = __ldg(cf + nuv * 4 + m);
                    const float2 cre = make_float2(c.x, c.y), cim = make_float2(c.z, c.w);
                    const LPair Sr = S3[nuv]->r[m], Si = S3[nuv]->i[m];
                    // F - (c_re + i c_im)(S_re + i S_im)
                    const LPair p1 = lp_mul(cre, Sr), p2 = lp_mul(cim, Si);
                    const LPair p3 = lp_mul(cre, Si), p4 = lp_mul(cim, Sr);
                    lp_add(ar, -p1.s, -p1.e);
                    lp_add(ar, p2);
                    lp_add(ai, -p3.s, -p3.e);
                    lp_add(ai, -p4.s, -p4.e);
                }
            }
            r32[k] = ar.s + ar.e;
            r32[nu + k] = ai.s + ai.e;
        }
        sm = s0;
        s0 = sp;
    }
}

// Side kinds the mixed-precision solve takes: Dirichlet (FP32 sine tiles) and
// Neumann on both faces of an axis (FP32 cosine tile, lengths with a compiled
// FFT); the quarter-wave axes have no FP32 tile.
bool mixed_sides_ok(const hs_zplan_s *Z, int x_kind, int y_kind) {
    const int k[2] = {x_kind, y_kind};
    const int N[2] = {Z->Nx, Z->Ny};
    for (int a = 0; a < 2; ++a) {
        if (k[a] == HS_SIDE_DIRICHLET) continue;
        if (k[a] != HS_SIDE_NEUMANN || !hs_dct32_size(N[a] + 1)) return false;
    }
    return true;
}

}  // namespace

extern "C" {

hs_status hs_zplan(hs_zplan_t *out, int Nx, int Ny, int Nz, double Lx, double Ly, double Lz,
                   int order) {
    if (!out) return HS_ERR_INVALID_ARG;
    *out = nullptr;
    if (Nx < 1 || Ny < 1 || Nz < 1 || !(Lx > 0) || !(Ly > 0) || !(Lz > 0)) return HS_ERR_INVALID_ARG;
    if (order != 2 && order != 4 && order != 6) return HS_ERR_INVALID_ARG;
    if (order == 6) {   // Section 3.4's rows assume one step in every direction
        const double hx = Lx / (Nx + 1), hy = Ly / (Ny + 1), hz = Lz / (Nz + 1);
        if (fabs(hx - hz) > 1e-12 * hz || fabs(hy - hz) > 1e-12 * hz) return HS_ERR_INVALID_ARG;
    }
    if (2.0 * (Nz + 2) * (double)(Nx + 2) * (Ny + 2) > 4.0e9) return HS_ERR_UNSUPPORTED;
    hs_zplan_s *Z = new (std::nothrow) hs_zplan_s();
    if (!Z) return HS_ERR_OOM;
    Z->Nx = Nx; Z->Ny = Ny; Z->Nz = Nz; Z->order = order;
    Z->Lx = Lx; Z->Ly = Ly; Z->Lz = Lz;
    Z->hx = Lx / (Nx + 1); Z->hy = Ly / (Ny + 1); Z->hz = Lz / (Nz + 1);
    Z->kind[0] = Z->kind[1] = HS_ZFACE_DIRICHLET;
    Z->alpha[0] = Z->alpha[1] = make_double2(1.0, 0.0);
    Z->beta[0] = Z->beta[1] = make_double2(0.0, 0.0);
    Z->side[0] = Z->side[1] = HS_SIDE_DIRICHLET;
    const hs_status st = layout(Z);
    if (st != HS_OK) {
        hs_zplan_destroy(Z);
        return st;
    }
    *out = Z;
    return HS_OK;
}

hs_status hs_zplan_set_coeff6(hs_zplan_t Z, const double *K, const double *Kz,
                              const double *Kzz) {
    if (!Z || !K || (Z->order == 6 && (!Kz || !Kzz))) return HS_ERR_INVALID_ARG;
    const int n = Z->Nz + 2;
    std::vector<double2> k(n), kz(n, make_double2(0.0, 0.0)), kzz(n, make_double2(0.0, 0.0));
    for (int l = 0; l < n; ++l) {
        if (!isfinite(K[2 * l]) || !isfinite(K[2 * l + 1])) return HS_ERR_INVALID_ARG;
        k[l] = make_double2(K[2 * l], K[2 * l + 1]);
        if (Z->order == 6) {
            if (!isfinite(Kz[2 * l]) || !isfinite(Kz[2 * l + 1]) || !isfinite(Kzz[2 * l]) ||
                !isfinite(Kzz[2 * l + 1]))
                return HS_ERR_INVALID_ARG;
            kz[l] = make_double2(Kz[2 * l], Kz[2 * l + 1]);
            kzz[l] = make_double2(Kzz[2 * l], Kzz[2 * l + 1]);
        }
    }
    if (Z->order == 6) {   // K and K_z for the right-hand side's K terms
        std::vector<double2> kk(2 * (size_t)n);
        for (int l = 0; l < n; ++l) {
            kk[l] = k[l];
            kk[n + l] = kz[l];
        }
        if (!Z->d_kk) ZCK(Z, cudaMalloc(&Z->d_kk, kk.size() * sizeof(double2)));
        ZCK(Z, cudaMemcpy(Z->d_kk, kk.data(), kk.size() * sizeof(double2),
                          cudaMemcpyHostToDevice));
    }
    Z->K = k;
    Z->Kz = kz;
    Z->Kzz = kzz;
    Z->have_coeff = 1;
    return build_rows(Z);
}

hs_status hs_zplan_set_precision(hs_zplan_t Z, int precision, int sweeps) {
    if (!Z || (precision != HS_FP64 && precision != HS_MIXED) || sweeps < 0 || sweeps > 8)
        return HS_ERR_INVALID_ARG;
    if (precision == HS_MIXED && !mixed_sides_ok(Z, Z->side[0], Z->side[1]))
        return HS_ERR_UNSUPPORTED;   // no FP32 quarter-wave tile; cosine lines need a compiled FFT
    Z->precision = precision;
    Z->sweeps = sweeps;
    return HS_OK;
}

hs_status hs_zplan_set_coeff(hs_zplan_t Z, const double *K) {
    if (!Z || !K || Z->order == 6) return HS_ERR_INVALID_ARG;   // order 6 needs K_z, K_zz
    return hs_zplan_set_coeff6(Z, K, nullptr, nullptr);
}

hs_status hs_zplan_set_faces(hs_zplan_t Z, int lo_kind, const double *alpha_lo,
                             const double *beta_lo, int hi_kind, const double *alpha_hi,
                             const double *beta_hi) {
    if (!Z) return HS_ERR_INVALID_ARG;
    const int kinds[2] = {lo_kind, hi_kind};
    const double *al[2] = {alpha_lo, alpha_hi}, *be[2] = {beta_lo, beta_hi};
    double2 na[2], nb[2];
    for (int s = 0; s < 2; ++s) {
        if (kinds[s] != HS_ZFACE_DIRICHLET && kinds[s] != HS_ZFACE_ROBIN) return HS_ERR_INVALID_ARG;
        na[s] = make_double2(1.0, 0.0);
        nb[s] = make_double2(0.0, 0.0);
        if (kinds[s] == HS_ZFACE_ROBIN) {
            if (!al[s] || !be[s]) return HS_ERR_INVALID_ARG;
            na[s] = make_double2(al[s][0], al[s][1]);
            nb[s] = make_double2(be[s][0], be[s][1]);
            if (!isfinite(na[s].x) || !isfinite(na[s].y) || !isfinite(nb[s].x) ||
                !isfinite(nb[s].y) || (na[s].x == 0.0 && na[s].y == 0.0))
                return HS_ERR_INVALID_ARG;
        }
    }
    for (int s = 0; s < 2; ++s) {
        Z->kind[s] = kinds[s];
        Z->alpha[s] = na[s];
        Z->beta[s] = nb[s];
    }
    const hs_status st = layout(Z);
    if (st != HS_OK) return st;
    return Z->have_coeff ? build_rows(Z) : HS_OK;
}

hs_status hs_zplan_set_sides(hs_zplan_t Z, int x_kind, int y_kind) {
    if (!Z) return HS_ERR_INVALID_ARG;
    const int k[2] = {x_kind, y_kind};
    for (int a = 0; a < 2; ++a)
        if (k[a] < HS_SIDE_DIRICHLET || k[a] > HS_SIDE_ND) return HS_ERR_INVALID_ARG;
    // the 6th-order right-hand side's ghosts are defined for Dirichlet side faces,
    // and the mixed-precision solve has FP32 sine and cosine tiles (no quarter-wave)
    if (Z->order == 6 && (x_kind != HS_SIDE_DIRICHLET || y_kind != HS_SIDE_DIRICHLET))
        return HS_ERR_UNSUPPORTED;
    if (Z->precision == HS_MIXED && !mixed_sides_ok(Z, x_kind, y_kind)) return HS_ERR_UNSUPPORTED;
    // lengths without a compiled FFT take the runtime-sized transforms (direct sums
    // for a cosine axis, the sine plan's own fallback for the extended lines of a
    // mixed axis); a layout that cannot be built leaves the previous kinds in place
    const int old[2] = {Z->side[0], Z->side[1]};
    Z->side[0] = x_kind;
    Z->side[1] = y_kind;
    const hs_status st = layout(Z);
    if (st != HS_OK) {
        Z->side[0] = old[0];
        Z->side[1] = old[1];
        if (layout(Z) == HS_OK && Z->have_coeff) (void)build_rows(Z);
        return st;
    }
    return Z->have_coeff ? build_rows(Z) : HS_OK;
}

hs_status hs_zsolve(hs_zplan_t Z, const double *f, const double *g_lo, const double *g_hi,
                    double *u, void *stream) {
    return hs_zsolve_ex(Z, f, g_lo, g_hi, nullptr, u, stream);
}

hs_status hs_zsolve_ex(hs_zplan_t Z, const double *f, const double *g_lo, const double *g_hi,
                       const double *const *side, double *u, void *stream) {
    return hs_zsolve_full(Z, f, g_lo, g_hi, side, nullptr, u, stream);
}

hs_status hs_zsolve_full(hs_zplan_t Z, const double *f, const double *g_lo, const double *g_hi,
                         const double *const *side, const double *const *fnn, double *u,
                         void *stream) {
    HsRange range("hs_zsolve");
    if (!Z || !f || !u) return HS_ERR_INVALID_ARG;
    if (!Z->layout_ok) {
        zerr(Z, "plan set-up incomplete: an earlier set-up call failed part-way");
        return HS_ERR_NO_COEFF;
    }
    if (!Z->have_coeff || !Z->rows_ok) return HS_ERR_NO_COEFF;
    if (!device_ptr(f) || !device_ptr(u) || (g_lo && !device_ptr(g_lo)) ||
        (g_hi && !device_ptr(g_hi)))
        return HS_ERR_INVALID_ARG;
    const double *sd[4] = {nullptr, nullptr, nullptr, nullptr};
    for (int k = 0; side && k < 4; ++k) {
        if (!side[k]) continue;
        // data on a Dirichlet face have no meaning
        const int kind = Z->side[k / 2];
        const bool neu = kind == HS_SIDE_NEUMANN || (kind == HS_SIDE_ND && k % 2 == 0) ||
                         (kind == HS_SIDE_DN && k % 2 == 1);
        if (!neu || !device_ptr(side[k])) return HS_ERR_INVALID_ARG;
        sd[k] = side[k];
    }
    const double *fd[6] = {nullptr, nullptr, nullptr, nullptr, nullptr, nullptr};
    for (int k = 0; fnn && Z->order == 6 && k < 6; ++k) {
        if (fnn[k] && !device_ptr(fnn[k])) return HS_ERR_INVALID_ARG;
        fd[k] = fnn[k];
    }
    Z->last_error[0] = 0;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    hs_plan_s *T = Z->T;
    const size_t plane = (size_t)Z->nx * Z->ny;
    const size_t nu = plane * Z->Nu;
    double *W = T->d_w64;
    ZRhsArgs a;
    a.Nx = Z->Nx; a.Ny = Z->Ny; a.Nz = Z->Nz; a.Nu = Z->Nu; a.l0 = Z->l0; a.order = Z->order;
    a.nx = Z->nx; a.ny = Z->ny; a.i0x = Z->i0x; a.i0y = Z->i0y;
    a.neu_x = Z->side[0] != HS_SIDE_DIRICHLET;
    a.neu_y = Z->side[1] != HS_SIDE_DIRICHLET;
    a.nlo_x = Z->side[0] == HS_SIDE_NEUMANN || Z->side[0] == HS_SIDE_ND;
    a.nhi_x = Z->side[0] == HS_SIDE_NEUMANN || Z->side[0] == HS_SIDE_DN;
    a.nlo_y = Z->side[1] == HS_SIDE_NEUMANN || Z->side[1] == HS_SIDE_ND;
    a.nhi_y = Z->side[1] == HS_SIDE_NEUMANN || Z->side[1] == HS_SIDE_DN;
    a.kind_lo = Z->kind[0]; a.kind_hi = Z->kind[1];
    a.hz = Z->hz;
    a.ga_lo = cscale(2.0 * Z->hz, cdiv_host(make_double2(1.0, 0.0), Z->alpha[0]));
    a.ga_hi = cscale(2.0 * Z->hz, cdiv_host(make_double2(1.0, 0.0), Z->alpha[1]));
    a.f = f; a.g_lo = g_lo; a.g_hi = g_hi; a.rows = Z->d_rows; a.W = W;
    for (int k = 0; k < 4; ++k) a.side[k] = sd[k];
    for (int k = 0; k < 6; ++k) a.fnn[k] = fd[k];
    a.kk = Z->d_kk;
    a.hx = Z->hx;
    a.hy = Z->hy;
    {
        const double h2 = Z->hz * Z->hz;
        a.k20 = -h2 * h2 / 20.0;
        a.k120 = h2 * h2 * Z->hz / 120.0;
    }
    (void)nu;
    const dim3 blocks((unsigned)((plane + 255) / 256), (unsigned)Z->Nu, 1);
    auto mark = [&](int k) -> hs_status {
        if (Z->timing && Z->have_ev) ZCK(Z, cudaEventRecord(Z->ev[k], s));
        return HS_OK;
    };
    hs_status mk;
    if ((mk = mark(0)) != HS_OK) return mk;
    // mixed precision at orders 2 and 4 without side-face data: the rows past the
    // first two and before the last two take the plain interior formula, formed
    // in pair arithmetic straight into the pair planes; the edge rows (Robin
    // rows, rows next to a Dirichlet face) in FP64 as usual, split afterwards
    const bool pair_rhs = Z->precision == HS_MIXED && Z->order <= 4 && !sd[0] && !sd[1] &&
                          !sd[2] && !sd[3];
    const int e0 = Z->Nu < 2 ? Z->Nu : 2, e1 = Z->Nu - 2 > e0 ? Z->Nu - 2 : e0;
    a.rbase = 0;
    if (!pair_rhs) {
        zrhs_kernel<<<blocks, 256, 0, s>>>(a);
        ZCK(Z, cudaGetLastError());
    } else {
        if (!Z->d_Fp) ZCK(Z, cudaMalloc(&Z->d_Fp, 4 * nu * sizeof(float)));
        zrhs_kernel<<<dim3(blocks.x, (unsigned)e0, 1), 256, 0, s>>>(a);
        ZCK(Z, cudaGetLastError());
        if (Z->Nu > e1) {
            a.rbase = e1;
            zrhs_kernel<<<dim3(blocks.x, (unsigned)(Z->Nu - e1), 1), 256, 0, s>>>(a);
            ZCK(Z, cudaGetLastError());
        }
        if (e1 > e0) {
            const double h2 = Z->hz * Z->hz;
            auto pair = [](double x) {
                const float hi = (float)x;
                return make_float2(hi, (float)(x - (double)hi));
            };
            a.rbase = e0;
            zrhs_pair_kernel<<<dim3(blocks.x, (unsigned)(e1 - e0), 1), 256, 0, s>>>(
                a, Z->d_Fp, pair(Z->order == 4 ? 0.5 * h2 : h2), pair(h2 / 12.0));
            ZCK(Z, cudaGetLastError());
        }
        a.rbase = 0;
    }
    if ((a.neu_x && (sd[0] || sd[1])) || (a.neu_y && (sd[2] || sd[3]))) {
        const size_t rows = 2 * (size_t)Z->Nu * (Z->nx + Z->ny);
        zside_kernel<<<(unsigned)((rows + 127) / 128), 128, 0, s>>>(a);
        ZCK(Z, cudaGetLastError());
    }
    if ((mk = mark(1)) != HS_OK) return mk;
    // one transform pass along an axis: the cosine kernel on a Neumann axis, the
    // quarter-wave gather / extended sine transform / scatter on a mixed one, else
    // the plan's sine transform; inverse passes carry 2 / (N + 1) for each kind
    auto pass = [&](int axis, bool fwd, double scale) -> hs_status {
        if (Z->side[axis] == HS_SIDE_DN || Z->side[axis] == HS_SIDE_ND) {
            hs_plan_s *Q = Z->TQ[axis];
            QArgs q;
            q.axis = axis;
            q.n = axis == HS_AXIS_X ? Z->nx : Z->ny;
            q.nx = Z->nx;
            q.ny = Z->ny;
            q.rev = Z->side[axis] == HS_SIDE_ND;
            q.lines = (long)2 * Z->Nu * (axis == HS_AXIS_X ? Z->ny : Z->nx);
            q.scale = scale;
            const long work = q.lines * (2 * q.n - 1);
            const unsigned qb = (unsigned)((work + 255) / 256 < 152 * 16 ? (work + 255) / 256 : 152 * 16);
            if (fwd)
                zq_gather_fwd<<<qb, 256, 0, s>>>(q, W, Q->d_w64);
            else
                zq_gather_inv<<<qb, 256, 0, s>>>(q, W, Q->d_w64);
            if (cudaGetLastError() != cudaSuccess) return HS_ERR_CUDA;
            const hs_status sq = hs_launch_dst(Q, axis, HS_T_F64, HS_T_F64, Q->d_w64, HS_T_F64,
                                               Q->d_w64, HS_MODE_WRITE, 1.0, s);
            if (sq != HS_OK) return sq;
            if (fwd)
                zq_scatter_fwd<<<qb, 256, 0, s>>>(q, Q->d_w64, W);
            else
                zq_scatter_inv<<<qb, 256, 0, s>>>(q, Q->d_w64, W);
            return cudaGetLastError() == cudaSuccess ? HS_OK : HS_ERR_CUDA;
        }
        if (Z->side[axis] == HS_SIDE_NEUMANN) {
            const int M = (axis == HS_AXIS_X ? Z->Nx : Z->Ny) + 1;
            const double2 *t = Z->d_dct[axis];
            return hs_launch_dct(axis, M, W, W, t, t + M, (long)Z->ny * 2 * Z->Nu, Z->nx,
                                 2 * Z->Nu, scale, s);
        }
        return hs_launch_dst(T, axis, HS_T_F64, HS_T_F64, W, HS_T_F64, W, HS_MODE_WRITE, scale, s);
    };
    hs_status st;
    const double *Wout = W;   // the unknown planes' solution
    if (Z->precision == HS_MIXED) {
        // U_0 = M F, U_{m+1} = U_m + M (F - A U_m) with M the FP32 solve (FP32
        // transforms and z-solves on FP32-rounded factors); F and U are FP32 pairs
        // and the residual is formed in pair arithmetic; the last correction is
        // added in FP64.  The stage events see the whole loop as the transform stage.
        const size_t n2 = 2 * nu;
        if (!Z->d_w32) ZCK(Z, cudaMalloc(&Z->d_w32, n2 * sizeof(float)));
        if (!Z->d_U) ZCK(Z, cudaMalloc(&Z->d_U, n2 * sizeof(double)));
        if (!Z->d_fac32) ZCK(Z, cudaMalloc(&Z->d_fac32, 3 * n2 * sizeof(float)));
        if (!Z->d_Fp) ZCK(Z, cudaMalloc(&Z->d_Fp, 2 * n2 * sizeof(float)));
        if (!Z->d_Up) ZCK(Z, cudaMalloc(&Z->d_Up, 2 * n2 * sizeof(float)));
        if (!Z->d_rows32) {
            ZCK(Z, cudaMalloc(&Z->d_rows32, (size_t)Z->Nu * 12 * sizeof(float4)));
            const hs_status rs = build_rows(Z);
            if (rs != HS_OK) return rs;
        }
        if (!Z->fac_ok) {
            zfactor_kernel<<<(unsigned)((plane + 127) / 128), 128, 0, s>>>(
                Z->d_fac, Z->d_rows, Z->d_cos, Z->d_cos + Z->nx, Z->nx, Z->ny, Z->Nu);
            ZCK(Z, cudaGetLastError());
            Z->fac_ok = 1;
            Z->fac32_ok = 0;
        }
        const unsigned eb = (unsigned)((n2 + 255) / 256 < 152 * 16 ? (n2 + 255) / 256 : 152 * 16);
        if (!Z->fac32_ok) {
            zround_kernel<double><<<eb, 256, 0, s>>>(Z->d_fac, Z->d_fac32, 3 * n2);
            ZCK(Z, cudaGetLastError());
            Z->fac32_ok = 1;
        }
        if (!pair_rhs) {
            zsplit_kernel<<<eb, 256, 0, s>>>(W, Z->d_Fp, n2);
            ZCK(Z, cudaGetLastError());
        } else {
            // the edge rows formed in FP64 (the others are pairs already)
            for (int side = 0; side < 2; ++side) {
                const int r0 = side == 0 ? 0 : e1, nr = side == 0 ? e0 : Z->Nu - e1;
                if (nr <= 0) continue;
                const int work = 2 * nr * (int)plane;
                zsplit_rows_kernel<<<(unsigned)((work + 255) / 256), 256, 0, s>>>(
                    W, Z->d_Fp, nu, (int)plane, r0, nr);
                ZCK(Z, cudaGetLastError());
            }
        }
        // the FP32 transforms take the fused tiles where the length is compiled
        // (the plan's own variant is for its FP64 passes)
        const int saved[2] = {T->dst_variant[0], T->dst_variant[1]};
        for (int a = 0; a < 2; ++a)
            if (hs_dst_fast_size(T->axf[a].M)) T->dst_variant[a] = HS_DST_FUSED;
        float *w = Z->d_w32;
        const double sx = 2.0 / (Z->Nx + 1), sy = 2.0 / (Z->Ny + 1);
        const dim3 rgrid((unsigned)((Z->nx + ZRX - 1) / ZRX), (unsigned)((Z->ny + ZRY - 1) / ZRY));
        const int sw = Z->sweeps;
        st = HS_OK;
        // one FP32 pass: the cosine tile on a Neumann axis, else the sine tiles
        auto pass32 = [&](int axis, const float *pin, int tout, void *pout, int mode,
                          double scale, double *paux) -> hs_status {
            if (Z->side[axis] == HS_SIDE_NEUMANN) {
                const int M = (axis == HS_AXIS_X ? Z->Nx : Z->Ny) + 1;
                const float2 *t = Z->d_dct32[axis];
                return hs_launch_dct32(axis, M, tout, mode, pin, pout, paux, n2, t, t + M,
                                       (long)Z->ny * 2 * Z->Nu, Z->nx, 2 * Z->Nu, scale, s);
            }
            return hs_launch_dst(T, axis, HS_T_F32, HS_T_F32, pin, tout, pout, mode, scale, s,
                                 paux);
        };
        const int rx = Z->side[0] == HS_SIDE_NEUMANN, ry = Z->side[1] == HS_SIDE_NEUMANN;
        // one sweep: the first solve writes only U's hi planes, and the residual and
        // the final update read only those (the lo parts are zero until the
        // correction is added); the results are those of the pair sequence
        const bool hi_only = sw == 1;
        for (int m = 0; m <= sw && st == HS_OK; ++m) {
            const float *in = w;
            if (m == 0) {
                in = Z->d_Fp;   // F_hi
            } else {
                auto kern = Z->resid_xy ? (hi_only ? zresid_df_kernel<true, false>
                                                   : zresid_df_kernel<true, true>)
                                        : (hi_only ? zresid_df_kernel<false, false>
                                                   : zresid_df_kernel<false, true>);
                kern<<<rgrid, ZRX * ZRY, 0, s>>>(Z->d_Fp, Z->d_Up, Z->d_rows32, w, Z->nx, Z->ny,
                                                 Z->Nu, rx, ry);
                if (cudaGetLastError() != cudaSuccess) st = HS_ERR_CUDA;
            }
            if (st == HS_OK) st = pass32(HS_AXIS_X, in, HS_T_F32, w, HS_MODE_WRITE, 1.0, nullptr);
            if (st == HS_OK) st = pass32(HS_AXIS_Y, w, HS_T_F32, w, HS_MODE_WRITE, 1.0, nullptr);
            if (st == HS_OK) {
                zthomas32_kernel<<<(unsigned)((plane + 127) / 128), 128, 0, s>>>(w, Z->d_fac32, Z->nx,
                                                                               Z->ny, Z->Nu);
                if (cudaGetLastError() != cudaSuccess) st = HS_ERR_CUDA;
            }
            if (st == HS_OK) st = pass32(HS_AXIS_Y, w, HS_T_F32, w, HS_MODE_WRITE, sy, nullptr);
            if (st != HS_OK) break;
            // the iterate: FP64 U straight away without refinement, else pairs (set,
            // add) and, on the last sweep, U + correction in FP64
            if (sw == 0)
                st = pass32(HS_AXIS_X, w, HS_T_F64, Z->d_U, HS_MODE_WRITE, sx, nullptr);
            else if (hi_only && m == 0)
                st = pass32(HS_AXIS_X, w, HS_T_F32, Z->d_Up, HS_MODE_WRITE, sx, nullptr);
            else if (hi_only)
                st = pass32(HS_AXIS_X, w, HS_T_DF, Z->d_Up, HS_MODE_DF_FINAL_HI, sx, Z->d_U);
            else
                st = pass32(HS_AXIS_X, w, HS_T_DF, Z->d_Up,
                            m == 0 ? HS_MODE_DF_SET : (m < sw ? HS_MODE_DF_ADD : HS_MODE_DF_FINAL),
                            sx, Z->d_U);
        }
        T->dst_variant[0] = saved[0];
        T->dst_variant[1] = saved[1];
        if (st != HS_OK) {
            zerr(Z, "mixed-precision solve: status %d", st);
            return st;
        }
        Wout = Z->d_U;
        if ((mk = mark(2)) != HS_OK || (mk = mark(3)) != HS_OK || (mk = mark(4)) != HS_OK) return mk;
    } else {
    if ((st = pass(HS_AXIS_X, true, 1.0)) != HS_OK || (st = pass(HS_AXIS_Y, true, 1.0)) != HS_OK) {
        zerr(Z, "forward transform: status %d", st);
        return st;
    }
    if ((mk = mark(2)) != HS_OK) return mk;
    if (!Z->fac_ok) {   // first solve after a change of coefficients, faces or sides
        zfactor_kernel<<<(unsigned)((plane + 127) / 128), 128, 0, s>>>(
            Z->d_fac, Z->d_rows, Z->d_cos, Z->d_cos + Z->nx, Z->nx, Z->ny, Z->Nu);
        ZCK(Z, cudaGetLastError());
        Z->fac_ok = 1;
    }
    zthomas_kernel<<<(unsigned)((plane + 127) / 128), 128, 0, s>>>(W, Z->d_fac, Z->nx, Z->ny,
                                                                 Z->Nu);
    ZCK(Z, cudaGetLastError());
    if ((mk = mark(3)) != HS_OK) return mk;
    if ((st = pass(HS_AXIS_Y, false, 2.0 / (Z->Ny + 1))) != HS_OK ||
        (st = pass(HS_AXIS_X, false, 2.0 / (Z->Nx + 1))) != HS_OK) {
        zerr(Z, "inverse transform: status %d", st);
        return st;
    }
    if ((mk = mark(4)) != HS_OK) return mk;
    }
    // unknown planes into u; Dirichlet planes receive their face data
    const size_t uplanes = (size_t)Z->Nz + 2;
    for (int comp = 0; comp < 2; ++comp) {
        double *uc = u + comp * uplanes * plane;
        ZCK(Z, cudaMemcpyAsync(uc + (size_t)Z->l0 * plane, Wout + comp * nu, nu * sizeof(double),
                               cudaMemcpyDeviceToDevice, s));
        for (int side = 0; side < 2; ++side) {
            if (Z->kind[side] != HS_ZFACE_DIRICHLET) continue;
            double *dst = uc + (side == 0 ? 0 : (size_t)(Z->Nz + 1) * plane);
            const double *g = side == 0 ? g_lo : g_hi;
            if (g)
                ZCK(Z, cudaMemcpyAsync(dst, g + comp * plane, plane * sizeof(double),
                                       cudaMemcpyDeviceToDevice, s));
            else
                ZCK(Z, cudaMemsetAsync(dst, 0, plane * sizeof(double), s));
        }
    }
    return mark(5);
}

hs_status hs_zplan_set_stage_timing(hs_zplan_t Z, int on) {
    if (!Z) return HS_ERR_INVALID_ARG;
    if (on && !Z->have_ev) {
        for (int k = 0; k < 6; ++k) {
            if (cudaEventCreate(&Z->ev[k]) != cudaSuccess) {
                cudaGetLastError();
                for (int j = 0; j < k; ++j) cudaEventDestroy(Z->ev[j]);
                return HS_ERR_CUDA;
            }
        }
        Z->have_ev = 1;
    }
    Z->timing = on ? 1 : 0;
    return HS_OK;
}

hs_status hs_zplan_stage_times(hs_zplan_t Z, float *ms) {
    if (!Z || !ms) return HS_ERR_INVALID_ARG;
    if (!Z->have_ev) return HS_ERR_INVALID_ARG;
    ZCK(Z, cudaEventSynchronize(Z->ev[5]));
    for (int k = 0; k < 5; ++k) ZCK(Z, cudaEventElapsedTime(&ms[k], Z->ev[k], Z->ev[k + 1]));
    return HS_OK;
}

size_t hs_zplan_workspace_bytes(hs_zplan_t Z) {
    if (!Z) return 0;
    size_t b = hs_workspace_bytes(Z->T) + (Z->d_rows ? (size_t)Z->Nu * 12 * sizeof(double2) : 0);
    for (int a = 0; a < 2; ++a) b += hs_workspace_bytes(Z->TQ[a]);
    b += (size_t)(Z->nx + Z->ny) * sizeof(double);
    if (Z->d_fac) b += (size_t)6 * Z->Nu * Z->nx * Z->ny * sizeof(double);
    if (Z->d_dct[0]) b += (2 * (size_t)Z->Nx + 3) * (sizeof(double2) + sizeof(float2));
    if (Z->d_dct[1]) b += (2 * (size_t)Z->Ny + 3) * (sizeof(double2) + sizeof(float2));
    return b;
}

const char *hs_zplan_last_error(hs_zplan_t Z) {
    if (!Z) return "no plan";
    if (Z->last_error[0]) return Z->last_error;
    return Z->T ? hs_last_error(Z->T) : "";
}

void hs_zplan_destroy(hs_zplan_t Z) {
    if (!Z) return;
    if (Z->T) hs_destroy(Z->T);
    for (int a = 0; a < 2; ++a)
        if (Z->TQ[a]) hs_destroy(Z->TQ[a]);
    if (Z->d_kk) cudaFree(Z->d_kk);
    free_mixed(Z);
    if (Z->d_rows) cudaFree(Z->d_rows);
    if (Z->d_cos) cudaFree(Z->d_cos);
    if (Z->d_fac) cudaFree(Z->d_fac);
    for (int a = 0; a < 2; ++a) {
        if (Z->d_dct[a]) cudaFree(Z->d_dct[a]);
        if (Z->d_dct32[a]) cudaFree(Z->d_dct32[a]);
    }
    if (Z->have_ev)
        for (int k = 0; k < 6; ++k) cudaEventDestroy(Z->ev[k]);
    delete Z;
}

}  // extern "C"
