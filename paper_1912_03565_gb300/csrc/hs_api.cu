// C ABI of the solver (declared in include/hs.h): plan creation, coefficient
// tables, the solve pipeline and diagnostics.  Host code only; the kernels
// live in k_dst.cu, k_rhs.cu and k_thomas.cu.
//
// Solve pipeline (Section 3.6 with Algorithm 1's three phases, per RHS):
//   FP64 path:  F = R_h f - lift          (k_rhs, FP64)
//               Fhat = DST_y DST_x F       (k_dst, FP64, in place)
//               W = T_pq^{-1} Fhat         (k_thomas, FP64, cached LU)
//               U = 4/((Nx+1)(Ny+1)) DST_x DST_y W
//   Mixed path: F as above, kept as FP32 pairs; U_0 = 0; for m = 0..sweeps:
//               r = F - A U_m (27-point, FP32-pair or FP64 arithmetic; r = F
//               for m = 0), rounded to FP32,
//               U_{m+1} = U_m + (FP32 DSTs, FP32 z-solves with FP32 or FP64
//               factors) r, U held as FP32 pairs.
#include <math.h>
#include <stdarg.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <new>
#include <vector>

#include "hs_internal.cuh"

namespace {

void set_err(hs_plan_s *P, const char *fmt, ...) {
    if (!P) return;
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(P->last_error, sizeof(P->last_error), fmt, ap);
    va_end(ap);
}

#define HS_CK(P, call)                                                                   \
    do {                                                                                 \
        cudaError_t e_ = (call);                                                         \
        if (e_ != cudaSuccess) {                                                         \
            set_err(P, "%s failed: %s", #call, cudaGetErrorString(e_));                  \
            return (e_ == cudaErrorMemoryAllocation) ? HS_ERR_OOM : HS_ERR_CUDA;         \
        }                                                                                \
    } while (0)

#define HS_TRY(P, expr)                                                                  \
    do {                                                                                 \
        hs_status st_ = (expr);                                                          \
        if (st_ < 0) {                                                                   \
            if (!P->last_error[0]) set_err(P, "%s failed (%d): %s", #expr, st_,           \
                                           cudaGetErrorString(cudaGetLastError()));      \
            return st_;                                                                  \
        }                                                                                \
    } while (0)

// Stages of M = 2^a 3^b (4s, then one 2, then 3s); 0 when M has another factor.
int plan_radix(int M, int *radix, int *nst) {
    int n = 0;
    while (M % 4 == 0 && n < HS_MAX_STAGES) { radix[n++] = 4; M /= 4; }
    while (M % 2 == 0 && n < HS_MAX_STAGES) { radix[n++] = 2; M /= 2; }
    while (M % 3 == 0 && n < HS_MAX_STAGES) { radix[n++] = 3; M /= 3; }
    *nst = n;
    return M == 1 ? 1 : 0;
}

// sin(pi * num / den) with the argument reduced exactly to [0, pi/2]
// before the FP64 sine (num, den integers, den > 0).
double sin_pi_ratio(long num, long den) {
    long m = num % (2 * den);
    if (m < 0) m += 2 * den;
    double sign = 1.0;
    if (m >= den) { m -= den; sign = -1.0; }        // sin(x + pi) = -sin x
    if (2 * m > den) m = den - m;                   // sin(pi - x) = sin x
    return sign * sin(M_PI * (double)m / (double)den);
}
double cos_pi_ratio(long num, long den) { return sin_pi_ratio(2 * num + den, 2 * den); }

bool is_device_ptr(const void *p) {
    if (!p) return true;
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

// The device alias of pinned (page-locked, mapped) host memory, else NULL.
void *mapped_host(const void *p) {
    cudaPointerAttributes a;
    if (!p || cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    return a.type == cudaMemoryTypeHost ? a.devicePointer : nullptr;
}

// The upload stream and events of the pipelined host-f copy (created once per plan).
hs_status ensure_upload(hs_plan_s *P) {
    if (P->have_up) return HS_OK;
    if (cudaStreamCreateWithFlags(&P->up_stream, cudaStreamNonBlocking) != cudaSuccess) {
        cudaGetLastError();
        return HS_ERR_CUDA;
    }
    const int nev = HS_UP_CHUNKS + 3 + P->max_rhs;
    P->up_rhs = new (std::nothrow) cudaEvent_t[P->max_rhs];
    if (!P->up_rhs) {
        cudaStreamDestroy(P->up_stream);
        return HS_ERR_OOM;
    }
    auto ev = [&](int k) -> cudaEvent_t & {
        return k < HS_UP_CHUNKS + 3 ? P->up_ev[k] : P->up_rhs[k - HS_UP_CHUNKS - 3];
    };
    for (int k = 0; k < nev; ++k) {
        if (cudaEventCreateWithFlags(&ev(k), cudaEventDisableTiming) != cudaSuccess) {
            cudaGetLastError();
            for (int j = 0; j < k; ++j) cudaEventDestroy(ev(j));
            delete[] P->up_rhs;
            P->up_rhs = nullptr;
            cudaStreamDestroy(P->up_stream);
            return HS_ERR_CUDA;
        }
    }
    P->f_buf = 0;
    P->have_up = 1;
    return HS_OK;
}

// The download stream and events of HS_HOST_U_LATE (created once per plan).
hs_status ensure_download(hs_plan_s *P) {
    if (P->have_dn) return HS_OK;
    if (cudaStreamCreateWithFlags(&P->dn_stream, cudaStreamNonBlocking) != cudaSuccess) {
        cudaGetLastError();
        return HS_ERR_CUDA;
    }
    for (int k = 0; k < 3; ++k) {
        if (cudaEventCreateWithFlags(&P->dn_ev[k], cudaEventDisableTiming) != cudaSuccess) {
            cudaGetLastError();
            for (int j = 0; j < k; ++j) cudaEventDestroy(P->dn_ev[j]);
            cudaStreamDestroy(P->dn_stream);
            return HS_ERR_CUDA;
        }
    }
    P->dn_pending[0] = P->dn_pending[1] = 0;
    P->dn_last = -1;
    P->u_buf = 0;
    P->have_dn = 1;
    return HS_OK;
}

// Work queued on s next may overwrite u staging buffer b: it waits for a
// queued copy of that buffer to the host.
hs_status guard_stage_u(hs_plan_s *P, int b, cudaStream_t s) {
    if (P->have_dn && P->dn_pending[b])
        HS_CK(P, cudaStreamWaitEvent(s, P->dn_ev[b], 0));
    return HS_OK;
}

template <typename T>
hs_status dev_alloc(hs_plan_s *P, T **p, size_t n) {
    *p = nullptr;
    if (n == 0) return HS_OK;
    HS_CK(P, cudaMalloc((void **)p, n * sizeof(T)));
    P->bytes += n * sizeof(T);
    return HS_OK;
}

void free_ytmp(hs_plan_s *P) {
    if (!P->d_ytmp) return;
    cudaFree(P->d_ytmp);
    P->bytes -= (size_t)P->Nz * P->axf[HS_AXIS_Y].M * P->Nx * 2 * sizeof(float);
    P->d_ytmp = nullptr;
}

// The tensor-core transform's split sine matrix of one axis (and the plan's
// error flag of those kernels), built on first use.
hs_status ensure_gemm_table(hs_plan_s *P, int axis) {
    if (!P->d_gemm_err) {
        HS_TRY(P, dev_alloc(P, &P->d_gemm_err, (size_t)1));
        HS_CK(P, cudaMemset(P->d_gemm_err, 0, sizeof(int)));
    }
    if (P->d_gemm[axis]) return HS_OK;
    const int M = P->axf[axis].M;
    const size_t bytes = hs_dst_gemm_table_bytes(M);
    std::vector<uint8_t> h(bytes);
    hs_dst_gemm_table(M, h.data());
    uint8_t *d = nullptr;
    HS_TRY(P, dev_alloc(P, &d, bytes));
    P->d_gemm[axis] = d;
    HS_CK(P, cudaMemcpy(d, h.data(), bytes, cudaMemcpyHostToDevice));
    return HS_OK;
}

// HS_ERR_TIMEOUT (and the flag cleared) when a tensor-core transform gave up a
// wait since the last check; synchronous.
hs_status check_gemm_err(hs_plan_s *P) {
    if (!P->d_gemm_err) return HS_OK;
    int e = 0;
    HS_CK(P, cudaMemcpy(&e, P->d_gemm_err, sizeof(int), cudaMemcpyDeviceToHost));
    if (!e) return HS_OK;
    HS_CK(P, cudaMemset(P->d_gemm_err, 0, sizeof(int)));
    set_err(P, "a tensor-core transform kernel gave up a wait");
    return HS_ERR_TIMEOUT;
}

void free_plan(hs_plan_s *P) {
    if (!P) return;
    void *ptrs[] = {P->d_coef, P->d_c0, P->d_c1, P->d_cx, P->d_cy, P->d_fac, P->d_red,
                    P->d_tables, P->d_w64, P->d_w32, P->d_dscr, P->d_stage_f, P->d_stage_u,
                    P->d_stage_bnd, P->d_fac32, P->d_coef_df, P->d_Fdf, P->d_Udf, P->d_rhs_df,
                    P->d_skip, P->d_ytmp, P->d_stage_u1, P->d_stage_f1, P->d_stage_bnd1,
                    P->d_gemm[0], P->d_gemm[1], P->d_gemm_err, P->d_ghost};
    for (void *q : ptrs)
        if (q) cudaFree(q);
    if (P->have_up) {
        for (int k = 0; k < HS_UP_CHUNKS + 3; ++k) cudaEventDestroy(P->up_ev[k]);
        for (int k = 0; k < P->max_rhs; ++k) cudaEventDestroy(P->up_rhs[k]);
        delete[] P->up_rhs;
        cudaStreamDestroy(P->up_stream);
    }
    if (P->have_dn) {
        for (int k = 0; k < 3; ++k) cudaEventDestroy(P->dn_ev[k]);
        cudaStreamDestroy(P->dn_stream);
    }
    if (P->have_events) {
        for (int k = 0; k < 2 * HS_EVENT_PAIRS; ++k) cudaEventDestroy(P->ev[k]);
        cudaEventDestroy(P->ev_total[0]);
        cudaEventDestroy(P->ev_total[1]);
    }
    delete P;
}

// Builds the FP64 and FP32 transform tables of both axes in one allocation.
hs_status build_tables(hs_plan_s *P) {
    const int Ns[2] = {P->Nx, P->Ny};
    size_t tot = 0;
    size_t off_d[2][3], off_f[2][3];
    for (int a = 0; a < 2; ++a) {
        const int M = Ns[a] + 1;
        off_d[a][0] = tot; tot += (size_t)M * 16;
        off_d[a][1] = tot; tot += (size_t)(M + 1) * 16;
        off_d[a][2] = tot; tot += (size_t)2 * M * 8;
        off_f[a][0] = tot; tot += (size_t)M * 8;
        off_f[a][1] = tot; tot += (size_t)(M + 1) * 8;
        off_f[a][2] = tot; tot += (size_t)2 * M * 4;
        tot = (tot + 255) & ~(size_t)255;
    }
    std::vector<unsigned char> host(tot, 0);
    for (int a = 0; a < 2; ++a) {
        const int N = Ns[a], M = N + 1;
        double *rd = reinterpret_cast<double *>(&host[off_d[a][0]]);
        double *hd = reinterpret_cast<double *>(&host[off_d[a][1]]);
        double *sd = reinterpret_cast<double *>(&host[off_d[a][2]]);
        float *rf = reinterpret_cast<float *>(&host[off_f[a][0]]);
        float *hf = reinterpret_cast<float *>(&host[off_f[a][1]]);
        float *sf = reinterpret_cast<float *>(&host[off_f[a][2]]);
        for (int k = 0; k < M; ++k) {   // exp(-2 pi i k / M)
            rd[2 * k] = cos_pi_ratio(2L * k, M);
            rd[2 * k + 1] = -sin_pi_ratio(2L * k, M);
            rf[2 * k] = (float)rd[2 * k];
            rf[2 * k + 1] = (float)rd[2 * k + 1];
        }
        for (int k = 0; k <= M; ++k) {  // (cos(pi k / M), sin(pi k / M))
            hd[2 * k] = cos_pi_ratio(k, M);
            hd[2 * k + 1] = sin_pi_ratio(k, M);
            hf[2 * k] = (float)hd[2 * k];
            hf[2 * k + 1] = (float)hd[2 * k + 1];
        }
        for (int m = 0; m < 2 * M; ++m) {
            sd[m] = sin_pi_ratio(m, M);
            sf[m] = (float)sd[m];
        }
    }
    HS_TRY(P, dev_alloc(P, (unsigned char **)&P->d_tables, tot));
    HS_CK(P, cudaMemcpy(P->d_tables, host.data(), tot, cudaMemcpyHostToDevice));
    unsigned char *base = static_cast<unsigned char *>(P->d_tables);
    for (int a = 0; a < 2; ++a) {
        const int N = Ns[a], M = N + 1;
        DstAxis ax;
        memset(&ax, 0, sizeof(ax));
        ax.N = N;
        ax.M = M;
        ax.fft = plan_radix(M, ax.radix, &ax.nst);
        DstAxis af = ax;
        ax.roots = base + off_d[a][0];
        ax.half = base + off_d[a][1];
        ax.sintab = base + off_d[a][2];
        af.roots = base + off_f[a][0];
        af.half = base + off_f[a][1];
        af.sintab = base + off_f[a][2];
        P->axd[a] = ax;
        P->axf[a] = af;
    }
    return HS_OK;
}

// Per-row stencil coefficients C[l][nu][a,b,c,d] (Sections 3.2-3.5).
void stencil_table(const hs_plan_s *P, const double *c0, const double *c1, const double *c2,
                   int cd_variant, double *C) {
    const int Nz = P->Nz;
    const double hx = P->hx, hy = P->hy, hz = P->hz;
    const double Rzx = hz * hz / (hx * hx), Rzy = hz * hz / (hy * hy);
    memset(C, 0, sizeof(double) * 12 * (size_t)Nz);
    for (int l = 1; l <= Nz; ++l) {
        double *lo = C + (size_t)(l - 1) * 12, *mid = lo + 4, *up = lo + 8;
        if (P->equation == HS_HELMHOLTZ) {
            const double K = c0[l], Km = c0[l - 1], Kp = c0[l + 1];
            if (P->order == 2) {
                mid[1] = Rzx;
                mid[2] = Rzy;
                lo[3] = up[3] = 1.0;
                mid[3] = -2.0 * (Rzx + Rzy + 1.0) + hz * hz * K;
            } else if (P->order == 4) {
                lo[1] = up[1] = (1.0 + Rzx) / 12.0;
                lo[2] = up[2] = (1.0 + Rzy) / 12.0;
                lo[3] = 2.0 / 3.0 - (Rzx + Rzy) / 6.0 + hz * hz * Km / 12.0;
                up[3] = 2.0 / 3.0 - (Rzx + Rzy) / 6.0 + hz * hz * Kp / 12.0;
                mid[0] = (Rzx + Rzy) / 12.0;
                mid[1] = (4.0 * Rzx - Rzy - 1.0 + hz * hz * K / 2.0) / 6.0;
                mid[2] = (4.0 * Rzy - Rzx - 1.0 + hz * hz * K / 2.0) / 6.0;
                mid[3] = -4.0 * (1.0 + Rzx + Rzy) / 3.0 + hz * hz * K / 2.0;
            } else {
                const double h = hz, h2 = h * h, h3 = h2 * h, h4 = h2 * h2;
                const double Kz = c1[l], Kzz = c2[l];
                lo[0] = up[0] = 1.0 / 30.0;
                lo[1] = lo[2] = 0.1 + h2 * Km / 90.0 - h3 * Kz / 120.0;
                up[1] = up[2] = 0.1 + h2 * Kp / 90.0 + h3 * Kz / 120.0;
                lo[3] = 7.0 / 15.0 - h2 * Km / 90.0 - (h3 * Kz / 20.0) * (1.0 / 3.0 + h2 * Km / 6.0);
                up[3] = 7.0 / 15.0 - h2 * Kp / 90.0 + (h3 * Kz / 20.0) * (1.0 / 3.0 + h2 * Kp / 6.0);
                mid[0] = 0.1 + h2 * K / 90.0;
                mid[1] = mid[2] = 7.0 / 15.0 - h2 * K / 90.0;
                mid[3] = -64.0 / 15.0 + 14.0 * h2 * K / 15.0 - h4 * K * K / 20.0 + h4 * Kzz / 20.0;
            }
        } else {
            const double g = c0[l];
            const double s[2] = {-1.0, 1.0};
            double *rows[2] = {lo, up};
            for (int k = 0; k < 2; ++k) {
                rows[k][1] = (1.0 + Rzx) * (2.0 + s[k] * g * hz) / 24.0;
                rows[k][2] = (1.0 + Rzy) * (2.0 + s[k] * g * hz) / 24.0;
                rows[k][3] = 2.0 / 3.0 - (Rzx + Rzy) / 6.0 +
                             s[k] * (hz * g / 12.0) * (4.0 - Rzx - Rzy + s[k] * hz * g);
            }
            mid[0] = (Rzx + Rzy) / 12.0;
            mid[1] = (4.0 * Rzx - Rzy - 1.0) / 6.0;
            mid[2] = (4.0 * Rzy - Rzx - 1.0) / 6.0;
            mid[3] = -4.0 * (1.0 + Rzx + Rzy) / 3.0 - hz * hz * g * g / 6.0;
            if (cd_variant == HS_CD_CORRECTED) {
                const double g1 = c1 ? c1[l] : 0.0, g2 = c2 ? c2[l] : 0.0;
                const double t3 = hz * hz * hz * (g2 + g * g1) / 24.0;
                const double t2 = hz * hz * g1 / 6.0;
                up[3] += t3 + t2;
                lo[3] += -t3 + t2;
                mid[3] += -hz * hz * g1 / 3.0;
            }
        }
    }
}

size_t node_count(const hs_plan_s *P) {
    return (size_t)(P->Nx + 2) * (P->Ny + 2) * (P->Nz + 2);
}
size_t interior_count(const hs_plan_s *P) { return (size_t)P->Nx * P->Ny * P->Nz; }
size_t face_count(const hs_plan_s *P, int k) {
    if (k < 2) return (size_t)(P->Nz + 2) * (P->Ny + 2);
    if (k < 4) return (size_t)(P->Nz + 2) * (P->Nx + 2);
    return (size_t)(P->Ny + 2) * (P->Nx + 2);
}

// Copies host-resident boundary arrays to the plan's staging buffer.
// Host boundary arrays are copied on stream s into boundary staging buffer bb
// (0 or 1); device ones are used in place.
hs_status stage_boundary(hs_plan_s *P, const hs_boundary *bnd, size_t esz, cudaStream_t s,
                         DevBoundary *out, int bb = 0) {
    memset(out, 0, sizeof(*out));
    if (!bnd) return HS_OK;
    size_t need = 0;
    for (int k = 0; k < 12; ++k) {
        const void *p = (k < 6) ? bnd->face[k] : bnd->fnn[k - 6];
        if (p && !is_device_ptr(p)) need += ((face_count(P, k % 6) * esz + 255) & ~(size_t)255);
    }
    void **buf = bb ? &P->d_stage_bnd1 : &P->d_stage_bnd;
    size_t *bytes = bb ? &P->stage_bnd1_bytes : &P->stage_bnd_bytes;
    if (need > *bytes) {
        if (*buf) {
            cudaFree(*buf);
            P->bytes -= *bytes;
        }
        *buf = nullptr;
        *bytes = 0;
        HS_TRY(P, dev_alloc(P, (unsigned char **)buf, need));
        *bytes = need;
    }
    size_t off = 0;
    for (int k = 0; k < 12; ++k) {
        const void *p = (k < 6) ? bnd->face[k] : bnd->fnn[k - 6];
        const void **dst = (k < 6) ? &out->face[k] : &out->fnn[k - 6];
        if (!p) continue;
        if (is_device_ptr(p)) {
            *dst = p;
            continue;
        }
        const size_t nb = face_count(P, k % 6) * esz;
        unsigned char *d = static_cast<unsigned char *>(*buf) + off;
        HS_CK(P, cudaMemcpyAsync(d, p, nb, cudaMemcpyHostToDevice, s));
        *dst = d;
        off += (nb + 255) & ~(size_t)255;
    }
    return HS_OK;
}

// Records an event pair around each stage launch without synchronising.  The
// pairs live in the plan; hs_stage_times (or a solve with hs_info) reads them
// once the stream has passed them, so timing does not change the launch
// stream.  When the pool is full it is drained first (one synchronisation).
void timer_drain(hs_plan_s *P) {
    if (P->timer_used == 0) return;
    cudaEventSynchronize(P->ev[2 * (P->timer_used - 1) + 1]);
    for (int k = 0; k < P->timer_used; ++k) {
        float ms = 0.f;
        cudaEventElapsedTime(&ms, P->ev[2 * k], P->ev[2 * k + 1]);
        P->timer_acc[P->timer_stage[k]] += ms;
    }
    P->timer_used = 0;
}

// Stage events (when timing is on) and an NVTX range per stage (always; a no-op
// without a profiler).
const char *const kStageName[HS_STAGE_TOTAL] = {"hs rhs", "hs dst_x", "hs dst_y", "hs thomas",
                                                "hs idst_y", "hs idst_x", "hs residual"};
struct StageTimer {
    hs_plan_s *P;
    cudaStream_t s;
    bool on;
    bool open = false;   // an NVTX stage range is pushed
    StageTimer(hs_plan_s *p, cudaStream_t st, bool o) : P(p), s(st), on(o) {}
    ~StageTimer() {
        if (open) nvtxRangePop();
    }
    void begin(int k) {
        if (open) nvtxRangePop();
        nvtxRangePushA(k >= 0 && k < HS_STAGE_TOTAL ? kStageName[k] : "hs stage");
        open = true;
        if (!on) return;
        if (P->timer_used == HS_EVENT_PAIRS) timer_drain(P);
        P->timer_stage[P->timer_used] = k;
        cudaEventRecord(P->ev[2 * P->timer_used], s);
    }
    void end(int k) {
        if (open) nvtxRangePop();
        open = false;
        if (!on) return;
        (void)k;
        cudaEventRecord(P->ev[2 * P->timer_used + 1], s);
        ++P->timer_used;
    }
};

void timer_reset(hs_plan_s *P) {
    P->timer_used = 0;
    for (int k = 0; k < HS_INFO_STAGES; ++k) P->timer_acc[k] = 0.f;
    P->timer_total_pending = 0;
}

// Drains the pending pairs and the total; fills ms[HS_INFO_STAGES].
void timer_read(hs_plan_s *P, float *ms) {
    timer_drain(P);
    if (P->timer_total_pending) {
        cudaEventSynchronize(P->ev_total[1]);
        float t = 0.f;
        cudaEventElapsedTime(&t, P->ev_total[0], P->ev_total[1]);
        P->timer_acc[HS_STAGE_TOTAL] = t;
        P->timer_total_pending = 0;
    }
    for (int k = 0; k < HS_INFO_STAGES; ++k) ms[k] = P->timer_acc[k];
}

// FP64 work arrays (lifted F and a residual/forward-sweep scratch): always
// present in FP64 plans, allocated on first need in mixed plans.
hs_status ensure_f64_work(hs_plan_s *P) {
    const size_t nint = interior_count(P);
    if (!P->d_w64) HS_TRY(P, dev_alloc(P, &P->d_w64, nint));
    if (!P->d_dscr) HS_TRY(P, dev_alloc(P, &P->d_dscr, nint));
    return HS_OK;
}

// ||F - A U||_2^2 and ||F||^2 into d_red[2], d_red[3] (synchronous).
hs_status residual_norms(hs_plan_s *P, const double *F, const double *U, cudaStream_t s,
                         double *res2, double *f2) {
    HS_CK(P, cudaMemsetAsync(P->d_red + 2, 0, 2 * sizeof(double), s));
    HS_TRY(P, hs_launch_residual(P, F, U, nullptr, P->d_dscr, s));
    HS_TRY(P, hs_launch_sumsq(P->d_dscr, nullptr, interior_count(P), P->d_red + 2, s));
    HS_TRY(P, hs_launch_sumsq(F, nullptr, interior_count(P), P->d_red + 3, s));
    double h[2];
    HS_CK(P, cudaMemcpyAsync(h, P->d_red + 2, 2 * sizeof(double), cudaMemcpyDeviceToHost, s));
    HS_CK(P, cudaStreamSynchronize(s));
    *res2 = h[0];
    *f2 = h[1];
    return HS_OK;
}

// One right-hand side: F (lifted, FP64) is in P->d_w64 on entry.
// Does a mixed solve accumulate ||F||^2 and ||r_m||^2 on the device (tolerance
// stop or the automatic residual precision, without hs_info)?
// Residual precision the mixed solve uses.  The automatic mode decides per sweep
// on the device (residual_use_f64): FP64 only after a pair residual that stopped
// shrinking.  Forcing FP64 from the first sweep on plans close to singular was
// measured to buy no accuracy on the batch workload (same worst errors) at a
// quarter of its time, so the pivot ratio does not enter the choice.
int effective_resid_mode(const hs_plan_s *P) { return P->resid_mode; }

bool refine_norms_on(const hs_plan_s *P, bool info) {
    if (P->precision != HS_MIXED || info || P->refine_sweeps < 1) return false;
    return P->refine_tol > 0 ||
           (effective_resid_mode(P) == HS_RESID_AUTO && P->refine_sweeps >= 2);
}

hs_status solve_one(hs_plan_s *P, double *u, cudaStream_t s, StageTimer &T, hs_info *info) {
    const double sx = 2.0 / (P->Nx + 1), sy = 2.0 / (P->Ny + 1);
    if (P->precision == HS_FP64) {
        double *w = P->d_w64;
        T.begin(HS_STAGE_DST_X);
        HS_TRY(P, hs_launch_dst(P, HS_AXIS_X, HS_T_F64, HS_T_F64, w, HS_T_F64, w, HS_MODE_WRITE, 1.0, s));
        T.end(HS_STAGE_DST_X);
        T.begin(HS_STAGE_DST_Y);
        HS_TRY(P, hs_launch_dst(P, HS_AXIS_Y, HS_T_F64, HS_T_F64, w, HS_T_F64, w, HS_MODE_WRITE, 1.0, s));
        T.end(HS_STAGE_DST_Y);
        T.begin(HS_STAGE_THOMAS);
        HS_TRY(P, hs_launch_thomas(P, HS_T_F64, w, nullptr, s));
        T.end(HS_STAGE_THOMAS);
        T.begin(HS_STAGE_IDST_Y);
        HS_TRY(P, hs_launch_dst(P, HS_AXIS_Y, HS_T_F64, HS_T_F64, w, HS_T_F64, w, HS_MODE_WRITE, sy, s));
        T.end(HS_STAGE_IDST_Y);
        T.begin(HS_STAGE_IDST_X);
        HS_TRY(P, hs_launch_dst(P, HS_AXIS_X, HS_T_F64, HS_T_F64, w, HS_T_F64, u, HS_MODE_WRITE, sx, s));
        T.end(HS_STAGE_IDST_X);
        if (info) {
            // residual norms use a copy of F: the FP64 path consumed it, so recompute
            info->iterations = 1;
        }
        return HS_OK;
    }
    // mixed path: F (double-float planes) in P->d_Fdf on entry; the iterate U
    // is kept as double-float in P->d_Udf and written to u (FP64) at the end.
    float *w = P->d_w32;
    const float *F = P->d_Fdf;
    float *U = P->d_Udf;
    const size_t n = interior_count(P);
    const int sweeps = P->refine_sweeps;
    // tolerance mode (no info): the device decides after each residual whether to
    // go on; converged sweeps' kernels return at once and u is written at the end
    const bool tol_mode = P->refine_tol > 0 && sweeps > 0 && !info;
    const bool norms = refine_norms_on(P, info != nullptr);
    double *nrm = P->d_red + 4;   // [||F||^2, ||r_1||^2, ...] when `norms`
    // info mode takes the automatic residual decision on the host, from the
    // same quantities (relative residuals; rel[-1] = 1)
    const int rmode = effective_resid_mode(P);
    // one fixed sweep: the FP32 solve writes only U's hi plane, and the
    // residual and the final update read only that (U's lo parts are zero until
    // a correction is added); results are those of the pair iterate bit for bit
    const bool hi_only = sweeps == 1 && !tol_mode && !info && rmode != HS_RESID_F64;
    auto host_use64 = [&](int m) {
        if (rmode == HS_RESID_F64) return true;
        if (rmode != HS_RESID_AUTO || m < 2) return false;
        const double prev = m >= 3 ? info->rel_residual[m - 3] : 1.0;
        return info->rel_residual[m - 2] > prev / 16.0;
    };
    for (int m = 0; m <= sweeps; ++m) {
        const bool last = (m == sweeps);
        if (m > 0) {
            if (tol_mode) P->cur_skip = P->d_skip;
            T.begin(HS_STAGE_RESIDUAL);
            double *r2 = norms ? nrm + m : nullptr;
            if (info) {
                HS_TRY(P, hs_launch_residual_df(P, F, U, w, s, nullptr,
                                                host_use64(m) ? HS_RESID_F64 : HS_RESID_DF));
            } else if (rmode == HS_RESID_AUTO && m >= 2) {
                HS_TRY(P, hs_launch_residual_df(P, F, U, w, s, r2, HS_RESID_SEL_DF, nrm, m));
                HS_TRY(P, hs_launch_residual_df(P, F, U, w, s, r2, HS_RESID_SEL_F64, nrm, m));
            } else {
                HS_TRY(P, hs_launch_residual_df(P, F, U, w, s, r2,
                                                rmode == HS_RESID_F64 ? HS_RESID_F64
                                                                      : HS_RESID_DF,
                                                nullptr, 0, hi_only));
            }
            T.end(HS_STAGE_RESIDUAL);
            if (tol_mode)
                HS_TRY(P, hs_launch_gate(P->d_red + 4 + m, P->d_red + 4, P->refine_tol, P->d_skip, s));
        }
        // m = 0 transforms F_hi (the first plane of F) directly
        T.begin(HS_STAGE_DST_X);
        HS_TRY(P, hs_launch_dst(P, HS_AXIS_X, HS_T_F32, HS_T_F32, m == 0 ? F : w, HS_T_F32, w,
                                HS_MODE_WRITE, 1.0, s));
        T.end(HS_STAGE_DST_X);
        T.begin(HS_STAGE_DST_Y);
        HS_TRY(P, hs_launch_dst(P, HS_AXIS_Y, HS_T_F32, HS_T_F32, w, HS_T_F32, w, HS_MODE_WRITE, 1.0, s));
        T.end(HS_STAGE_DST_Y);
        T.begin(HS_STAGE_THOMAS);
        HS_TRY(P, hs_launch_thomas(P, HS_T_F32, w, P->d_dscr, s));
        T.end(HS_STAGE_THOMAS);
        T.begin(HS_STAGE_IDST_Y);
        HS_TRY(P, hs_launch_dst(P, HS_AXIS_Y, HS_T_F32, HS_T_F32, w, HS_T_F32, w, HS_MODE_WRITE, sy, s));
        T.end(HS_STAGE_IDST_Y);
        T.begin(HS_STAGE_IDST_X);
        if (tol_mode) {
            HS_TRY(P, hs_launch_dst(P, HS_AXIS_X, HS_T_F32, HS_T_F32, w, HS_T_DF, U,
                                    m == 0 ? HS_MODE_DF_SET : HS_MODE_DF_ADD, sx, s));
        } else if (sweeps == 0 && !info) {
            HS_TRY(P, hs_launch_dst(P, HS_AXIS_X, HS_T_F32, HS_T_F32, w, HS_T_F64, u,
                                    HS_MODE_WRITE, sx, s));
        } else if (hi_only) {
            if (m == 0)
                HS_TRY(P, hs_launch_dst(P, HS_AXIS_X, HS_T_F32, HS_T_F32, w, HS_T_F32, U,
                                        HS_MODE_WRITE, sx, s));
            else
                HS_TRY(P, hs_launch_dst(P, HS_AXIS_X, HS_T_F32, HS_T_F32, w, HS_T_DF, U,
                                        HS_MODE_DF_FINAL_HI, sx, s, u));
        } else if (last && !info) {
            HS_TRY(P, hs_launch_dst(P, HS_AXIS_X, HS_T_F32, HS_T_F32, w, HS_T_DF, U,
                                    HS_MODE_DF_FINAL, sx, s, u));
        } else {
            HS_TRY(P, hs_launch_dst(P, HS_AXIS_X, HS_T_F32, HS_T_F32, w, HS_T_DF, U,
                                    m == 0 ? HS_MODE_DF_SET : HS_MODE_DF_ADD, sx, s));
        }
        T.end(HS_STAGE_IDST_X);
        if (info && m < HS_INFO_MAX_ITERS) {
            // ||F - A U|| with the double-float residual, ||F|| from F_hi
            HS_CK(P, cudaMemsetAsync(P->d_red + 2, 0, 2 * sizeof(double), s));
            HS_TRY(P, hs_launch_residual_df(P, F, U, w, s, nullptr,
                                            host_use64(m + 1) ? HS_RESID_F64 : HS_RESID_DF));
            HS_TRY(P, hs_launch_sumsq(nullptr, w, n, P->d_red + 2, s));
            HS_TRY(P, hs_launch_sumsq(nullptr, F, n, P->d_red + 3, s));
            double h[2];
            HS_CK(P, cudaMemcpyAsync(h, P->d_red + 2, sizeof(h), cudaMemcpyDeviceToHost, s));
            HS_CK(P, cudaStreamSynchronize(s));
            info->rel_residual[m] = h[1] > 0 ? sqrt(h[0] / h[1]) : sqrt(h[0]);
            info->iterations = m + 1;
            if (P->refine_tol > 0 && info->rel_residual[m] <= P->refine_tol) break;
        }
    }
    P->cur_skip = nullptr;
    if (info || tol_mode) HS_TRY(P, hs_launch_df_to_f64(U, n, u, s));
    return HS_OK;
}

}  // namespace

bool hs_is_device_ptr(const void *p) { return is_device_ptr(p); }

namespace {

// Factor precision of the mixed path's z-solves: FP32 factors (the FP32 sweep)
// when allowed -- by default only when no z-system is close to singular (min
// pivot ratio >= 1e-4) -- else the FP64 factors are built (and kept) as well
// and the sweep runs in FP64 with FP32 data.
hs_status choose_factors(hs_plan_s *P) {
    const bool f32 = P->factor_mode == HS_FACTOR_F32 ||
                     (P->factor_mode == HS_FACTOR_AUTO && P->min_pivot_ratio >= HS_ILL_PIVOT);
    P->thomas32 = (P->precision == HS_MIXED && f32) ? 1 : 0;
    if (P->precision == HS_MIXED && !P->thomas32) {
        const double init[2] = {__builtin_inf(), 0.0};
        if (!P->d_fac) HS_TRY(P, dev_alloc(P, &P->d_fac, 3 * interior_count(P)));
        HS_TRY(P, ensure_f64_work(P));
        HS_CK(P, cudaMemcpy(P->d_red, init, sizeof(init), cudaMemcpyHostToDevice));
        HS_TRY(P, hs_launch_factor(P, 0));
        HS_CK(P, cudaDeviceSynchronize());
    }
    return HS_OK;
}

}  // namespace

// Exposed for the fixed-scratch residual entry point (k_noalloc.cu).
void hs_stencil_table(const hs_plan_s *P, const double *c0, const double *c1, const double *c2,
                      int cd_variant, double *C) {
    stencil_table(P, c0, c1, c2, cd_variant, C);
}

extern "C" {

hs_status hs_plan(hs_plan_t *out, int Nx, int Ny, int Nz, double Lx, double Ly, double Lz,
                  int order, int equation, int bc, int precision, int max_rhs) {
    return hs_plan_ex(out, Nx, Ny, Nz, Lx, Ly, Lz, order, equation, bc, precision, max_rhs, 0);
}

hs_status hs_plan_ex(hs_plan_t *out, int Nx, int Ny, int Nz, double Lx, double Ly, double Lz,
                     int order, int equation, int bc, int precision, int max_rhs, int lean) {
    if (!out) return HS_ERR_INVALID_ARG;
    *out = nullptr;
    if (Nx < 1 || Ny < 1 || Nz < 1 || !(Lx > 0) || !(Ly > 0) || !(Lz > 0) || max_rhs < 1)
        return HS_ERR_INVALID_ARG;
    if (bc != HS_BC_DIRICHLET) return HS_ERR_UNSUPPORTED;
    if (equation != HS_HELMHOLTZ && equation != HS_CONVDIFF) return HS_ERR_INVALID_ARG;
    if (equation == HS_HELMHOLTZ && order != 2 && order != 4 && order != 6)
        return HS_ERR_INVALID_ARG;
    if (equation == HS_CONVDIFF && order != 4) return HS_ERR_INVALID_ARG;
    if (precision != HS_FP64 && precision != HS_MIXED) return HS_ERR_INVALID_ARG;
    if ((double)Nx * Ny * Nz > 4.0e9 || Nx > 16383 || Ny > 16383) return HS_ERR_UNSUPPORTED;
    const double hx = Lx / (Nx + 1), hy = Ly / (Ny + 1), hz = Lz / (Nz + 1);
    if (order == 6) {
        const double tol = 1e-12 * hz;
        if (fabs(hx - hz) > tol || fabs(hy - hz) > tol) return HS_ERR_INVALID_ARG;
    }
    hs_plan_s *P = new (std::nothrow) hs_plan_s;
    if (!P) return HS_ERR_OOM;
    memset(P, 0, sizeof(*P));
    P->Nx = Nx; P->Ny = Ny; P->Nz = Nz;
    P->Lx = Lx; P->Ly = Ly; P->Lz = Lz;
    P->hx = hx; P->hy = hy; P->hz = hz;
    P->order = order; P->equation = equation; P->precision = precision; P->max_rhs = max_rhs;
    {
        // constant weight of the sum-factorised right-hand side: h^2 / 720 (6th
        // order), h^2 / 12 (4th order, CD), h^2 (2nd order); h = h_z
        const double w = hz * hz / (order == 6 ? 720.0 : (order == 2 ? 1.0 : 12.0));
        const float wh = (float)w;
        P->rhs_sf_W = make_float2(wh, (float)(w - (double)wh));
    }
    P->refine_sweeps = 2;
    P->resid_mode = HS_RESID_AUTO;
    P->host_io_mapped = 0;
    P->cd_variant = HS_CD_CORRECTED;
    if (cudaGetDevice(&P->device) != cudaSuccess) {
        cudaGetLastError();
        delete P;
        return HS_ERR_CUDA;
    }
    for (int a = 0; a < 2; ++a) {
        DstAxis ax;
        memset(&ax, 0, sizeof(ax));
        ax.N = a == 0 ? Nx : Ny;
        ax.M = ax.N + 1;
        ax.fft = plan_radix(ax.M, ax.radix, &ax.nst);
        const int tc = precision == HS_FP64 ? HS_T_F64 : HS_T_F32;
        if (!hs_dst_fits(ax, a, tc) || !hs_dst_fits(ax, a, HS_T_F64)) {
            delete P;
            return HS_ERR_UNSUPPORTED;
        }
    }
    const size_t nint = (size_t)Nx * Ny * Nz;
    hs_status st = HS_OK;
    if ((st = dev_alloc(P, &P->d_coef, (size_t)Nz * 12)) ||
        (st = dev_alloc(P, &P->d_c0, (size_t)Nz + 2)) ||
        (st = dev_alloc(P, &P->d_c1, (size_t)Nz + 2)) ||
        (st = dev_alloc(P, &P->d_cx, (size_t)Nx)) || (st = dev_alloc(P, &P->d_cy, (size_t)Ny)) ||
        (precision == HS_FP64 && !lean && (st = dev_alloc(P, &P->d_fac, 3 * nint))) ||
        (st = dev_alloc(P, &P->d_red, (size_t)64)) || (st = dev_alloc(P, &P->d_skip, (size_t)1)) ||
        (precision == HS_FP64 && (st = dev_alloc(P, &P->d_w64, nint))) ||
        (precision == HS_FP64 && (st = dev_alloc(P, &P->d_dscr, nint))) ||
        (precision == HS_MIXED && (st = dev_alloc(P, &P->d_w32, nint))) ||
        (precision == HS_MIXED && (st = dev_alloc(P, &P->d_Fdf, 2 * nint))) ||
        (precision == HS_MIXED && (st = dev_alloc(P, &P->d_Udf, 2 * nint))) ||
        (precision == HS_MIXED && (st = dev_alloc(P, &P->d_fac32, 3 * nint))) ||
        (precision == HS_MIXED && (st = dev_alloc(P, &P->d_coef_df, (size_t)Nz * 12))) ||
        (precision == HS_MIXED && (st = dev_alloc(P, &P->d_rhs_df, 2 * ((size_t)Nz + 2)))) ||
        (precision == HS_MIXED && order == 6 &&
         (st = dev_alloc(P, &P->d_ghost,
                         2 * (((size_t)Nz + 2) * (Ny + 2) + ((size_t)Nz + 2) * (Nx + 2) +
                              ((size_t)Ny + 2) * (Nx + 2))))) ||
        (st = build_tables(P))) {
        free_plan(P);
        return st;
    }
    std::vector<double> cxh(Nx), cyh(Ny);
    for (int p = 1; p <= Nx; ++p) cxh[p - 1] = cos_pi_ratio(p, Nx + 1);
    for (int q = 1; q <= Ny; ++q) cyh[q - 1] = cos_pi_ratio(q, Ny + 1);
    if (cudaMemcpy(P->d_cx, cxh.data(), Nx * sizeof(double), cudaMemcpyHostToDevice) !=
            cudaSuccess ||
        cudaMemcpy(P->d_cy, cyh.data(), Ny * sizeof(double), cudaMemcpyHostToDevice) !=
            cudaSuccess) {
        cudaGetLastError();
        free_plan(P);
        return HS_ERR_CUDA;
    }
    {
        int ok = 1, k = 0;
        for (; k < 2 * HS_EVENT_PAIRS && ok; ++k) ok = cudaEventCreate(&P->ev[k]) == cudaSuccess;
        ok = ok && cudaEventCreate(&P->ev_total[0]) == cudaSuccess;
        ok = ok && cudaEventCreate(&P->ev_total[1]) == cudaSuccess;
        if (!ok) {
            cudaGetLastError();
            free_plan(P);  // events are not destroyed: have_events is still 0
            return HS_ERR_CUDA;
        }
        P->have_events = 1;
    }
    *out = P;
    return HS_OK;
}

hs_status hs_set_coeff_fn(hs_plan_t P, hs_coeff_fn fn, void *user, int cd_variant) {
    if (!P || !fn) return HS_ERR_INVALID_ARG;
    const int n = P->Nz + 2;
    std::vector<double> c0(n), c1(n), c2(n);
    for (int l = 0; l < n; ++l) {
        const double z = l * P->hz;
        c0[l] = fn(z, 0, user);
        c1[l] = fn(z, 1, user);
        c2[l] = fn(z, 2, user);
    }
    return hs_set_coeff(P, c0.data(), c1.data(), c2.data(), cd_variant);
}

hs_status hs_set_coeff(hs_plan_t P, const double *c0, const double *c1, const double *c2,
                       int cd_variant) {
    if (!P || !c0) return HS_ERR_INVALID_ARG;
    if (P->equation == HS_HELMHOLTZ && P->order == 6 && (!c1 || !c2)) {
        set_err(P, "order 6 needs (k^2)' and (k^2)''");
        return HS_ERR_INVALID_ARG;
    }
    if (P->equation == HS_CONVDIFF && cd_variant != HS_CD_PAPER && cd_variant != HS_CD_CORRECTED)
        return HS_ERR_INVALID_ARG;
    const int Nz = P->Nz;
    for (int l = 0; l < Nz + 2; ++l)
        if (!isfinite(c0[l]) || (c1 && !isfinite(c1[l])) || (c2 && !isfinite(c2[l])))
            return HS_ERR_NONFINITE;
    P->last_error[0] = 0;
    P->have_coeff = 0;   // until every table below is in place
    std::vector<double> C((size_t)Nz * 12), c1v(Nz + 2, 0.0);
    stencil_table(P, c0, c1, c2, cd_variant, C.data());
    if (c1)
        for (int l = 0; l < Nz + 2; ++l) c1v[l] = c1[l];
    HS_CK(P, cudaMemcpy(P->d_coef, C.data(), C.size() * sizeof(double), cudaMemcpyHostToDevice));
    P->resid_xy = 1;
    for (int l = 0; l < Nz; ++l)
        for (int nu = 0; nu < 3; ++nu)
            if (C[(size_t)l * 12 + nu * 4 + 1] != C[(size_t)l * 12 + nu * 4 + 2]) P->resid_xy = 0;
    if (P->d_coef_df) {
        std::vector<float2> Cdf(C.size());
        for (size_t k = 0; k < C.size(); ++k) {
            const float hi = (float)C[k];
            Cdf[k] = make_float2(hi, (float)(C[k] - (double)hi));
        }
        HS_CK(P, cudaMemcpy(P->d_coef_df, Cdf.data(), Cdf.size() * sizeof(float2),
                            cudaMemcpyHostToDevice));
    }
    if (P->d_rhs_df) {
        // per-row weights of the double-float right-hand side, formed in FP64
        std::vector<float4> w(2 * ((size_t)Nz + 2));
        const double h = P->hz, h2 = h * h;
        auto pair4 = [](double a, double e) {
            const float ah = (float)a, eh = (float)e;
            return make_float4(ah, (float)(a - (double)ah), eh, (float)(e - (double)eh));
        };
        for (int l = 0; l < Nz + 2; ++l) {
            double a = 0.0, e = 0.0;
            if (P->equation == HS_CONVDIFF) {
                e = h * c0[l] / 24.0;
            } else if (P->order == 6) {
                a = 67.0 / 120.0 - h2 * c0[l] / 20.0;
                e = h2 * h * (c1 ? c1[l] : 0.0) / 120.0;
            }
            w[l] = pair4(a, e);
            w[Nz + 2 + l] = pair4(h2 * a, h2 * e);   // the sum-factorised kernel's weights
        }
        HS_CK(P, cudaMemcpy(P->d_rhs_df, w.data(), w.size() * sizeof(float4),
                            cudaMemcpyHostToDevice));
    }
    HS_CK(P, cudaMemcpy(P->d_c0, c0, (Nz + 2) * sizeof(double), cudaMemcpyHostToDevice));
    HS_CK(P, cudaMemcpy(P->d_c1, c1v.data(), (Nz + 2) * sizeof(double), cudaMemcpyHostToDevice));
    const double init[2] = {__builtin_inf(), 0.0};
    HS_CK(P, cudaMemcpy(P->d_red, init, sizeof(init), cudaMemcpyHostToDevice));
    HS_TRY(P, hs_launch_factor(P, 0));
    double red[2];
    HS_CK(P, cudaMemcpy(red, P->d_red, sizeof(red), cudaMemcpyDeviceToHost));
    P->min_pivot_ratio = red[1] > 0 ? red[0] / red[1] : 0.0;
    HS_TRY(P, choose_factors(P));
    P->cd_variant = cd_variant;
    P->have_coeff = 1;
    return P->min_pivot_ratio < 1e-13 ? HS_WARN_NEAR_SINGULAR : HS_OK;
}

hs_status hs_set_refinement(hs_plan_t P, int sweeps) {
    if (!P || sweeps < 0 || sweeps >= HS_INFO_MAX_ITERS) return HS_ERR_INVALID_ARG;
    P->refine_sweeps = sweeps;
    return HS_OK;
}

hs_status hs_set_refinement_tol(hs_plan_t P, double tol) {
    if (!P || !(tol >= 0.0)) return HS_ERR_INVALID_ARG;
    P->refine_tol = tol;
    return HS_OK;
}

hs_status hs_set_residual_precision(hs_plan_t P, int mode) {
    if (!P || (mode != HS_RESID_DF && mode != HS_RESID_F64 && mode != HS_RESID_AUTO))
        return HS_ERR_INVALID_ARG;
    P->resid_mode = mode;
    return HS_OK;
}

hs_status hs_set_transform_variant(hs_plan_t P, int axis, int variant) {
    if (!P || (axis != HS_AXIS_X && axis != HS_AXIS_Y)) return HS_ERR_INVALID_ARG;
    if (variant < HS_DST_STAGED || variant > HS_DST_HALF) return HS_ERR_INVALID_ARG;
    if (variant == HS_DST_HALF &&
        (P->precision != HS_FP64 || !hs_dst_half_size(P->axd[axis].M)))
        return HS_ERR_UNSUPPORTED;
    if (variant == HS_DST_GEMM) {
        if (P->precision != HS_MIXED || !hs_dst_gemm_size(P->axf[axis].M)) return HS_ERR_UNSUPPORTED;
        HS_TRY(P, ensure_gemm_table(P, axis));
    }
    const bool fast = hs_dst_fast_size(P->axd[axis].M) != 0;
    if (variant == HS_DST_FUSED && (!fast || P->precision != HS_MIXED)) return HS_ERR_UNSUPPORTED;
    if (variant == HS_DST_FUSED_WIDE) {
        const int M = P->axf[axis].M;
        if (!fast || P->precision != HS_MIXED ||
            (axis == HS_AXIS_X ? hs_dst_fused_lines_x(M, 1) : hs_dst_fused_lines_y(M, 1)) == 0)
            return HS_ERR_UNSUPPORTED;
    }
    if (variant == HS_DST_STAGED && !fast) return HS_ERR_UNSUPPORTED;
    if (variant == HS_DST_TWOPASS) {
        if (axis != HS_AXIS_Y || P->precision != HS_MIXED ||
            !hs_dst_twopass_size(P->axf[HS_AXIS_Y].M))
            return HS_ERR_UNSUPPORTED;
        if (!P->d_ytmp) {
            const size_t n = (size_t)P->Nz * P->axf[HS_AXIS_Y].M * P->Nx * 2;   // floats
            float *t = nullptr;
            HS_TRY(P, dev_alloc(P, &t, n));
            P->d_ytmp = t;
        }
    } else if (axis == HS_AXIS_Y && P->d_ytmp) {
        free_ytmp(P);
    }
    P->dst_variant[axis] = variant;
    return HS_OK;
}

hs_status hs_set_thomas_variant(hs_plan_t P, int variant) {
    if (!P || variant < HS_THOMAS_PIPE16_256 || variant > HS_THOMAS_BAL16_256)
        return HS_ERR_INVALID_ARG;
    P->thomas_variant = variant;
    return HS_OK;
}

hs_status hs_get_thomas_variant(hs_plan_t P, int *variant) {
    if (!P || !variant) return HS_ERR_INVALID_ARG;
    *variant = P->thomas_variant;
    return HS_OK;
}

hs_status hs_get_transform_variant(hs_plan_t P, int axis, int *variant) {
    if (!P || !variant || (axis != HS_AXIS_X && axis != HS_AXIS_Y)) return HS_ERR_INVALID_ARG;
    *variant = P->dst_variant[axis];
    return HS_OK;
}

hs_status hs_autotune(hs_plan_t P, void *stream, int reps, float *ms_x, float *ms_y) {
    HsRange range("hs_autotune");
    if (!P || reps < 1) return HS_ERR_INVALID_ARG;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const bool mixed = P->precision == HS_MIXED;
    const bool tune_thomas = mixed && P->have_coeff && P->thomas32;
    {   // a plan of the same class was tuned before: take its choices
        int cx, cy, ct;
        float mx, my;
        if (hs_tune_lookup(P, &cx, &cy, &ct, &mx, &my) &&
            hs_set_transform_variant(P, HS_AXIS_X, cx) == HS_OK &&
            hs_set_transform_variant(P, HS_AXIS_Y, cy) == HS_OK &&
            (!tune_thomas || hs_set_thomas_variant(P, ct) == HS_OK)) {
            if (ms_x) *ms_x = mx;
            if (ms_y) *ms_y = my;
            return HS_OK;
        }
    }
    const int tc = mixed ? HS_T_F32 : HS_T_F64;
    void *w = mixed ? (void *)P->d_w32 : (void *)P->d_w64;
    if (!w) return HS_ERR_INVALID_ARG;
    const size_t n = interior_count(P);
    HS_CK(P, cudaMemsetAsync(w, 0, n * (mixed ? sizeof(float) : sizeof(double)), s));
    if (mixed && P->d_Udf) HS_CK(P, cudaMemsetAsync(P->d_Udf, 0, 2 * n * sizeof(float), s));
    cudaEvent_t e0, e1;
    HS_CK(P, cudaEventCreate(&e0));
    if (cudaEventCreate(&e1) != cudaSuccess) {
        cudaEventDestroy(e0);
        return HS_ERR_CUDA;
    }
    hs_status st = HS_OK;
    float best_ms[2] = {0.f, 0.f};
    for (int axis = 0; axis < 2 && st == HS_OK; ++axis) {
        const int saved = P->dst_variant[axis];
        int best = -1;
        for (int v = HS_DST_STAGED; v <= HS_DST_HALF && st == HS_OK; ++v) {
            if (hs_set_transform_variant(P, axis, v) != HS_OK) continue;
            // one untimed round (first launch, attribute set-up), then `reps`
            // timed.  x of a mixed plan: a forward pass and an inverse pass that
            // adds into the pair iterate (the two uses of the x kernels per sweep)
            auto one_round = [&]() {
                hs_status q = hs_launch_dst(P, axis, tc, tc, w, tc, w, HS_MODE_WRITE, 1.0, s);
                if (q == HS_OK && mixed && axis == HS_AXIS_X && P->d_Udf && P->d_Fdf) {
                    // the inverse x passes of a refined solve: set the pair iterate, then
                    // the final u = U + correction (written into F's storage, which
                    // holds n doubles and is rebuilt by every solve)
                    q = hs_launch_dst(P, axis, tc, tc, w, HS_T_DF, P->d_Udf, HS_MODE_DF_SET,
                                      1.0, s);
                    if (q == HS_OK)
                        q = hs_launch_dst(P, axis, tc, tc, w, HS_T_DF, P->d_Udf,
                                          HS_MODE_DF_FINAL, 1.0, s,
                                          reinterpret_cast<double *>(P->d_Fdf));
                }
                return q;
            };
            st = one_round();
            if (st != HS_OK) break;
            cudaEventRecord(e0, s);
            for (int r = 0; r < reps && st == HS_OK; ++r) st = one_round();
            cudaEventRecord(e1, s);
            if (cudaEventSynchronize(e1) != cudaSuccess) st = HS_ERR_CUDA;
            if (st == HS_OK && v == HS_DST_GEMM) st = check_gemm_err(P);
            float ms = 0.f;
            cudaEventElapsedTime(&ms, e0, e1);
            ms /= reps;
            if (st == HS_OK && (best < 0 || ms < best_ms[axis])) {
                best = v;
                best_ms[axis] = ms;
            }
        }
        // through the setter: the two-pass scratch is kept only when chosen
        if (hs_set_transform_variant(P, axis, best >= 0 ? best : saved) != HS_OK)
            P->dst_variant[axis] = saved;
    }
    if (st == HS_OK && mixed && P->have_coeff && P->thomas32) {
        int best = -1;
        float best_t = 0.f;
        for (int v = HS_THOMAS_PIPE16_256; v <= HS_THOMAS_BAL16_256 && st == HS_OK; ++v) {
            P->thomas_variant = v;
            st = hs_launch_thomas(P, HS_T_F32, w, P->d_dscr, s);
            if (st != HS_OK) break;
            cudaEventRecord(e0, s);
            for (int r = 0; r < reps && st == HS_OK; ++r)
                st = hs_launch_thomas(P, HS_T_F32, w, P->d_dscr, s);
            cudaEventRecord(e1, s);
            if (cudaEventSynchronize(e1) != cudaSuccess) st = HS_ERR_CUDA;
            float ms = 0.f;
            cudaEventElapsedTime(&ms, e0, e1);
            if (st == HS_OK && (best < 0 || ms < best_t)) {
                best = v;
                best_t = ms;
            }
        }
        P->thomas_variant = best >= 0 ? best : HS_THOMAS_PIPE16_256;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (st != HS_OK) {
        cudaGetLastError();
        return st;
    }
    if (ms_x) *ms_x = best_ms[0];
    if (ms_y) *ms_y = best_ms[1];
    hs_tune_store(P, P->dst_variant[0], P->dst_variant[1], tune_thomas ? P->thomas_variant : -1,
                  best_ms[0], best_ms[1]);
    return HS_OK;
}

hs_status hs_set_factor_precision(hs_plan_t P, int mode) {
    if (!P || mode < HS_FACTOR_AUTO || mode > HS_FACTOR_F64) return HS_ERR_INVALID_ARG;
    P->factor_mode = mode;
    if (P->have_coeff) HS_TRY(P, choose_factors(P));
    return HS_OK;
}

hs_status hs_set_host_io(hs_plan_t P, int mapped) {
    if (!P) return HS_ERR_INVALID_ARG;
    if (mapped < 0 || mapped > 15) return HS_ERR_INVALID_ARG;
    P->host_io_mapped = mapped;
    return HS_OK;
}

hs_status hs_host_io_wait(hs_plan_t P, void *stream) {
    if (!P) return HS_ERR_INVALID_ARG;
    // copies on the download stream run in order: the latest covers the others
    if (P->have_dn && P->dn_last >= 0)
        HS_CK(P, cudaStreamWaitEvent(static_cast<cudaStream_t>(stream), P->dn_ev[P->dn_last], 0));
    return HS_OK;
}

hs_status hs_set_stage_timing(hs_plan_t P, int on) {
    if (!P) return HS_ERR_INVALID_ARG;
    P->stage_timing = on ? 1 : 0;
    return HS_OK;
}

hs_status hs_solve(hs_plan_t P, const void *f, int f_dtype, int rhs_kind, const hs_boundary *bnd,
                   double *u, int nrhs, void *stream, hs_info *info) {
    HsRange range("hs_solve");
    if (!P || !f || !u) return HS_ERR_INVALID_ARG;
    if (f_dtype != HS_F64 && f_dtype != HS_F32) return HS_ERR_INVALID_ARG;
    if (rhs_kind != HS_RHS_NODAL && rhs_kind != HS_RHS_ASSEMBLED) return HS_ERR_INVALID_ARG;
    if (nrhs < 1 || nrhs > P->max_rhs) return HS_ERR_INVALID_ARG;
    if (!P->have_coeff) return HS_ERR_NO_COEFF;
    P->last_error[0] = 0;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const size_t esz = f_dtype == HS_F64 ? 8 : 4;
    const size_t fcount = rhs_kind == HS_RHS_NODAL ? node_count(P) : interior_count(P);
    const size_t ucount = interior_count(P);

    // host buffers: pinned ones are read / written in place through their device
    // alias when the plan allows it (the kernels then move the bytes over the
    // host link themselves), pageable ones are staged
    const unsigned char *fd = static_cast<const unsigned char *>(f);
    const void *f_mapped =
        (!is_device_ptr(f) && (P->host_io_mapped & HS_HOST_F_MAPPED)) ? mapped_host(f) : nullptr;
    bool piped = false;   // staged host f uploaded in chunks overlapping the first RHS kernel
    int fb = 0;           // f and boundary staging buffers of this call
    if (f_mapped) {
        fd = static_cast<const unsigned char *>(f_mapped);
    } else if (!is_device_ptr(f)) {
        const size_t nb = fcount * esz * nrhs;
        piped = rhs_kind == HS_RHS_NODAL && ensure_upload(P) == HS_OK;
        // HS_HOST_F_EARLY: two staging buffers in turn, so a call's upload waits
        // only for the solve before the previous one
        if (piped && (P->host_io_mapped & HS_HOST_F_EARLY)) fb = P->f_buf;
        void **buf = fb ? &P->d_stage_f1 : &P->d_stage_f;
        size_t *bytes = fb ? &P->stage_f1_bytes : &P->stage_f_bytes;
        if (nb > *bytes) {
            if (*buf) { cudaFree(*buf); P->bytes -= *bytes; }
            *buf = nullptr;
            *bytes = 0;
            HS_TRY(P, dev_alloc(P, (unsigned char **)buf, nb));
            *bytes = nb;
        }
        if (!piped) HS_CK(P, cudaMemcpyAsync(*buf, f, nb, cudaMemcpyHostToDevice, s));
        fd = static_cast<const unsigned char *>(*buf);
        if (piped) P->f_buf = (P->host_io_mapped & HS_HOST_F_EARLY) ? fb ^ 1 : 0;
    }
    double *ud = u;
    bool u_host = !is_device_ptr(u);
    double *u_mapped =
        (u_host && (P->host_io_mapped & HS_HOST_U_MAPPED)) ? static_cast<double *>(mapped_host(u))
                                                           : nullptr;
    if (u_mapped) {
        ud = u_mapped;
        u_host = false;
    }
    // HS_HOST_U_LATE: the copy back runs on the download stream and overlaps the
    // work queued after this call; the solves use the staging buffers in turn
    const bool u_late = u_host && (P->host_io_mapped & HS_HOST_U_LATE) && !info &&
                        ensure_download(P) == HS_OK;
    // copies of u per right-hand side on the download stream (late ones, or
    // several right-hand sides, each copied while the next is solved)
    const bool u_down = u_late || (u_host && nrhs > 1 && ensure_download(P) == HS_OK);
    int ub = 0;
    if (u_host) {
        const size_t nb = ucount * sizeof(double) * nrhs;
        ub = u_late ? P->u_buf : 0;
        double **buf = ub ? &P->d_stage_u1 : &P->d_stage_u;
        size_t *bytes = ub ? &P->stage_u1_bytes : &P->stage_u_bytes;
        if (nb > *bytes) {
            if (*buf) { cudaFree(*buf); P->bytes -= *bytes; }
            *buf = nullptr;
            *bytes = 0;
            HS_TRY(P, dev_alloc(P, buf, ucount * (size_t)nrhs));
            *bytes = nb;
        }
        HS_TRY(P, guard_stage_u(P, ub, s));
        ud = *buf;
    }
    DevBoundary db;
    const bool early = piped && (P->host_io_mapped & HS_HOST_F_EARLY);
    if (piped) {
        if (early) {
            // the caller vouches that no work queued on s writes the host f or
            // boundary arrays: their copies wait only until the last
            // right-hand-side kernel that read staging buffers fb is done (a
            // never-recorded event is complete), so they may overlap the solves
            // before it; the boundary goes first, the f chunks' events cover it
            HS_CK(P, cudaStreamWaitEvent(P->up_stream, P->up_ev[HS_UP_CHUNKS + 1 + fb], 0));
            HS_TRY(P, stage_boundary(P, bnd, esz, P->up_stream, &db, fb));
        } else {
            // stream order: the copies start after everything queued on s so far
            HS_CK(P, cudaEventRecord(P->up_ev[HS_UP_CHUNKS], s));
            HS_CK(P, cudaStreamWaitEvent(P->up_stream, P->up_ev[HS_UP_CHUNKS], 0));
            HS_TRY(P, stage_boundary(P, bnd, esz, s, &db));
        }
    } else {
        HS_TRY(P, stage_boundary(P, bnd, esz, s, &db));
    }

    if (info) {
        // synchronous mode: NaN or infinite samples of f are reported instead of
        // solved (a device reduction over device f, a scan of host f)
        unsigned long long bad = 0;
        if (is_device_ptr(f)) {
            HS_TRY(P, hs_check_finite(P, f, f_dtype, fcount * nrhs, stream, &bad));
        } else if (f_dtype == HS_F64) {
            const double *h = static_cast<const double *>(f);
            for (size_t i = 0; i < fcount * nrhs; ++i) bad += !isfinite(h[i]);
        } else {
            const float *h = static_cast<const float *>(f);
            for (size_t i = 0; i < fcount * nrhs; ++i) bad += !isfinite(h[i]);
        }
        if (bad) {
            set_err(P, "hs_solve: f holds %llu NaN or infinite value(s)", bad);
            return HS_ERR_NONFINITE;
        }
    }
    StageTimer T(P, s, P->stage_timing != 0 && P->have_events);
    timer_reset(P);
    if (T.on) cudaEventRecord(P->ev_total[0], s);
    for (int r = 0; r < nrhs; ++r) {
        const void *fr = fd + (size_t)r * fcount * esz;
        double *ur = ud + (size_t)r * ucount;
        hs_info *ir = (info && r == nrhs - 1) ? info : nullptr;
        if (ir) memset(ir, 0, sizeof(*ir));
        const bool norms = refine_norms_on(P, ir != nullptr);
        if (norms) {
            HS_CK(P, cudaMemsetAsync(P->d_red + 4, 0, (HS_INFO_MAX_ITERS + 1) * sizeof(double), s));
            HS_CK(P, cudaMemsetAsync(P->d_skip, 0, sizeof(int), s));
        }
        T.begin(HS_STAGE_RHS);
        void *Fout = P->precision == HS_MIXED ? (void *)P->d_Fdf : (void *)P->d_w64;
        if (piped && r == 0) {
            // early uploads usually finish during the previous solve: one chunk,
            // so the right-hand-side kernel runs as one launch
            HS_TRY(P, hs_upload_rhs(P, f, const_cast<unsigned char *>(fd),
                                    early ? 1 : HS_UP_CHUNKS, f_dtype, db, Fout,
                                    P->precision == HS_MIXED, s, norms ? P->d_red + 4 : nullptr));
            // the other right-hand sides one copy each, overlapping the solves before them
            const size_t one = fcount * esz;
            for (int q = 1; q < nrhs; ++q) {
                HS_CK(P, cudaMemcpyAsync(const_cast<unsigned char *>(fd) + q * one,
                                         static_cast<const unsigned char *>(f) + q * one, one,
                                         cudaMemcpyHostToDevice, P->up_stream));
                HS_CK(P, cudaEventRecord(P->up_rhs[q], P->up_stream));
            }
        } else {
            if (piped) HS_CK(P, cudaStreamWaitEvent(s, P->up_rhs[r], 0));
            HS_TRY(P, hs_launch_rhs(P, fr, f_dtype, rhs_kind, db, Fout, P->precision == HS_MIXED,
                                    s, norms ? P->d_red + 4 : nullptr));
        }
        // the last reader of staging buffers fb (f, boundary) is queued: a later
        // early upload into them may start
        if (P->have_up && r == nrhs - 1)
            HS_CK(P, cudaEventRecord(P->up_ev[HS_UP_CHUNKS + 1 + fb], s));
        T.end(HS_STAGE_RHS);
        HS_TRY(P, solve_one(P, ur, s, T, ir));
        if (ir && P->precision == HS_FP64) {
            HS_TRY(P, hs_launch_rhs(P, fr, f_dtype, rhs_kind, db, P->d_w64, 0, s));
            if (P->have_up) HS_CK(P, cudaEventRecord(P->up_ev[HS_UP_CHUNKS + 1 + fb], s));
            double r2, f2;
            HS_TRY(P, residual_norms(P, P->d_w64, ur, s, &r2, &f2));
            ir->rel_residual[0] = f2 > 0 ? sqrt(r2 / f2) : sqrt(r2);
        }
        if (u_down) {
            // this right-hand side's u goes back while the next ones are solved
            HS_CK(P, cudaEventRecord(P->dn_ev[2], s));
            HS_CK(P, cudaStreamWaitEvent(P->dn_stream, P->dn_ev[2], 0));
            HS_CK(P, cudaMemcpyAsync(u + (size_t)r * ucount, ur, ucount * sizeof(double),
                                     cudaMemcpyDeviceToHost, P->dn_stream));
        }
    }
    if (u_down) {
        HS_CK(P, cudaEventRecord(P->dn_ev[ub], P->dn_stream));
        P->dn_pending[ub] = 1;
        P->dn_last = ub;
        if (u_late)
            P->u_buf = ub ^ 1;
        else   // the caller's stream is done only when u is on the host
            HS_CK(P, cudaStreamWaitEvent(s, P->dn_ev[ub], 0));
    } else if (u_host) {
        HS_CK(P, cudaMemcpyAsync(u, ud, ucount * sizeof(double) * nrhs, cudaMemcpyDeviceToHost, s));
    }
    if (T.on) {
        cudaEventRecord(P->ev_total[1], s);
        P->timer_total_pending = 1;
    }
    if (info) {
        info->min_pivot_ratio = P->min_pivot_ratio;
        HS_TRY(P, check_gemm_err(P));
        HS_CK(P, cudaStreamSynchronize(s));
        if (T.on) timer_read(P, info->stage_ms);
    }
    HS_CK(P, cudaGetLastError());
    return (P->min_pivot_ratio < 1e-13) ? HS_WARN_NEAR_SINGULAR : HS_OK;
}

hs_status hs_residual(hs_plan_t P, const void *f, int f_dtype, int rhs_kind,
                      const hs_boundary *bnd, const double *u, void *stream, double *res_norm,
                      double *rhs_norm) {
    if (!P || !f || !u) return HS_ERR_INVALID_ARG;
    if (!P->have_coeff) return HS_ERR_NO_COEFF;
    if (f_dtype != HS_F64 && f_dtype != HS_F32) return HS_ERR_INVALID_ARG;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const size_t esz = f_dtype == HS_F64 ? 8 : 4;
    const size_t fcount = rhs_kind == HS_RHS_NODAL ? node_count(P) : interior_count(P);
    const size_t ucount = interior_count(P);
    const void *fd = f;
    if (!is_device_ptr(f)) {
        const size_t nb = fcount * esz;
        if (nb > P->stage_f_bytes) {
            if (P->d_stage_f) { cudaFree(P->d_stage_f); P->bytes -= P->stage_f_bytes; }
            P->d_stage_f = nullptr;
            P->stage_f_bytes = 0;
            HS_TRY(P, dev_alloc(P, (unsigned char **)&P->d_stage_f, nb));
            P->stage_f_bytes = nb;
        }
        HS_CK(P, cudaMemcpyAsync(P->d_stage_f, f, nb, cudaMemcpyHostToDevice, s));
        fd = P->d_stage_f;
    }
    const double *ud = u;
    if (!is_device_ptr(u)) {
        const size_t nb = ucount * sizeof(double);
        if (nb > P->stage_u_bytes) {
            if (P->d_stage_u) { cudaFree(P->d_stage_u); P->bytes -= P->stage_u_bytes; }
            P->d_stage_u = nullptr;
            P->stage_u_bytes = 0;
            HS_TRY(P, dev_alloc(P, &P->d_stage_u, ucount));
            P->stage_u_bytes = nb;
        }
        HS_TRY(P, guard_stage_u(P, 0, s));
        HS_CK(P, cudaMemcpyAsync(P->d_stage_u, u, nb, cudaMemcpyHostToDevice, s));
        ud = P->d_stage_u;
    }
    DevBoundary db;
    HS_TRY(P, stage_boundary(P, bnd, esz, s, &db));
    HS_TRY(P, ensure_f64_work(P));
    HS_TRY(P, hs_launch_rhs(P, fd, f_dtype, rhs_kind, db, P->d_w64, 0, s));
    // staging buffers 0 (f, boundary) read: an early upload of a later solve may reuse them
    if (P->have_up) HS_CK(P, cudaEventRecord(P->up_ev[HS_UP_CHUNKS + 1], s));
    double r2, f2;
    HS_TRY(P, residual_norms(P, P->d_w64, ud, s, &r2, &f2));
    if (res_norm) *res_norm = sqrt(r2);
    if (rhs_norm) *rhs_norm = sqrt(f2);
    return HS_OK;
}

hs_status hs_rhs_apply(hs_plan_t P, const void *f, int f_dtype, int rhs_kind,
                       const hs_boundary *bnd, void *F, void *stream) {
    if (!P || !f || !F) return HS_ERR_INVALID_ARG;
    if (!P->have_coeff) return HS_ERR_NO_COEFF;
    if (f_dtype != HS_F64 && f_dtype != HS_F32) return HS_ERR_INVALID_ARG;
    if (rhs_kind != HS_RHS_NODAL && rhs_kind != HS_RHS_ASSEMBLED) return HS_ERR_INVALID_ARG;
    if (!is_device_ptr(f) || !is_device_ptr(F)) return HS_ERR_INVALID_ARG;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    DevBoundary db;
    HS_TRY(P, stage_boundary(P, bnd, f_dtype == HS_F64 ? 8 : 4, s, &db));
    HS_TRY(P, hs_launch_rhs(P, f, f_dtype, rhs_kind, db, F, P->precision == HS_MIXED, s));
    // staging buffers 0 (boundary) read: an early upload of a later solve may reuse them
    if (P->have_up) HS_CK(P, cudaEventRecord(P->up_ev[HS_UP_CHUNKS + 1], s));
    return HS_OK;
}

hs_status hs_stage_times(hs_plan_t P, float *ms) {
    if (!P || !ms) return HS_ERR_INVALID_ARG;
    if (!P->have_events) return HS_ERR_CUDA;
    timer_read(P, ms);
    return HS_OK;
}

size_t hs_workspace_bytes(hs_plan_t P) { return P ? P->bytes : 0; }

hs_status hs_destroy(hs_plan_t P) {
    if (!P) return HS_OK;
    int cur = 0;
    cudaGetDevice(&cur);
    const int dev = P->device;
    if (cur != dev) cudaSetDevice(dev);
    cudaDeviceSynchronize();
    free_plan(P);
    if (cur != dev) cudaSetDevice(cur);
    return HS_OK;
}

const char *hs_status_str(hs_status s) {
    switch (s) {
        case HS_OK: return "HS_OK";
        case HS_WARN_NEAR_SINGULAR: return "HS_WARN_NEAR_SINGULAR: a z-system has a pivot below 1e-13 of its diagonal";
        case HS_WARN_NOT_CONVERGED: return "HS_WARN_NOT_CONVERGED: refinement ended above its tolerance";
        case HS_ERR_INVALID_ARG: return "HS_ERR_INVALID_ARG: invalid argument";
        case HS_ERR_UNSUPPORTED: return "HS_ERR_UNSUPPORTED: unsupported configuration";
        case HS_ERR_OOM: return "HS_ERR_OOM: out of device memory";
        case HS_ERR_CUDA: return "HS_ERR_CUDA: CUDA error";
        case HS_ERR_NO_COEFF: return "HS_ERR_NO_COEFF: hs_set_coeff was not called";
        case HS_ERR_TIMEOUT: return "HS_ERR_TIMEOUT: a bounded device wait gave up";
        case HS_ERR_NONFINITE: return "HS_ERR_NONFINITE: non-finite input";
        default: return "unknown hs_status";
    }
}

const char *hs_last_error(hs_plan_t P) { return P ? P->last_error : "no plan"; }

}  // extern "C"
