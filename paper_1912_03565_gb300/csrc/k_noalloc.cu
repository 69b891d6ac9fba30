// hs_residual_static: the L2 residual ||F - A U||_2 (L2-res of Section 5.1) (and ||F||_2) of an
// assembled right-hand side, for callers that cannot allocate device memory.
//
// Who needs it: code that runs where cudaMalloc is not allowed or not
// possible -- a caller whose device memory is owned by its own pool
// allocator or framework, a plugin that may only use the buffers it is
// handed, or a real-time loop that must not allocate -- and that wants to
// check a solution (for example inside its own iteration around this
// solver) without creating a plan, because hs_plan allocates workspace.
//
// How: the only device scratch is one file-scope array below.  Its size is
// fixed at build time (the coefficient table of up to HS_STATIC_MAX_NZ rows
// plus the partial sums of a fixed-size grid), every GPU that loads the
// library holds it until the process exits, and every call shares it.
// The computation is the same as hs_residual's for an assembled right-hand
// side with zero Dirichlet data, but the residual is reduced on the fly
// (the plan path writes it to a full-size workspace array first).
#include <math.h>
#include <string.h>

#include <mutex>

#include "hs_internal.cuh"

#define HS_STATIC_PARTS 1024
#define HS_STATIC_COEF (HS_STATIC_MAX_NZ * 12)
#define HS_STATIC_DOUBLES (HS_STATIC_COEF + 2 * HS_STATIC_PARTS + 2)
#define HS_STATIC_MAX_DEVICES 64

// Layout: [0, 12 Nz) coefficient table C[l][nu][a,b,c,d];
//         [HS_STATIC_COEF, + PARTS) per-block sums of r^2;
//         [.. + PARTS, + 2 PARTS) per-block sums of F^2; last 2: the totals.
static __device__ __align__(256) double g_hs_static_scratch[HS_STATIC_DOUBLES];

namespace {

std::mutex g_setup_mu;
double *g_scratch_addr[HS_STATIC_MAX_DEVICES];

// Device address of the static array on the current device.  The host-side
// symbol g_hs_static_scratch is only a stand-in; the address the kernels
// need comes from cudaGetSymbolAddress, looked up once per device.
hs_status static_scratch(double **out) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) {
        cudaGetLastError();
        return HS_ERR_CUDA;
    }
    if (dev < 0 || dev >= HS_STATIC_MAX_DEVICES) return HS_ERR_UNSUPPORTED;
    std::lock_guard<std::mutex> lock(g_setup_mu);
    if (!g_scratch_addr[dev]) {
        void *p = nullptr;
        if (cudaGetSymbolAddress(&p, g_hs_static_scratch) != cudaSuccess || !p) {
            cudaGetLastError();
            return HS_ERR_CUDA;
        }
        g_scratch_addr[dev] = static_cast<double *>(p);
    }
    *out = g_scratch_addr[dev];
    return HS_OK;
}

// Memory the kernels may dereference: device or managed memory of the current
// device `dev` (a pointer into another GPU's memory would be a peer access,
// which faults without peer access enabled).
bool on_device(const void *p, int dev) {
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    if (a.type == cudaMemoryTypeDevice) return a.device == dev;
    return a.type == cudaMemoryTypeManaged;
}

// Each block adds r^2 = (F - A U)^2 and F^2 over a grid-stride range of
// interior points (U = 0 outside the interior) and writes its two sums.
__global__ void __launch_bounds__(256) residual_parts_kernel(int Nx, int Ny, int Nz,
                                                              const double *__restrict__ coef,
                                                              const double *__restrict__ F,
                                                              const double *__restrict__ U,
                                                              double *__restrict__ parts) {
    const size_t plane = (size_t)Nx * Ny;
    const size_t n = plane * Nz;
    double rr = 0.0, ff = 0.0;
    for (size_t o = (size_t)blockIdx.x * blockDim.x + threadIdx.x; o < n;
         o += (size_t)gridDim.x * blockDim.x) {
        const int l = (int)(o / plane);
        const size_t c = o - (size_t)l * plane;
        const int j = (int)(c / Nx);
        const int i = (int)(c - (size_t)j * Nx);
        const double *cf = coef + (size_t)l * 12;
        double acc = 0.0;
        for (int dl = -1; dl <= 1; ++dl) {
            const int ll = l + dl;
            if (ll < 0 || ll >= Nz) continue;
            const double *P = U + (size_t)ll * plane;
            double corners = 0.0, xn = 0.0, yn = 0.0;
            if (j > 0) {
                if (i > 0) corners += P[c - Nx - 1];
                if (i < Nx - 1) corners += P[c - Nx + 1];
                yn += P[c - Nx];
            }
            if (j < Ny - 1) {
                if (i > 0) corners += P[c + Nx - 1];
                if (i < Nx - 1) corners += P[c + Nx + 1];
                yn += P[c + Nx];
            }
            if (i > 0) xn += P[c - 1];
            if (i < Nx - 1) xn += P[c + 1];
            const double *k = cf + (dl + 1) * 4;
            acc += k[0] * corners + k[1] * xn + k[2] * yn + k[3] * P[c];
        }
        const double Fo = F[o];
        const double r = Fo - acc;
        rr += r * r;
        ff += Fo * Fo;
    }
    for (int s = 16; s > 0; s >>= 1) {
        rr += __shfl_down_sync(0xffffffffu, rr, s);
        ff += __shfl_down_sync(0xffffffffu, ff, s);
    }
    __shared__ double wr[8], wf[8];
    if ((threadIdx.x & 31) == 0) {
        wr[threadIdx.x >> 5] = rr;
        wf[threadIdx.x >> 5] = ff;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double a = 0.0, b = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) {
            a += wr[w];
            b += wf[w];
        }
        parts[blockIdx.x] = a;
        parts[HS_STATIC_PARTS + blockIdx.x] = b;
    }
}

// One block: totals of the per-block sums (fixed order, so repeatable).
__global__ void __launch_bounds__(256) residual_total_kernel(const double *__restrict__ parts,
                                                              double *__restrict__ out) {
    __shared__ double sr[256], sf[256];
    double a = 0.0, b = 0.0;
    for (int k = threadIdx.x; k < HS_STATIC_PARTS; k += blockDim.x) {
        a += parts[k];
        b += parts[HS_STATIC_PARTS + k];
    }
    sr[threadIdx.x] = a;
    sf[threadIdx.x] = b;
    __syncthreads();
    for (int w = blockDim.x / 2; w > 0; w >>= 1) {
        if ((int)threadIdx.x < w) {
            sr[threadIdx.x] += sr[threadIdx.x + w];
            sf[threadIdx.x] += sf[threadIdx.x + w];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        out[0] = sr[0];
        out[1] = sf[0];
    }
}

}  // namespace

extern "C" hs_status hs_residual_static(int Nx, int Ny, int Nz, double Lx, double Ly, double Lz,
                                        int order, int equation, int cd_variant,
                                        const double *c0, const double *c1, const double *c2,
                                        const double *F, const double *u, void *stream,
                                        double *res_norm, double *rhs_norm) {
    if (Nx < 1 || Ny < 1 || Nz < 1 || !(Lx > 0) || !(Ly > 0) || !(Lz > 0) || !c0 || !F || !u ||
        !res_norm || !rhs_norm)
        return HS_ERR_INVALID_ARG;
    if (equation != HS_HELMHOLTZ && equation != HS_CONVDIFF) return HS_ERR_INVALID_ARG;
    if (equation == HS_HELMHOLTZ && order != 2 && order != 4 && order != 6)
        return HS_ERR_INVALID_ARG;
    if (equation == HS_CONVDIFF && order != 4) return HS_ERR_INVALID_ARG;
    if (equation == HS_HELMHOLTZ && order == 6 && (!c1 || !c2)) return HS_ERR_INVALID_ARG;
    if (equation == HS_CONVDIFF && cd_variant != HS_CD_PAPER && cd_variant != HS_CD_CORRECTED)
        return HS_ERR_INVALID_ARG;
    if (Nz > HS_STATIC_MAX_NZ) return HS_ERR_UNSUPPORTED;  // beyond the fixed scratch
    const double hx = Lx / (Nx + 1), hy = Ly / (Ny + 1), hz = Lz / (Nz + 1);
    if (equation == HS_HELMHOLTZ && order == 6) {
        // the sixth-order table assumes one spacing (Section 3.4), as hs_plan does
        const double tol = 1e-12 * hz;
        if (fabs(hx - hz) > tol || fabs(hy - hz) > tol) return HS_ERR_INVALID_ARG;
    }
    for (int l = 0; l < Nz + 2; ++l)
        if (!isfinite(c0[l]) || (c1 && !isfinite(c1[l])) || (c2 && !isfinite(c2[l])))
            return HS_ERR_NONFINITE;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) {
        cudaGetLastError();
        return HS_ERR_CUDA;
    }
    if (!on_device(F, dev) || !on_device(u, dev)) return HS_ERR_INVALID_ARG;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    {
        // the synchronous copies below are not allowed on a capturing stream
        cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
        if (cudaStreamIsCapturing(s, &cap) != cudaSuccess) {
            cudaGetLastError();
            return HS_ERR_CUDA;
        }
        if (cap != cudaStreamCaptureStatusNone) return HS_ERR_INVALID_ARG;
    }

    double *scratch = nullptr;
    hs_status st = static_scratch(&scratch);
    if (st != HS_OK) return st;

    // Coefficient table in chunks of rows built on the host stack and copied
    // into the static array: row l depends on c0..c2 at l-1, l, l+1 only, so a
    // chunk is the table of a sub-grid whose profile arrays start at row l0.
    hs_plan_s sub;
    memset(&sub, 0, sizeof(sub));
    sub.Nx = Nx;
    sub.Ny = Ny;
    sub.hx = hx;
    sub.hy = hy;
    sub.hz = hz;
    sub.order = order;
    sub.equation = equation;
    const int CH = 128;
    double rows[CH * 12];
    for (int l0 = 0; l0 < Nz; l0 += CH) {
        sub.Nz = (Nz - l0) < CH ? (Nz - l0) : CH;
        hs_stencil_table(&sub, c0 + l0, c1 ? c1 + l0 : nullptr, c2 ? c2 + l0 : nullptr,
                         cd_variant, rows);
        if (cudaMemcpyAsync(scratch + (size_t)l0 * 12, rows, sizeof(double) * 12 * sub.Nz,
                            cudaMemcpyHostToDevice, s) != cudaSuccess) {
            cudaGetLastError();
            return HS_ERR_CUDA;
        }
        // the host buffer is reused by the next chunk: wait for this copy
        if (cudaStreamSynchronize(s) != cudaSuccess) {
            cudaGetLastError();
            return HS_ERR_CUDA;
        }
    }
    double *parts = scratch + HS_STATIC_COEF;
    double *tot = parts + 2 * HS_STATIC_PARTS;
    residual_parts_kernel<<<HS_STATIC_PARTS, 256, 0, s>>>(Nx, Ny, Nz, scratch, F, u, parts);
    residual_total_kernel<<<1, 256, 0, s>>>(parts, tot);
    double h[2] = {0.0, 0.0};
    if (cudaGetLastError() != cudaSuccess ||
        cudaMemcpyAsync(h, tot, sizeof(h), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess) {
        cudaGetLastError();
        return HS_ERR_CUDA;
    }
    *res_norm = sqrt(h[0]);
    *rhs_norm = sqrt(h[1]);
    return HS_OK;
}
