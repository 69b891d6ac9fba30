// Batched solves in one persistent launch (no paper counterpart; each problem
// is Section 3.6's solve): host side (plans, work and item lists, kernel
// variant and grid, graph capture).  The device side and the scheduling scheme
// are in hs_batch.cuh.
#include <string.h>

#include <algorithm>
#include <new>
#include <vector>

#include "hs_batch.cuh"

using namespace hs_batch;

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
    int nitems, nworks;
    int variant;                      // index into kVariants
    int grid[5];                      // resident CTAs of each variant (graph mode: 1)
    int graph_warm;                   // graph mode: plans have solved once outside capture
    int graph_kernels;                // kernel nodes in the captured graph
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

// The kernel variants: 0/1 staged transform tiles, registers capped for 2/3
// CTAs per SM; 2/3 the same with the fused transform tiles.
constexpr int kNumVariants = 5;
constexpr int kGraphVariant = 4;   // stand-alone solves in one graph (no persistent kernel)
constexpr int kGraphBranches = 8;
const void *variant_fn(int v) {
    switch (v) {
        case 0: return batch_kernel_v2();
        case 1: return batch_kernel_v3();
        case 2: return batch_kernel_v2f();
        case 3: return batch_kernel_v3f();
        default: return nullptr;
    }
}

void drop_graph(hs_batch_s *B) {
    if (B->have_graph) {
        cudaGraphExecDestroy(B->graph);
        B->have_graph = 0;
    }
}

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


int count_kernel_nodes(cudaGraph_t g) {
    size_t n = 0;
    if (cudaGraphGetNodes(g, nullptr, &n) != cudaSuccess) return -1;
    std::vector<cudaGraphNode_t> nodes(n);
    if (n && cudaGraphGetNodes(g, nodes.data(), &n) != cudaSuccess) return -1;
    int k = 0;
    for (cudaGraphNode_t v : nodes) {
        cudaGraphNodeType t;
        if (cudaGraphNodeGetType(v, &t) == cudaSuccess && t == cudaGraphNodeTypeKernel) ++k;
    }
    return k;
}

// The persistent launch: counter resets and one kernel, captured as a graph.
hs_status capture_persistent(hs_batch_s *B) {
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
        void *args[] = {&A};
        cudaLaunchKernel(variant_fn(B->variant), dim3(B->grid[B->variant]), dim3(256), args,
                         B->smem, cs);
        ok = cudaStreamEndCapture(cs, &g) == cudaSuccess && g;
    }
    if (ok) B->graph_kernels = count_kernel_nodes(g);
    ok = ok && cudaGraphInstantiate(&B->graph, g, 0) == cudaSuccess;
    if (g) cudaGraphDestroy(g);
    cudaStreamDestroy(cs);
    if (!ok) {
        cudaGetLastError();
        return HS_ERR_CUDA;
    }
    B->have_graph = 1;
    return HS_OK;
}

// The other execution: every problem's stand-alone mixed solve (one per RHS,
// the plans the batch already holds) captured into one graph on up to 8
// parallel branches, problems assigned largest first to the least-loaded
// branch.  Each stage then runs at its own kernel's occupancy and small
// problems overlap; the queue, counters and waits are not used.
hs_status capture_solves(hs_batch_s *B) {
    const int nb = B->n < kGraphBranches ? B->n : kGraphBranches;
    for (hs_plan_t P : B->plans) {
        hs_status st;
        if ((st = hs_set_refinement(P, B->sweeps)) != HS_OK ||
            (st = hs_set_refinement_tol(P, B->tol)) != HS_OK ||
            (st = hs_set_residual_precision(P, B->resid_mode)) != HS_OK)
            return st;
    }
    if (!B->graph_warm) {
        // each plan picks its own transform kernels and z-solve mapping (timed on
        // its work buffers), then solves once outside capture: first-launch
        // attributes and any lazily created buffers exist before the capture
        for (int k = 0; k < B->n; ++k) {
            const hs_status st = hs_autotune(B->plans[k], nullptr, 2, nullptr, nullptr);
            if (st < 0) return st;
        }
        for (int k = 0; k < B->n; ++k) {
            const BatchWork &W = B->works[B->work_of[k]];
            const hs_status st = hs_solve(B->plans[k], W.f, B->f_dtype, HS_RHS_NODAL, nullptr,
                                          W.u, 1, nullptr, nullptr);
            if (st < 0) return st;
        }
        if (cudaDeviceSynchronize() != cudaSuccess) {
            cudaGetLastError();
            return HS_ERR_CUDA;
        }
        B->graph_warm = 1;
    }
    std::vector<int> order(B->n);
    for (int k = 0; k < B->n; ++k) order[k] = k;
    auto work = [&](int k) {
        const hs_plan_s *P = B->plans[k];
        return (double)P->Nx * P->Ny * P->Nz * B->nrhs[k];
    };
    std::sort(order.begin(), order.end(), [&](int a, int b) { return work(a) > work(b); });
    std::vector<double> load(nb, 0.0);
    std::vector<int> branch_of(B->n, 0);
    for (int k : order) {
        int best = 0;
        for (int b = 1; b < nb; ++b)
            if (load[b] < load[best]) best = b;
        branch_of[k] = best;
        load[best] += work(k);
    }
    cudaStream_t cs;
    std::vector<cudaStream_t> br(nb, nullptr);
    std::vector<cudaEvent_t> ev(nb + 1, nullptr);
    bool ok = cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking) == cudaSuccess;
    for (int b = 0; ok && b < nb; ++b)
        ok = cudaStreamCreateWithFlags(&br[b], cudaStreamNonBlocking) == cudaSuccess;
    for (int b = 0; ok && b <= nb; ++b)
        ok = cudaEventCreateWithFlags(&ev[b], cudaEventDisableTiming) == cudaSuccess;
    cudaGraph_t g = nullptr;
    hs_status st = HS_OK;
    if (ok) ok = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal) == cudaSuccess;
    if (ok) {
        cudaMemsetAsync(B->d_ctr + 1, 0, sizeof(int), cs);   // no stale timeout flag
        cudaEventRecord(ev[nb], cs);
        for (int b = 0; b < nb; ++b) cudaStreamWaitEvent(br[b], ev[nb], 0);
        for (int k : order) {
            for (int r = 0; r < B->nrhs[k] && st >= 0; ++r) {
                const BatchWork &W = B->works[B->work_of[k] + r];
                st = hs_solve(B->plans[k], W.f, B->f_dtype, HS_RHS_NODAL, nullptr, W.u, 1,
                              br[branch_of[k]], nullptr);
            }
        }
        for (int b = 0; b < nb; ++b) {
            cudaEventRecord(ev[b], br[b]);
            cudaStreamWaitEvent(cs, ev[b], 0);
        }
        ok = cudaStreamEndCapture(cs, &g) == cudaSuccess && g && st >= 0;
    }
    if (ok) B->graph_kernels = count_kernel_nodes(g);
    ok = ok && cudaGraphInstantiate(&B->graph, g, 0) == cudaSuccess;
    if (g) cudaGraphDestroy(g);
    for (int b = 0; b <= nb; ++b)
        if (ev[b]) cudaEventDestroy(ev[b]);
    for (int b = 0; b < nb; ++b)
        if (br[b]) cudaStreamDestroy(br[b]);
    cudaStreamDestroy(cs);
    if (!ok) {
        cudaGetLastError();
        return st < 0 ? st : HS_ERR_CUDA;
    }
    B->have_graph = 1;
    return HS_OK;
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
    B->graph_warm = 0;
    B->graph_kernels = 0;
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
    size_t smem = sf_smem_bytes<2, double>();   // the largest right-hand-side ring
    const size_t res_smem = 2 * QHY * QHX * sizeof(double);   // FP64 residual tile
    if (res_smem > smem) smem = res_smem;
    if (2 * RSHX * RSHY * sizeof(float2) > smem) smem = 2 * RSHX * RSHY * sizeof(float2);
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
            ra.zt = SFZ;   // the persistent kernel's tile grid (W.gz) uses full-depth tiles
            ra.ghost = nullptr;   // ghost nodes formed in the tile (same values)
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
            // right-hand-side and residual tiles share one grid (SFX = RSX, SFY = RSY,
            // SFZ = RSZ = 2 QZ)
            static_assert(SFX == RSX && SFY == RSY && SFZ == RSZ && RSZ == 2 * QZ, "tile grids");
            W.gx = (d.Nx + SFX - 1) / SFX;
            W.gy = (d.Ny + SFY - 1) / SFY;
            W.gz = (d.Nz + SFZ - 1) / SFZ;
            W.rw = P->d_rhs_df + (d.Nz + 2);
            W.rhsW = P->rhs_sf_W;
            W.resid_xy = P->resid_xy;
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
                   cudaMemcpyHostToDevice) != cudaSuccess) {
        cudaGetLastError();
        free_batch(B);
        return HS_ERR_CUDA;
    }
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    B->variant = -1;
    for (int v = 0; v < kNumVariants; ++v) {
        int per = 0;
        B->grid[v] = 0;
        if (v == kGraphVariant) {
            B->grid[v] = 1;
            continue;
        }
        if (cudaFuncSetAttribute(variant_fn(v), cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)smem) != cudaSuccess ||
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, variant_fn(v), 256, smem) !=
                cudaSuccess) {
            cudaGetLastError();
            continue;
        }
        B->grid[v] = sms * per;  // every CTA resident: waits only on items already taken
        if (per >= 1 && B->variant < 0) B->variant = v;
    }
    if (B->variant < 0) {
        free_batch(B);
        return HS_ERR_UNSUPPORTED;
    }
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
    drop_graph(B);   // the graph mode captures the pointers
    return HS_OK;
}

hs_status hs_batch_set_wait_limit(hs_batch_t B, long long spins) {
    if (!B || spins < 1) return HS_ERR_INVALID_ARG;
    B->spin_limit = spins;
    drop_graph(B);
    return HS_OK;
}

hs_status hs_batch_set_tol(hs_batch_t B, double tol) {
    if (!B || !(tol >= 0.0)) return HS_ERR_INVALID_ARG;
    B->tol = tol;
    drop_graph(B);
    return HS_OK;
}

hs_status hs_batch_set_residual_precision(hs_batch_t B, int mode) {
    if (!B || (mode != HS_RESID_DF && mode != HS_RESID_F64 && mode != HS_RESID_AUTO))
        return HS_ERR_INVALID_ARG;
    B->resid_mode = mode;
    drop_graph(B);
    return HS_OK;
}

hs_status hs_batch_set_variant(hs_batch_t B, int variant) {
    if (!B || variant < 0 || variant >= kNumVariants) return HS_ERR_INVALID_ARG;
    if (B->grid[variant] < 1) return HS_ERR_UNSUPPORTED;
    if (variant != B->variant) drop_graph(B);
    B->variant = variant;
    return HS_OK;
}

hs_status hs_batch_get_variant(hs_batch_t B, int *variant, int *grid) {
    if (!B) return HS_ERR_INVALID_ARG;
    if (variant) *variant = B->variant;
    if (grid) *grid = B->grid[B->variant];
    return HS_OK;
}

hs_status hs_batch_graph_kernels(hs_batch_t B, int *kernels) {
    if (!B || !kernels) return HS_ERR_INVALID_ARG;
    *kernels = B->have_graph ? B->graph_kernels : 0;
    return HS_OK;
}

hs_status hs_batch_autotune(hs_batch_t B, void *stream, int reps, float *ms_out) {
    if (!B || reps < 1) return HS_ERR_INVALID_ARG;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    cudaEvent_t e0, e1;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
        cudaGetLastError();
        return HS_ERR_CUDA;
    }
    int best = -1;
    float best_ms = 0.f;
    hs_status st = HS_OK;
    for (int v = 0; v < kNumVariants && st == HS_OK; ++v) {
        if (B->grid[v] < 1) continue;
        if ((st = hs_batch_set_variant(B, v)) != HS_OK) break;
        if ((st = hs_batch_solve(B, stream, 1)) != HS_OK) break;  // capture + warm-up
        float tot = 0.f;
        for (int r = 0; r < reps && st == HS_OK; ++r) {
            cudaEventRecord(e0, s);
            st = hs_batch_solve(B, stream, 0);
            cudaEventRecord(e1, s);
            if (cudaEventSynchronize(e1) != cudaSuccess) st = HS_ERR_CUDA;
            float ms = 0.f;
            cudaEventElapsedTime(&ms, e0, e1);
            tot += ms;
        }
        if (st == HS_OK && (best < 0 || tot < best_ms)) {
            best = v;
            best_ms = tot;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (st != HS_OK) return st;
    if (best < 0) return HS_ERR_UNSUPPORTED;
    if (ms_out) *ms_out = best_ms / reps;
    return hs_batch_set_variant(B, best);
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
    HsRange range("hs_batch_solve");
    if (!B) return HS_ERR_INVALID_ARG;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    if (!B->have_graph || B->graph_stream != s) {
        if (B->have_graph) cudaGraphExecDestroy(B->graph);
        B->have_graph = 0;
        const hs_status st = B->variant == kGraphVariant ? capture_solves(B) : capture_persistent(B);
        if (st != HS_OK) return st;
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
