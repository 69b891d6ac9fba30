// Tile functions (Sections 3.2-3.6) shared by the stand-alone kernels and the
// batched persistent kernel: one CTA's work for the transforms (k_dst_fast.cu),
// the double-float right-hand side and residual (k_rhs.cu) and the z-solves
// (k_thomas.cu).
// Each takes its tile index and, where it needs one, a pointer to the CTA's
// shared memory instead of reading blockIdx or declaring shared arrays, so a
// persistent CTA can run tiles of different stages one after another.
#pragma once

#include "hs_internal.cuh"

namespace hs_tiles {

// Load that bypasses L1 when COH: data written by other CTAs earlier in the
// same launch must not be served from a stale L1 line.
template <bool COH, typename T>
__device__ __forceinline__ T ldc(const T *p) {
    if constexpr (COH)
        return __ldcg(p);
    else
        return *p;
}

// =================================================================== transforms
// cos(2 pi k / 48) and sin(2 pi k / 48), the constant twiddles of the compiled
// radix stages (R divides 48).  The first quadrant cos(pi m / 24), m = 0..12,
// is tabulated correctly rounded (the exact values rounded to the nearest
// FP64 number); every other k is mapped onto it by the exact symmetries
// cos(pi - x) = -cos x, cos(pi + x) = -cos x, cos(2 pi - x) = cos x, and
// sin x = cos(x - pi / 2).
__device__ __forceinline__ double cos_q24(int m) {
    switch (m) {
        case 0: return 1.0;
        case 1: return 0.9914448613738104;
        case 2: return 0.9659258262890683;
        case 3: return 0.9238795325112867;
        case 4: return 0.8660254037844386;
        case 5: return 0.7933533402912352;
        case 6: return 0.7071067811865476;
        case 7: return 0.6087614290087207;
        case 8: return 0.5;
        case 9: return 0.3826834323650898;
        case 10: return 0.25881904510252074;
        case 11: return 0.1305261922200516;
        default: return 0.0;   // m = 12
    }
}
__device__ __forceinline__ double cos48(int k) {
    k = ((k % 48) + 48) % 48;
    if (k <= 12) return cos_q24(k);
    if (k <= 24) return -cos_q24(24 - k);
    if (k <= 36) return -cos_q24(k - 24);
    return cos_q24(48 - k);
}
__device__ __forceinline__ double sin48(int k) { return cos48(k - 12); }

template <typename T> struct Cx;
template <> struct Cx<double> { typedef double2 t; };
template <> struct Cx<float> { typedef float2 t; };

template <typename T2, typename T>
__device__ __forceinline__ T2 mk2(T x, T y) {
    T2 r;
    r.x = x;
    r.y = y;
    return r;
}

// y * W_R^m (forward sign): W = cos(2 pi m/R) - i sin(2 pi m/R)
template <typename Tc, int R>
__device__ __forceinline__ typename Cx<Tc>::t twiddle_const(typename Cx<Tc>::t y, int m) {
    const int k = (m % R) * (48 / R);
    if (k == 0) return y;
    if (k == 12) return mk2<typename Cx<Tc>::t>(y.y, -y.x);     // -i
    if (k == 24) return mk2<typename Cx<Tc>::t>(-y.x, -y.y);    // -1
    if (k == 36) return mk2<typename Cx<Tc>::t>(-y.y, y.x);     // +i
    const Tc c = (Tc)cos48(k), s = (Tc)sin48(k);
    return mk2<typename Cx<Tc>::t>(y.x * c + y.y * s, y.y * c - y.x * s);
}

template <typename Tc, int R> struct Dft;

template <typename Tc> struct Dft<Tc, 2> {
    typedef typename Cx<Tc>::t T2;
    static __device__ __forceinline__ void run(T2 *v) {
        const T2 a = v[0], b = v[1];
        v[0] = mk2<T2>(a.x + b.x, a.y + b.y);
        v[1] = mk2<T2>(a.x - b.x, a.y - b.y);
    }
};

template <typename Tc> struct Dft<Tc, 3> {
    typedef typename Cx<Tc>::t T2;
    static __device__ __forceinline__ void run(T2 *v) {
        const Tc k3 = (Tc)0.86602540378443864676;
        const T2 a = v[0];
        const T2 s = mk2<T2>(v[1].x + v[2].x, v[1].y + v[2].y);
        const T2 d = mk2<T2>(v[1].x - v[2].x, v[1].y - v[2].y);
        const T2 t = mk2<T2>(a.x - (Tc)0.5 * s.x, a.y - (Tc)0.5 * s.y);
        v[0] = mk2<T2>(a.x + s.x, a.y + s.y);
        v[1] = mk2<T2>(t.x + k3 * d.y, t.y - k3 * d.x);
        v[2] = mk2<T2>(t.x - k3 * d.y, t.y + k3 * d.x);
    }
};

template <typename Tc> struct Dft<Tc, 4> {
    typedef typename Cx<Tc>::t T2;
    static __device__ __forceinline__ void run(T2 *v) {
        const T2 s02 = mk2<T2>(v[0].x + v[2].x, v[0].y + v[2].y);
        const T2 d02 = mk2<T2>(v[0].x - v[2].x, v[0].y - v[2].y);
        const T2 s13 = mk2<T2>(v[1].x + v[3].x, v[1].y + v[3].y);
        const T2 d13 = mk2<T2>(v[1].y - v[3].y, v[3].x - v[1].x);  // -i (v1 - v3)
        v[0] = mk2<T2>(s02.x + s13.x, s02.y + s13.y);
        v[2] = mk2<T2>(s02.x - s13.x, s02.y - s13.y);
        v[1] = mk2<T2>(d02.x + d13.x, d02.y + d13.y);
        v[3] = mk2<T2>(d02.x - d13.x, d02.y - d13.y);
    }
};

// R = R1 * R2 with R1 = 4 when possible, else 2, else 3.
template <typename Tc, int R> struct Dft {
    typedef typename Cx<Tc>::t T2;
    static constexpr int R1 = (R % 4 == 0) ? 4 : ((R % 2 == 0) ? 2 : 3);
    static constexpr int R2 = R / R1;
    static __device__ __forceinline__ void run(T2 *x) {
        T2 y[R];
#pragma unroll
        for (int n2 = 0; n2 < R2; ++n2) {
            T2 t[R1];
#pragma unroll
            for (int n1 = 0; n1 < R1; ++n1) t[n1] = x[R2 * n1 + n2];
            Dft<Tc, R1>::run(t);
#pragma unroll
            for (int k1 = 0; k1 < R1; ++k1) y[n2 * R1 + k1] = twiddle_const<Tc, R>(t[k1], n2 * k1);
        }
#pragma unroll
        for (int k1 = 0; k1 < R1; ++k1) {
            T2 t[R2];
#pragma unroll
            for (int n2 = 0; n2 < R2; ++n2) t[n2] = y[n2 * R1 + k1];
            Dft<Tc, R2>::run(t);
#pragma unroll
            for (int k2 = 0; k2 < R2; ++k2) x[k1 + R1 * k2] = t[k2];
        }
    }
};

// Shared-memory layout of a line: complex element i lives at PAD(i) = i + i/16,
// so the stride-16 writes of a first radix-16 stage fall in distinct banks.
__device__ __forceinline__ int PAD(int i) { return i + (i >> 4); }
template <int M> struct LineStride { static constexpr int value = M + (M >> 4) + 1; };

// One Stockham stage of radix R on S lines of length M (line stride LS).
template <typename Tc, int M, int S, int R, int Ns>
__device__ __forceinline__ void fstage(const typename Cx<Tc>::t *__restrict__ src,
                                       typename Cx<Tc>::t *__restrict__ dst,
                                       const typename Cx<Tc>::t *__restrict__ roots) {
    typedef typename Cx<Tc>::t T2;
    constexpr int LS = LineStride<M>::value;
    constexpr int MR = M / R;
    constexpr int stride = M / (Ns * R);
    for (int t = threadIdx.x; t < S * MR; t += blockDim.x) {
        const int s = t / MR;
        const int j = t - s * MR;
        const int k = j % Ns;
        const T2 *x = src + s * LS;
        T2 *y = dst + s * LS;
        T2 v[R];
#pragma unroll
        for (int r = 0; r < R; ++r) v[r] = x[PAD(j + r * MR)];
        if (Ns > 1 && k > 0) {
#pragma unroll
            for (int r = 1; r < R; ++r) {
                const T2 w = roots[k * r * stride];
                const T2 a = v[r];
                v[r] = mk2<T2>(a.x * w.x - a.y * w.y, a.x * w.y + a.y * w.x);
            }
        }
        Dft<Tc, R>::run(v);
        const int idxD = (j / Ns) * Ns * R + k;
#pragma unroll
        for (int r = 0; r < R; ++r) y[PAD(idxD + r * Ns)] = v[r];
    }
}

template <typename Tc, int M, int S, int Ns>
__device__ __forceinline__ void fstages(typename Cx<Tc>::t *&src, typename Cx<Tc>::t *&dst,
                                        const typename Cx<Tc>::t *roots) {}

template <typename Tc, int M, int S, int Ns, int R, int... Rest>
__device__ __forceinline__ void fstages(typename Cx<Tc>::t *&src, typename Cx<Tc>::t *&dst,
                                        const typename Cx<Tc>::t *roots) {
    fstage<Tc, M, S, R, Ns>(src, dst, roots);
    __syncthreads();
    typename Cx<Tc>::t *t = src;
    src = dst;
    dst = t;
    fstages<Tc, M, S, Ns * R, Rest...>(src, dst, roots);
}

// Real element m of a line's odd extension, stored inside the padded complex layout.
__device__ __forceinline__ int ZPAD(int m) { return 2 * PAD(m >> 1) + (m & 1); }

// FP32 tiles use up to ~74 KB of shared memory, so three CTAs fit an SM; the
// register cap keeps the third one resident.
// One CTA's work of the transform: S whole lines (see the file comment of
// k_dst_fast.cu).  COH: loads of data written earlier in the same launch go
// through L2 only (the batched persistent kernel); smem_raw is the CTA's
// dynamic shared memory; (bx, by) the tile index.
template <typename Tc, typename Tin, typename Tout, int AXIS, int MODE, int M, int S, bool COH,
          int... Rs>
__device__ __forceinline__ void dst_fast_tile(const Tin *in, Tout *out, double *aux,
                                              const typename Cx<Tc>::t *roots_g,
                                              const typename Cx<Tc>::t *half_g, int Nx, int Ny,
                                              int Nz, Tc scale, unsigned char *smem_raw, int bx,
                                              int by) {
    typedef typename Cx<Tc>::t T2;
    constexpr int N = M - 1;
    constexpr int LS = LineStride<M>::value;
    constexpr int twoM = 2 * M;
    constexpr int NT = 256;
    constexpr int ITER = (S * N + NT - 1) / NT;  // elements per thread in load/store phases
    const size_t lo_off = (size_t)Nx * Ny * Nz;  // lo plane of a double-float output
    (void)lo_off;
    T2 *roots = reinterpret_cast<T2 *>(smem_raw);
    T2 *half = roots + M;
    T2 *buf0 = half + (M + 1);
    T2 *buf1 = buf0 + S * LS;
    for (int t = threadIdx.x; t < M; t += NT) roots[t] = roots_g[t];
    for (int t = threadIdx.x; t <= M; t += NT) half[t] = half_g[t];

    Tc *z = reinterpret_cast<Tc *>(buf0);
    for (int s = threadIdx.x; s < S; s += NT) {
        z[s * 2 * LS + ZPAD(0)] = (Tc)0;
        z[s * 2 * LS + ZPAD(M)] = (Tc)0;
    }
    size_t base;
    int nvalid;
    // all global loads of the tile are issued before any shared-memory store
    Tc v[ITER];
    if (AXIS == HS_AXIS_X) {
        const long nrows = (long)Ny * Nz;
        const long row0 = (long)bx * S;
        base = (size_t)row0 * N;
        nvalid = (int)min((long)S, nrows - row0);
        const int nel = nvalid * N;
#pragma unroll
        for (int it = 0; it < ITER; ++it) {
            const int e = threadIdx.x + it * NT;
            v[it] = (e < nel) ? (Tc)ldc<COH>(in + base + e) : (Tc)0;
        }
#pragma unroll
        for (int it = 0; it < ITER; ++it) {
            const int e = threadIdx.x + it * NT;
            if (e < S * N) {
                const int s = e / N;
                const int i = e - s * N;
                z[s * 2 * LS + ZPAD(i + 1)] = v[it];
                z[s * 2 * LS + ZPAD(twoM - 1 - i)] = -v[it];
            }
        }
    } else {
        const int p0 = bx * S;
        base = (size_t)by * N * Nx + p0;
        nvalid = min(S, Nx - p0);
#pragma unroll
        for (int it = 0; it < ITER; ++it) {
            const int e = threadIdx.x + it * NT;
            const int j = e / S;
            const int s = e - j * S;
            v[it] = (e < S * N && s < nvalid) ? (Tc)ldc<COH>(in + base + (size_t)j * Nx + s) : (Tc)0;
        }
#pragma unroll
        for (int it = 0; it < ITER; ++it) {
            const int e = threadIdx.x + it * NT;
            if (e < S * N) {
                const int j = e / S;
                const int s = e - j * S;
                z[s * 2 * LS + ZPAD(j + 1)] = v[it];
                z[s * 2 * LS + ZPAD(twoM - 1 - j)] = -v[it];
            }
        }
    }
    __syncthreads();

    T2 *src = buf0, *dst = buf1;
    fstages<Tc, M, S, 1, Rs...>(src, dst, roots);

    const Tc q = scale * (Tc)0.25;
    if (AXIS == HS_AXIS_X) {
        const int nel = nvalid * N;
        if constexpr (MODE == HS_MODE_DF_ADD || MODE == HS_MODE_DF_FINAL ||
                      MODE == HS_MODE_DF_FINAL_HI) {
            // read every (hi, lo) of the tile before any store
            float uh[ITER], ul[ITER];
#pragma unroll
            for (int it = 0; it < ITER; ++it) {
                const int e = threadIdx.x + it * NT;
                uh[it] = (e < nel) ? ldc<COH>(out + base + e) : 0.f;
                ul[it] = (e < nel && MODE != HS_MODE_DF_FINAL_HI) ? ldc<COH>(out + base + e + lo_off)
                                                                  : 0.f;
            }
#pragma unroll
            for (int it = 0; it < ITER; ++it) {
                const int e = threadIdx.x + it * NT;
                if (e < nel) {
                    const int s = e / N;
                    const int k = e - s * N + 1;
                    const T2 Wk = src[s * LS + PAD(k)];
                    const T2 Wm = src[s * LS + PAD(M - k)];
                    const T2 cs = half[k];
                    const Tc X = ((Wm.y - Wk.y) + cs.x * (Wk.x - Wm.x) + cs.y * (Wk.y + Wm.y)) * q;
                    dfloat a;
                    a.hi = uh[it];
                    a.lo = ul[it];
                    const dfloat r = df_add(a, df_of((float)X));
                    if constexpr (MODE == HS_MODE_DF_ADD) {
                        out[base + e] = r.hi;
                        out[base + e + lo_off] = r.lo;
                    } else {
                        aux[base + e] = (double)r.hi + (double)r.lo;
                    }
                }
            }
        } else {
#pragma unroll
            for (int it = 0; it < ITER; ++it) {
                const int e = threadIdx.x + it * NT;
                if (e < nel) {
                    const int s = e / N;
                    const int k = e - s * N + 1;
                    const T2 Wk = src[s * LS + PAD(k)];
                    const T2 Wm = src[s * LS + PAD(M - k)];
                    const T2 cs = half[k];
                    const Tc X = ((Wm.y - Wk.y) + cs.x * (Wk.x - Wm.x) + cs.y * (Wk.y + Wm.y)) * q;
                    hs_emit<Tout, MODE>(out, aux, lo_off, base + e, (double)X);
                }
            }
        }
    } else {
#pragma unroll
        for (int it = 0; it < ITER; ++it) {
            const int e = threadIdx.x + it * NT;
            const int kk = e / S;
            const int s = e - kk * S;
            if (e < S * N && s < nvalid) {
                const int k = kk + 1;
                const T2 Wk = src[s * LS + PAD(k)];
                const T2 Wm = src[s * LS + PAD(M - k)];
                const T2 cs = half[k];
                const Tc X = ((Wm.y - Wk.y) + cs.x * (Wk.x - Wm.x) + cs.y * (Wk.y + Wm.y)) * q;
                hs_emit<Tout, MODE>(out, aux, lo_off, base + (size_t)kk * Nx + s, (double)X);
            }
        }
    }
}


// Lines per CTA: about 4096 (FP32) or 2048 (FP64) complex points per buffer;
// y-lines at least 16 (FP32) / 8 (FP64) so each row segment is 64 bytes; never
// more than fits in 227 KB of shared memory.
template <typename Tc, int M, int AXIS>
struct Lines {
    static constexpr int pts = (sizeof(Tc) == 4) ? 4096 : 2048;
    static constexpr int base = (pts / M) > 0 ? (pts / M) : 1;
    static constexpr int ymin = (sizeof(Tc) == 4) ? 16 : 8;
    static constexpr int want = (AXIS == HS_AXIS_Y && base < ymin) ? ymin : base;
    static constexpr int fit = (int)((227 * 1024 / (2 * sizeof(Tc)) - (2 * M + 1)) /
                                     (2 * (M + (M >> 4) + 1)));
    static constexpr int value = want < fit ? want : fit;
};

template <typename Tc, int M, int S>
constexpr size_t fast_smem() {
    return sizeof(typename Cx<Tc>::t) * ((size_t)2 * M + 1 + (size_t)2 * S * LineStride<M>::value);
}


// ============================================================ right-hand side
struct RhsArgs {
    int Nx, Ny, Nz;
    double hz;           // h_z (the uniform h for order 6)
    int order, equation, rhs_kind;
    const double *coef;  // [Nz][3][4]
    const double *c0;    // [Nz+2]
    const double *c1;    // [Nz+2]
    const float4 *rc;    // [Nz+2]: per-row double-float RHS weights (hs_api.cu, hs_set_coeff)
    int has_faces;       // 0: every Dirichlet face is zero, so the lifting vanishes
    int bz0;             // first z-tile of the launch (slab launches of the tiled kernels)
    int zt;              // planes per z-tile of the sum-factorised kernel (runtime depth)
    const double *ghost; // precomputed ghost nodes (layout of hs_plan_s::d_ghost), or null
    DevBoundary b;
};

template <typename T>
__device__ __forceinline__ double ld(const T *p, size_t i) {
    return (double)__ldg(p + i);
}

template <typename T>
__device__ double boundary_value(const RhsArgs &a, int i, int j, int l) {
    const int Nx2 = a.Nx + 2, Ny2 = a.Ny + 2;
    const T *p;
    size_t idx;
    if (l == 0 || l == a.Nz + 1) {
        p = static_cast<const T *>(a.b.face[l == 0 ? 4 : 5]);
        idx = (size_t)j * Nx2 + i;
    } else if (j == 0 || j == a.Ny + 1) {
        p = static_cast<const T *>(a.b.face[j == 0 ? 2 : 3]);
        idx = (size_t)l * Nx2 + i;
    } else {
        p = static_cast<const T *>(a.b.face[i == 0 ? 0 : 1]);
        idx = (size_t)l * Ny2 + j;
    }
    return p ? ld(p, idx) : 0.0;
}

// Adds a per-thread value over the CTA and atomically to *out (thread 0).
__device__ __forceinline__ void block_sum_to(double v, double *out) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    __shared__ double part[32];
    const int tid = threadIdx.x + threadIdx.y * blockDim.x;
    const int nw = (blockDim.x * blockDim.y + 31) >> 5;
    __syncthreads();
    if ((tid & 31) == 0) part[tid >> 5] = v;
    __syncthreads();
    if (tid == 0) {
        double s = 0.0;
        for (int w = 0; w < nw; ++w) s += part[w];
        atomicAdd(out, s);
    }
}

// Subtract the boundary-node terms of row (i, j, l) (node indices, interior).
template <typename T>
__device__ double lift_terms(const RhsArgs &a, int i, int j, int l) {
    double acc = 0.0;
    const double *cf = a.coef + (size_t)(l - 1) * 12;
    for (int dl = -1; dl <= 1; ++dl) {
        const int ll = l + dl;
        for (int dj = -1; dj <= 1; ++dj) {
            const int jj = j + dj;
            for (int di = -1; di <= 1; ++di) {
                const int ii = i + di;
                const bool bnd = (ll == 0 || ll == a.Nz + 1 || jj == 0 || jj == a.Ny + 1 ||
                                  ii == 0 || ii == a.Nx + 1);
                if (!bnd) continue;
                const int m = (di != 0 && dj != 0) ? 0 : (di != 0 ? 1 : (dj != 0 ? 2 : 3));
                const double c = cf[(dl + 1) * 4 + m];
                if (c != 0.0) acc += c * boundary_value<T>(a, ii, jj, ll);
            }
        }
    }
    return acc;
}

// OUT_DF = 0: F is FP64; OUT_DF = 1: F is stored as a double-float pair (hi, lo).
// ---------------------------------------------------------------------------
// Tiled right-hand side for nodal f: a CTA owns a TX x TY patch of interior
// points and marches over RZ planes in z with a ring of five f-planes in
// shared memory (halo 2 in x and y; the second neighbours beyond a face are
// the ghosts 2 f_0 - f_1 + h^2 (f_nn)_face, filled in at load time).  The
// 6th-order operator is evaluated in the summed form
//   F6 / h^2 = (67/120 - h^2 K_l / 20) f + S1 / 18 - S2 / 240 + E / 90
//              + (h^3 K_{z,l} / 120) (f_{l+1} - f_{l-1}),
// where S1 sums the 6 face neighbours, S2 the 6 second neighbours and E the 12
// edge mid-points (the same operator as the expanded form above:
// Dx+Dy+Dz = S1 - 6 f, Dx^2+Dy^2+Dz^2 = S2 - 4 S1 + 18 f,
// DxDy+DxDz+DyDz = E - 4 S1 + 12 f).
constexpr int RTX = 32, RTY = 8, RZ = 16;
constexpr int RHX = RTX + 4, RHY = RTY + 4;

template <typename T>
__device__ double node_or_ghost(const RhsArgs &a, const T *f, int i, int j, int l) {
    const int Nx = a.Nx, Ny = a.Ny, Nz = a.Nz;
    const size_t sy = (size_t)(Nx + 2), sz = sy * (Ny + 2);
    const bool xin = i >= 0 && i <= Nx + 1, yin = j >= 0 && j <= Ny + 1, zin = l >= 0 && l <= Nz + 1;
    if (xin && yin && zin) return ld(f, (size_t)l * sz + (size_t)j * sy + i);
    // ghosts exist one node beyond a face, along that face's normal only
    if (!xin && yin && zin && (i == -1 || i == Nx + 2)) {
        const int i0 = (i == -1) ? 0 : Nx + 1, i1 = (i == -1) ? 1 : Nx;
        const T *fnn = static_cast<const T *>(a.b.fnn[i == -1 ? 0 : 1]);
        const size_t r = (size_t)l * sz + (size_t)j * sy;
        return 2.0 * ld(f, r + i0) - ld(f, r + i1) +
               (fnn ? (a.hz * a.hz) * ld(fnn, (size_t)l * (Ny + 2) + j) : 0.0);
    }
    if (xin && !yin && zin && (j == -1 || j == Ny + 2)) {
        const int j0 = (j == -1) ? 0 : Ny + 1, j1 = (j == -1) ? 1 : Ny;
        const T *fnn = static_cast<const T *>(a.b.fnn[j == -1 ? 2 : 3]);
        const size_t r = (size_t)l * sz + i;
        return 2.0 * ld(f, r + (size_t)j0 * sy) - ld(f, r + (size_t)j1 * sy) +
               (fnn ? (a.hz * a.hz) * ld(fnn, (size_t)l * (Nx + 2) + i) : 0.0);
    }
    if (xin && yin && !zin && (l == -1 || l == Nz + 2)) {
        const int l0 = (l == -1) ? 0 : Nz + 1, l1 = (l == -1) ? 1 : Nz;
        const T *fnn = static_cast<const T *>(a.b.fnn[l == -1 ? 4 : 5]);
        const size_t r = (size_t)j * sy + i;
        return 2.0 * ld(f, (size_t)l0 * sz + r) - ld(f, (size_t)l1 * sz + r) +
               (fnn ? (a.hz * a.hz) * ld(fnn, (size_t)j * (Nx + 2) + i) : 0.0);
    }
    return 0.0;  // never read by an interior point
}

// =================================================================== residual
// One term of the double-float residual's row sum (hs_resid_sf.cuh): the
// coefficient pair k times the plane sum v + vl (hi sum v; vl its two_sum error
// plus the sum of the lo parts, formed once per plane) added to the
// unnormalised pair (S, E): the leading product exactly (two_prod into two_sum),
// cross terms in FP32.
__device__ __forceinline__ void acc_term(float &S, float &E, float2 k, float v, float vl) {
    // S + E += (k.x + k.y) * (v + vl)
    const float p = k.x * v;
    const float pe = fmaf(k.x, v, -p);
    float s, t;
    df_two_sum(S, p, s, t);
    S = s;
    E += t + pe + fmaf(k.x, vl, k.y * v);
}

// The same term for a plane sum with no low-order part (vl = 0): the cross
// term k.y v is rounded on its own (not contracted into the sum), so the result
// is acc_term's with vl = 0 bit for bit.
__device__ __forceinline__ void acc_term_hi(float &S, float &E, float2 k, float v) {
    const float p = k.x * v;
    const float pe = fmaf(k.x, v, -p);
    float s, t;
    df_two_sum(S, p, s, t);
    S = s;
    E += t + pe + __fmul_rn(k.y, v);
}

constexpr int QTX = 32, QTY = 8, QZ = 16;
constexpr int QHX = QTX + 2, QHY = QTY + 2;

// FP64 residual of a double-float iterate: the same z-march as residual_sf_tile,
// with U = U_hi + U_lo and F = F_hi + F_lo formed in FP64 and the 12 products
// and the subtraction in FP64 (rounding 2^-53 instead of the pair's ~2^-47).
// Used where the double-float residual has stopped the refinement short.
// smem holds 2 planes of (QTY + 2) x (QTX + 2) doubles; r is written in FP32
// (it only feeds the next correction solve).
template <bool COH>
__device__ __forceinline__ void residual64_tile(int Nx, int Ny, int Nz,
                                                const double *__restrict__ coef,
                                                const float *__restrict__ F,
                                                const float *__restrict__ U, float *__restrict__ r,
                                                double *r2out, unsigned char *smem, int bx, int by,
                                                int bz) {
    double(*ud)[QHY][QHX] = reinterpret_cast<double(*)[QHY][QHX]>(smem);
    constexpr int NT = QTX * QTY;
    constexpr int PER = (QHX * QHY + NT - 1) / NT;
    const int tid = threadIdx.x + threadIdx.y * blockDim.x;
    const int tx = tid & (QTX - 1), ty = tid / QTX;
    const int i0 = bx * QTX, j0 = by * QTY;
    const int lbeg = bz * QZ;
    const int lend = min(lbeg + QZ, Nz);
    const size_t plane = (size_t)Nx * Ny;
    const size_t n = plane * Nz;
    const int i = i0 + tx, j = j0 + ty;
    const bool active = i < Nx && j < Ny;

    double rv[PER];
    auto fetch = [&](int l) {
#pragma unroll
        for (int k = 0; k < PER; ++k) {
            const int e = tid + k * NT;
            const int ey = e / QHX, ex = e - ey * QHX;
            const int ii = i0 - 1 + ex, jj = j0 - 1 + ey;
            rv[k] = 0.0;
            if (e < QHX * QHY && l >= 0 && l < Nz && ii >= 0 && ii < Nx && jj >= 0 && jj < Ny) {
                const size_t o = (size_t)l * plane + (size_t)jj * Nx + ii;
                rv[k] = (double)ldc<COH>(U + o) + (double)ldc<COH>(U + n + o);
            }
        }
    };
    auto store = [&](int l) {
        const int slot = (l + 2) & 1;
#pragma unroll
        for (int k = 0; k < PER; ++k) {
            const int e = tid + k * NT;
            if (e < QHX * QHY) {
                const int ey = e / QHX, ex = e - ey * QHX;
                ud[slot][ey][ex] = rv[k];
            }
        }
    };
    struct Sums {
        double C, X, Y, U;
    };
    auto sums = [&](int l, Sums &ps) {
        const int sl = (l + 2) & 1;
        const int cx = tx + 1, cy = ty + 1;
        ps.C = (ud[sl][cy - 1][cx - 1] + ud[sl][cy - 1][cx + 1]) +
               (ud[sl][cy + 1][cx - 1] + ud[sl][cy + 1][cx + 1]);
        ps.X = ud[sl][cy][cx - 1] + ud[sl][cy][cx + 1];
        ps.Y = ud[sl][cy - 1][cx] + ud[sl][cy + 1][cx];
        ps.U = ud[sl][cy][cx];
    };

    Sums pm, p0, pp;
    double rsq = 0.0;
    fetch(lbeg - 1);
    store(lbeg - 1);
    __syncthreads();
    sums(lbeg - 1, pm);
    fetch(lbeg);
    __syncthreads();
    store(lbeg);
    __syncthreads();
    sums(lbeg, p0);
    fetch(lbeg + 1);
    for (int l = lbeg; l < lend; ++l) {
        __syncthreads();
        store(l + 1);
        __syncthreads();
        fetch(l + 2);
        sums(l + 1, pp);
        if (active) {
            const double *cf = coef + (size_t)l * 12;
            double S = 0.0;
            const Sums *q[3] = {&pm, &p0, &pp};
#pragma unroll
            for (int nu = 0; nu < 3; ++nu) {
                const int ll = l + nu - 1;
                if (ll < 0 || ll >= Nz) continue;
                const Sums &ps = *q[nu];
                S = fma(cf[nu * 4 + 0], ps.C, S);
                S = fma(cf[nu * 4 + 1], ps.X, S);
                S = fma(cf[nu * 4 + 2], ps.Y, S);
                S = fma(cf[nu * 4 + 3], ps.U, S);
            }
            const size_t o = (size_t)l * plane + (size_t)j * Nx + i;
            const double res = ((double)ldc<COH>(F + o) + (double)ldc<COH>(F + o + n)) - S;
            r[o] = (float)res;
            rsq = fma(res, res, rsq);
        }
        pm = p0;
        p0 = pp;
    }
    if (r2out) block_sum_to(rsq, r2out);
}

// Residual precision of the refinement: the device-side rule of the automatic
// mode.  `norms` holds squared norms [||F||^2, ||r_1||^2, ...].  Sweep m's
// residual (m >= 2) is taken in FP64 when the previous one shrank by less than
// 16x (||r_{m-1}|| > ||r_{m-2}|| / 16, r_0 = F): a correction solve in FP32
// contracts far more than that unless the double-float residual has reached
// its rounding floor.
__device__ __forceinline__ bool residual_use_f64(const double *norms, int m) {
    if (m < 2) return false;
    const double prev = __ldcg(norms + m - 2), cur = __ldcg(norms + m - 1);
    return cur > prev * (1.0 / 256.0);
}

// ==================================================================== z-solves
// The sweeps walk the column CH planes at a time: all loads of a chunk are
// issued before its dependent chain and its stores (the in-place stores would
// otherwise keep the next plane's load from starting early), so each thread has
// 2-3 x CH loads in flight.
constexpr int CH = 16;

// Loads of the cached factors in the pipelined sweeps.  STREAM: each factor is
// read once per solve, so it is loaded with the streaming (evict-first) policy and
// does not push the forward sweep's values, which the backward sweep reads again,
// out of L2 -- worth it where those values fit in L2 (255^3: 405 -> 299 MB of DRAM
// traffic per launch); at 511^3 and above they cannot, and plain loads are faster.
template <bool STREAM, typename Tf>
__device__ __forceinline__ Tf ldfac(const Tf *p) {
    if constexpr (STREAM) return __ldcs(p);
    else return *p;
}

// One z-solve with cached factors.  Td: data type (in place); Tf: factor type;
// Ts: type of the forward-sweep values (kept in `scratch` when it is not null,
// else in `data`); Ta: arithmetic type.
template <typename Td, typename Tf, typename Ta, bool COH = false, bool PIPE = true, int CH = hs_tiles::CH,
          bool STREAM = false>
__device__ __forceinline__ void thomas_column(int Nz, size_t plane, size_t idx, Td *data,
                                              Ta *scratch, const Tf *cpr, const Tf *alpha,
                                              const Tf *beta) {
    if constexpr (!PIPE) {
        // chunked, not pipelined (kernels whose register budget cannot hold two
        // chunks, e.g. the persistent batch kernel)
        Ta d = (Ta)0;
        int l = 0;
        for (; l + CH <= Nz; l += CH) {
            Ta r[CH], a[CH], b[CH];
    #pragma unroll
            for (int k = 0; k < CH; ++k) {
                const size_t o = (size_t)(l + k) * plane + idx;
                r[k] = (Ta)ldc<COH>(data + o);
                a[k] = (Ta)alpha[o];
                b[k] = (Ta)beta[o];
            }
    #pragma unroll
            for (int k = 0; k < CH; ++k) {
                d = a[k] * r[k] - b[k] * d;
                r[k] = d;
            }
    #pragma unroll
            for (int k = 0; k < CH; ++k) {
                const size_t o = (size_t)(l + k) * plane + idx;
                if (scratch)
                    scratch[o] = r[k];
                else
                    data[o] = (Td)r[k];
            }
        }
        for (; l < Nz; ++l) {
            const size_t o = (size_t)l * plane + idx;
            d = (Ta)alpha[o] * (Ta)ldc<COH>(data + o) - (Ta)beta[o] * d;
            if (scratch)
                scratch[o] = d;
            else
                data[o] = (Td)d;
        }
        Ta w = d;
        data[(size_t)(Nz - 1) * plane + idx] = (Td)w;
        int top = Nz - 2;  // next plane to solve, going down
        for (; top - CH + 1 >= 0; top -= CH) {
            Ta dv[CH], c[CH];
    #pragma unroll
            for (int k = 0; k < CH; ++k) {
                const size_t o = (size_t)(top - k) * plane + idx;
                dv[k] = scratch ? ldc<COH>(scratch + o) : (Ta)ldc<COH>(data + o);
                c[k] = (Ta)cpr[o];
            }
    #pragma unroll
            for (int k = 0; k < CH; ++k) {
                w = dv[k] - c[k] * w;
                dv[k] = w;
            }
    #pragma unroll
            for (int k = 0; k < CH; ++k) data[(size_t)(top - k) * plane + idx] = (Td)dv[k];
        }
        for (; top >= 0; --top) {
            const size_t o = (size_t)top * plane + idx;
            const Ta dd = scratch ? ldc<COH>(scratch + o) : (Ta)ldc<COH>(data + o);
            w = dd - (Ta)cpr[o] * w;
            data[o] = (Td)w;
        }
    } else {
        // software-pipelined: the loads of chunk c + 1 are issued before the
        // dependent chain and the stores of chunk c (the in-place stores would
        // otherwise keep the compiler from moving them up)
        Ta d = (Ta)0;
        const int nfull = Nz / CH;
        {
            Ta r[CH], a[CH], b[CH];
            if (nfull > 0) {
    #pragma unroll
                for (int k = 0; k < CH; ++k) {
                    const size_t o = (size_t)k * plane + idx;
                    r[k] = (Ta)ldc<COH>(data + o);
                    a[k] = (Ta)ldfac<STREAM>(alpha + o);
                    b[k] = (Ta)ldfac<STREAM>(beta + o);
                }
            }
            for (int c = 0; c < nfull; ++c) {
                const bool more = c + 1 < nfull;
                Ta r2[CH], a2[CH], b2[CH];
    #pragma unroll
                for (int k = 0; k < CH; ++k) {
                    const size_t o = (size_t)((c + 1) * CH + k) * plane + idx;
                    r2[k] = more ? (Ta)ldc<COH>(data + o) : (Ta)0;
                    a2[k] = more ? (Ta)ldfac<STREAM>(alpha + o) : (Ta)0;
                    b2[k] = more ? (Ta)ldfac<STREAM>(beta + o) : (Ta)0;
                }
    #pragma unroll
                for (int k = 0; k < CH; ++k) {
                    d = a[k] * r[k] - b[k] * d;
                    r[k] = d;
                }
    #pragma unroll
                for (int k = 0; k < CH; ++k) {
                    const size_t o = (size_t)(c * CH + k) * plane + idx;
                    if (scratch)
                        scratch[o] = r[k];
                    else
                        data[o] = (Td)r[k];
                }
    #pragma unroll
                for (int k = 0; k < CH; ++k) {
                    r[k] = r2[k];
                    a[k] = a2[k];
                    b[k] = b2[k];
                }
            }
        }
        for (int l = nfull * CH; l < Nz; ++l) {
            const size_t o = (size_t)l * plane + idx;
            d = (Ta)ldfac<STREAM>(alpha + o) * (Ta)ldc<COH>(data + o) - (Ta)ldfac<STREAM>(beta + o) * d;
            if (scratch)
                scratch[o] = d;
            else
                data[o] = (Td)d;
        }
        Ta w = d;
        data[(size_t)(Nz - 1) * plane + idx] = (Td)w;
        // back substitution, planes Nz-2 down to 0, in chunks of CH (tail first)
        const int nb = Nz - 1;             // planes left to solve
        const int ntail = nb % CH;
        int top = Nz - 2;
        for (int t = 0; t < ntail; ++t, --top) {
            const size_t o = (size_t)top * plane + idx;
            const Ta dd = scratch ? ldc<COH>(scratch + o) : (Ta)ldc<COH>(data + o);
            w = dd - (Ta)ldfac<STREAM>(cpr + o) * w;
            data[o] = (Td)w;
        }
        const int nbf = nb / CH;           // full chunks, top planes first
        {
            Ta dv[CH], cc[CH];
            if (nbf > 0) {
    #pragma unroll
                for (int k = 0; k < CH; ++k) {
                    const size_t o = (size_t)(top - k) * plane + idx;
                    dv[k] = scratch ? ldc<COH>(scratch + o) : (Ta)ldc<COH>(data + o);
                    cc[k] = (Ta)ldfac<STREAM>(cpr + o);
                }
            }
            for (int c = 0; c < nbf; ++c, top -= CH) {
                const bool more = c + 1 < nbf;
                Ta dv2[CH], cc2[CH];
    #pragma unroll
                for (int k = 0; k < CH; ++k) {
                    const size_t o = (size_t)(more ? top - CH - k : top - k) * plane + idx;
                    dv2[k] = more ? (scratch ? ldc<COH>(scratch + o) : (Ta)ldc<COH>(data + o)) : (Ta)0;
                    cc2[k] = more ? (Ta)ldfac<STREAM>(cpr + o) : (Ta)0;
                }
    #pragma unroll
                for (int k = 0; k < CH; ++k) {
                    w = dv[k] - cc[k] * w;
                    dv[k] = w;
                }
    #pragma unroll
                for (int k = 0; k < CH; ++k) data[(size_t)(top - k) * plane + idx] = (Td)dv[k];
    #pragma unroll
                for (int k = 0; k < CH; ++k) {
                    dv[k] = dv2[k];
                    cc[k] = cc2[k];
                }
            }
        }
    }
}

}  // namespace hs_tiles
