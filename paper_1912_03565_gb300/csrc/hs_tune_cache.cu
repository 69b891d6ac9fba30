// Autotune cache: the kernel choices hs_autotune made (transform kernel per
// axis, z-solve mapping) keyed by the device and the problem class -- device
// name and SM count, Nx, Ny, Nz, scheme order, equation, precision and whether
// the z-solves run on FP32 factors -- so a later plan of the same class takes
// them without timing.  Kept for the process (thread-safe) and saved to or
// loaded from a text file, one entry per line:
//   <device> <sms> <Nx> <Ny> <Nz> <order> <equation> <precision> <f32_factors>
//   <variant_x> <variant_y> <thomas_variant> <ms_x> <ms_y>
// (spaces in the device name become '_'; thomas_variant and f32_factors are -1
// where they do not apply).  Host code only; no paper counterpart.
#include <stdio.h>
#include <string.h>

#include <map>
#include <mutex>
#include <string>
#include <tuple>
#include <vector>

#include "hs_internal.cuh"

namespace {

struct TuneKey {
    std::string dev;
    int sms, Nx, Ny, Nz, order, equation, precision, f32fac;
    bool operator<(const TuneKey &o) const {
        return std::tie(dev, sms, Nx, Ny, Nz, order, equation, precision, f32fac) <
               std::tie(o.dev, o.sms, o.Nx, o.Ny, o.Nz, o.order, o.equation, o.precision,
                        o.f32fac);
    }
};

struct TuneVal {
    int vx, vy, thomas;
    float msx, msy;
};

std::mutex g_mu;
std::map<TuneKey, TuneVal> g_cache;

bool key_of(const hs_plan_s *P, TuneKey *k) {
    cudaDeviceProp prop;
    if (cudaGetDeviceProperties(&prop, P->device) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    std::string name(prop.name);
    for (char &c : name)
        if (c == ' ' || c == '\t') c = '_';
    k->dev = name.empty() ? std::string("unknown") : name;
    k->sms = prop.multiProcessorCount;
    k->Nx = P->Nx;
    k->Ny = P->Ny;
    k->Nz = P->Nz;
    k->order = P->order;
    k->equation = P->equation;
    k->precision = P->precision;
    k->f32fac = (P->precision == HS_MIXED && P->have_coeff) ? P->thomas32 : -1;
    return true;
}

bool valid(const TuneKey &k, const TuneVal &v) {
    return k.sms > 0 && k.Nx > 0 && k.Ny > 0 && k.Nz > 0 &&
           (k.order == 2 || k.order == 4 || k.order == 6) &&
           (k.equation == HS_HELMHOLTZ || k.equation == HS_CONVDIFF) &&
           (k.precision == HS_FP64 || k.precision == HS_MIXED) && k.f32fac >= -1 &&
           k.f32fac <= 1 && v.vx >= HS_DST_STAGED && v.vx <= HS_DST_HALF &&
           v.vy >= HS_DST_STAGED && v.vy <= HS_DST_HALF && v.thomas >= -1 &&
           v.thomas <= HS_THOMAS_BAL16_256 && v.msx >= 0.f && v.msy >= 0.f;
}

}  // namespace

bool hs_tune_lookup(const hs_plan_s *P, int *vx, int *vy, int *thomas, float *msx, float *msy) {
    TuneKey k;
    if (!key_of(P, &k)) return false;
    std::lock_guard<std::mutex> g(g_mu);
    const auto it = g_cache.find(k);
    if (it == g_cache.end()) return false;
    *vx = it->second.vx;
    *vy = it->second.vy;
    *thomas = it->second.thomas;
    *msx = it->second.msx;
    *msy = it->second.msy;
    return true;
}

void hs_tune_store(const hs_plan_s *P, int vx, int vy, int thomas, float msx, float msy) {
    TuneKey k;
    if (!key_of(P, &k)) return;
    const TuneVal v{vx, vy, thomas, msx, msy};
    if (!valid(k, v)) return;
    std::lock_guard<std::mutex> g(g_mu);
    g_cache[k] = v;
}

extern "C" hs_status hs_autotune_cache_save(const char *path) {
    if (!path) return HS_ERR_INVALID_ARG;
    FILE *fp = fopen(path, "w");
    if (!fp) return HS_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> g(g_mu);
    fprintf(fp, "# hs autotune cache v1\n");
    for (const auto &e : g_cache) {
        const TuneKey &k = e.first;
        const TuneVal &v = e.second;
        fprintf(fp, "%s %d %d %d %d %d %d %d %d %d %d %d %.6g %.6g\n", k.dev.c_str(), k.sms, k.Nx,
                k.Ny, k.Nz, k.order, k.equation, k.precision, k.f32fac, v.vx, v.vy, v.thomas,
                (double)v.msx, (double)v.msy);
    }
    const bool ok = fflush(fp) == 0;
    return (fclose(fp) == 0 && ok) ? HS_OK : HS_ERR_INVALID_ARG;
}

extern "C" hs_status hs_autotune_cache_load(const char *path) {
    if (!path) return HS_ERR_INVALID_ARG;
    FILE *fp = fopen(path, "r");
    if (!fp) return HS_ERR_INVALID_ARG;
    std::vector<std::pair<TuneKey, TuneVal>> add;
    char line[512];
    bool bad = false;
    while (!bad && fgets(line, sizeof(line), fp)) {
        if (!strchr(line, '\n') && !feof(fp)) {   // longer than any valid entry
            bad = true;
            break;
        }
        const char *p = line;
        while (*p == ' ' || *p == '\t') ++p;
        if (*p == '#' || *p == '\n' || *p == '\r' || *p == 0) continue;
        char dev[256];
        TuneKey k;
        TuneVal v;
        double mx = 0.0, my = 0.0;
        char extra[2];
        const int n = sscanf(p, "%255s %d %d %d %d %d %d %d %d %d %d %d %lf %lf %1s", dev, &k.sms,
                             &k.Nx, &k.Ny, &k.Nz, &k.order, &k.equation, &k.precision, &k.f32fac,
                             &v.vx, &v.vy, &v.thomas, &mx, &my, extra);
        v.msx = (float)mx;
        v.msy = (float)my;
        k.dev = dev;
        if (n != 14 || !valid(k, v)) bad = true;
        else add.emplace_back(k, v);
    }
    fclose(fp);
    if (bad) return HS_ERR_INVALID_ARG;   // nothing merged
    std::lock_guard<std::mutex> g(g_mu);
    for (const auto &e : add) g_cache[e.first] = e.second;
    return HS_OK;
}

extern "C" hs_status hs_autotune_cache_clear(void) {
    std::lock_guard<std::mutex> g(g_mu);
    g_cache.clear();
    return HS_OK;
}

extern "C" hs_status hs_autotune_cache_count(int *count) {
    if (!count) return HS_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> g(g_mu);
    *count = (int)g_cache.size();
    return HS_OK;
}
