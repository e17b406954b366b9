// pstd_tune.cu -- plan-time autotuner of the axis-pass schedules.
//
// The register-FFT passes of an axis can run several schedules (variant: how
// many elements each lane holds and how many passes the FFT takes; line pairs
// per CTA), and which is fastest depends on the axis length, its line count
// and the device.  pstd_plan_autotune times the candidates on the device with
// CUDA events around graph-replayed steps on scratch fields and keeps the
// fastest, axis by axis (coordinate descent from the plan's default choice,
// which stays unless a candidate is at least 2% faster).  The winner is cached
// per (device, grid, walls, form) for the life of the process, so a second
// plan of the same shape costs nothing.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdio>
#include <map>
#include <mutex>
#include <string>
#include <vector>

#include "../../include/pstd.h"
#include "pstd_wkernels.cuh"

namespace {

struct Tuned {
    pstd_plan_opts opts;
    double us, us_default;
};

std::map<std::string, Tuned> g_cache;
std::mutex g_cache_mu;

std::string key_of(const pstd_desc* d, const pstd_plan_opts& o, int dev) {
    char buf[256];
    int n = std::snprintf(buf, sizeof buf, "%d|%d|%d", dev, d->ndim, o.form);
    std::string k(buf, (size_t)n);
    for (int i = 0; i < d->ndim; ++i) {
        n = std::snprintf(buf, sizeof buf, "|%lld:%d%d", (long long)d->ncells[i], d->bc[i][0], d->bc[i][1]);
        k.append(buf, (size_t)n);
    }
    return k;
}

// FFT length of an axis's register passes (0: the axis has none).
int fft_length(const pstd_desc* d, int i) {
    const int l = d->bc[i][0], r = d->bc[i][1];
    if (r == PSTD_NEUMANN_MID || r == PSTD_DIRICHLET_MID) return 0;
    return l == PSTD_PERIODIC ? (int)d->ncells[i] : (int)(2 * d->ncells[i]);
}

// Mean time of one leapfrog step of a plan built with `o` (microseconds; a
// negative value if the plan cannot be built with these options).
double time_step(const pstd_desc* d, const pstd_plan_opts& o, cudaStream_t st, float* p, float* const* u) {
    pstd_plan_t* P = nullptr;
    if (pstd_plan_ex(d, st, &o, &P) != PSTD_OK) return -1.0;
    double us = -1.0;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (cudaEventCreate(&e0) == cudaSuccess && cudaEventCreate(&e1) == cudaSuccess &&
        pstd_run(P, p, u, 32) == PSTD_OK && pstd_sync(P) == PSTD_OK) {
        // two runs of 32 and 96 steps: the difference cancels the per-run
        // conversions of the velocity
        float ms32 = 0, ms96 = 0;
        bool ok = cudaEventRecord(e0, st) == cudaSuccess && pstd_run(P, p, u, 32) == PSTD_OK &&
                  cudaEventRecord(e1, st) == cudaSuccess && cudaEventSynchronize(e1) == cudaSuccess &&
                  cudaEventElapsedTime(&ms32, e0, e1) == cudaSuccess;
        ok = ok && cudaEventRecord(e0, st) == cudaSuccess && pstd_run(P, p, u, 96) == PSTD_OK &&
             cudaEventRecord(e1, st) == cudaSuccess && cudaEventSynchronize(e1) == cudaSuccess &&
             cudaEventElapsedTime(&ms96, e0, e1) == cudaSuccess;
        if (ok && pstd_sync(P) == PSTD_OK && ms96 > ms32) us = 1e3 * (ms96 - ms32) / 64.0;
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    pstd_free(P);
    return us;
}

}  // namespace

extern "C" int pstd_plan_autotune(const pstd_desc* desc, void* stream, const pstd_plan_opts* base,
                                  pstd_plan_t** out, double times_us[2]) {
    if (!desc || !out) return PSTD_EINVAL;
    *out = nullptr;
    pstd_plan_opts o{{-1, -1, -1}, {-1, -1, -1}, 0, 0, 0, 0};
    if (base) o = *base;
    // only the FFT form's register passes have schedules to choose
    if (o.form != 0 || o.persistent) {
        if (times_us) times_us[0] = times_us[1] = -1.0;
        return pstd_plan_ex(desc, stream, &o, out);
    }
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return PSTD_ECUDA;
    const std::string key = key_of(desc, o, dev);
    {
        std::lock_guard<std::mutex> lock(g_cache_mu);
        auto it = g_cache.find(key);
        if (it != g_cache.end()) {
            if (times_us) {
                times_us[0] = it->second.us;
                times_us[1] = it->second.us_default;
            }
            return pstd_plan_ex(desc, stream, &it->second.opts, out);
        }
    }
    // scratch fields of the plan's shapes (zeros: the timing does not depend
    // on the values)
    pstd_plan_t* P0 = nullptr;
    int rc = pstd_plan_ex(desc, stream, &o, &P0);
    if (rc != PSTD_OK) return rc;
    std::vector<float*> f((size_t)desc->ndim + 1, nullptr);
    for (int i = 0; i <= desc->ndim && rc == PSTD_OK; ++i) {
        const size_t bytes = (size_t)pstd_field_numel(P0, i) * sizeof(float);
        if (cudaMalloc((void**)&f[i], bytes) != cudaSuccess || cudaMemset(f[i], 0, bytes) != cudaSuccess)
            rc = PSTD_ENOMEM;
    }
    pstd_free(P0);
    cudaStream_t st = (cudaStream_t)stream;
    Tuned best{o, -1.0, -1.0};
    if (rc == PSTD_OK) {
        best.us = best.us_default = time_step(desc, o, st, f[0], f.data() + 1);
        if (best.us < 0) rc = PSTD_ECUDA;
    }
    for (int a = 0; a < desc->ndim && rc == PSTD_OK; ++a) {
        const int L = fft_length(desc, a);
        if (L <= 0 || pstd::wlanes(L) == 0) continue;
        const int lanes[6] = {pstd::wlanes(L), pstd::wlanes_latency(L), pstd::wlanes_v2(L), pstd::wlanes_v3(L),
                              pstd::wlanes_v4(L), pstd::wlanes_v5(L)};
        for (int v = 0; v < 6; ++v) {
            if (lanes[v] == 0) continue;
            for (int sq = 1; sq * lanes[v] <= 256; sq *= 2) {
                if (sq * lanes[v] < 32) continue;
                pstd_plan_opts c = best.opts;
                c.variant[a] = v;
                c.seqs_per_cta[a] = sq;
                const double us = time_step(desc, c, st, f[0], f.data() + 1);
                if (us > 0 && us < 0.98 * best.us) {
                    best.us = us;
                    best.opts = c;
                }
            }
        }
    }
    for (float* b : f) cudaFree(b);
    if (rc != PSTD_OK) return rc;
    {
        std::lock_guard<std::mutex> lock(g_cache_mu);
        g_cache[key] = best;
    }
    if (times_us) {
        times_us[0] = best.us;
        times_us[1] = best.us_default;
    }
    return pstd_plan_ex(desc, stream, &best.opts, out);
}
