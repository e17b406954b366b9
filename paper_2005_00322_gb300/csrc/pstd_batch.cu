// pstd_batch.cu -- batched runs and the reflection-coefficient combination
// of Section 5.
//
// A batch is a set of independent simulations (members), each a plan with
// its own stream.  pstd_batch_run records, per pointer set, one CUDA graph
// of a block of steps in which every member is a parallel branch (fork and
// join events on the batch stream), so one graph launch advances all members
// and small members fill the GPU side by side.
//
// Section 5 realises walls of arbitrary real reflection coefficient R by
// summing 4 basic runs per axis (NN, ND, DN, DD) with weights
// w = (1/4) M^T r, r = [R_L, 1, R_R, R_L R_R]; in d dimensions the 4^d runs
// carry the product of the per-axis weights.  pstd_batch_combine forms
// sum_c w_c p_c on the full node lattice shared by the members.
#include <cuda_runtime.h>

#include <cmath>
#include <new>
#include <vector>

#include "../../include/pstd.h"
#include "pstd_internal.h"

namespace {

constexpr int kBatchGraphSteps = 32;
constexpr int kCombineMax = 64;

struct CombineArgs {
    int n, ndim, accumulate;
    int64_t full[3];            // N_i + 1 nodes per axis (1 for unused axes)
    int64_t total;
    const float* p[kCombineMax];
    int lo[kCombineMax][3];
    int64_t shape[kCombineMax][3];
    double w[kCombineMax];
    float* out;
};

// out[node] (+)= sum_c w_c p_c[node - lo_c], nodes a member does not store
// (Dirichlet walls) contributing zero.  Accumulates in FP64.
__global__ void k_combine(CombineArgs a) {
    for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < a.total;
         idx += (int64_t)gridDim.x * blockDim.x) {
        const int64_t j2 = idx % a.full[2];
        const int64_t r = idx / a.full[2];
        const int64_t j1 = r % a.full[1];
        const int64_t j0 = r / a.full[1];
        double acc = a.accumulate ? (double)a.out[idx] : 0.0;
        for (int c = 0; c < a.n; ++c) {
            const int64_t q0 = j0 - a.lo[c][0], q1 = j1 - a.lo[c][1], q2 = j2 - a.lo[c][2];
            if (q0 < 0 || q0 >= a.shape[c][0] || q1 < 0 || q1 >= a.shape[c][1] || q2 < 0 ||
                q2 >= a.shape[c][2])
                continue;
            acc += a.w[c] * (double)a.p[c][(q0 * a.shape[c][1] + q1) * a.shape[c][2] + q2];
        }
        a.out[idx] = (float)acc;
    }
}

}  // namespace

struct pstd_batch_s {
    int n = 0;
    cudaStream_t stream = nullptr;
    std::vector<pstd_plan_t*> plans;
    std::vector<cudaStream_t> streams;
    cudaEvent_t fork = nullptr;
    std::vector<cudaEvent_t> joins;
    std::vector<pstd_desc> descs;
    // graph of kBatchGraphSteps steps for one pointer set
    std::vector<float*> gptrs;
    cudaGraphExec_t exec = nullptr;
    int64_t graph_launches = 0;
    int64_t last_launches = 0;
    // one cooperative kernel per run (pstd_batch_set_persistent)
    int persistent = 0;
    long long spin_limit = 0;
    unsigned withhold = 0;
    pstd_batch_persist_s* ps = nullptr;
};

namespace {

#define BCK(call)                                                          \
    do {                                                                   \
        cudaError_t _e = (call);                                           \
        if (_e != cudaSuccess) return pstd_internal_cuda_fail(_e, #call);  \
    } while (0)

void batch_release(pstd_batch_s* B) {
    pstd_internal_batch_persist_free(B->ps);
    if (B->exec) cudaGraphExecDestroy(B->exec);
    for (auto* p : B->plans) pstd_free(p);
    for (auto s : B->streams) cudaStreamDestroy(s);
    for (auto e : B->joins) cudaEventDestroy(e);
    if (B->fork) cudaEventDestroy(B->fork);
}

// One block of `k` steps of every member as parallel branches of the batch
// stream (captured when the caller is capturing).
int launch_block(pstd_batch_s* B, float* const* p, float* const* u, int64_t k, int64_t* launches) {
    BCK(cudaEventRecord(B->fork, B->stream));
    for (int m = 0; m < B->n; ++m) {
        BCK(cudaStreamWaitEvent(B->streams[m], B->fork, 0));
        int rc = pstd_internal_launch_steps(B->plans[m], p[m], u + 3 * m, k, launches);
        if (rc != PSTD_OK) return rc;
        BCK(cudaEventRecord(B->joins[m], B->streams[m]));
        BCK(cudaStreamWaitEvent(B->stream, B->joins[m], 0));
    }
    return PSTD_OK;
}

// Every member's register-FFT velocities to their spectrum form or back
// (parallel branches of the batch stream, like the steps).
int convert_block(pstd_batch_s* B, float* const* u, int to_spectrum, int64_t* launches) {
    BCK(cudaEventRecord(B->fork, B->stream));
    for (int m = 0; m < B->n; ++m) {
        BCK(cudaStreamWaitEvent(B->streams[m], B->fork, 0));
        int rc = pstd_internal_convert_velocity(B->plans[m], u + 3 * m, to_spectrum, launches);
        if (rc != PSTD_OK) return rc;
        BCK(cudaEventRecord(B->joins[m], B->streams[m]));
        BCK(cudaStreamWaitEvent(B->stream, B->joins[m], 0));
    }
    return PSTD_OK;
}

bool check_ptrs(const pstd_batch_s* B, float* const* p, float* const* u) {
    if (!p || !u) return false;
    for (int m = 0; m < B->n; ++m) {
        if (!p[m]) return false;
        for (int a = 0; a < B->descs[m].ndim; ++a)
            if (!u[3 * m + a]) return false;
    }
    return true;
}

}  // namespace

extern "C" {

int pstd_batch_plan(const pstd_desc* descs, int n, void* stream, pstd_batch_t** out) {
    if (!out) return PSTD_EINVAL;
    *out = nullptr;
    if (!descs || n < 1) return PSTD_EINVAL;
    pstd_batch_s* B = new (std::nothrow) pstd_batch_s();
    if (!B) return PSTD_ENOMEM;
    B->n = n;
    B->stream = (cudaStream_t)stream;
    B->descs.assign(descs, descs + n);
    int rc = PSTD_OK;
    cudaError_t e = cudaEventCreateWithFlags(&B->fork, cudaEventDisableTiming);
    if (e != cudaSuccess) rc = pstd_internal_cuda_fail(e, "cudaEventCreate");
    for (int m = 0; m < n && rc == PSTD_OK; ++m) {
        cudaStream_t s = nullptr;
        cudaEvent_t j = nullptr;
        e = cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking);
        if (e != cudaSuccess) { rc = pstd_internal_cuda_fail(e, "cudaStreamCreate"); break; }
        B->streams.push_back(s);
        e = cudaEventCreateWithFlags(&j, cudaEventDisableTiming);
        if (e != cudaSuccess) { rc = pstd_internal_cuda_fail(e, "cudaEventCreate"); break; }
        B->joins.push_back(j);
        pstd_plan_t* P = nullptr;
        rc = pstd_plan(&descs[m], s, &P);
        if (rc == PSTD_OK) B->plans.push_back(P);
    }
    if (rc != PSTD_OK) {
        batch_release(B);
        delete B;
        return rc;
    }
    *out = B;
    return PSTD_OK;
}

int pstd_batch_member(const pstd_batch_t* B, int i, pstd_plan_t** plan) {
    if (!B || !plan || i < 0 || i >= B->n) return PSTD_EINVAL;
    *plan = B->plans[i];
    return PSTD_OK;
}

int pstd_batch_init_velocity(pstd_batch_t* B, float* const* p, float* const* u) {
    if (!B || !check_ptrs(B, p, u)) return PSTD_EINVAL;
    B->last_launches = 0;
    BCK(cudaEventRecord(B->fork, B->stream));
    for (int m = 0; m < B->n; ++m) {
        BCK(cudaStreamWaitEvent(B->streams[m], B->fork, 0));
        int rc = pstd_init_velocity(B->plans[m], p[m], u + 3 * m);
        if (rc != PSTD_OK) return rc;
        B->last_launches += pstd_last_launch_count(B->plans[m]);
        BCK(cudaEventRecord(B->joins[m], B->streams[m]));
        BCK(cudaStreamWaitEvent(B->stream, B->joins[m], 0));
    }
    return PSTD_OK;
}

namespace {
int batch_steps(pstd_batch_t* B, float* const* p, float* const* u, int64_t nsteps);
}

int pstd_batch_run(pstd_batch_t* B, float* const* p, float* const* u, int64_t nsteps) {
    if (!B || nsteps < 0 || !check_ptrs(B, p, u)) return PSTD_EINVAL;
    B->last_launches = 0;
    if (nsteps == 0) return PSTD_OK;
    int64_t conv = 0;
    if (B->persistent) {
        // every member's steps in one cooperative kernel on the batch stream;
        // the register-FFT kernel works on the velocities' spectrum form
        const int kind = pstd_internal_batch_persist_kind(B->plans.data(), B->n);
        int rc = kind == 1 ? convert_block(B, u, 1, &conv) : PSTD_OK;
        if (rc == PSTD_OK)
            rc = pstd_internal_batch_persist_run(&B->ps, B->plans.data(), B->n, p, u, nsteps, B->spin_limit,
                                                 B->withhold, B->stream);
        if (rc == PSTD_OK && kind == 1) rc = convert_block(B, u, 0, &conv);
        B->last_launches = conv + 1;
        return rc;
    }
    int rc = convert_block(B, u, 1, &conv);
    if (rc == PSTD_OK) rc = batch_steps(B, p, u, nsteps);
    if (rc == PSTD_OK) rc = convert_block(B, u, 0, &conv);
    B->last_launches += conv;
    return rc;
}

namespace {
// The steps of pstd_batch_run, velocities in spectrum form.
int batch_steps(pstd_batch_t* B, float* const* p, float* const* u, int64_t nsteps) {
    int64_t done = 0;
    if (B->stream != nullptr && nsteps >= kBatchGraphSteps) {
        std::vector<float*> key;
        for (int m = 0; m < B->n; ++m) {
            key.push_back(p[m]);
            for (int a = 0; a < 3; ++a) key.push_back(a < B->descs[m].ndim ? u[3 * m + a] : nullptr);
        }
        if (!B->exec || key != B->gptrs) {
            if (B->exec) { cudaGraphExecDestroy(B->exec); B->exec = nullptr; }
            BCK(cudaStreamBeginCapture(B->stream, cudaStreamCaptureModeThreadLocal));
            int64_t nl = 0;
            int rc = launch_block(B, p, u, kBatchGraphSteps, &nl);
            cudaGraph_t g = nullptr;
            cudaError_t e = cudaStreamEndCapture(B->stream, &g);
            if (rc != PSTD_OK) { if (g) cudaGraphDestroy(g); return rc; }
            if (e != cudaSuccess) return pstd_internal_cuda_fail(e, "cudaStreamEndCapture");
            e = cudaGraphInstantiate(&B->exec, g, 0);
            cudaGraphDestroy(g);
            if (e != cudaSuccess) { B->exec = nullptr; return pstd_internal_cuda_fail(e, "cudaGraphInstantiate"); }
            B->gptrs = key;
            B->graph_launches = nl;
        }
        while (nsteps - done >= kBatchGraphSteps) {
            BCK(cudaGraphLaunch(B->exec, B->stream));
            done += kBatchGraphSteps;
            B->last_launches += B->graph_launches;
        }
    }
    if (done < nsteps) return launch_block(B, p, u, nsteps - done, &B->last_launches);
    return PSTD_OK;
}
}  // namespace

int pstd_batch_combine(pstd_batch_t* B, const double* w, float* const* p, float* out) {
    if (!B || !w || !p || !out) return PSTD_EINVAL;
    const pstd_desc& d0 = B->descs[0];
    for (int m = 0; m < B->n; ++m) {
        if (!p[m]) return PSTD_EINVAL;
        const pstd_desc& d = B->descs[m];
        if (d.ndim != d0.ndim) return PSTD_EINVAL;
        for (int a = 0; a < d.ndim; ++a)
            if (d.ncells[a] != d0.ncells[a]) return PSTD_EINVAL;
    }
    B->last_launches = 0;
    CombineArgs a{};
    a.ndim = d0.ndim;
    a.total = 1;
    for (int i = 0; i < 3; ++i) {
        a.full[i] = i < d0.ndim ? d0.ncells[i] + 1 : 1;
        a.total *= a.full[i];
    }
    a.out = out;
    for (int c0 = 0; c0 < B->n; c0 += kCombineMax) {
        a.n = (B->n - c0) < kCombineMax ? (B->n - c0) : kCombineMax;
        a.accumulate = c0 > 0;
        for (int c = 0; c < a.n; ++c) {
            a.p[c] = p[c0 + c];
            a.w[c] = w[c0 + c];
            pstd_internal_layout(B->plans[c0 + c], a.lo[c], a.shape[c]);
        }
        const int threads = 256;
        int64_t blocks = (a.total + threads - 1) / threads;
        if (blocks > 152 * 16) blocks = 152 * 16;
        k_combine<<<(unsigned)blocks, threads, 0, B->stream>>>(a);
        BCK(cudaGetLastError());
        ++B->last_launches;
    }
    return PSTD_OK;
}

int pstd_batch_free(pstd_batch_t* B) {
    if (!B) return PSTD_OK;
    cudaStreamSynchronize(B->stream);
    batch_release(B);
    delete B;
    return PSTD_OK;
}

int64_t pstd_batch_last_launch_count(const pstd_batch_t* B) { return B ? B->last_launches : 0; }

int pstd_batch_set_persistent(pstd_batch_t* B, int enable, long long spin_limit, int withhold_arrivals) {
    if (!B || spin_limit < 0 || withhold_arrivals < 0) return PSTD_EINVAL;
    if (enable && pstd_internal_batch_persist_kind(B->plans.data(), B->n) == 0) return PSTD_EUNSUPPORTED;
    B->persistent = enable ? 1 : 0;
    B->spin_limit = spin_limit;
    B->withhold = (unsigned)withhold_arrivals;
    return PSTD_OK;
}

int pstd_batch_persistent_kind(const pstd_batch_t* B) {
    if (!B) return PSTD_EINVAL;
    return pstd_internal_batch_persist_kind(B->plans.data(), B->n);
}

int pstd_batch_sync(pstd_batch_t* B) {
    if (!B) return PSTD_EINVAL;
    BCK(cudaStreamSynchronize(B->stream));
    BCK(cudaGetLastError());
    return pstd_internal_batch_persist_status(B->ps);
}

int pstd_reflection_combos(const pstd_desc* tmpl, const double* refl, pstd_desc* descs, double* w) {
    if (!tmpl || !refl || !descs || !w || tmpl->ndim < 1 || tmpl->ndim > 3) return PSTD_EINVAL;
    const int d = tmpl->ndim;
    // image-source polarity matrix of Section 5; columns are NN, ND, DN, DD
    static const double M[4][4] = {{1, 1, -1, -1}, {1, 1, 1, 1}, {1, -1, 1, -1}, {1, -1, -1, 1}};
    static const int BC[4][2] = {{PSTD_NEUMANN, PSTD_NEUMANN}, {PSTD_NEUMANN, PSTD_DIRICHLET},
                                 {PSTD_DIRICHLET, PSTD_NEUMANN}, {PSTD_DIRICHLET, PSTD_DIRICHLET}};
    double wa[3][4];
    for (int i = 0; i < d; ++i) {
        const double rl = refl[2 * i], rr = refl[2 * i + 1];
        if (!std::isfinite(rl) || !std::isfinite(rr)) return PSTD_EINVAL;
        const double r[4] = {rl, 1.0, rr, rl * rr};
        for (int c = 0; c < 4; ++c) {
            double s = 0;
            for (int k = 0; k < 4; ++k) s += M[k][c] * r[k];   // (M^T r)_c
            wa[i][c] = 0.25 * s;
        }
    }
    int count = 1;
    for (int i = 0; i < d; ++i) count *= 4;
    for (int c = 0; c < count; ++c) {
        pstd_desc x = *tmpl;
        double wt = 1.0;
        int rem = c;
        for (int i = d - 1; i >= 0; --i) {   // axis 0 slowest
            const int b = rem % 4;
            rem /= 4;
            x.bc[i][0] = BC[b][0];
            x.bc[i][1] = BC[b][1];
            wt *= wa[i][b];
        }
        descs[c] = x;
        w[c] = wt;
    }
    return PSTD_OK;
}

}  // extern "C"
