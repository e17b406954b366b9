// pstd_noalloc.cu -- pstd_step_noalloc: leapfrog steps that allocate nothing.
//
// Some callers cannot allocate device memory when they call us: a host
// application whose device memory is owned by a memory manager (a framework's
// caching allocator or a budget fixed at start-up) that forbids allocations
// behind its back, or a latency-critical loop that must not pay for
// cudaMalloc / cudaFree (they can synchronise the device).  pstd_plan()
// allocates its tables and a pressure-shaped scratch accumulator, so this
// entry point instead keeps both in file-scope device arrays of fixed size,
// which every GPU that loads the library holds until the process exits:
//
//   g_noalloc_acc     PSTD_NOALLOC_MAX_POINTS floats (16 MiB): the running
//                     pressure sum over axes of one step (the scratch).
//   g_noalloc_tables  3 axes x 4 tables x PSTD_NOALLOC_MAX_FFT complex (384 KiB):
//                     twiddles, group-II shifts and the two folded k-space
//                     coefficient tables, recomputed in FP64 on the device by
//                     every call.
//
// Host code may not use these names as device addresses (on the host they are
// stand-ins, not device pointers), so every call looks their addresses up with
// cudaGetSymbolAddress on the current device, a host-side query that
// allocates nothing; nothing is cached, so a device reset or a new primary
// context (which may load the module at new addresses) cannot leave a stale
// pointer behind.  Under lazy module loading the arrays are committed when the
// first call on a device loads the module.  Every call shares the arrays and
// leaves them holding its own tables and partial sums; two calls whose work
// overlaps on the GPU (two streams, or two host threads) race on them.
#include <cuda_runtime.h>

#include <cmath>

#include "../../include/pstd.h"
#include "pstd_cta.cuh"

namespace pstd {
cudaError_t launch_k_step(unsigned grid, size_t smem, cudaStream_t st, const StepArgs& a);
cudaError_t set_max_smem(int bytes);
}  // namespace pstd

namespace {

constexpr int kMaxFft = PSTD_NOALLOC_MAX_FFT;
constexpr size_t kSmemBudget = 100 * 1024;

static __device__ __align__(256) float g_noalloc_acc[PSTD_NOALLOC_MAX_POINTS];
static __device__ __align__(256) float2 g_noalloc_tables[3][4][kMaxFft];

// Device addresses of the arrays on the current device, and the step
// kernels' shared-memory limit (both host-side calls that allocate nothing).
cudaError_t resolve_arrays(float** acc, float2** tables) {
    void* a = nullptr;
    void* t = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&a, g_noalloc_acc);
    if (e != cudaSuccess) return e;
    e = cudaGetSymbolAddress(&t, g_noalloc_tables);
    if (e != cudaSuccess) return e;
    e = pstd::set_max_smem((int)kSmemBudget);
    if (e != cudaSuccess) return e;
    *acc = (float*)a;
    *tables = (float2*)t;
    return cudaSuccess;
}

struct AxisSpec {
    int N, L, group2;
    double dx, scaleP, scaleU;
};

// FP64 tables of one axis: [0] exp(-2 pi i m / L), [1] exp(-i pi m / L),
// [2] / [3] the folded coefficients of the p -> u and u -> p derivatives
// (i k exp(+-i k dx / 2) / L times the time-step factor; Table 1 wavenumbers).
__global__ void k_noalloc_tables(AxisSpec a, float2* tab) {
    const int L = a.L, N = a.N;
    for (int m = blockIdx.x * blockDim.x + threadIdx.x; m < L; m += gridDim.x * blockDim.x) {
        double s, c;
        sincospi(2.0 * m / L, &s, &c);
        tab[m] = make_float2((float)c, (float)-s);
        sincospi((double)m / L, &s, &c);
        tab[kMaxFft + m] = make_float2((float)c, (float)-s);
        double kap, phase;      // kap * (dx / 2) = pi * phase
        bool nyq = false;
        if (!a.group2) {
            const int nn = m <= N ? m : m - L;
            kap = 2.0 * M_PI * nn / (L * a.dx);
            phase = (double)nn / L;
            nyq = (m == N);
        } else {
            const int nn = m < N ? m : m - L;
            kap = M_PI * (2.0 * nn + 1.0) / (L * a.dx);
            phase = (2.0 * nn + 1.0) / (2.0 * L);
        }
        sincospi(phase, &s, &c);
        // dir 0 (shift +dx/2): i kap e^{+i kap dx/2} = (-kap s, kap c)
        // dir 1 (shift -dx/2): i kap e^{-i kap dx/2} = (+kap s, kap c)
        const double im = nyq ? 0.0 : kap * c;
        tab[2 * kMaxFft + m] = make_float2((float)(-kap * s * a.scaleP / L), (float)(im * a.scaleP / L));
        tab[3 * kMaxFft + m] = make_float2((float)(kap * s * a.scaleU / L), (float)(im * a.scaleU / L));
    }
}

bool radix_plan(int L, pstd::FftPlan& P) {
    int r = L, twos = 0, threes = 0, fives = 0;
    while (r % 2 == 0) { r /= 2; ++twos; }
    while (r % 3 == 0) { r /= 3; ++threes; }
    while (r % 5 == 0) { r /= 5; ++fives; }
    if (r != 1 || L < 2) return false;
    P.L = L;
    P.npass = 0;
    int rad[64];
    int n = 0;
    while (twos >= 3) { rad[n++] = 8; twos -= 3; }
    if (twos == 2) rad[n++] = 4;
    if (twos == 1) rad[n++] = 2;
    for (int i = 0; i < threes; ++i) rad[n++] = 3;
    for (int i = 0; i < fives; ++i) rad[n++] = 5;
    if (n > pstd::kMaxPasses) return false;
    for (int i = 0; i < n; ++i) P.radix[i] = rad[i];
    P.npass = n;
    return true;
}

}  // namespace

extern "C" int pstd_step_noalloc(const pstd_desc* d, float* p, float* const* u, int64_t nsteps,
                                 void* stream) {
    if (!d || !p || !u || nsteps < 0 || d->ndim < 1 || d->ndim > 3) return PSTD_EINVAL;
    if (!(d->c0 > 0) || !(d->rho0 > 0) || !(d->dt > 0) || !std::isfinite(d->dt)) return PSTD_EINVAL;
    int64_t pshape[3] = {1, 1, 1};
    int64_t points = 1;
    double k2 = 0;
    for (int i = 0; i < d->ndim; ++i) {
        const int64_t N = d->ncells[i];
        if (!u[i] || N < 1 || !(d->dx[i] > 0)) return PSTD_EINVAL;
        for (int s = 0; s < 2; ++s) {
            const int b = d->bc[i][s];
            // valid wall types this call has no schedule for: periodic axes and
            // mid-cell right walls
            if (b == PSTD_PERIODIC || (s == 1 && (b == PSTD_NEUMANN_MID || b == PSTD_DIRICHLET_MID)))
                return PSTD_EUNSUPPORTED;
            if (b != PSTD_NEUMANN && b != PSTD_DIRICHLET) return PSTD_EINVAL;
        }
        const int64_t lo = d->bc[i][0] == PSTD_DIRICHLET ? 1 : 0;
        const int64_t hi = d->bc[i][1] == PSTD_DIRICHLET ? N - 1 : N;
        if (hi < lo) return PSTD_EINVAL;
        pshape[i] = hi - lo + 1;
        points *= pshape[i];
        const double L = N * d->dx[i];
        double kmax;
        if (d->bc[i][0] == PSTD_NEUMANN && d->bc[i][1] == PSTD_NEUMANN) kmax = M_PI * N / L;
        else if (d->bc[i][0] != d->bc[i][1]) kmax = M_PI * (N - 0.5) / L;
        else kmax = M_PI * (N - 1.0) / L;
        k2 += kmax * kmax;
    }
    if (d->c0 * d->dt * std::sqrt(k2) / 2.0 > 1.0) return PSTD_EUNSTABLE;
    // fixed capacity of the file-scope arrays
    if (points > PSTD_NOALLOC_MAX_POINTS) return PSTD_EUNSUPPORTED;
    pstd::FftPlan plans[3];
    for (int i = 0; i < d->ndim; ++i) {
        if (2 * d->ncells[i] > kMaxFft || !radix_plan((int)(2 * d->ncells[i]), plans[i]))
            return PSTD_EUNSUPPORTED;
    }

    float* acc = nullptr;
    float2* tables = nullptr;
    if (resolve_arrays(&acc, &tables) != cudaSuccess) return PSTD_ECUDA;
    cudaStream_t st = (cudaStream_t)stream;

    pstd::StepArgs args[3];
    unsigned grids[3];
    size_t smem[3];
    for (int i = 0; i < d->ndim; ++i) {
        const int N = (int)d->ncells[i], L = 2 * N;
        const int bcl = d->bc[i][0], bcr = d->bc[i][1];
        const int lo = bcl == PSTD_DIRICHLET ? 1 : 0;
        const int lp = (int)pshape[i];
        float2* tab = tables + (size_t)i * 4 * kMaxFft;
        AxisSpec spec{N, L, bcl != bcr, d->dx[i], -d->dt / d->rho0, -d->dt * d->rho0 * d->c0 * d->c0};
        k_noalloc_tables<<<(L + 255) / 256, 256, 0, st>>>(spec, tab);
        if (cudaGetLastError() != cudaSuccess) return PSTD_ECUDA;
        plans[i].tw = tab;
        for (int dir = 0; dir < 2; ++dir) {
            pstd::LineOp& op = dir == 0 ? args[i].opP : args[i].opU;
            op = pstd::LineOp{};
            op.kind = 0;
            op.N = N;
            op.R2 = 2 * N;
            op.L = L;
            op.group2 = bcl != bcr;
            op.dir = dir;
            op.in_half = dir;
            op.out_half = 1 - dir;
            op.nin = dir == 0 ? lp : N;
            op.nout = dir == 0 ? N : lp;
            op.in_lo = lo;
            op.out_lo = lo;
            op.s_right = dir == 0 ? (bcr == PSTD_NEUMANN ? 1.0f : -1.0f) : (bcr == PSTD_NEUMANN ? -1.0f : 1.0f);
            op.f = tab + (size_t)(2 + dir) * kMaxFft;
            op.shift = tab + kMaxFft;
            op.dense = nullptr;
            op.seqlen = L;
            op.fold = 1.0f;
            op.fft = plans[i];
        }
        int64_t nl = 1, inner = 1;
        for (int j = 0; j < d->ndim; ++j) {
            if (j == i) continue;
            nl *= pshape[j];
            if (j > i) inner *= pshape[j];
        }
        const int rs = lp > N ? lp : N;
        int G = 16;
        while (G > 2 && pstd::cta_smem_bytes(G, L, rs) > kSmemBudget) G -= 2;
        if ((int64_t)G > nl) G = (int)nl;
        if (G < 1) G = 1;
        smem[i] = pstd::cta_smem_bytes(G, L, rs);
        if (smem[i] > 227 * 1024) return PSTD_EUNSUPPORTED;
        args[i].nlines = nl;
        args[i].inner = inner;
        args[i].G = G;
        args[i].rs = rs;
        args[i].p = p;
        args[i].u = u[i];
        args[i].acc_in = (i == d->ndim - 1) ? p : acc;
        args[i].acc_out = (i == 0) ? p : acc;
        grids[i] = (unsigned)((nl + G - 1) / G);
    }
    for (int64_t s = 0; s < nsteps; ++s) {
        for (int a = d->ndim - 1; a >= 0; --a) {
            if (pstd::launch_k_step(grids[a], smem[a], st, args[a]) != cudaSuccess) return PSTD_ECUDA;
        }
    }
    return PSTD_OK;
}
