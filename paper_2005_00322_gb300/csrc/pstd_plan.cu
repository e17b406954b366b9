// pstd_plan.cu -- host side of the C ABI declared in include/pstd.h.
//
// A plan holds, per axis, the FP64-built / FP32-stored tables of the two
// staggered derivatives (Section 3.4 with Table 1's wavenumbers and Table 2's
// transform choice, evaluated as the Fourier multiplier on the symmetric-
// periodic extension), the launch geometry of the axis pass, and one scratch
// accumulator of the pressure shape.  A leapfrog step (Eq. dtt_pstd_solution,
// n-D form of Section 4.3) launches one fused pass per axis, last axis first:
//     axis d-1:     u_{d-1} += f_P(p);  S = p + f_U(u_{d-1})
//     axis 1..d-2:  u_a     += f_P(p);  S = S + f_U(u_a)
//     axis 0:       u_0     += f_P(p);  p = S + f_U(u_0)
// (1-D: u += f_P(p); p = p + f_U(u)).  Every pass reads p^n, which no pass of
// the same step overwrites before the last one, and the last pass writes each
// p line only after the CTA that owns it has read it.
#include <cuda_runtime.h>

#include <cmath>
#include <complex>
#include <cstdio>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "../../include/pstd.h"
#include "pstd_cta.cuh"
#include "pstd_energy.h"
#include "pstd_gemm.h"
#include "pstd_internal.h"
#include "pstd_tc16.h"
#include <cuda_fp16.h>
#include "pstd_wkernels.cuh"

namespace pstd {
// Launchers and attribute setup, defined with the kernels (pstd_kernels.cu).
cudaError_t launch_k_step(unsigned grid, size_t smem, cudaStream_t st, const StepArgs& a);
cudaError_t launch_k_grad(unsigned grid, size_t smem, cudaStream_t st, const GradArgs& a);
cudaError_t set_max_smem(int bytes);
cudaError_t launch_k_step_persist(unsigned grid, size_t smem, cudaStream_t st, const StepPersistArgs& a,
                                  const GridSync& sync);
cudaError_t k_step_persist_blocks(size_t smem, int* blocks);
cudaError_t launch_k_axpby(int64_t n, float alpha, const float* x, float beta, float* y, cudaStream_t st);
// register-FFT passes, one dispatcher per translation unit (pstd_wkernels_*.cu)
cudaError_t wsmall_step(int L, int V, bool s, const WLaunch& g, cudaStream_t st, const WStep& a);
cudaError_t wsmall_grad(int L, int V, bool s, const WLaunch& g, cudaStream_t st, const WGrad& a);
cudaError_t wsmall_smem(int L, int V, int bytes);
bool wsmall_twiddles(int L, int V, std::vector<float2>& out);
cudaError_t wsmall_persist(int L, int V, const WLaunch& g, cudaStream_t st, const PersistArgs& a);
cudaError_t wsmall_persist_blocks(int L, int V, int threads, size_t smem, int* blocks);
cudaError_t w64_step(int L, int V, bool s, const WLaunch& g, cudaStream_t st, const WStep& a);
cudaError_t w64_grad(int L, int V, bool s, const WLaunch& g, cudaStream_t st, const WGrad& a);
cudaError_t w64_smem(int L, int V, int bytes);
bool w64_twiddles(int L, int V, std::vector<float2>& out);
cudaError_t w64_persist(int L, int V, const WLaunch& g, cudaStream_t st, const PersistArgs& a);
cudaError_t w64_persist_blocks(int L, int V, int threads, size_t smem, int* blocks);
cudaError_t w1024t_step(int L, int V, bool s, const WLaunch& g, cudaStream_t st, const WStep& a);
cudaError_t w1024t_grad(int L, int V, bool s, const WLaunch& g, cudaStream_t st, const WGrad& a);
cudaError_t w1024t_smem(int L, int V, int bytes);
bool w1024t_twiddles(int L, int V, std::vector<float2>& out);
cudaError_t w1024t_persist(int L, int V, const WLaunch& g, cudaStream_t st, const PersistArgs& a);
cudaError_t w1024t_persist_blocks(int L, int V, int threads, size_t smem, int* blocks);
cudaError_t w256_step(int L, int V, bool s, const WLaunch& g, cudaStream_t st, const WStep& a);
cudaError_t w256_grad(int L, int V, bool s, const WLaunch& g, cudaStream_t st, const WGrad& a);
cudaError_t w256_smem(int L, int V, int bytes);
bool w256_twiddles(int L, int V, std::vector<float2>& out);
cudaError_t w256_persist(int L, int V, const WLaunch& g, cudaStream_t st, const PersistArgs& a);
cudaError_t w256_persist_blocks(int L, int V, int threads, size_t smem, int* blocks);
cudaError_t w512_step(int L, int V, bool s, const WLaunch& g, cudaStream_t st, const WStep& a);
cudaError_t w512_grad(int L, int V, bool s, const WLaunch& g, cudaStream_t st, const WGrad& a);
cudaError_t w512_smem(int L, int V, int bytes);
bool w512_twiddles(int L, int V, std::vector<float2>& out);
cudaError_t w512_persist(int L, int V, const WLaunch& g, cudaStream_t st, const PersistArgs& a);
cudaError_t w512_persist_blocks(int L, int V, int threads, size_t smem, int* blocks);
cudaError_t w768_step(int L, int V, bool s, const WLaunch& g, cudaStream_t st, const WStep& a);
cudaError_t w768_grad(int L, int V, bool s, const WLaunch& g, cudaStream_t st, const WGrad& a);
cudaError_t w768_smem(int L, int V, int bytes);
bool w768_twiddles(int L, int V, std::vector<float2>& out);
cudaError_t w768_persist(int L, int V, const WLaunch& g, cudaStream_t st, const PersistArgs& a);
cudaError_t w768_persist_blocks(int L, int V, int threads, size_t smem, int* blocks);
cudaError_t w1024_step(int L, int V, bool s, const WLaunch& g, cudaStream_t st, const WStep& a);
cudaError_t w1024_grad(int L, int V, bool s, const WLaunch& g, cudaStream_t st, const WGrad& a);
cudaError_t w1024_smem(int L, int V, int bytes);
bool w1024_twiddles(int L, int V, std::vector<float2>& out);
cudaError_t w1024_persist(int L, int V, const WLaunch& g, cudaStream_t st, const PersistArgs& a);
cudaError_t w1024_persist_blocks(int L, int V, int threads, size_t smem, int* blocks);
}  // namespace pstd

using pstd::FftPlan;
using pstd::GradArgs;
using pstd::LineOp;
using pstd::StepArgs;
using pstd::WAxis;
using pstd::WGrad;
using pstd::WLaunch;
using pstd::WStep;
using pstd::PersistArgs;
using pstd::GridSync;
using pstd::StepPersistArgs;

namespace {

thread_local std::string g_cuda_err;

constexpr int kDenseMaxN = 64;       // dense operator below this, convolution route above
constexpr int kConvMaxFft = 8192;    // largest power-of-two FFT of the convolution route
constexpr int kGraphSteps = 32;
constexpr int kGraphCache = 4;
constexpr size_t kSmemBudget = 100 * 1024;

enum { OP_GRAD_P = 0, OP_GRAD_U = 1, OP_STEP_P = 2, OP_STEP_U = 3, OP_INIT_P = 4, OP_COUNT = 5 };

struct Axis {
    int N = 0, L = 0, group2 = 0, kind = 0, M2 = 0, periodic = 0;
    int lp = 0, lo = 0;               // stored pressure length, first stored node
    int mid = 0;                      // right wall at mid-cell, x = (N - 1/2) dx (types V-VIII)
    int R2 = 0;                       // twice the right wall's position in cells (2N or 2N - 1)
    int nu = 0;                       // stored velocity half-nodes (N, or N - 1 next to a
                                      // Neumann mid-cell wall)
    double dx = 0;
    int bcl = 0, bcr = 0;
    FftPlan fft{};
    float2* d_tw = nullptr;
    float2* d_shift = nullptr;
    float2* d_f[OP_COUNT] = {};
    float* d_dense[OP_COUNT] = {};
    LineOp op[OP_COUNT];
    int64_t nlines = 0, inner = 1;
    int G = 2, rs = 1;
    size_t smem = 0;
    // register-FFT passes (wl > 0: lanes per sequence)
    int wl = 0, wv = 0;
    bool strided = false;
    float2* d_wtw = nullptr;
    float2* d_sym = nullptr;          // velocity-spectrum symmetry factors (WAxis::sym)
    float2* d_fUL = nullptr;          // L x the u -> p step coefficients (spectral velocity)
    float* d_ph = nullptr;            // phantom partner lines of unpaired velocity lines
    float* d_tc = nullptr;            // tensor-core split form: D1 hi | D1 lo | D2 hi | D2 lo
    // plain differentiation and staggered interpolation (pstd_apply), built on
    // first use: [op][input field kind]
    LineOp xop[2][4];
    int xok[2][4] = {};
    int xG[2][4] = {};
    size_t xsmem[2][4] = {};
    float2* d_xf[2][4] = {};
    float* d_xdense[2][4] = {};
    // second-order form (pstd_run2), built on first use: (c0 dt)^2 D_u D_p
    // on the pressure nodes
    int ok2 = 0;
    LineOp op2{};
    float2* d_f2 = nullptr;
    float* d_dense2 = nullptr;
    WAxis wax{};
    WLaunch wgeo{};
    // BF16 three-way split form on tcgen05: the two operators' BF16 slices
    // (D1: N x lp, D2: lp x N) and their TMA tensor maps
    uint16_t* d_tc16[2] = {nullptr, nullptr};
    int tc16_MT[2] = {0, 0}, tc16_KC[2] = {0, 0};
    // the padded fields along this axis: X maps of p and u_a, Y (and Cin)
    // maps of u_a, p and the accumulator; line tiles
    CUtensorMap tc16_x[2], tc16_y[3];
    int64_t tc16_tiles = 0, tc16_tpo = 0;
    // split-precision dense form
    uint4* d_gemm = nullptr;          // A1h | A1l | A2h | A2l fragments
    pstd::GemmAxis gax{};
    unsigned ggrid = 0;
    size_t gsmem = 0;
};

// register-FFT dispatch by length and schedule variant: the translation unit
// that instantiates (L, V)
#define PSTD_WBY_LENGTH(CALL)                      \
    switch (L) {                                   \
        case 1024:                                 \
            if (V == 0 || V == 2) return pstd::w1024t_##CALL; \
            return pstd::w1024_##CALL;             \
        case 768: case 384: return pstd::w768_##CALL; \
        case 512: return pstd::w512_##CALL;        \
        case 256: return pstd::w256_##CALL;        \
        case 64: case 128: case 96: case 192:      \
            return pstd::w64_##CALL;               \
        default: return pstd::wsmall_##CALL;       \
    }
cudaError_t wstep(int L, int V, bool s, const WLaunch& g, cudaStream_t st, const WStep& a) {
    PSTD_WBY_LENGTH(step(L, V, s, g, st, a))
}
cudaError_t wgrad(int L, int V, bool s, const WLaunch& g, cudaStream_t st, const WGrad& a) {
    PSTD_WBY_LENGTH(grad(L, V, s, g, st, a))
}
cudaError_t wsmem(int L, int V, int bytes) { PSTD_WBY_LENGTH(smem(L, V, bytes)) }
cudaError_t wpersist(int L, int V, const WLaunch& g, cudaStream_t st, const pstd::PersistArgs& a) {
    PSTD_WBY_LENGTH(persist(L, V, g, st, a))
}
cudaError_t wpersist_blocks(int L, int V, int threads, size_t smem, int* blocks) {
    PSTD_WBY_LENGTH(persist_blocks(L, V, threads, smem, blocks))
}
bool wtw(int L, int V, std::vector<float2>& out) { PSTD_WBY_LENGTH(twiddles(L, V, out)) }
#undef PSTD_WBY_LENGTH

struct GraphEntry {
    int kind = 0;                     // 0: leapfrog steps (u: velocities), 1: second-order steps (u[0]: q)
    float* p = nullptr;
    float* u[3] = {nullptr, nullptr, nullptr};
    cudaGraphExec_t exec = nullptr;
    int steps = 0;
    int64_t launches = 0;
    uint64_t stamp = 0;
};

int cuda_fail(cudaError_t e, const char* what) {
    g_cuda_err = std::string(what) + ": " + cudaGetErrorString(e);
    return PSTD_ECUDA;
}

#define CK(call)                                         \
    do {                                                 \
        cudaError_t _e = (call);                         \
        if (_e != cudaSuccess) return cuda_fail(_e, #call); \
    } while (0)

// Radix schedule of L over {8, 4, 2, 3, 5}; false if L has another factor.
bool radix_schedule(int L, FftPlan& P) {
    int r = L;
    P.L = L;
    P.npass = 0;
    int twos = 0;
    while (r % 2 == 0) { r /= 2; ++twos; }
    int threes = 0;
    while (r % 3 == 0) { r /= 3; ++threes; }
    int fives = 0;
    while (r % 5 == 0) { r /= 5; ++fives; }
    if (r != 1 || L < 2) return false;
    auto push = [&](int R) {
        if (P.npass >= pstd::kMaxPasses) return false;
        P.radix[P.npass++] = R;
        return true;
    };
    while (twos >= 3) { if (!push(8)) return false; twos -= 3; }
    if (twos == 2) { if (!push(4)) return false; }
    if (twos == 1) { if (!push(2)) return false; }
    for (int i = 0; i < threes; ++i) if (!push(3)) return false;
    for (int i = 0; i < fives; ++i) if (!push(5)) return false;
    return true;
}

}  // namespace

struct pstd_plan_s {
    pstd_desc desc{};
    pstd_plan_opts opts{{-1, -1, -1}, {-1, -1, -1}, 0, 0, 0, 0};
    unsigned* d_sync = nullptr;       // grid barrier: count, generation, status
    int nsm = 152;                    // SMs of the plan's device (queried at plan time)
    int persist_ok = 0;
    WLaunch pgeo{};
    cudaStream_t stream = nullptr;
    int ndim = 0;
    int64_t shape[4][3] = {};
    Axis ax[3];
    float* d_S = nullptr;
    double* d_energy = nullptr;       // pstd_energy's FP64 partial sums, on first use
    // BF16 split form: plan-owned copies of p, u_0.. and the accumulator with
    // the last dimension padded to a multiple of 4 floats (TMA strides)
    float* d_pad[4] = {};
    float* d_Spad = nullptr;
    int64_t pitch[4] = {};
    int64_t last_launches = 0;
    GraphEntry graphs[kGraphCache];
    uint64_t stamp = 0;
};

namespace {

// Folded coefficient f_n of the extension's Fourier multiplier (Table 1
// wavenumbers; shift +dx/2 for p -> u, -dx/2 for u -> p), including 1/M.
// Wavenumber of bin n of the extension's FFT and whether it is the Nyquist
// bin (the bin that pairs with itself, whose value is real for real lines).
// Period L = M: 2N (groups I, II), 2N - 1 (groups III, IV: odd), N (periodic).
// Periodic groups: k = 2 pi n / (L dx); antiperiodic groups, pre-twiddled:
// k = pi (2n + 1) / (L dx); n above the middle stands for n - L.
double wavenumber(const Axis& a, int n, bool& nyquist) {
    const int L = a.L;
    if (a.periodic) {
        // n in [-N/2, N/2 - 1] (even N), [-(N-1)/2, (N-1)/2] (odd)
        const int nn = n < (L + 1) / 2 ? n : n - L;
        nyquist = (L % 2 == 0 && n == L / 2);
        return 2.0 * M_PI * nn / (L * a.dx);
    }
    if (!a.group2) {
        const int nn = 2 * n <= L ? n : n - L;
        nyquist = 2 * n == L;
        return 2.0 * M_PI * nn / (L * a.dx);
    }
    const int nn = 2 * n + 1 <= L ? n : n - L;
    nyquist = 2 * n + 1 == L;
    return M_PI * (2.0 * nn + 1.0) / (L * a.dx);
}

std::complex<double> coeff(const Axis& a, int n, int dir, double scale) {
    const int L = a.L;
    bool nyquist = false;
    const double kap = wavenumber(a, n, nyquist);
    const double s = dir == 0 ? 0.5 * a.dx : -0.5 * a.dx;
    // i kap exp(i kap s) = (-kap sin(kap s), kap cos(kap s))
    double re = -kap * std::sin(kap * s);
    double im = nyquist ? 0.0 : kap * std::cos(kap * s);
    return std::complex<double>(re, im) * (scale / L);
}

template <class T>
int upload(const std::vector<T>& h, T** d) {
    CK(cudaMalloc((void**)d, h.size() * sizeof(T)));
    CK(cudaMemcpy(*d, h.data(), h.size() * sizeof(T), cudaMemcpyHostToDevice));
    return PSTD_OK;
}

// Dense operator (rows: stored outputs, cols: stored inputs) of the same
// multiplier, FP64, for axes with no FFT schedule.
std::vector<double> dense_operator64(const Axis& a, int dir, double scale) {
    const int L = a.L;
    std::vector<std::complex<double>> K(L);
    for (int d = 0; d < L; ++d) {
        std::complex<double> acc = 0;
        for (int n = 0; n < L; ++n) {
            const double ang = 2.0 * M_PI * (double)((int64_t)d * n % L) / L;
            acc += coeff(a, n, dir, scale) * std::complex<double>(std::cos(ang), std::sin(ang));
        }
        K[d] = acc;
    }
    const int nin = dir == 0 ? a.lp : a.nu;
    const int nout = dir == 0 ? a.nu : a.lp;
    const double sR = dir == 0 ? (a.bcr == PSTD_NEUMANN ? 1.0 : -1.0)
                               : (a.bcr == PSTD_NEUMANN ? -1.0 : 1.0);
    std::vector<double> D((size_t)nout * nin);
    for (int i = 0; i < nout; ++i) {
        const int pos = dir == 0 ? i : i + a.lo;
        for (int j = 0; j < nin; ++j) {
            // positions of stored input j in one period of the extension: itself
            // and its reflection about the right wall (R2 - q, R2 - 1 - m) unless
            // it lies on a wall
            int src[2];
            double sg[2];
            int nimg = 0;
            if (a.periodic) {
                src[nimg] = j; sg[nimg++] = 1.0;
            } else if (dir == 0) {
                const int q = j + a.lo;
                src[nimg] = q; sg[nimg++] = 1.0;
                if (q > 0 && 2 * q < a.R2) { src[nimg] = a.R2 - q; sg[nimg++] = sR; }
            } else {
                src[nimg] = j; sg[nimg++] = 1.0;
                if (2 * j + 1 < a.R2) { src[nimg] = a.R2 - 1 - j; sg[nimg++] = sR; }
            }
            double v = 0;
            for (int m = 0; m < nimg; ++m) {
                const int delta = pos - src[m];
                std::complex<double> k = K[((delta % L) + L) % L];
                if (a.group2) {
                    const double ang = M_PI * delta / L;
                    k *= std::complex<double>(std::cos(ang), std::sin(ang));
                }
                v += sg[m] * k.real();
            }
            D[(size_t)i * nin + j] = v;
        }
    }
    return D;
}

std::vector<float> dense_operator(const Axis& a, int dir, double scale) {
    std::vector<double> d = dense_operator64(a, dir, scale);
    return std::vector<float>(d.begin(), d.end());
}

// Fragment-ordered hi / lo copies of D / max|D| (rows m < M, cols k < K)
// for mma m16n8k16: per (16-row tile, 16-column tile) 32 lanes x 4 words,
// FP16 with the low part stored multiplied by 2^11 (see pstd_gemm.cu).
void gemm_fragments(const std::vector<double>& D, int M, int K, std::vector<uint4>& hi,
                    std::vector<uint4>& lo, double& scale) {
    double mx = 0;
    for (double v : D) mx = std::fabs(v) > mx ? std::fabs(v) : mx;
    scale = mx > 0 ? mx : 1.0;
    const int MT = (M + 15) / 16, KT = (K + 15) / 16;
    hi.assign((size_t)MT * KT * 32, uint4{0, 0, 0, 0});
    lo.assign(hi.size(), uint4{0, 0, 0, 0});
    auto el = [&](int m, int k, bool low) -> uint16_t {
        double x = (m < M && k < K) ? D[(size_t)m * K + k] / scale : 0.0;
        const __half h = __float2half_rn((float)x);
        __half r = h;
        if (low) r = __float2half_rn((float)((x - (double)__half2float(h)) * 2048.0));
        uint16_t bits;
        std::memcpy(&bits, &r, 2);
        return bits;
    };
    auto pack = [&](int m, int k, bool low) -> unsigned {
        return (unsigned)el(m, k, low) | ((unsigned)el(m, k + 1, low) << 16);
    };
    for (int mt = 0; mt < MT; ++mt)
        for (int kt = 0; kt < KT; ++kt)
            for (int lane = 0; lane < 32; ++lane) {
                const int g = lane >> 2, t = lane & 3;
                const int m0 = mt * 16 + g, k0 = kt * 16 + 2 * t;
                for (int part = 0; part < 2; ++part) {
                    const bool low = part == 1;
                    uint4 r;
                    r.x = pack(m0, k0, low);
                    r.y = pack(m0 + 8, k0, low);
                    r.z = pack(m0, k0 + 8, low);
                    r.w = pack(m0 + 8, k0 + 8, low);
                    (low ? lo : hi)[((size_t)mt * KT + kt) * 32 + lane] = r;
                }
            }
}

void host_fft_pow2(std::vector<std::complex<double>>& x);

// Forward DFT X_k = sum_j x_j e^{-2 pi i j k / n} (FP64, host) of any length:
// radix 2 for powers of two, otherwise decimation in time over the smallest
// prime factor p (p interleaved sub-transforms of length n / p, combined with
// the twiddles e^{-2 pi i r k / n}), down to direct sums at prime lengths.
void host_fft(std::vector<std::complex<double>>& x) {
    const size_t n = x.size();
    if (n <= 1) return;
    if ((n & (n - 1)) == 0) {
        host_fft_pow2(x);
        return;
    }
    size_t p = 2;
    while (n % p) ++p;
    auto unit = [n](size_t e) {   // e^{-2 pi i e / n}, e reduced mod n
        const double ang = -2.0 * M_PI * (double)(e % n) / (double)n;
        return std::complex<double>(std::cos(ang), std::sin(ang));
    };
    std::vector<std::complex<double>> y(n);
    if (p == n) {
        for (size_t k = 0; k < n; ++k) {
            std::complex<double> acc = 0;
            for (size_t j = 0; j < n; ++j) acc += x[j] * unit(j * k);
            y[k] = acc;
        }
        x.swap(y);
        return;
    }
    const size_t m = n / p;
    std::vector<std::vector<std::complex<double>>> sub(p, std::vector<std::complex<double>>(m));
    for (size_t r = 0; r < p; ++r) {
        for (size_t j = 0; j < m; ++j) sub[r][j] = x[j * p + r];
        host_fft(sub[r]);
    }
    for (size_t k = 0; k < n; ++k) {
        std::complex<double> acc = 0;
        for (size_t r = 0; r < p; ++r) acc += sub[r][k % m] * unit(r * k);
        y[k] = acc;
    }
    x.swap(y);
}

// In-place radix-2 FFT of a power-of-two length (FP64, host), same sign.
void host_fft_pow2(std::vector<std::complex<double>>& x) {
    const size_t n = x.size();
    for (size_t i = 1, j = 0; i < n; ++i) {
        size_t bit = n >> 1;
        for (; j & bit; bit >>= 1) j ^= bit;
        j ^= bit;
        if (i < j) std::swap(x[i], x[j]);
    }
    for (size_t len = 2; len <= n; len <<= 1) {
        const double ang = -2.0 * M_PI / (double)len;
        for (size_t i = 0; i < n; i += len)
            for (size_t k = 0; k < len / 2; ++k) {
                const std::complex<double> w(std::cos(ang * k), std::sin(ang * k));
                const std::complex<double> u = x[i + k], v = x[i + k + len / 2] * w;
                x[i + k] = u + v;
                x[i + k + len / 2] = u - v;
            }
    }
}

// Convolution-route table of one direction at unit scale (see LineOp kind 2):
// H = FFT_M2(h~) / M2 with h~[d] = sum_n f_n e^{2 pi i d n / L} (times
// e^{i pi d / L} for group II), d < L, zero-padded to M2.
std::vector<std::complex<double>> conv_table(const Axis& a, int dir) {
    const int L = a.L;
    std::vector<std::complex<double>> f(L), wl(L), h(a.M2, 0.0);
    for (int n = 0; n < L; ++n) {
        f[n] = coeff(a, n, dir, 1.0);
        wl[n] = std::complex<double>(std::cos(2.0 * M_PI * n / L), std::sin(2.0 * M_PI * n / L));
    }
    for (int d = 0; d < L; ++d) {
        std::complex<double> acc = 0;
        int64_t idx = 0;
        for (int n = 0; n < L; ++n) {
            acc += f[n] * wl[idx];
            idx += d;
            if (idx >= L) idx -= L;
        }
        if (a.group2) acc *= std::complex<double>(std::cos(M_PI * d / L), std::sin(M_PI * d / L));
        h[d] = acc;
    }
    host_fft(h);
    for (auto& x : h) x /= (double)a.M2;
    return h;
}

// ---- plain differentiation and staggered interpolation (pstd_apply) --------
// Field kinds along one axis: grid (nodes or half-nodes) and parity class
// (pressure-like: symmetric at a Neumann wall, antisymmetric at a Dirichlet
// one; velocity-like: the reverse).  A node where the field is antisymmetric
// about a wall is zero and not stored.
struct KindGeo {
    int half, lo, len;
    float sR;                 // sign of the field reflected about the right wall
};

bool kind_geo(const Axis& a, int kind, KindGeo& g) {
    const bool half = kind == PSTD_HALF_U || kind == PSTD_HALF_P;
    const bool ppar = kind == PSTD_NODES_P || kind == PSTD_HALF_P;
    g.half = half ? 1 : 0;
    if (a.periodic) {
        g.lo = 0;
        g.len = a.N;
        g.sR = 1.0f;
        return true;
    }
    const bool rightS = ppar == (a.bcr == PSTD_NEUMANN);
    const bool leftS = ppar == (a.bcl == PSTD_NEUMANN);
    g.sR = rightS ? 1.0f : -1.0f;
    if (half) {
        // half-nodes m = 0..N-1; with a mid-cell right wall m = N-1 lies on it
        g.lo = 0;
        g.len = a.mid && !rightS ? a.N - 1 : a.N;
    } else {
        // nodes up to N (wall node), or N - 1 before a mid-cell wall
        g.lo = leftS ? 0 : 1;
        g.len = (a.mid ? a.N - 1 : (rightS ? a.N : a.N - 1)) - g.lo + 1;
    }
    return g.len > 0;
}

// Output kind: differentiation keeps the grid and swaps the parity class,
// interpolation keeps the parity class and swaps the grid (Section 3.3).
int out_kind(int op, int kind) {
    static const int diff[4] = {PSTD_NODES_U, PSTD_HALF_P, PSTD_NODES_P, PSTD_HALF_U};
    static const int interp[4] = {PSTD_HALF_P, PSTD_NODES_U, PSTD_HALF_U, PSTD_NODES_P};
    return op == PSTD_OP_DIFF ? diff[kind] : interp[kind];
}

// Folded multiplier of the extension, including 1/L: (i k if `deriv`) times
// e^{i k shift}; at the Nyquist bin of an even period only its real part,
// which keeps real lines real (the bin the tables drop or pad with zero).
std::complex<double> coeff_gen(const Axis& a, int n, bool deriv, double shift) {
    const int L = a.L;
    bool nyquist = false;
    const double kap = wavenumber(a, n, nyquist);
    std::complex<double> m = std::polar(1.0, kap * shift);
    if (deriv) m *= std::complex<double>(0.0, kap);
    if (nyquist) m = m.real();
    return m / (double)L;
}

// The convolution-route table of a multiplier f (as conv_table).
std::vector<std::complex<double>> conv_table_of(const Axis& a, const std::vector<std::complex<double>>& f) {
    const int L = a.L;
    std::vector<std::complex<double>> wl(L), h(a.M2, 0.0);
    for (int n = 0; n < L; ++n)
        wl[n] = std::complex<double>(std::cos(2.0 * M_PI * n / L), std::sin(2.0 * M_PI * n / L));
    for (int d = 0; d < L; ++d) {
        std::complex<double> acc = 0;
        int64_t idx = 0;
        for (int n = 0; n < L; ++n) {
            acc += f[n] * wl[idx];
            idx += d;
            if (idx >= L) idx -= L;
        }
        if (a.group2) acc *= std::complex<double>(std::cos(M_PI * d / L), std::sin(M_PI * d / L));
        h[d] = acc;
    }
    host_fft(h);
    for (auto& x : h) x /= (double)a.M2;
    return h;
}

// Dense operator (rows: stored outputs, cols: stored inputs) of a multiplier
// f between two field kinds (as dense_operator64).
std::vector<float> dense_operator_of(const Axis& a, const std::vector<std::complex<double>>& f, const KindGeo& gi,
                                     const KindGeo& go) {
    const int L = a.L;
    std::vector<std::complex<double>> K(L);
    for (int d = 0; d < L; ++d) {
        std::complex<double> acc = 0;
        for (int n = 0; n < L; ++n) {
            const double ang = 2.0 * M_PI * (double)((int64_t)d * n % L) / L;
            acc += f[n] * std::complex<double>(std::cos(ang), std::sin(ang));
        }
        K[d] = acc;
    }
    std::vector<float> D((size_t)go.len * gi.len);
    for (int i = 0; i < go.len; ++i) {
        const int pos = go.half ? i : i + go.lo;
        for (int j = 0; j < gi.len; ++j) {
            int src[2];
            double sg[2];
            int nimg = 0;
            if (a.periodic) {
                src[nimg] = j; sg[nimg++] = 1.0;
            } else if (!gi.half) {
                const int q = j + gi.lo;
                src[nimg] = q; sg[nimg++] = 1.0;
                if (q > 0 && 2 * q < a.R2) { src[nimg] = a.R2 - q; sg[nimg++] = gi.sR; }
            } else {
                src[nimg] = j; sg[nimg++] = 1.0;
                if (2 * j + 1 < a.R2) { src[nimg] = a.R2 - 1 - j; sg[nimg++] = gi.sR; }
            }
            double v = 0;
            for (int m = 0; m < nimg; ++m) {
                const int delta = pos - src[m];
                std::complex<double> k = K[((delta % L) + L) % L];
                if (a.group2) k *= std::complex<double>(std::cos(M_PI * delta / L), std::sin(M_PI * delta / L));
                v += sg[m] * k.real();
            }
            D[(size_t)i * gi.len + j] = (float)v;
        }
    }
    return D;
}

// Build (once) the line operation `op` on input kind `kind` of axis `i`.
int build_xop(pstd_plan_s* P, int i, int op, int kind) {
    Axis& a = P->ax[i];
    if (a.xok[op][kind]) return PSTD_OK;
    KindGeo gi, go;
    const int ok = out_kind(op, kind);
    if (!kind_geo(a, kind, gi) || !kind_geo(a, ok, go)) return PSTD_EINVAL;
    const bool deriv = op == PSTD_OP_DIFF;
    const double shift = gi.half == go.half ? 0.0 : (gi.half ? -0.5 * a.dx : 0.5 * a.dx);
    std::vector<std::complex<double>> f(a.L);
    for (int n = 0; n < a.L; ++n) f[n] = coeff_gen(a, n, deriv, shift);
    LineOp o = a.op[OP_GRAD_P];     // route, FFT plan, shifts, sequence length
    o.dir = gi.half;
    o.in_half = gi.half;
    o.out_half = go.half;
    o.nin = gi.len;
    o.nout = go.len;
    o.in_lo = gi.lo;
    o.out_lo = go.lo;
    o.s_right = gi.sR;
    o.f = nullptr;
    o.dense = nullptr;
    int rc;
    if (a.kind == 0) {
        std::vector<float2> t(a.L);
        for (int n = 0; n < a.L; ++n) t[n] = make_float2((float)f[n].real(), (float)f[n].imag());
        if ((rc = upload(t, &a.d_xf[op][kind])) != PSTD_OK) return rc;
        o.f = a.d_xf[op][kind];
    } else if (a.kind == 2) {
        const std::vector<std::complex<double>> h = conv_table_of(a, f);
        std::vector<float2> t(a.M2);
        for (int n = 0; n < a.M2; ++n) t[n] = make_float2((float)h[n].real(), (float)h[n].imag());
        if ((rc = upload(t, &a.d_xf[op][kind])) != PSTD_OK) return rc;
        o.f = a.d_xf[op][kind];
    } else {
        const std::vector<float> D = dense_operator_of(a, f, gi, go);
        if ((rc = upload(D, &a.d_xdense[op][kind])) != PSTD_OK) return rc;
        o.dense = a.d_xdense[op][kind];
    }
    int G = 16;
    while (G > 1 && pstd::cta_smem_bytes(G, o.seqlen, gi.len) > kSmemBudget) --G;
    const size_t bytes = pstd::cta_smem_bytes(G, o.seqlen, gi.len);
    if (bytes > 227 * 1024) return PSTD_EUNSUPPORTED;
    CK(pstd::set_max_smem((int)bytes));
    a.xop[op][kind] = o;
    a.xG[op][kind] = G;
    a.xsmem[op][kind] = bytes;
    a.xok[op][kind] = 1;
    return PSTD_OK;
}

// ---- second-order pressure-only form (pstd_run2) ----------------------------
// Eliminating u from the leapfrog gives p^{n+1} = 2 p^n - p^{n-1}
// + (c0 dt)^2 sum_a D_{u,a} D_{p,a} p^n.  On the extension D_u D_p is the
// product of the two staggered multipliers, -kappa^2 (the half-cell shifts
// cancel, and at the Nyquist bin the real parts multiply to the same value),
// so each axis needs one real table on the pressure nodes.
int build_order2(pstd_plan_s* P, int i) {
    Axis& a = P->ax[i];
    if (a.ok2) return PSTD_OK;
    const pstd_desc& d = P->desc;
    const double s2 = (d.c0 * d.dt) * (d.c0 * d.dt);
    std::vector<std::complex<double>> f(a.L);
    for (int n = 0; n < a.L; ++n)
        f[n] = (coeff(a, n, 0, 1.0) * coeff(a, n, 1, 1.0) * (double)a.L * s2).real();
    KindGeo g;
    if (!kind_geo(a, PSTD_NODES_P, g)) return PSTD_EINVAL;
    LineOp o = a.op[OP_GRAD_P];     // route, FFT plan, shifts, sequence length
    o.dir = 0;
    o.in_half = 0;
    o.out_half = 0;
    o.nin = g.len;
    o.nout = g.len;
    o.in_lo = g.lo;
    o.out_lo = g.lo;
    o.s_right = g.sR;
    o.f = nullptr;
    o.dense = nullptr;
    int rc;
    if (a.kind == 0 || a.kind == 2) {
        const std::vector<std::complex<double>> h = a.kind == 0 ? f : conv_table_of(a, f);
        std::vector<float2> t(h.size());
        for (size_t n = 0; n < h.size(); ++n) t[n] = make_float2((float)h[n].real(), (float)h[n].imag());
        if ((rc = upload(t, &a.d_f2)) != PSTD_OK) return rc;
        o.f = a.d_f2;
    } else {
        const std::vector<float> D = dense_operator_of(a, f, g, g);
        if ((rc = upload(D, &a.d_dense2)) != PSTD_OK) return rc;
        o.dense = a.d_dense2;
    }
    a.op2 = o;
    a.ok2 = 1;
    return PSTD_OK;
}

int build_axis(pstd_plan_s* P, int i) {
    Axis& a = P->ax[i];
    const pstd_desc& d = P->desc;
    a.N = (int)d.ncells[i];
    a.dx = d.dx[i];
    a.bcl = d.bc[i][0];
    a.bcr = d.bc[i][1];
    // a mid-cell right wall keeps its parity (Neumann / Dirichlet) in bcr
    a.mid = a.bcr == PSTD_NEUMANN_MID || a.bcr == PSTD_DIRICHLET_MID;
    if (a.mid) a.bcr = a.bcr == PSTD_NEUMANN_MID ? PSTD_NEUMANN : PSTD_DIRICHLET;
    if (a.mid && P->opts.form != 0) return PSTD_EUNSUPPORTED;
    a.periodic = a.bcl == PSTD_PERIODIC;
    // period of the extension: 2N (groups I, II), 2N - 1 (groups III, IV:
    // right wall at mid-cell) or N (periodic axis)
    a.R2 = a.mid ? 2 * a.N - 1 : 2 * a.N;
    a.L = a.periodic ? a.N : a.R2;
    a.group2 = !a.periodic && a.bcl != a.bcr;
    a.lo = a.bcl == PSTD_DIRICHLET ? 1 : 0;
    const int hi = (a.periodic || a.mid) ? a.N - 1 : (a.bcr == PSTD_DIRICHLET ? a.N - 1 : a.N);
    a.lp = hi - a.lo + 1;
    // velocity half-nodes: the one on a mid-cell wall is stored only where u
    // is symmetric about it (Dirichlet)
    a.nu = a.mid && a.bcr == PSTD_NEUMANN ? a.N - 1 : a.N;
    const bool fft_ok = radix_schedule(a.L, a.fft);
    a.kind = fft_ok ? 0 : (a.N <= kDenseMaxN ? 1 : 2);
    if (a.kind == 2) {
        // The linear convolution needs a circular length M2 >= 2L - 1.  Of the
        // lengths with an FFT schedule (2^a 3^b 5^c) up to the next power of
        // two, take the one with the least shared-memory traffic in the
        // Stockham passes, M2 x passes (the power of two on a tie).
        int pow2 = 1;
        while (pow2 < 2 * a.L - 1) pow2 *= 2;
        int M2 = 0;
        int64_t best = 0;
        pstd::FftPlan cand{};
        for (int m = pow2; m >= 2 * a.L - 1; --m) {
            if (m > kConvMaxFft || !radix_schedule(m, cand)) continue;
            const int64_t cost = (int64_t)m * cand.npass;
            if (M2 == 0 || cost < best) {
                M2 = m;
                best = cost;
            }
        }
        if (M2 == 0 || !radix_schedule(M2, a.fft)) return PSTD_EUNSUPPORTED;
        a.M2 = M2;
    }

    // twiddles and group-II shifts, FP64 -> FP32 once
    const int FL = a.kind == 2 ? a.M2 : a.L;   // FFT length of the route
    std::vector<float2> tw(FL), sh(a.L);
    for (int m = 0; m < FL; ++m) {
        const double ang = 2.0 * M_PI * m / FL;
        tw[m] = make_float2((float)std::cos(ang), (float)-std::sin(ang));
    }
    for (int m = 0; m < a.L; ++m) {
        const double ang2 = M_PI * m / a.L;
        sh[m] = make_float2((float)std::cos(ang2), (float)-std::sin(ang2));
    }
    int rc;
    if ((rc = upload(tw, &a.d_tw)) != PSTD_OK) return rc;
    if ((rc = upload(sh, &a.d_shift)) != PSTD_OK) return rc;
    a.fft.tw = a.d_tw;

    const double scales[OP_COUNT] = {1.0, 1.0, -d.dt / d.rho0, -d.dt * d.rho0 * d.c0 * d.c0,
                                     d.dt / (2.0 * d.rho0)};
    const int dirs[OP_COUNT] = {0, 1, 0, 1, 0};
    std::vector<std::complex<double>> conv[2];
    if (a.kind == 2) {
        conv[0] = conv_table(a, 0);
        conv[1] = conv_table(a, 1);
    }
    for (int o = 0; o < OP_COUNT; ++o) {
        const int dir = dirs[o];
        LineOp& op = a.op[o];
        std::memset(&op, 0, sizeof(op));
        op.kind = a.kind;
        op.N = a.N;
        op.R2 = a.R2;
        op.L = a.L;
        op.group2 = a.group2;
        op.dir = dir;
        op.in_half = dir;
        op.out_half = 1 - dir;
        op.nin = dir == 0 ? a.lp : a.nu;
        op.nout = dir == 0 ? a.nu : a.lp;
        op.in_lo = a.lo;
        op.out_lo = a.lo;
        op.s_right = dir == 0 ? (a.bcr == PSTD_NEUMANN ? 1.0f : -1.0f)
                              : (a.bcr == PSTD_NEUMANN ? -1.0f : 1.0f);
        op.shift = a.d_shift;
        op.fft = a.fft;
        op.seqlen = FL;
        op.fold = a.group2 ? -1.0f : 1.0f;
        if (a.kind == 2) {
            std::vector<float2> H(a.M2);
            for (int n = 0; n < a.M2; ++n) {
                const std::complex<double> c = conv[dir][n] * scales[o];
                H[n] = make_float2((float)c.real(), (float)c.imag());
            }
            if ((rc = upload(H, &a.d_f[o])) != PSTD_OK) return rc;
            op.f = a.d_f[o];
        } else if (a.kind == 0) {
            std::vector<float2> f(a.L);
            for (int n = 0; n < a.L; ++n) {
                std::complex<double> c = coeff(a, n, dir, scales[o]);
                f[n] = make_float2((float)c.real(), (float)c.imag());
            }
            if ((rc = upload(f, &a.d_f[o])) != PSTD_OK) return rc;
            op.f = a.d_f[o];
        } else {
            std::vector<float> D = dense_operator(a, dir, scales[o]);
            if ((rc = upload(D, &a.d_dense[o])) != PSTD_OK) return rc;
            op.dense = a.d_dense[o];
        }
    }

    // lines of this axis: extents of p on the other axes
    int64_t nl = 1, inner = 1;
    for (int j = 0; j < P->ndim; ++j) {
        if (j == i) continue;
        nl *= P->shape[0][j];
        if (j > i) inner *= P->shape[0][j];
    }
    a.nlines = nl;
    a.inner = inner;
    a.rs = a.lp > a.nu ? a.lp : a.nu;
    int G = 16;
    while (G > 2 && pstd::cta_smem_bytes(G, FL, a.rs) > kSmemBudget) G -= 2;
    if ((int64_t)G > nl) G = (int)nl;
    if (G < 1) G = 1;
    a.G = G;
    a.smem = pstd::cta_smem_bytes(G, FL, a.rs);
    if (a.smem > 227 * 1024) return PSTD_EUNSUPPORTED;

    // register-FFT passes where a schedule exists.  Measured on GB300 (512^2,
    // 256^3, 384^3): the latency schedules (8 or 12 elements per lane) beat
    // the throughput ones wherever they exist, with 2 line pairs per CTA once
    // the axis has enough lines to keep 2 CTAs per SM busy.
    int T = pstd::wlanes(a.L);
    int V = 0;
    int os = P->opts.seqs_per_cta[i];
    const int ov = P->opts.variant[i];
    // schedules 3, 4 and 5 are compiled for walled axes, L = 2 N (their
    // passes fix N = L / 2)
    if (ov == 5) {
        if (pstd::wlanes_v5(a.L) == 0 || a.periodic) return PSTD_EINVAL;
        V = 5;
        T = pstd::wlanes_v5(a.L);
    } else if (ov == 4) {
        if (pstd::wlanes_v4(a.L) == 0 || a.periodic) return PSTD_EINVAL;
        V = 4;
        T = pstd::wlanes_v4(a.L);
    } else if (ov == 3) {
        if (pstd::wlanes_v3(a.L) == 0 || a.periodic) return PSTD_EINVAL;
        V = 3;
        T = pstd::wlanes_v3(a.L);
    } else if (ov == 2) {
        if (pstd::wlanes_v2(a.L) == 0) return PSTD_EINVAL;
        V = 2;
        T = pstd::wlanes_v2(a.L);
    } else if (ov == 1 || (ov < 0 && pstd::wlanes_latency(a.L) > 0)) {
        if (pstd::wlanes_latency(a.L) == 0) return PSTD_EINVAL;
        V = 1;
        T = pstd::wlanes_latency(a.L);
    }
    // length-512/1024 axes with few lines (the 2-D sizes): 128 / 256 lanes of
    // 4 elements shorten each lane's dependent chain; measured 13.7 -> 12.2 us
    // per 512^2 step and 14.2 -> 9.3 us per 256^2 step (with many lines, as
    // in 256^3, the 8-element schedule stays faster: 0.69 vs 0.94 ms)
    const int64_t nsm = P->nsm;
    if (ov < 0 && V == 1 && !a.periodic && pstd::wlanes_v3(a.L) > 0 && (a.nlines + 1) / 2 < 2 * 2 * nsm) {
        V = 3;
        T = pstd::wlanes_v3(a.L);
    }
    // many lines (the 3-D sizes), walled axes: the latency radices with the
    // tables read from memory instead of registers (V=5: global through L1,
    // 64 registers; V=4 at 768: shared memory) and N = L / 2 fixed at compile
    // time; measured on 256^3 0.660 (V=1) -> 0.572 (V=4) -> 0.482 ms per step
    // (V=5, 4 line pairs per CTA on strided axes, 1 on the contiguous one)
    if (ov < 0 && V == 1 && !a.periodic && pstd::wlanes_v4(a.L) > 0 && (a.nlines + 1) / 2 >= 4 * 2 * nsm) {
        V = pstd::wlanes_v5(a.L) > 0 ? 5 : 4;
        T = V == 5 ? pstd::wlanes_v5(a.L) : pstd::wlanes_v4(a.L);
    }
    if (os == 0 || os > 256 || (os > 0 && (os & (os - 1)))) return PSTD_EINVAL;
    const bool auto_os = os < 0;
    if (os < 0 && V >= 1 && T <= 128 && (a.nlines + 1) / 2 >= 2 * 2 * nsm) os = 2;
    // strided axes stage tiles of 2 os lines: 4 sequences make each staged
    // run 8 words (one 32-byte sector); measured 0.815 -> 0.768 ms per 256^3
    // step.  The shared-table schedule takes 4 on contiguous axes too, the
    // global-table one 1 (64-thread CTAs, 16 per SM).  Not
    // for the persistent run, whose axes share one CTA size.
    if (auto_os && os == 2 && !P->opts.persistent && (inner > 1 || V >= 4) && T <= 64 &&
        (a.nlines + 1) / 2 >= 4 * 2 * nsm)
        os = inner == 1 && V == 5 ? 1 : 4;
    if (a.kind == 0 && T > 0) {
        std::vector<float2> wt;
        if (!wtw(a.L, V, wt)) return PSTD_EUNSUPPORTED;
        if ((rc = upload(wt, &a.d_wtw)) != PSTD_OK) return rc;
        // The passes keep u_a as its spectrum (bins of the FFT of its
        // extension, / L): the u -> p coefficients carry the factor L, and the
        // symmetry of the extension gives the factor on the stored bin of each
        // non-owner bin: group I  U[k] = sR_u e^{2 pi i k/L} U[L-k]  (k > N),
        // group II U[k] = sR_u e^{-i pi (L-1)/L} e^{2 pi i k/L} U[L-1-k]  (k >= N),
        // and the vanishing bin (U[0] for sR_u = -1, U[N] for sR_u = +1) gets 0.
        {
            const double sRu = a.bcr == PSTD_NEUMANN ? -1.0 : 1.0;
            std::vector<float2> sym(a.L), fUL(a.L);
            for (int k = 0; k < a.L; ++k) {
                std::complex<double> g = 1.0;
                if (!a.periodic) {
                    if (a.group2) {
                        if (k >= a.N)
                            g = sRu * std::polar(1.0, -M_PI * (a.L - 1) / a.L + 2.0 * M_PI * k / a.L);
                    } else if (k == 0) {
                        g = sRu < 0 ? 0.0 : 1.0;
                    } else if (k == a.N) {
                        g = sRu < 0 ? 1.0 : 0.0;
                    } else if (k > a.N) {
                        g = sRu * std::polar(1.0, 2.0 * M_PI * k / a.L);
                    }
                }
                sym[k] = make_float2((float)g.real(), (float)g.imag());
                const std::complex<double> c = coeff(a, k, 1, scales[OP_STEP_U]) * (double)a.L;
                fUL[k] = make_float2((float)c.real(), (float)c.imag());
            }
            if ((rc = upload(sym, &a.d_sym)) != PSTD_OK) return rc;
            if ((rc = upload(fUL, &a.d_fUL)) != PSTD_OK) return rc;
        }
        WAxis& w = a.wax;
        w.N = a.N;
        w.L = a.L;
        w.lp = a.lp;
        w.lo = a.lo;
        w.group2 = a.group2;
        w.sR_p = a.bcr == PSTD_NEUMANN ? 1.0f : -1.0f;
        w.sR_u = a.bcr == PSTD_NEUMANN ? -1.0f : 1.0f;
        w.tw = a.d_wtw;
        w.shift = a.d_shift;
        w.nlines = a.nlines;
        w.inner = a.inner;
        w.sym = a.d_sym;
        a.strided = a.inner > 1;
        // unpaired velocity lines: the last line of a contiguous axis with an
        // odd line count, or of every outer block of a strided axis whose
        // inner extent is odd (tiles hold an even number G of lines)
        {
            const int64_t nph = a.strided ? ((a.inner & 1) ? a.nlines / a.inner : 0) : (a.nlines & 1);
            if (nph > 0) {
                CK(cudaMalloc((void**)&a.d_ph, (size_t)nph * a.N * sizeof(float)));
                CK(cudaMemset(a.d_ph, 0, (size_t)nph * a.N * sizeof(float)));
            }
            w.ph = a.d_ph;
        }
        const int64_t nseq = (a.nlines + 1) / 2;
        const int64_t want = 2 * nsm;
        int threads = V >= 1 ? T : 128;
        if (os > 0) {
            threads = os * T;
            if (threads < 32 || threads > 256) return PSTD_EINVAL;
        }
        if (!a.strided) {
            while (os < 0 && threads > 32 && threads > T && (nseq * T + threads - 1) / threads < want)
                threads /= 2;
            w.seqs = threads / T;
            w.G = 2 * w.seqs;
            a.wgeo.grid = (unsigned)((nseq + w.seqs - 1) / w.seqs);
            a.wgeo.smem = (size_t)w.seqs * pstd::wseq_words(a.L) * sizeof(float2);
            a.wgeo.smem += pstd::wk::contig_stage_floats(w) * sizeof(float);  // staged slots and accumulator
            if (V != 5) a.wgeo.smem += (wt.size() + 4 * (size_t)a.L) * sizeof(float2);   // staged tables
        } else {
            const int64_t outer = a.nlines / a.inner;
            auto tiles = [&](int th) {
                const int G2 = 2 * (th / T);
                return outer * ((a.inner + G2 - 1) / G2);
            };
            while (os < 0 && threads > 32 && threads > T && tiles(threads) < want) threads /= 2;
            w.seqs = threads / T;
            w.G = 2 * w.seqs;
            a.wgeo.grid = (unsigned)tiles(threads);
            a.wgeo.smem = pstd::wk::strided_step_floats(w, pstd::wseq_words(a.L), true) * sizeof(float);
            if (V != 5) a.wgeo.smem += (wt.size() + 4 * (size_t)a.L) * sizeof(float2);   // staged tables
        }
        a.wgeo.threads = threads;
        if (a.wgeo.smem > 200 * 1024) return PSTD_EUNSUPPORTED;
        a.wl = T;
        a.wv = V;
    }

    // tensor-core split form: the dense operators of the two derivatives
    // (FP64-built, scales folded in) as TF32 hi + lo parts
    if (P->opts.form == 2) {
        if (a.N > 1024) return PSTD_EUNSUPPORTED;
        auto tf32 = [](double x) {
            float f = (float)x;
            uint32_t u;
            std::memcpy(&u, &f, 4);
            u = (u + 0x1000u) & 0xFFFFE000u;     // round to 10 mantissa bits, ties away
            std::memcpy(&f, &u, 4);
            return f;
        };
        const std::vector<double> D1 = dense_operator64(a, 0, scales[OP_STEP_P]);   // N x lp
        const std::vector<double> D2 = dense_operator64(a, 1, scales[OP_STEP_U]);   // lp x N
        std::vector<float> all;
        for (const auto* D : {&D1, &D2}) {
            std::vector<float> hi(D->size()), lo(D->size());
            for (size_t j = 0; j < D->size(); ++j) {
                hi[j] = tf32((*D)[j]);
                lo[j] = tf32((*D)[j] - (double)hi[j]);
            }
            all.insert(all.end(), hi.begin(), hi.end());
            all.insert(all.end(), lo.begin(), lo.end());
        }
        if ((rc = upload(all, &a.d_tc)) != PSTD_OK) return rc;
    }

    // BF16 three-way split form: both dense operators (FP64-built, scales
    // folded in) as exact BF16 slices with their tensor maps
    if (P->opts.form == 3) {
        if (a.N > 1024) return PSTD_EUNSUPPORTED;
        const std::vector<double> D1 = dense_operator64(a, 0, scales[OP_STEP_P]);   // nu x lp
        const std::vector<double> D2 = dense_operator64(a, 1, scales[OP_STEP_U]);   // lp x nu
        const int dims[2][2] = {{a.nu, a.lp}, {a.lp, a.nu}};
        for (int o = 0; o < 2; ++o) {
            const int r = pstd::tc16_operator(o == 0 ? D1 : D2, dims[o][0], dims[o][1], &a.d_tc16[o]);
            if (r != 0) return cuda_fail((cudaError_t)r, "BF16 operator slices");
            a.tc16_MT[o] = (dims[o][0] + 127) / 128;
            a.tc16_KC[o] = pstd::tc16_chunks(dims[o][1]);
        }
    }

    // split-precision dense form
    if (P->opts.form == 1) {
        if (a.N > 1024) return PSTD_EUNSUPPORTED;
        std::vector<uint4> h1, l1, h2, l2;
        double s1, s2;
        gemm_fragments(dense_operator64(a, 0, scales[OP_STEP_P]), a.N, a.lp, h1, l1, s1);
        gemm_fragments(dense_operator64(a, 1, scales[OP_STEP_U]), a.lp, a.N, h2, l2, s2);
        std::vector<uint4> all;
        all.insert(all.end(), h1.begin(), h1.end());
        all.insert(all.end(), l1.begin(), l1.end());
        all.insert(all.end(), h2.begin(), h2.end());
        all.insert(all.end(), l2.begin(), l2.end());
        if ((rc = upload(all, &a.d_gemm)) != PSTD_OK) return rc;
        pstd::GemmAxis& g = a.gax;
        g.N = a.N;
        g.lp = a.lp;
        g.MT1 = (a.N + 15) / 16;
        g.KT1 = (a.lp + 15) / 16;
        g.MT2 = (a.lp + 15) / 16;
        g.KT2 = (a.N + 15) / 16;
        g.A1h = a.d_gemm;
        g.A1l = g.A1h + h1.size();
        g.A2h = g.A1l + l1.size();
        g.A2l = g.A2h + h2.size();
        g.s1 = (float)s1;
        g.s2 = (float)s2;
        g.nlines = a.nlines;
        g.inner = a.inner;
        // lines per CTA: fit shared memory, and shrink until the axis has at
        // least one CTA per SM
        int G = 64;
        while (G > 8 && pstd::gemm_smem_bytes(G, g.KT1, g.KT2, a.N) > 200 * 1024) G /= 2;
        auto ctas = [&](int gg) {
            return a.inner == 1 ? (a.nlines + gg - 1) / gg : (a.nlines / a.inner) * ((a.inner + gg - 1) / gg);
        };
        while (G > 8 && ctas(G) < P->nsm) G /= 2;
        g.G = G;
        a.gsmem = pstd::gemm_smem_bytes(G, g.KT1, g.KT2, a.N);
        if (a.inner == 1) a.ggrid = (unsigned)((a.nlines + G - 1) / G);
        else a.ggrid = (unsigned)((a.nlines / a.inner) * ((a.inner + G - 1) / G));
    }
    return PSTD_OK;
}

void free_plan_memory(pstd_plan_s* P) {
    for (auto& a : P->ax) {
        cudaFree(a.d_tw);
        cudaFree(a.d_shift);
        cudaFree(a.d_wtw);
        cudaFree(a.d_sym);
        cudaFree(a.d_fUL);
        cudaFree(a.d_ph);
        cudaFree(a.d_tc);
        cudaFree(a.d_f2);
        cudaFree(a.d_dense2);
        for (int o = 0; o < 2; ++o)
            for (int k = 0; k < 4; ++k) {
                cudaFree(a.d_xf[o][k]);
                cudaFree(a.d_xdense[o][k]);
            }
        cudaFree(a.d_gemm);
        cudaFree(a.d_tc16[0]);
        cudaFree(a.d_tc16[1]);
        for (int o = 0; o < OP_COUNT; ++o) {
            cudaFree(a.d_f[o]);
            cudaFree(a.d_dense[o]);
        }
    }
    cudaFree(P->d_S);
    cudaFree(P->d_energy);
    for (auto* b : P->d_pad) cudaFree(b);
    cudaFree(P->d_Spad);
    cudaFree(P->d_sync);
    for (auto& g : P->graphs)
        if (g.exec) cudaGraphExecDestroy(g.exec);
}

// BF16 split form: the padded copies of p, u_0.. and the accumulator (last
// dimension rounded up to 4 floats, zero-filled) and every axis's tensor maps.
int tc16_setup(pstd_plan_s* P) {
    const int d = P->ndim;
    auto rows_of = [&](int f) {
        int64_t r = 1;
        for (int j = 0; j < d - 1; ++j) r *= P->shape[f][j];
        return r;
    };
    for (int f = 0; f <= d; ++f) {
        P->pitch[f] = (P->shape[f][d - 1] + 3) / 4 * 4;
        const size_t bytes = (size_t)rows_of(f) * P->pitch[f] * sizeof(float);
        cudaError_t e = cudaMalloc((void**)&P->d_pad[f], bytes);
        if (e == cudaSuccess) e = cudaMemset(P->d_pad[f], 0, bytes);
        if (e == cudaSuccess && f == 0) e = cudaMalloc((void**)&P->d_Spad, bytes);
        if (e == cudaSuccess && f == 0) e = cudaMemset(P->d_Spad, 0, bytes);
        if (e != cudaSuccess) return e == cudaErrorMemoryAllocation ? PSTD_ENOMEM : cuda_fail(e, "cudaMalloc(padded)");
    }
    for (int a = 0; a < d; ++a) {
        Axis& A = P->ax[a];
        const int contig = a == d - 1;
        // fields along this axis: 0 = p (and S), a + 1 = u_a
        auto map = [&](int f, float* base, int ymap, CUtensorMap* m) {
            const int64_t len = P->shape[f][a];
            if (contig) return pstd::tc16_field_map(base, 1, len, rows_of(f), 1, P->pitch[f], ymap, m);
            int64_t inner = P->pitch[f], outer = 1;
            for (int j = a + 1; j < d - 1; ++j) inner *= P->shape[f][j];
            for (int j = 0; j < a; ++j) outer *= P->shape[f][j];
            return pstd::tc16_field_map(base, 0, len, inner, outer, P->pitch[f], ymap, m);
        };
        int r = map(0, P->d_pad[0], 0, &A.tc16_x[0]);
        if (r == 0) r = map(a + 1, P->d_pad[a + 1], 0, &A.tc16_x[1]);
        if (r == 0) r = map(a + 1, P->d_pad[a + 1], 1, &A.tc16_y[0]);
        if (r == 0) r = map(0, P->d_pad[0], 1, &A.tc16_y[1]);
        if (r == 0) r = map(0, P->d_Spad, 1, &A.tc16_y[2]);
        if (r != 0) return cuda_fail(cudaErrorNotSupported, "cuTensorMapEncodeTiled(field)");
        if (contig) {
            A.tc16_tpo = 0;
            A.tc16_tiles = (rows_of(0) + 127) / 128;
        } else {
            int64_t inner = P->pitch[0], outer = 1;
            for (int j = a + 1; j < d - 1; ++j) inner *= P->shape[0][j];
            for (int j = 0; j < a; ++j) outer *= P->shape[0][j];
            A.tc16_tpo = (inner + 127) / 128;
            A.tc16_tiles = outer * A.tc16_tpo;
        }
    }
    return PSTD_OK;
}

// Copy the caller's fields into the padded copies (in = true) or back.
int tc16_copy(pstd_plan_s* P, float* p, float* const* u, bool in) {
    const int d = P->ndim;
    for (int f = 0; f <= d; ++f) {
        float* user = f == 0 ? p : u[f - 1];
        int64_t rows = 1;
        for (int j = 0; j < d - 1; ++j) rows *= P->shape[f][j];
        const size_t w = (size_t)P->shape[f][d - 1] * sizeof(float), pw = (size_t)P->pitch[f] * sizeof(float);
        cudaError_t e = in ? cudaMemcpy2DAsync(P->d_pad[f], pw, user, w, w, (size_t)rows, cudaMemcpyDeviceToDevice,
                                               P->stream)
                           : cudaMemcpy2DAsync(user, w, P->d_pad[f], pw, w, (size_t)rows, cudaMemcpyDeviceToDevice,
                                               P->stream);
        if (e != cudaSuccess) return cuda_fail(e, "cudaMemcpy2DAsync(padded field)");
    }
    return PSTD_OK;
}

int validate(const pstd_desc* d) {
    if (!d || d->ndim < 1 || d->ndim > 3) return PSTD_EINVAL;
    if (!(d->c0 > 0) || !(d->rho0 > 0) || !(d->dt > 0)) return PSTD_EINVAL;
    if (!std::isfinite(d->c0) || !std::isfinite(d->rho0) || !std::isfinite(d->dt)) return PSTD_EINVAL;
    if (d->uinit != PSTD_U_HALFSTEP && d->uinit != PSTD_U_AS_GIVEN) return PSTD_EINVAL;
    for (int i = 0; i < d->ndim; ++i) {
        if (d->ncells[i] < 1 || d->ncells[i] > (1 << 20)) return PSTD_EINVAL;
        if (!(d->dx[i] > 0) || !std::isfinite(d->dx[i])) return PSTD_EINVAL;
        const int l = d->bc[i][0], r = d->bc[i][1];
        if (l != PSTD_NEUMANN && l != PSTD_DIRICHLET && l != PSTD_PERIODIC) return PSTD_EINVAL;
        if (r != PSTD_NEUMANN && r != PSTD_DIRICHLET && r != PSTD_PERIODIC && r != PSTD_NEUMANN_MID &&
            r != PSTD_DIRICHLET_MID)
            return PSTD_EINVAL;
        if ((l == PSTD_PERIODIC) != (r == PSTD_PERIODIC)) return PSTD_EINVAL;
        if (l == PSTD_PERIODIC && d->ncells[i] < 2) return PSTD_EINVAL;
        if (d->ncells[i] == 1 && l == PSTD_DIRICHLET && r == PSTD_DIRICHLET) return PSTD_EINVAL;
        if (d->ncells[i] < 2 && (r == PSTD_NEUMANN_MID || r == PSTD_DIRICHLET_MID)) return PSTD_EINVAL;
    }
    // leapfrog limit: c0 dt |k|_max / 2 <= 1 with the largest stored-mode
    // wavenumber of each axis (NN keeps k = pi/dx; ND/DN pi(N-1/2)/L; DD pi(N-1)/L;
    // mid-cell right wall, M = 2N - 1: same parity 2 pi (N-1) / (M dx), ND-mid
    // pi / dx, DN-mid pi (M - 2) / (M dx))
    double k2 = 0;
    for (int i = 0; i < d->ndim; ++i) {
        const double N = (double)d->ncells[i], L = N * d->dx[i];
        const int l = d->bc[i][0], r = d->bc[i][1];
        double kmax;
        if (r == PSTD_NEUMANN_MID || r == PSTD_DIRICHLET_MID) {
            const double M = 2.0 * N - 1.0, dx = d->dx[i];
            const bool same = (l == PSTD_NEUMANN) == (r == PSTD_NEUMANN_MID);
            if (same) kmax = 2.0 * M_PI * (N - 1.0) / (M * dx);
            else if (l == PSTD_NEUMANN) kmax = M_PI / dx;
            else kmax = M_PI * (M - 2.0) / (M * dx);
        } else if (l == PSTD_PERIODIC) kmax = 2.0 * M_PI * std::floor(N / 2.0) / L;
        else if (d->bc[i][0] == PSTD_NEUMANN && d->bc[i][1] == PSTD_NEUMANN) kmax = M_PI * N / L;
        else if (d->bc[i][0] != d->bc[i][1]) kmax = M_PI * (N - 0.5) / L;
        else kmax = M_PI * (N - 1.0) / L;
        k2 += kmax * kmax;
    }
    if (d->c0 * d->dt * std::sqrt(k2) / 2.0 > 1.0) return PSTD_EUNSTABLE;
    return PSTD_OK;
}

StepArgs step_args(pstd_plan_s* P, int a, float* p, float* const* u) {
    Axis& A = P->ax[a];
    StepArgs s;
    s.opP = A.op[OP_STEP_P];
    s.opU = A.op[OP_STEP_U];
    s.nlines = A.nlines;
    s.inner = A.inner;
    s.G = A.G;
    s.rs = A.rs;
    s.p = p;
    s.u = u[a];
    const int d = P->ndim;
    s.acc_in = (a == d - 1) ? p : P->d_S;
    s.acc_out = (a == 0) ? p : P->d_S;
    return s;
}

int launch_step(pstd_plan_s* P, float* p, float* const* u, int64_t* launches) {
    for (int a = P->ndim - 1; a >= 0; --a) {
        Axis& A = P->ax[a];
        if (P->opts.form == 2) {
            // u_a += p D1^T, then acc_out = acc_in + u_a D2^T, as GEMMs over the
            // lines of the axis (outer blocks as the batch on strided axes)
            const int64_t inner = A.inner, outer = A.nlines / A.inner;
            const int N = A.N, lp = A.lp;
            const size_t n1 = (size_t)N * lp;
            const float* D1h = A.d_tc;
            const float* D1l = D1h + n1;
            const float* D2h = D1l + n1;
            const float* D2l = D2h + n1;
            float* acc_in = (a == P->ndim - 1) ? p : P->d_S;
            float* acc_out = (a == 0) ? p : P->d_S;
            int* status = (int*)(P->d_sync + 2);
            auto lines = [&](pstd_gemm_desc& g, const float* X, int xlen, float* Y, int ylen) {
                if (inner > 1) {
                    g.batch = outer;
                    g.M = (int)inner;
                    g.sAb = (int64_t)xlen * inner; g.sAm = 1; g.sAk = inner;
                    g.sCb = (int64_t)ylen * inner; g.sCm = 1; g.sCn = inner;
                } else {
                    g.batch = 1;
                    g.M = (int)A.nlines;
                    g.sAb = 0; g.sAm = xlen; g.sAk = 1;
                    g.sCb = 0; g.sCm = ylen; g.sCn = 1;
                }
                g.A = X;
                g.C = Y;
                g.K = xlen;
                g.N = ylen;
                g.sBb = 0; g.sBk = 1; g.sBn = xlen;
                g.alpha = 1.0f;
                g.beta = 1.0f;
                g.batch2 = 1;
                g.K_last = xlen;
            };
            pstd_gemm_desc g1{};
            lines(g1, p, lp, u[a], N);
            g1.B = D1h;
            int rc = pstd_internal_tc_gemm_split(&g1, D1l, status, P->stream);
            if (rc != PSTD_OK) return rc;
            ++*launches;
            if (acc_in != acc_out)
                CK(cudaMemcpyAsync(acc_out, acc_in, (size_t)pstd_field_numel(P, 0) * sizeof(float),
                                   cudaMemcpyDeviceToDevice, P->stream));
            pstd_gemm_desc g2{};
            lines(g2, u[a], N, acc_out, lp);
            g2.B = D2h;
            rc = pstd_internal_tc_gemm_split(&g2, D2l, status, P->stream);
            if (rc != PSTD_OK) return rc;
            ++*launches;
            continue;
        }
        if (P->opts.form == 3) {
            // on the plan's padded fields: u_a += D1 p, then acc_out = acc_in + D2 u_a
            int* status = (int*)(P->d_sync + 2);
            const int contig = a == P->ndim - 1;
            pstd::Tc16Gemm g1{};
            g1.K = A.lp; g1.Mout = A.nu; g1.MT = A.tc16_MT[0]; g1.KC = A.tc16_KC[0];
            g1.contiguous = contig; g1.tiles = A.tc16_tiles; g1.tpo = A.tc16_tpo; g1.status = status;
            g1.op = (const uint8_t*)A.d_tc16[0];
            CK(pstd::tc16_launch(A.tc16_x[0], A.tc16_y[0], A.tc16_y[0], g1, P->stream));
            pstd::Tc16Gemm g2 = g1;
            g2.K = A.nu; g2.Mout = A.lp; g2.MT = A.tc16_MT[1]; g2.KC = A.tc16_KC[1];
            g2.op = (const uint8_t*)A.d_tc16[1];
            const CUtensorMap& cin = (a == P->ndim - 1) ? A.tc16_y[1] : A.tc16_y[2];
            const CUtensorMap& out = (a == 0) ? A.tc16_y[1] : A.tc16_y[2];
            CK(pstd::tc16_launch(A.tc16_x[1], cin, out, g2, P->stream));
            *launches += 2;
            continue;
        }
        if (P->opts.form == 1) {
            pstd::GemmStep g;
            g.ax = A.gax;
            g.p = p;
            g.u = u[a];
            g.acc_in = (a == P->ndim - 1) ? p : P->d_S;
            g.acc_out = (a == 0) ? p : P->d_S;
            CK(pstd::launch_gemm_step(A.ggrid, A.gsmem, P->stream, g));
            ++*launches;
            continue;
        }
        if (A.wl) {
            WStep w;
            w.ax = A.wax;
            w.fP = A.d_f[OP_STEP_P];
            w.fU = A.d_fUL;
            w.p = p;
            w.u = u[a];
            w.acc_in = (a == P->ndim - 1) ? p : P->d_S;
            w.acc_out = (a == 0) ? p : P->d_S;
            CK(wstep(A.L, A.wv, A.strided, A.wgeo, P->stream, w));
            ++*launches;
            continue;
        }
        StepArgs s = step_args(P, a, p, u);
        const unsigned grid = (unsigned)((A.nlines + A.G - 1) / A.G);
        CK(pstd::launch_k_step(grid, A.smem, P->stream, s));
        ++*launches;
    }
    return PSTD_OK;
}

int launch_grad(pstd_plan_s* P, int axis, int opi, const float* in, float* out, int acc) {
    Axis& A = P->ax[axis];
    if (A.wl) {
        WGrad g;
        g.ax = A.wax;
        g.dir = A.op[opi].dir;
        g.f = A.d_f[opi];
        g.in = in;
        g.out = out;
        g.accumulate = acc;
        g.scale = 1.0f;
        CK(wgrad(A.L, A.wv, A.strided, A.wgeo, P->stream, g));
        return PSTD_OK;
    }
    GradArgs g;
    g.op = A.op[opi];
    g.nlines = A.nlines;
    g.inner = A.inner;
    g.G = A.G;
    g.rs = A.rs;
    g.in = in;
    g.out = out;
    g.accumulate = acc;
    const unsigned grid = (unsigned)((A.nlines + A.G - 1) / A.G);
    CK(pstd::launch_k_grad(grid, A.smem, P->stream, g));
    return PSTD_OK;
}

// One second-order pass of `axis`: out += (c0 dt)^2 D_u D_p in along the
// axis, and pout = in + out (the new value) where pout is given.
int launch_order2(pstd_plan_s* P, int axis, const float* in, float* out, float* pout) {
    Axis& A = P->ax[axis];
    if (A.wl) {
        WGrad g{};
        g.ax = A.wax;
        g.dir = 4;
        g.f = A.d_f2;
        g.in = in;
        g.out = out;
        g.accumulate = 1;
        g.scale = 1.0f;
        g.pout = pout;
        CK(wgrad(A.L, A.wv, A.strided, A.wgeo, P->stream, g));
        return PSTD_OK;
    }
    GradArgs g;
    g.op = A.op2;
    g.nlines = A.nlines;
    g.inner = A.inner;
    g.G = A.G;
    g.rs = A.rs;
    g.in = in;
    g.out = out;
    g.accumulate = 1;
    g.pout = pout;
    const unsigned grid = (unsigned)((A.nlines + A.G - 1) / A.G);
    CK(pstd::launch_k_grad(grid, A.smem, P->stream, g));
    return PSTD_OK;
}

// One second-order step on (p, q = p^n - p^{n-1}), last axis first:
// q += (c0 dt)^2 sum_a D_{u,a} D_{p,a} p, and the pass of axis 0 also writes
// p = p + q.  Each pass reads p^n, which only the last pass overwrites, and
// that pass writes each p line after the CTA that owns it has read it.
int launch_order2_step(pstd_plan_s* P, float* p, float* q, int64_t* launches) {
    for (int a = P->ndim - 1; a >= 0; --a) {
        int rc = launch_order2(P, a, p, q, a == 0 ? p : nullptr);
        if (rc != PSTD_OK) return rc;
        ++*launches;
    }
    return PSTD_OK;
}

// Replay graphs of kGraphSteps steps for this pointer set (kind 0: leapfrog
// steps on p and the velocities; kind 1: second-order steps on p and q),
// recording one on first use (least recently used entry replaced); `done`
// counts the steps replayed.
template <class StepFn>
int replay_graphs(pstd_plan_t* P, int kind, float* p, float* const* u, int nu, int64_t nsteps, int64_t& done,
                  StepFn&& one_step) {
    GraphEntry* ge = nullptr;
    for (auto& g : P->graphs) {
        bool same = g.exec && g.kind == kind && g.p == p;
        for (int a = 0; a < nu && same; ++a) same = g.u[a] == u[a];
        if (same) { ge = &g; break; }
    }
    if (!ge) {
        GraphEntry* victim = &P->graphs[0];
        for (auto& g : P->graphs) {
            if (!g.exec) { victim = &g; break; }
            if (g.stamp < victim->stamp) victim = &g;
        }
        if (victim->exec) { cudaGraphExecDestroy(victim->exec); victim->exec = nullptr; }
        CK(cudaStreamBeginCapture(P->stream, cudaStreamCaptureModeThreadLocal));
        int64_t nl = 0;
        int rc = PSTD_OK;
        for (int s = 0; s < kGraphSteps && rc == PSTD_OK; ++s) rc = one_step(&nl);
        cudaGraph_t graph = nullptr;
        cudaError_t e = cudaStreamEndCapture(P->stream, &graph);
        if (rc != PSTD_OK) { if (graph) cudaGraphDestroy(graph); return rc; }
        if (e != cudaSuccess) return cuda_fail(e, "cudaStreamEndCapture");
        e = cudaGraphInstantiate(&victim->exec, graph, 0);
        cudaGraphDestroy(graph);
        if (e != cudaSuccess) { victim->exec = nullptr; return cuda_fail(e, "cudaGraphInstantiate"); }
        victim->kind = kind;
        victim->p = p;
        for (int a = 0; a < 3; ++a) victim->u[a] = a < nu ? u[a] : nullptr;
        victim->steps = kGraphSteps;
        victim->launches = nl;
        ge = victim;
    }
    ge->stamp = ++P->stamp;
    while (nsteps - done >= ge->steps) {
        CK(cudaGraphLaunch(ge->exec, P->stream));
        done += ge->steps;
        P->last_launches += ge->launches;
    }
    return PSTD_OK;
}

// Register-FFT axes keep u_a as its spectrum between the passes of a run:
// dir 2 converts u_a to it in place before the first step, dir 3 back after
// the last.  Other axes (and the split form) step u_a itself.
int convert_velocity(pstd_plan_s* P, float* const* u, int dir, int64_t* launches) {
    if (P->opts.form != 0) return PSTD_OK;
    for (int a = 0; a < P->ndim; ++a) {
        Axis& A = P->ax[a];
        if (!A.wl) continue;
        WGrad g;
        g.ax = A.wax;
        g.dir = dir;
        g.f = nullptr;
        g.in = u[a];
        g.out = u[a];
        g.accumulate = 0;
        g.scale = (float)(1.0 / A.L);
        CK(wgrad(A.L, A.wv, A.strided, A.wgeo, P->stream, g));
        ++*launches;
    }
    return PSTD_OK;
}

}  // namespace

int pstd_internal_convert_velocity(pstd_plan_t* P, float* const* u, int to_spectrum, int64_t* launches) {
    return convert_velocity(P, u, to_spectrum ? 2 : 3, launches);
}

int pstd_internal_launch_steps(pstd_plan_t* P, float* p, float* const* u, int64_t n, int64_t* launches) {
    if (P->opts.form == 3) return PSTD_EUNSUPPORTED;     // steps on the plan's padded copies only
    for (int64_t s = 0; s < n; ++s) {
        int rc = launch_step(P, p, u, launches);
        if (rc != PSTD_OK) return rc;
    }
    return PSTD_OK;
}

// ---- batch of plans as one cooperative kernel ------------------------------
struct pstd_batch_persist_s {
    std::vector<unsigned char> h_args;   // WStep or StepArgs, [members][3]
    std::vector<int64_t> h_prefix;       // [3][members + 1]
    void* d_args = nullptr;
    int64_t* d_prefix = nullptr;
    size_t args_cap = 0, prefix_cap = 0;
    unsigned* d_sync = nullptr;          // count, generation, status
};

int pstd_internal_batch_persist_kind(pstd_plan_t* const* plans, int n) {
    if (n < 1) return 0;
    for (int m = 0; m < n; ++m)
        if (plans[m]->opts.form != 0) return 0;
    const Axis& A0 = plans[0]->ax[0];
    bool reg = true;
    for (int m = 0; m < n && reg; ++m)
        for (int a = 0; a < plans[m]->ndim && reg; ++a) {
            const Axis& A = plans[m]->ax[a];
            reg = A.wl > 0 && A0.wl > 0 && A.L == A0.L && A.wv == A0.wv && A.wgeo.threads == A0.wgeo.threads;
        }
    return reg ? 1 : 2;
}

void pstd_internal_batch_persist_free(pstd_batch_persist_s* S) {
    if (!S) return;
    if (S->d_args) cudaFree(S->d_args);
    if (S->d_prefix) cudaFree(S->d_prefix);
    if (S->d_sync) cudaFree(S->d_sync);
    delete S;
}

int pstd_internal_batch_persist_status(pstd_batch_persist_s* S) {
    if (!S || !S->d_sync) return PSTD_OK;
    int status = 0;
    CK(cudaMemcpy(&status, S->d_sync + 2, sizeof(int), cudaMemcpyDeviceToHost));
    if (status != 0) {
        CK(cudaMemset(S->d_sync, 0, 4 * sizeof(unsigned)));
        return PSTD_ETIMEOUT;
    }
    return PSTD_OK;
}

int pstd_internal_batch_persist_run(pstd_batch_persist_s** state, pstd_plan_t* const* plans, int n, float* const* p,
                                    float* const* u, int64_t nsteps, long long spin_limit, unsigned withhold,
                                    cudaStream_t st) {
    const int kind = pstd_internal_batch_persist_kind(plans, n);
    if (kind == 0) return PSTD_EUNSUPPORTED;
    if (!*state) {
        *state = new (std::nothrow) pstd_batch_persist_s();
        if (!*state) return PSTD_ENOMEM;
        CK(cudaMalloc((void**)&(*state)->d_sync, 4 * sizeof(unsigned)));
        CK(cudaMemset((*state)->d_sync, 0, 4 * sizeof(unsigned)));
    }
    pstd_batch_persist_s* S = *state;
    int npass = 0;
    for (int m = 0; m < n; ++m) npass = plans[m]->ndim > npass ? plans[m]->ndim : npass;
    const size_t esz = kind == 1 ? sizeof(WStep) : sizeof(StepArgs);
    S->h_args.assign((size_t)n * 3 * esz, 0);
    S->h_prefix.assign((size_t)3 * (n + 1), 0);
    size_t smem = 0;
    int64_t most = 0;
    for (int k = 0; k < npass; ++k) {
        int64_t* pre = S->h_prefix.data() + (size_t)k * (n + 1);
        for (int m = 0; m < n; ++m) {
            pstd_plan_s* P = plans[m];
            int64_t items = 0;
            const int a = P->ndim - 1 - k;
            if (a >= 0) {
                Axis& A = P->ax[a];
                unsigned char* slot = S->h_args.data() + ((size_t)m * 3 + k) * esz;
                if (kind == 1) {
                    WStep w;
                    w.ax = A.wax;
                    w.fP = A.d_f[OP_STEP_P];
                    w.fU = A.d_fUL;
                    w.p = p[m];
                    w.u = u[3 * m + a];
                    w.acc_in = (a == P->ndim - 1) ? p[m] : P->d_S;
                    w.acc_out = (a == 0) ? p[m] : P->d_S;
                    std::memcpy(slot, &w, sizeof w);
                    items = A.wgeo.grid;
                    smem = A.wgeo.smem > smem ? A.wgeo.smem : smem;
                } else {
                    const StepArgs sa = step_args(P, a, p[m], u + 3 * m);
                    std::memcpy(slot, &sa, sizeof sa);
                    items = (A.nlines + A.G - 1) / A.G;
                    smem = A.smem > smem ? A.smem : smem;
                }
            }
            pre[m + 1] = pre[m] + items;
        }
        most = pre[n] > most ? pre[n] : most;
    }
    if (S->h_args.size() > S->args_cap) {
        if (S->d_args) cudaFree(S->d_args);
        S->d_args = nullptr;
        S->args_cap = 0;
        CK(cudaMalloc(&S->d_args, S->h_args.size()));
        S->args_cap = S->h_args.size();
    }
    if (S->h_prefix.size() > S->prefix_cap) {
        if (S->d_prefix) cudaFree(S->d_prefix);
        S->d_prefix = nullptr;
        S->prefix_cap = 0;
        CK(cudaMalloc((void**)&S->d_prefix, S->h_prefix.size() * sizeof(int64_t)));
        S->prefix_cap = S->h_prefix.size();
    }
    // pageable sources: each copy has consumed its source when the call returns
    CK(cudaMemcpyAsync(S->d_args, S->h_args.data(), S->h_args.size(), cudaMemcpyHostToDevice, st));
    CK(cudaMemcpyAsync(S->d_prefix, S->h_prefix.data(), S->h_prefix.size() * sizeof(int64_t),
                       cudaMemcpyHostToDevice, st));
    CK(cudaMemsetAsync(S->d_sync, 0, sizeof(unsigned), st));   // arrival count
    int dev = 0, nsm = 0, per_sm = 0;
    CK(cudaGetDevice(&dev));
    CK(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
    const Axis& A0 = plans[0]->ax[0];
    if (kind == 1) CK(wpersist_blocks(A0.L, A0.wv, A0.wgeo.threads, smem, &per_sm));
    else {
        CK(pstd::set_max_smem((int)smem));
        CK(pstd::k_step_persist_blocks(smem, &per_sm));
    }
    if (per_sm < 1) return PSTD_EUNSUPPORTED;
    int64_t grid = (int64_t)per_sm * nsm;
    if (grid > most) grid = most;
    if (grid < 1) grid = 1;
    GridSync sync;
    sync.count = S->d_sync;
    sync.gen = S->d_sync + 1;
    sync.status = (int*)(S->d_sync + 2);
    sync.expected = (unsigned)grid + withhold;
    sync.spin_limit = spin_limit > 0 ? spin_limit : 2000000LL;
    if (kind == 1) {
        PersistArgs pa{};
        pa.ndim = npass;
        pa.nsteps = nsteps;
        pa.sync = sync;
        pa.members = n;
        pa.mem = (const WStep*)S->d_args;
        pa.prefix = S->d_prefix;
        WLaunch g;
        g.grid = (unsigned)grid;
        g.threads = A0.wgeo.threads;
        g.smem = smem;
        CK(wpersist(A0.L, A0.wv, g, st, pa));
    } else {
        StepPersistArgs sa;
        sa.mem = (const StepArgs*)S->d_args;
        sa.prefix = S->d_prefix;
        sa.members = n;
        sa.npass = npass;
        sa.nsteps = nsteps;
        CK(pstd::launch_k_step_persist((unsigned)grid, smem, st, sa, sync));
    }
    return PSTD_OK;
}

cudaStream_t pstd_internal_stream(const pstd_plan_t* P) { return P->stream; }

void pstd_internal_layout(const pstd_plan_t* P, int lo[3], int64_t shape[3]) {
    for (int i = 0; i < 3; ++i) {
        lo[i] = i < P->ndim ? P->ax[i].lo : 0;
        shape[i] = P->shape[0][i];
    }
}

int pstd_internal_cuda_fail(cudaError_t e, const char* what) { return cuda_fail(e, what); }

extern "C" {

const char* pstd_version(void) { return "pstd-gb300 0.1 (sm_103a)"; }

double pstd_dt_from_cfl(double cfl, double dx, double c0) { return cfl * dx / c0; }

const char* pstd_strerror(int code) {
    switch (code) {
        case PSTD_OK: return "ok";
        case PSTD_EINVAL: return "invalid argument";
        case PSTD_EUNSTABLE: return "time step beyond the leapfrog stability limit";
        case PSTD_ENOMEM: return "out of memory";
        case PSTD_ECUDA: return "CUDA runtime error";
        case PSTD_ETIMEOUT: return "device-side wait timed out";
        case PSTD_EUNSUPPORTED: return "unsupported size";
        default: return "unknown error";
    }
}

const char* pstd_last_cuda_error(void) { return g_cuda_err.c_str(); }

int pstd_plan(const pstd_desc* desc, void* stream, pstd_plan_t** out) {
    return pstd_plan_ex(desc, stream, nullptr, out);
}

int pstd_plan_persistent(const pstd_plan_t* P, int out[3]) {
    if (!P || !out) return PSTD_EINVAL;
    out[0] = P->persist_ok;
    out[1] = (int)P->pgeo.grid;
    out[2] = P->pgeo.threads;
    return PSTD_OK;
}

int pstd_plan_schedule(const pstd_plan_t* P, int axis, int out[4]) {
    if (!P || !out || axis < 0 || axis >= P->ndim) return PSTD_EINVAL;
    const Axis& A = P->ax[axis];
    if (!A.wl) {
        out[0] = out[1] = out[2] = out[3] = -1;
        return PSTD_OK;
    }
    out[0] = A.wv;
    out[1] = A.wl;
    out[2] = A.wax.seqs;
    out[3] = (int)A.wgeo.grid;
    return PSTD_OK;
}

int pstd_plan_ex(const pstd_desc* desc, void* stream, const pstd_plan_opts* opts, pstd_plan_t** out) {
    if (!out) return PSTD_EINVAL;
    *out = nullptr;
    int rc = validate(desc);
    if (rc != PSTD_OK) return rc;
    pstd_plan_s* P = new (std::nothrow) pstd_plan_s();
    if (!P) return PSTD_ENOMEM;
    P->desc = *desc;
    if (opts) P->opts = *opts;
    {
        int dev = 0, n = 0;
        if (cudaGetDevice(&dev) == cudaSuccess &&
            cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) == cudaSuccess && n > 0)
            P->nsm = n;
    }
    if (P->opts.form < 0 || P->opts.form > 3) {
        delete P;
        return PSTD_EINVAL;
    }
    P->stream = (cudaStream_t)stream;
    P->ndim = desc->ndim;
    for (int f = 0; f < 4; ++f)
        for (int j = 0; j < 3; ++j) P->shape[f][j] = 1;
    for (int i = 0; i < P->ndim; ++i) {
        const int64_t N = desc->ncells[i];
        const int r = desc->bc[i][1];
        const bool mid = r == PSTD_NEUMANN_MID || r == PSTD_DIRICHLET_MID;
        const int64_t lo = desc->bc[i][0] == PSTD_DIRICHLET ? 1 : 0;
        const int64_t hi = (desc->bc[i][0] == PSTD_PERIODIC || mid) ? N - 1 : (r == PSTD_DIRICHLET ? N - 1 : N);
        P->shape[0][i] = hi - lo + 1;
    }
    for (int f = 1; f <= P->ndim; ++f) {
        for (int j = 0; j < P->ndim; ++j) P->shape[f][j] = P->shape[0][j];
        // velocity half-nodes; N - 1 next to a Neumann mid-cell wall
        P->shape[f][f - 1] = desc->ncells[f - 1] - (desc->bc[f - 1][1] == PSTD_NEUMANN_MID ? 1 : 0);
    }
    for (int i = 0; i < P->ndim && rc == PSTD_OK; ++i) rc = build_axis(P, i);
    if (rc == PSTD_OK && P->opts.form == 3) rc = tc16_setup(P);
    if (rc == PSTD_OK && (P->opts.form == 2 || P->opts.form == 3)) {
        // status word of the tensor-core GEMMs' bounded waits (read by pstd_sync)
        cudaError_t e = cudaMalloc((void**)&P->d_sync, 4 * sizeof(unsigned));
        if (e == cudaSuccess) e = cudaMemset(P->d_sync, 0, 4 * sizeof(unsigned));
        if (e != cudaSuccess) rc = cuda_fail(e, "cudaMalloc(status)");
    }
    if (rc == PSTD_OK && P->ndim >= 2) {
        cudaError_t e = cudaMalloc((void**)&P->d_S, (size_t)pstd_field_numel(P, 0) * sizeof(float));
        if (e != cudaSuccess) rc = e == cudaErrorMemoryAllocation ? PSTD_ENOMEM : cuda_fail(e, "cudaMalloc(S)");
    }
    if (rc == PSTD_OK) {
        size_t mx = 0;
        for (int i = 0; i < P->ndim; ++i) mx = P->ax[i].smem > mx ? P->ax[i].smem : mx;
        cudaError_t e = pstd::set_max_smem((int)mx);
        if (e != cudaSuccess) rc = cuda_fail(e, "cudaFuncSetAttribute");
        if (rc == PSTD_OK && P->opts.form == 3) {
            e = pstd::tc16_set_smem();
            if (e != cudaSuccess) rc = cuda_fail(e, "cudaFuncSetAttribute(BF16 split pass)");
        }
        if (rc == PSTD_OK && P->opts.form == 1) {
            int dev = 0, optin = 0;
            cudaGetDevice(&dev);
            cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
            e = pstd::gemm_set_smem(optin);
            if (e != cudaSuccess) rc = cuda_fail(e, "cudaFuncSetAttribute(split-precision pass)");
        }
        for (int i = 0; i < P->ndim && rc == PSTD_OK; ++i) {
            if (!P->ax[i].wl) continue;
            int dev = 0, optin = 0;
            cudaGetDevice(&dev);
            cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
            e = wsmem(P->ax[i].L, P->ax[i].wv, optin);
            if (e != cudaSuccess) rc = cuda_fail(e, "cudaFuncSetAttribute(register-FFT pass)");
        }
    }
    // persistent run: every axis on the same register-FFT schedule and CTA size
    if (rc == PSTD_OK && P->opts.persistent) {
        bool same = P->opts.form == 0;
        for (int i = 0; i < P->ndim && same; ++i)
            same = P->ax[i].wl > 0 && P->ax[i].L == P->ax[0].L && P->ax[i].wv == P->ax[0].wv &&
                   P->ax[i].wgeo.threads == P->ax[0].wgeo.threads;
        if (same) {
            size_t smem = 0;
            int64_t items = 0;
            for (int i = 0; i < P->ndim; ++i) {
                smem = P->ax[i].wgeo.smem > smem ? P->ax[i].wgeo.smem : smem;
                items = (int64_t)P->ax[i].wgeo.grid > items ? (int64_t)P->ax[i].wgeo.grid : items;
            }
            int per_sm = 0, dev = 0, nsm = 0;
            cudaError_t e = cudaGetDevice(&dev);
            if (e == cudaSuccess) e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
            if (e == cudaSuccess)
                e = wpersist_blocks(P->ax[0].L, P->ax[0].wv, P->ax[0].wgeo.threads, smem, &per_sm);
            if (e == cudaSuccess) e = cudaMalloc((void**)&P->d_sync, 4 * sizeof(unsigned));
            if (e == cudaSuccess) e = cudaMemset(P->d_sync, 0, 4 * sizeof(unsigned));
            if (e != cudaSuccess) rc = cuda_fail(e, "persistent set-up");
            else if (per_sm > 0) {
                int64_t grid = (int64_t)per_sm * nsm;
                if (grid > items) grid = items;
                P->pgeo.grid = (unsigned)grid;
                P->pgeo.threads = P->ax[0].wgeo.threads;
                P->pgeo.smem = smem;
                P->persist_ok = 1;
            }
        }
    }
    if (rc != PSTD_OK) {
        free_plan_memory(P);
        delete P;
        return rc;
    }
    *out = P;
    return PSTD_OK;
}

int pstd_field_shape(const pstd_plan_t* P, int field, int64_t shape[3]) {
    if (!P || !shape || field < 0 || field > P->ndim) return PSTD_EINVAL;
    for (int j = 0; j < 3; ++j) shape[j] = P->shape[field][j];
    return PSTD_OK;
}

int64_t pstd_field_numel(const pstd_plan_t* P, int field) {
    if (!P || field < 0 || field > P->ndim) return 0;
    return P->shape[field][0] * P->shape[field][1] * P->shape[field][2];
}

int pstd_apply_shape(const pstd_plan_t* P, int axis, int kind, int64_t shape[3]) {
    if (!P || !shape || axis < 0 || axis >= P->ndim || kind < 0 || kind > 3) return PSTD_EINVAL;
    KindGeo g;
    if (!kind_geo(P->ax[axis], kind, g)) return PSTD_EINVAL;
    for (int j = 0; j < 3; ++j) shape[j] = P->shape[0][j];
    shape[axis] = g.len;
    return PSTD_OK;
}

int pstd_apply(pstd_plan_t* P, int axis, int op, int kind, const float* in, float* out) {
    if (!P || axis < 0 || axis >= P->ndim || (op != PSTD_OP_DIFF && op != PSTD_OP_INTERP) || kind < 0 ||
        kind > 3 || !in || !out)
        return PSTD_EINVAL;
    P->last_launches = 0;
    int rc = build_xop(P, axis, op, kind);
    if (rc != PSTD_OK) return rc;
    Axis& A = P->ax[axis];
    GradArgs g;
    g.op = A.xop[op][kind];
    g.nlines = A.nlines;
    g.inner = A.inner;
    g.G = A.xG[op][kind];
    g.rs = g.op.nin;
    g.in = in;
    g.out = out;
    g.accumulate = 0;
    const unsigned grid = (unsigned)((A.nlines + g.G - 1) / g.G);
    CK(pstd::launch_k_grad(grid, A.xsmem[op][kind], P->stream, g));
    P->last_launches = 1;
    return PSTD_OK;
}

int pstd_grad(pstd_plan_t* P, int axis, int dir, const float* in, float* out) {
    if (!P || axis < 0 || axis >= P->ndim || (dir != 0 && dir != 1) || !in || !out) return PSTD_EINVAL;
    P->last_launches = 0;
    int rc = launch_grad(P, axis, dir == 0 ? OP_GRAD_P : OP_GRAD_U, in, out, 0);
    if (rc == PSTD_OK) P->last_launches = 1;
    return rc;
}

int pstd_init_velocity(pstd_plan_t* P, const float* p0, float* const* u) {
    if (!P || !p0 || !u) return PSTD_EINVAL;
    for (int a = 0; a < P->ndim; ++a)
        if (!u[a]) return PSTD_EINVAL;
    P->last_launches = 0;
    if (P->desc.uinit == PSTD_U_AS_GIVEN) return PSTD_OK;
    for (int a = 0; a < P->ndim; ++a) {
        int rc = launch_grad(P, a, OP_INIT_P, p0, u[a], 1);
        if (rc != PSTD_OK) return rc;
        ++P->last_launches;
    }
    return PSTD_OK;
}

int pstd_step(pstd_plan_t* P, float* p, float* const* u) {
    if (!P || !p || !u) return PSTD_EINVAL;
    for (int a = 0; a < P->ndim; ++a)
        if (!u[a]) return PSTD_EINVAL;
    P->last_launches = 0;
    if (P->opts.form == 3) {
        // the step runs on the plan's padded copies
        int rc = tc16_copy(P, p, u, true);
        if (rc == PSTD_OK) rc = launch_step(P, P->d_pad[0], P->d_pad + 1, &P->last_launches);
        if (rc == PSTD_OK) rc = tc16_copy(P, p, u, false);
        return rc;
    }
    int rc = convert_velocity(P, u, 2, &P->last_launches);
    if (rc == PSTD_OK) rc = launch_step(P, p, u, &P->last_launches);
    if (rc == PSTD_OK) rc = convert_velocity(P, u, 3, &P->last_launches);
    return rc;
}

namespace {
int run_steps(pstd_plan_t* P, float* p, float* const* u, int64_t nsteps);
}

int pstd_run(pstd_plan_t* P, float* p, float* const* u, int64_t nsteps) {
    if (!P || !p || !u || nsteps < 0) return PSTD_EINVAL;
    for (int a = 0; a < P->ndim; ++a)
        if (!u[a]) return PSTD_EINVAL;
    P->last_launches = 0;
    if (nsteps == 0) return PSTD_OK;
    if (P->opts.form == 3) {
        // the steps run on the plan's padded copies (one graph for every call)
        int rc = tc16_copy(P, p, u, true);
        if (rc == PSTD_OK) rc = run_steps(P, P->d_pad[0], P->d_pad + 1, nsteps);
        if (rc == PSTD_OK) rc = tc16_copy(P, p, u, false);
        return rc;
    }
    int64_t conv = 0;
    int rc = convert_velocity(P, u, 2, &conv);
    if (rc == PSTD_OK) rc = run_steps(P, p, u, nsteps);
    if (rc == PSTD_OK) rc = convert_velocity(P, u, 3, &conv);
    P->last_launches += conv;
    return rc;
}

namespace {
// The steps of pstd_run with every register-FFT velocity in spectrum form.
int run_steps(pstd_plan_t* P, float* p, float* const* u, int64_t nsteps) {
    if (P->persist_ok && nsteps > 0) {
        PersistArgs pa{};
        pa.ndim = P->ndim;
        pa.nsteps = nsteps;
        for (int a = 0; a < P->ndim; ++a) {
            Axis& A = P->ax[a];
            WStep& w = pa.ax[a];
            w.ax = A.wax;
            w.fP = A.d_f[OP_STEP_P];
            w.fU = A.d_fUL;
            w.p = p;
            w.u = u[a];
            w.acc_in = (a == P->ndim - 1) ? p : P->d_S;
            w.acc_out = (a == 0) ? p : P->d_S;
            pa.strided[a] = A.strided ? 1 : 0;
            pa.items[a] = A.wgeo.grid;
        }
        pa.sync.count = P->d_sync;
        pa.sync.gen = P->d_sync + 1;
        pa.sync.status = (int*)(P->d_sync + 2);
        pa.sync.expected = P->pgeo.grid + (unsigned)(P->opts.withhold_arrivals > 0 ? P->opts.withhold_arrivals : 0);
        pa.sync.spin_limit = P->opts.spin_limit > 0 ? P->opts.spin_limit : 2000000LL;   // ~0.2-1 s of polls
        CK(cudaMemsetAsync(P->d_sync, 0, sizeof(unsigned), P->stream));   // arrival count
        CK(wpersist(P->ax[0].L, P->ax[0].wv, P->pgeo, P->stream, pa));
        P->last_launches = 1;
        return PSTD_OK;
    }
    int64_t done = 0;
    if (P->stream != nullptr && nsteps >= kGraphSteps) {
        int rc = replay_graphs(P, 0, p, u, P->ndim, nsteps, done,
                               [&](int64_t* nl) { return launch_step(P, p, u, nl); });
        if (rc != PSTD_OK) return rc;
    }
    while (done < nsteps) {
        int rc = launch_step(P, p, u, &P->last_launches);
        if (rc != PSTD_OK) return rc;
        ++done;
    }
    return PSTD_OK;
}
}  // namespace

int pstd_init_prev(pstd_plan_t* P, const float* p0, float* p_prev) {
    if (!P || !p0 || !p_prev || p0 == p_prev) return PSTD_EINVAL;
    P->last_launches = 0;
    const int64_t n = pstd_field_numel(P, 0);
    if (P->desc.uinit == PSTD_U_AS_GIVEN) {
        // u^{-1/2} = 0: p^{-1} = p^0
        CK(cudaMemcpyAsync(p_prev, p0, (size_t)n * sizeof(float), cudaMemcpyDeviceToDevice, P->stream));
        return PSTD_OK;
    }
    // half-step start: p^{-1} = p^0 + (c0 dt)^2 / 2 sum_a D_{u,a} D_{p,a} p^0
    for (int a = 0; a < P->ndim; ++a) {
        int rc = build_order2(P, a);
        if (rc != PSTD_OK) return rc;
    }
    CK(cudaMemsetAsync(p_prev, 0, (size_t)n * sizeof(float), P->stream));
    for (int a = P->ndim - 1; a >= 0; --a) {
        int rc = launch_order2(P, a, p0, p_prev, nullptr);
        if (rc != PSTD_OK) return rc;
        ++P->last_launches;
    }
    CK(pstd::launch_k_axpby(n, 1.0f, p0, 0.5f, p_prev, P->stream));
    ++P->last_launches;
    return PSTD_OK;
}

int pstd_run2(pstd_plan_t* P, float* p, float* p_prev, int64_t nsteps) {
    if (!P || !p || !p_prev || p == p_prev || nsteps < 0) return PSTD_EINVAL;
    P->last_launches = 0;
    if (nsteps == 0) return PSTD_OK;
    for (int a = 0; a < P->ndim; ++a) {
        int rc = build_order2(P, a);
        if (rc != PSTD_OK) return rc;
    }
    // carry q = p^n - p^{n-1} in the p_prev buffer during the run
    const int64_t n = pstd_field_numel(P, 0);
    float* q = p_prev;
    CK(pstd::launch_k_axpby(n, 1.0f, p, -1.0f, q, P->stream));
    int64_t conv = 1;
    int64_t done = 0;
    if (P->stream != nullptr && nsteps >= kGraphSteps) {
        int rc = replay_graphs(P, 1, p, &q, 1, nsteps, done,
                               [&](int64_t* nl) { return launch_order2_step(P, p, q, nl); });
        if (rc != PSTD_OK) return rc;
    }
    while (done < nsteps) {
        int rc = launch_order2_step(P, p, q, &P->last_launches);
        if (rc != PSTD_OK) return rc;
        ++done;
    }
    CK(pstd::launch_k_axpby(n, 1.0f, p, -1.0f, q, P->stream));   // p^{n-1} = p^n - q
    ++conv;
    P->last_launches += conv;
    return PSTD_OK;
}

int pstd_energy(pstd_plan_t* P, const float* p, float* const* u_prev, float* const* u_next, double* energy) {
    if (!P || !p || !u_prev || !u_next || !energy) return PSTD_EINVAL;
    const int d = P->ndim;
    for (int i = 0; i < d; ++i)
        if (!u_prev[i] || !u_next[i]) return PSTD_EINVAL;
    constexpr int kBlocks = 304;
    if (!P->d_energy) {
        cudaError_t e = cudaMalloc((void**)&P->d_energy, (4 * kBlocks + 1) * sizeof(double));
        if (e != cudaSuccess) return e == cudaErrorMemoryAllocation ? PSTD_ENOMEM : cuda_fail(e, "cudaMalloc(energy)");
    }
    pstd::EnergyField f[4];
    pstd::EnergyScales sc{};
    for (int fi = 0; fi <= d; ++fi) {
        f[fi].a = fi == 0 ? p : u_prev[fi - 1];
        f[fi].b = fi == 0 ? p : u_next[fi - 1];
        for (int j = 0; j < 3; ++j) f[fi].n[j] = P->shape[fi][j];
        f[fi].first_half = f[fi].last_half = 0;
        for (int a = 0; a < d; ++a) {
            const int l = P->desc.bc[a][0], r = P->desc.bc[a][1];
            if (fi == a + 1) {
                // the velocity's own axis: the half-node on a Dirichlet mid-cell wall
                if (r == PSTD_DIRICHLET_MID) f[fi].last_half |= 1 << a;
            } else {
                // pressure nodes on Neumann walls (a mid-cell wall has no node)
                if (l == PSTD_NEUMANN) f[fi].first_half |= 1 << a;
                if (r == PSTD_NEUMANN) f[fi].last_half |= 1 << a;
            }
        }
        sc.s[fi] = fi == 0 ? 1.0 / (2.0 * P->desc.rho0 * P->desc.c0 * P->desc.c0) : 0.5 * P->desc.rho0;
    }
    CK(pstd::energy_launch(f, d + 1, sc, kBlocks, P->d_energy, P->stream));
    CK(cudaMemcpyAsync(energy, P->d_energy + 4 * kBlocks, sizeof(double), cudaMemcpyDeviceToHost, P->stream));
    CK(cudaStreamSynchronize(P->stream));
    return PSTD_OK;
}

int pstd_sync(pstd_plan_t* P) {
    if (!P) return PSTD_EINVAL;
    CK(cudaStreamSynchronize(P->stream));
    CK(cudaGetLastError());
    if (P->d_sync) {
        int status = 0;
        CK(cudaMemcpy(&status, P->d_sync + 2, sizeof(int), cudaMemcpyDeviceToHost));
        if (status != 0) {
            CK(cudaMemset(P->d_sync, 0, 4 * sizeof(unsigned)));
            return PSTD_ETIMEOUT;
        }
    }
    return PSTD_OK;
}

int pstd_free(pstd_plan_t* P) {
    if (!P) return PSTD_OK;
    cudaStreamSynchronize(P->stream);
    free_plan_memory(P);
    delete P;
    return PSTD_OK;
}

int64_t pstd_last_launch_count(const pstd_plan_t* P) { return P ? P->last_launches : 0; }

}  // extern "C"
