// pstd_ops.cuh -- per-line staggered spectral derivative, as CTA phases.
//
// One staggered derivative along an axis (Section 3.4, Tables A3 / A6) maps a
// line of pressure nodes to the velocity half-nodes (dir 0) or back (dir 1).
// The line's symmetric-periodic extension (Section 3.2, Fig. 3) has period
// M = 2N (groups I: NN, DD) or is antiperiodic with period M (groups II: ND,
// DN).  The paper's T2^{-1} a1 T1 (resp. T1^{-1} a2 T2) is, in exact
// arithmetic, the Fourier multiplier i k e^{+-i k dx/2} applied to that
// extension and sampled on the other grid (Table 2's periodic row with the
// shift of Eq. fourier_shift_property); the DTT pair only restricts it to the
// representative samples.  This file evaluates it that way:
//
//   extend (reflect with the wall signs; group II: multiply by e^{-i pi j/M})
//   -> length-M complex FFT (mixed-radix Stockham passes in shared memory)
//   -> multiply by the folded coefficient table f_n (k_n of Table 1)
//   -> inverse FFT -> (group II: multiply by e^{+i pi j/M}) -> sample.
//
// The multiplier is complex-linear and maps real lines to real lines, so two
// real lines ride in one complex sequence (real and imaginary parts).
//
// Every phase is a loop "for t = tid; t < work; t += nthr" and touches only
// shared memory (`smem` pointers) and the global pointers it is given, so a
// CTA runs it with (threadIdx.x, blockDim.x) between barriers.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#ifdef __CUDA_ARCH__
#define PSTD_LDG(p) __ldg(p)
#else
#define PSTD_LDG(p) (*(p))
#endif
#define PSTD_HD __host__ __device__ __forceinline__

namespace pstd {

constexpr int kMaxPasses = 8;

// Radix schedule and tables of one length-L complex FFT.
struct FftPlan {
    int L;
    int npass;
    int radix[kMaxPasses];
    const float2* tw;       // tw[m] = exp(-2 pi i m / L), m < L   (FP64 -> FP32)
};

// One staggered derivative along one axis in one direction.
//
// kind 2 (convolution route, any N): the multiplier acting on the period-M
// extension is a circular (group I) or skew-circular (group II) convolution
// of length M = L with kernel h~[d] = sum_n f_n e^{2 pi i d n / L}
// (times e^{i pi d / L} for group II).  It is evaluated as the linear
// convolution of the extension with h~ through a power-of-two FFT of length
// M2 >= 2L - 1 (table H = FFT_M2(h~) / M2), folded back as
// y[pos] = y_lin[pos] + fold * y_lin[pos + L], fold = +1 (I) or -1 (II).
struct LineOp {
    int kind;               // 0: FFT route, 1: dense matrix route, 2: convolution route
    int N;                  // cells along the axis
    int L;                  // FFT length M = 2N
    int group2;             // 1: antiperiodic extension (ND, DN)
    int dir;                // 0: pressure nodes -> half-nodes, 1: half-nodes -> nodes
    int in_half, out_half;  // grid of the input / output: 0 nodes, 1 half-nodes
    int nin, nout;          // stored input / output line lengths
    int R2;                 // twice the right wall's position in cells: 2N (wall at a node),
                            // 2N - 1 (wall at mid-cell, Table 1 groups III / IV); the
                            // reflection about it maps node j to R2 - j, half-node m to R2 - 1 - m
    int in_lo;              // input on nodes: first stored node (0 or 1)
    int out_lo;             // output on nodes: first stored node (0 or 1)
    float s_right;          // sign of the input reflected about the right wall
                            // (pressure-like on nodes: +1 N, -1 D; velocity: -1 N, +1 D)
    const float2* f;        // L folded coefficients (complex)
    const float2* shift;    // group II: exp(-i pi j / L), j < L
    const float* dense;     // kind 1: nout x nin row-major operator
    int seqlen;             // buffer length of one sequence: L (kinds 0, 1) or M2 (kind 2)
    float fold;             // kind 2: +1 (group I) or -1 (group II)
    FftPlan fft;            // kinds 0 (length L) and 2 (length M2)
};

// Scalar arithmetic whose rounding is fixed by the source: each product,
// sum and fused multiply-add below is one IEEE operation that the compiler
// may neither merge with a neighbour into a fused multiply-add nor split, so a
// pass inlined into different kernels (the per-axis launches, the
// cooperative run) rounds identically.  Where a product feeds a sum, the
// fused form is written out (rfma), so nothing is lost against contraction.
PSTD_HD float rmul(float a, float b) {
#ifdef __CUDA_ARCH__
    return __fmul_rn(a, b);
#else
    return a * b;
#endif
}
PSTD_HD float radd(float a, float b) {
#ifdef __CUDA_ARCH__
    return __fadd_rn(a, b);
#else
    return a + b;
#endif
}
PSTD_HD float rsub(float a, float b) {
#ifdef __CUDA_ARCH__
    return __fsub_rn(a, b);
#else
    return a - b;
#endif
}
PSTD_HD float rfma(float a, float b, float c) {  // a * b + c, rounded once
#ifdef __CUDA_ARCH__
    return __fmaf_rn(a, b, c);
#else
    return fmaf(a, b, c);
#endif
}

PSTD_HD float2 cmul(float2 a, float2 b) {
    return make_float2(rfma(a.x, b.x, -rmul(a.y, b.y)), rfma(a.x, b.y, rmul(a.y, b.x)));
}
PSTD_HD float2 cmulc(float2 a, float2 b) {  // a * conj(b)
    return make_float2(rfma(a.x, b.x, rmul(a.y, b.y)), rfma(a.y, b.x, -rmul(a.x, b.y)));
}
PSTD_HD float2 cadd(float2 a, float2 b) { return make_float2(radd(a.x, b.x), radd(a.y, b.y)); }
PSTD_HD float2 csub(float2 a, float2 b) { return make_float2(rsub(a.x, b.x), rsub(a.y, b.y)); }
PSTD_HD float2 cscale(float2 a, float s) { return make_float2(rmul(a.x, s), rmul(a.y, s)); }
// a * s + b (real s), each component rounded once
PSTD_HD float2 cfma(float2 a, float s, float2 b) { return make_float2(rfma(a.x, s, b.x), rfma(a.y, s, b.y)); }
// multiply by sigma * i, sigma = -1 (forward) or +1 (inverse)
PSTD_HD float2 cmuli(float2 a, float sigma) { return make_float2(rmul(-sigma, a.y), rmul(sigma, a.x)); }

// ---- small DFTs: y_k = sum_q a_q exp(sigma 2 pi i q k / R) -----------------
PSTD_HD void dft2(float2* a) {
    float2 t = a[0];
    a[0] = cadd(t, a[1]);
    a[1] = csub(t, a[1]);
}
PSTD_HD void dft3(float2* a, float sigma) {
    const float c = -0.5f;
    const float s = 0.86602540378443864676f;  // sqrt(3)/2
    float2 t1 = cadd(a[1], a[2]);
    float2 t2 = cmuli(cscale(csub(a[1], a[2]), s), sigma);
    float2 m = cfma(t1, c, a[0]);
    a[0] = cadd(a[0], t1);
    a[1] = cadd(m, t2);
    a[2] = csub(m, t2);
}
PSTD_HD void dft4(float2* a, float sigma) {
    float2 s02 = cadd(a[0], a[2]), d02 = csub(a[0], a[2]);
    float2 s13 = cadd(a[1], a[3]), d13 = cmuli(csub(a[1], a[3]), sigma);
    a[0] = cadd(s02, s13);
    a[2] = csub(s02, s13);
    a[1] = cadd(d02, d13);
    a[3] = csub(d02, d13);
}
PSTD_HD void dft5(float2* a, float sigma) {
    const float c1 = 0.30901699437494742410f;   // cos(2 pi / 5)
    const float c2 = -0.80901699437494742410f;  // cos(4 pi / 5)
    const float s1 = 0.95105651629515357212f;   // sin(2 pi / 5)
    const float s2 = 0.58778525229247312917f;   // sin(4 pi / 5)
    float2 t1 = cadd(a[1], a[4]), d1 = csub(a[1], a[4]);
    float2 t2 = cadd(a[2], a[3]), d2 = csub(a[2], a[3]);
    float2 m1 = cadd(a[0], cfma(t1, c1, cscale(t2, c2)));
    float2 m2 = cadd(a[0], cfma(t1, c2, cscale(t2, c1)));
    float2 r1 = cmuli(cfma(d1, s1, cscale(d2, s2)), sigma);
    float2 r2 = cmuli(cfma(d1, s2, cscale(d2, -s1)), sigma);
    a[0] = cadd(a[0], cadd(t1, t2));
    a[1] = cadd(m1, r1);
    a[4] = csub(m1, r1);
    a[2] = cadd(m2, r2);
    a[3] = csub(m2, r2);
}
PSTD_HD void dft8(float2* a, float sigma) {
    float2 e[4] = {a[0], a[2], a[4], a[6]};
    float2 o[4] = {a[1], a[3], a[5], a[7]};
    dft4(e, sigma);
    dft4(o, sigma);
    const float h = 0.70710678118654752440f;  // sqrt(1/2)
    // w^k = exp(sigma 2 pi i k / 8)
    float2 w1 = make_float2(h, sigma * h);
    float2 w3 = make_float2(-h, sigma * h);
    float2 o1 = cmul(o[1], w1);
    float2 o2 = cmuli(o[2], sigma);
    float2 o3 = cmul(o[3], w3);
    a[0] = cadd(e[0], o[0]);
    a[4] = csub(e[0], o[0]);
    a[1] = cadd(e[1], o1);
    a[5] = csub(e[1], o1);
    a[2] = cadd(e[2], o2);
    a[6] = csub(e[2], o2);
    a[3] = cadd(e[3], o3);
    a[7] = csub(e[3], o3);
}

// One Stockham autosort pass of radix R over nseq sequences of length L.
// Input x in natural order of the previous passes (span Ns), output span Ns*R.
template <int R>
PSTD_HD void stockham_pass(const float2* src, float2* dst, int nseq, int L, int Ns,
                           const float2* tw, float sigma, int tid, int nthr) {
    const int LR = L / R;
    const int twstride = L / (Ns * R);
    const int total = nseq * LR;
    for (int t = tid; t < total; t += nthr) {
        const int s = t / LR;
        const int j = t - s * LR;
        const float2* x = src + (size_t)s * L;
        float2* y = dst + (size_t)s * L;
        float2 a[R];
#pragma unroll
        for (int k = 0; k < R; ++k) a[k] = x[j + k * LR];
        const int jm = j % Ns;
        if (jm != 0) {
#pragma unroll
            for (int k = 1; k < R; ++k) {
                float2 w = PSTD_LDG(&tw[jm * k * twstride]);
                w.y *= -sigma;  // table holds exp(-2 pi i m / L); conjugate for the inverse
                a[k] = cmul(a[k], w);
            }
        }
        if constexpr (R == 2) dft2(a);
        else if constexpr (R == 3) dft3(a, sigma);
        else if constexpr (R == 4) dft4(a, sigma);
        else if constexpr (R == 5) dft5(a, sigma);
        else dft8(a, sigma);
        const int idxD = (j - jm) * R + jm;
#pragma unroll
        for (int k = 0; k < R; ++k) y[idxD + k * Ns] = a[k];
    }
}

// Run pass `p` of the schedule (caller alternates buffers and barriers).
PSTD_HD void fft_pass(const FftPlan& P, int p, int& Ns, const float2* src, float2* dst,
                      int nseq, float sigma, int tid, int nthr) {
    const int R = P.radix[p];
    switch (R) {
        case 2: stockham_pass<2>(src, dst, nseq, P.L, Ns, P.tw, sigma, tid, nthr); break;
        case 3: stockham_pass<3>(src, dst, nseq, P.L, Ns, P.tw, sigma, tid, nthr); break;
        case 4: stockham_pass<4>(src, dst, nseq, P.L, Ns, P.tw, sigma, tid, nthr); break;
        case 5: stockham_pass<5>(src, dst, nseq, P.L, Ns, P.tw, sigma, tid, nthr); break;
        default: stockham_pass<8>(src, dst, nseq, P.L, Ns, P.tw, sigma, tid, nthr); break;
    }
    Ns *= R;
}

// ---- phases of one LineOp over G lines held in shared memory ---------------
//
// raw:   G lines of input, stride `rs` floats (line g at raw + g*rs)
// bufA/B: nseq = ceil(G/2) complex sequences of length L each

// Build the extension of line pairs (2s, 2s+1) from raw into buf (FFT route).
PSTD_HD void phase_extend(const LineOp& op, const float* raw, int rs, int G, float2* buf,
                          int tid, int nthr) {
    const int L = op.L, SL = op.seqlen;
    const int nseq = (G + 1) / 2;
    const int total = nseq * SL;
    for (int t = tid; t < total; t += nthr) {
        const int s = t / SL;
        const int j = t - s * SL;
        if (j >= L) {   // kind 2: zero padding of the linear convolution
            buf[(size_t)s * SL + j] = make_float2(0.0f, 0.0f);
            continue;
        }
        // position in the stored line and sign, or -1 for a zero
        int src;
        float sg;
        if (!op.in_half) {
            // input on nodes: node q (2 q <= R2) is stored at q - in_lo
            int q = j;
            sg = 1.0f;
            if (2 * j > op.R2) { q = op.R2 - j; sg = op.s_right; }
            src = q - op.in_lo;
            if (src < 0 || src >= op.nin) src = -1;
        } else {
            // input on half-nodes: m (2 m + 1 <= R2) stored at m; a half-node on
            // a mid-cell wall past the stored ones is a zero
            src = j;
            sg = 1.0f;
            if (2 * j + 1 > op.R2) { src = op.R2 - 1 - j; sg = op.s_right; }
            if (src >= op.nin) src = -1;
        }
        const int g0 = 2 * s, g1 = 2 * s + 1;
        float re = 0.0f, im = 0.0f;
        if (src >= 0) {
            re = sg * raw[(size_t)g0 * rs + src];
            if (g1 < G) im = sg * raw[(size_t)g1 * rs + src];
        }
        float2 v = make_float2(re, im);
        if (op.group2 && op.kind == 0) v = cmul(v, PSTD_LDG(&op.shift[j]));
        buf[(size_t)s * SL + j] = v;
    }
}

// Multiply every sequence by the coefficient table.
PSTD_HD void phase_multiply(const LineOp& op, float2* buf, int G, int tid, int nthr) {
    const int SL = op.seqlen;
    const int total = ((G + 1) / 2) * SL;
    for (int t = tid; t < total; t += nthr) {
        const int n = t % SL;
        buf[t] = cmul(buf[t], PSTD_LDG(&op.f[n]));
    }
}

// Dense route: y[2s + {0,1}] at output positions, written like the FFT result
// (sequence s, index pos) so that phase_value reads both routes alike.
PSTD_HD void phase_dense(const LineOp& op, const float* raw, int rs, int G, float2* buf,
                         int tid, int nthr) {
    const int nseq = (G + 1) / 2;
    const int total = nseq * op.nout;
    const int base = op.out_half ? 0 : op.out_lo;
    for (int t = tid; t < total; t += nthr) {
        const int s = t / op.nout;
        const int i = t - s * op.nout;
        const float* row = op.dense + (size_t)i * op.nin;
        const float* x0 = raw + (size_t)(2 * s) * rs;
        const bool two = 2 * s + 1 < G;
        const float* x1 = two ? raw + (size_t)(2 * s + 1) * rs : x0;
        float a0 = 0.0f, a1 = 0.0f;
        for (int j = 0; j < op.nin; ++j) {
            const float d = PSTD_LDG(&row[j]);
            a0 = fmaf(d, x0[j], a0);
            a1 = fmaf(d, x1[j], a1);
        }
        buf[(size_t)s * op.seqlen + base + i] = make_float2(a0, two ? a1 : 0.0f);
    }
}

// Output value of line g at stored output index i (after the inverse FFT).
PSTD_HD float op_value(const LineOp& op, const float2* buf, int g, int i) {
    const int pos = op.out_half ? i : i + op.out_lo;
    const float2* seq = buf + (size_t)(g >> 1) * op.seqlen;
    float2 v = seq[pos];
    if (op.kind == 0 && op.group2) v = cmulc(v, PSTD_LDG(&op.shift[pos]));
    if (op.kind == 2) v = cadd(v, cscale(seq[pos + op.L], op.fold));
    return (g & 1) ? v.y : v.x;
}

}  // namespace pstd
