// pstd_wcta.cuh -- axis passes on register FFTs (pstd_wfft.cuh).
//
// Each complex sequence carries a pair of real lines (real and imaginary
// parts) through one staggered derivative: symmetric-periodic extension
// (pre-twiddled for the antiperiodic group II), forward FFT, multiply by the
// folded coefficient table, inverse FFT, post-twiddle.  After the inverse FFT
// lane t holds positions t + T e of both lines, which is where it samples the
// output grid.
//
// Two layouts of the lines of an axis:
//  * contiguous (the last axis, stride 1): lanes read and write the lines in
//    global memory directly (consecutive lanes, consecutive words); warps are
//    independent and never meet at a block barrier.
//  * strided (stride `inner` > 1): a CTA owns a tile of G lines that are
//    adjacent in memory, loads the tile (p, u_a and the accumulator) into
//    shared memory with the line index fastest, computes, and stores it back
//    the same way, so every global access is a run of G consecutive words.
#pragma once

#include "pstd_wfft.cuh"

#ifndef PSTD_SYNCWARP
#ifdef __CUDA_ARCH__
#define PSTD_SYNCWARP() __syncwarp()
#else
#define PSTD_SYNCWARP() \
    do {                \
    } while (0)
#endif
#endif
#ifndef PSTD_SYNCCTA
#ifdef __CUDA_ARCH__
#define PSTD_SYNCCTA() __syncthreads()
#else
#define PSTD_SYNCCTA() \
    do {               \
    } while (0)
#endif
#endif

namespace pstd {

struct WAxis {
    int N, L, lp, lo, group2;
    float sR_p;              // sign of p reflected about the right wall (+1 N, -1 D)
    float sR_u;              // sign of u reflected about the right wall (-1 N, +1 D)
    const float2* tw;        // pass twiddles (wf::fill_pass_twiddles layout)
    const float2* shift;     // exp(-i pi j / L), j < L
    int64_t nlines;          // lines of this axis
    int64_t inner;           // stride of the axis
    int G;                   // strided layout: lines per tile (even)
    int seqs;                // sequences per CTA
};

struct WStep {
    WAxis ax;
    const float2* fP;        // -(dt/rho0) derivative coefficients, p -> u
    const float2* fU;        // -(dt rho0 c0^2) derivative coefficients, u -> p
    const float* p;
    float* u;
    const float* acc_in;
    float* acc_out;
};

struct WGrad {
    WAxis ax;
    int dir;                 // 0: p -> u, 1: u -> p
    const float2* f;
    const float* in;
    float* out;
    int accumulate;
};

namespace wk {

// Barrier among the lanes of one sequence (and, above a warp, the CTA).
template <class S>
PSTD_HD void seq_sync() {
    if constexpr (S::T > 32) PSTD_SYNCCTA();
    else PSTD_SYNCWARP();
}

template <class S, bool INV, int p = 0>
PSTD_HD void fft(float2 (&v)[S::E], int t, float2* sm, const float2* tw) {
    wf::pass_compute<S, p, INV>(v, t, tw);
    if constexpr (p + 1 < S::P) {
        wf::pass_scatter<S, p>(v, t, sm);
        seq_sync<S>();
        wf::gather<S>(v, t, sm);
        seq_sync<S>();
        fft<S, INV, p + 1>(v, t, sm, tw);
    }
}

// One staggered derivative of a line pair.  `src(i)` returns the pair's
// stored input at index i; on return v[e] holds the pair's output at
// extension position t + T e.  All lanes of the warp must call it together.
template <class S, int DIR, class Src>
PSTD_HD void derivative(float2 (&v)[S::E], int t, float2* sm, const WAxis& A, const float2* f,
                        Src&& src) {
    constexpr int T = S::T, E = S::E;
    const int N = A.N;
#pragma unroll
    for (int e = 0; e < E; ++e) {
        const int j = t + T * e;
        float2 val;
        if (DIR == 0) {
            const bool mirror = j > N;
            const int i = (mirror ? 2 * N - j : j) - A.lo;
            val = (i >= 0 && i < A.lp) ? src(i) : make_float2(0.0f, 0.0f);
            if (mirror) val = cscale(val, A.sR_p);
        } else {
            const bool mirror = j >= N;
            val = src(mirror ? 2 * N - 1 - j : j);
            if (mirror) val = cscale(val, A.sR_u);
        }
        if (A.group2) val = cmul(val, PSTD_LDG(&A.shift[j]));
        v[e] = val;
    }
    seq_sync<S>();   // the source may be this sequence's buffer
    fft<S, false>(v, t, sm, A.tw);
#pragma unroll
    for (int e = 0; e < E; ++e) v[e] = cmul(v[e], PSTD_LDG(&f[t + T * e]));
    fft<S, true>(v, t, sm, A.tw);
    if (A.group2) {
#pragma unroll
        for (int e = 0; e < E; ++e) v[e] = cmulc(v[e], PSTD_LDG(&A.shift[t + T * e]));
    }
}

// Lane geometry of a CTA: sequence (within the CTA) and lane within it.
template <class S>
PSTD_HD void lane_of(int tid, int& seq, int& t) {
    seq = tid / S::T;
    t = tid - seq * S::T;
}

// ---- contiguous layout ------------------------------------------------------
template <class S>
PSTD_HD void step_contig(const WStep& a, int64_t block, float2* smem, int tid) {
    constexpr int T = S::T, E = S::E;
    int sq, t;
    lane_of<S>(tid, sq, t);
    const WAxis& A = a.ax;
    const int64_t seq = block * A.seqs + sq;
    const int64_t la = 2 * seq, lb = 2 * seq + 1;
    const bool va = la < A.nlines, vb = lb < A.nlines;
    float2* sm = smem + (size_t)sq * wf::seq_words<S::L>();
    const int N = A.N, lp = A.lp;
    const float* pa = a.p + (va ? la : 0) * lp;
    const float* pb = a.p + (vb ? lb : 0) * lp;
    float2 v[E];
    derivative<S, 0>(v, t, sm, A, a.fP, [&](int i) {
        return make_float2(va ? pa[i] : 0.0f, vb ? pb[i] : 0.0f);
    });
    // u^{n+1/2} = u^{n-1/2} + f_P(p^n); the pair goes to the buffer for f_U
    float* ua = a.u + (va ? la : 0) * N;
    float* ub = a.u + (vb ? lb : 0) * N;
    seq_sync<S>();
#pragma unroll
    for (int e = 0; e < E; ++e) {
        const int m = t + T * e;
        if (m < N) {
            float2 w = make_float2(0.0f, 0.0f);
            if (va) { w.x = ua[m] + v[e].x; ua[m] = w.x; }
            if (vb) { w.y = ub[m] + v[e].y; ub[m] = w.y; }
            sm[m] = w;
        }
    }
    seq_sync<S>();
    derivative<S, 1>(v, t, sm, A, a.fU, [&](int m) { return sm[m]; });
    const float* ia = a.acc_in + (va ? la : 0) * lp;
    const float* ib = a.acc_in + (vb ? lb : 0) * lp;
    float* oa = a.acc_out + (va ? la : 0) * lp;
    float* ob = a.acc_out + (vb ? lb : 0) * lp;
#pragma unroll
    for (int e = 0; e < E; ++e) {
        const int i = t + T * e - A.lo;
        if (i >= 0 && i < lp) {
            if (va) oa[i] = ia[i] + v[e].x;
            if (vb) ob[i] = ib[i] + v[e].y;
        }
    }
}

template <class S>
PSTD_HD void grad_contig(const WGrad& a, int64_t block, float2* smem, int tid) {
    constexpr int T = S::T, E = S::E;
    int sq, t;
    lane_of<S>(tid, sq, t);
    const WAxis& A = a.ax;
    const int64_t seq = block * A.seqs + sq;
    const int64_t la = 2 * seq, lb = 2 * seq + 1;
    const bool va = la < A.nlines, vb = lb < A.nlines;
    float2* sm = smem + (size_t)sq * wf::seq_words<S::L>();
    const int nin = a.dir == 0 ? A.lp : A.N;
    const int nout = a.dir == 0 ? A.N : A.lp;
    const float* xa = a.in + (va ? la : 0) * nin;
    const float* xb = a.in + (vb ? lb : 0) * nin;
    float2 v[E];
    auto src = [&](int i) { return make_float2(va ? xa[i] : 0.0f, vb ? xb[i] : 0.0f); };
    if (a.dir == 0) derivative<S, 0>(v, t, sm, A, a.f, src);
    else derivative<S, 1>(v, t, sm, A, a.f, src);
    float* oa = a.out + (va ? la : 0) * nout;
    float* ob = a.out + (vb ? lb : 0) * nout;
    const int off = a.dir == 0 ? 0 : A.lo;
#pragma unroll
    for (int e = 0; e < E; ++e) {
        const int i = t + T * e - off;
        if (i >= 0 && i < nout) {
            if (va) oa[i] = a.accumulate ? oa[i] + v[e].x : v[e].x;
            if (vb) ob[i] = a.accumulate ? ob[i] + v[e].y : v[e].y;
        }
    }
}

// ---- strided layout ---------------------------------------------------------
// Tile `block`: outer block o, first inner index i0, Gv valid lines.
PSTD_HD void tile_of(const WAxis& A, int64_t block, int64_t& o, int64_t& i0, int& Gv) {
    const int64_t per = (A.inner + A.G - 1) / A.G;
    o = block / per;
    i0 = (block - o * per) * A.G;
    const int64_t left = A.inner - i0;
    Gv = (int)(left < A.G ? left : A.G);
}

// Row stride in shared memory for a line of `len` words (odd: conflict-free
// transposed staging).
PSTD_HD int row_stride(int len) { return len | 1; }

PSTD_HD void tile_load(const float* f, int len, const WAxis& A, int64_t o, int64_t i0, int Gv,
                       float* raw, int tid, int nthr) {
    const int rs = row_stride(len);
    const int64_t base = o * (int64_t)len * A.inner + i0;
    const int total = len * Gv;
    for (int idx = tid; idx < total; idx += nthr) {
        const int pos = idx / Gv, g = idx - pos * Gv;
        raw[g * rs + pos] = f[base + (int64_t)pos * A.inner + g];
    }
}

PSTD_HD void tile_store(float* f, int len, const WAxis& A, int64_t o, int64_t i0, int Gv,
                        const float* raw, int tid, int nthr) {
    const int rs = row_stride(len);
    const int64_t base = o * (int64_t)len * A.inner + i0;
    const int total = len * Gv;
    for (int idx = tid; idx < total; idx += nthr) {
        const int pos = idx / Gv, g = idx - pos * Gv;
        f[base + (int64_t)pos * A.inner + g] = raw[g * rs + pos];
    }
}

// shared memory of a strided step tile, in floats
PSTD_HD size_t strided_step_floats(const WAxis& A, int seq_words, bool separate_acc) {
    const size_t fft = (size_t)A.seqs * seq_words * 2;
    const size_t p = (size_t)A.G * row_stride(A.lp);
    const size_t u = (size_t)A.G * row_stride(A.N);
    return fft + p + u + (separate_acc ? p : 0);
}

template <class S>
PSTD_HD void step_strided(const WStep& a, int64_t block, float2* smem, int tid, int nthr) {
    constexpr int T = S::T, E = S::E;
    const WAxis& A = a.ax;
    int64_t o, i0;
    int Gv;
    tile_of(A, block, o, i0, Gv);
    const int N = A.N, lp = A.lp;
    const bool sep = a.acc_in != a.p;
    float* rawP = (float*)(smem + (size_t)A.seqs * wf::seq_words<S::L>());
    float* rawU = rawP + (size_t)A.G * row_stride(lp);
    float* rawA = sep ? rawU + (size_t)A.G * row_stride(N) : rawP;
    tile_load(a.p, lp, A, o, i0, Gv, rawP, tid, nthr);
    tile_load(a.u, N, A, o, i0, Gv, rawU, tid, nthr);
    if (sep) tile_load(a.acc_in, lp, A, o, i0, Gv, rawA, tid, nthr);
    PSTD_SYNCCTA();
    int sq, t;
    lane_of<S>(tid, sq, t);
    if (sq < A.seqs) {
        const int ga = 2 * sq, gb = 2 * sq + 1;
        const bool va = ga < Gv, vb = gb < Gv;
        float2* sm = smem + (size_t)sq * wf::seq_words<S::L>();
        const float* pa = rawP + (va ? ga : 0) * row_stride(lp);
        const float* pb = rawP + (vb ? gb : 0) * row_stride(lp);
        float2 v[E];
        derivative<S, 0>(v, t, sm, A, a.fP, [&](int i) {
            return make_float2(va ? pa[i] : 0.0f, vb ? pb[i] : 0.0f);
        });
        float* ua = rawU + (va ? ga : 0) * row_stride(N);
        float* ub = rawU + (vb ? gb : 0) * row_stride(N);
        seq_sync<S>();
#pragma unroll
        for (int e = 0; e < E; ++e) {
            const int m = t + T * e;
            if (m < N) {
                if (va) ua[m] += v[e].x;
                if (vb) ub[m] += v[e].y;
            }
        }
        seq_sync<S>();
        derivative<S, 1>(v, t, sm, A, a.fU, [&](int m) {
            return make_float2(va ? ua[m] : 0.0f, vb ? ub[m] : 0.0f);
        });
        float* aa = rawA + (va ? ga : 0) * row_stride(lp);
        float* ab = rawA + (vb ? gb : 0) * row_stride(lp);
        seq_sync<S>();
#pragma unroll
        for (int e = 0; e < E; ++e) {
            const int i = t + T * e - A.lo;
            if (i >= 0 && i < lp) {
                if (va) aa[i] += v[e].x;
                if (vb) ab[i] += v[e].y;
            }
        }
    }
    PSTD_SYNCCTA();
    tile_store(a.u, N, A, o, i0, Gv, rawU, tid, nthr);
    tile_store(a.acc_out, lp, A, o, i0, Gv, rawA, tid, nthr);
}

template <class S>
PSTD_HD void grad_strided(const WGrad& a, int64_t block, float2* smem, int tid, int nthr) {
    constexpr int T = S::T, E = S::E;
    const WAxis& A = a.ax;
    int64_t o, i0;
    int Gv;
    tile_of(A, block, o, i0, Gv);
    const int nin = a.dir == 0 ? A.lp : A.N;
    const int nout = a.dir == 0 ? A.N : A.lp;
    float* rawI = (float*)(smem + (size_t)A.seqs * wf::seq_words<S::L>());
    float* rawO = rawI + (size_t)A.G * row_stride(nin);
    tile_load(a.in, nin, A, o, i0, Gv, rawI, tid, nthr);
    if (a.accumulate) tile_load(a.out, nout, A, o, i0, Gv, rawO, tid, nthr);
    PSTD_SYNCCTA();
    int sq, t;
    lane_of<S>(tid, sq, t);
    if (sq < A.seqs) {
        const int ga = 2 * sq, gb = 2 * sq + 1;
        const bool va = ga < Gv, vb = gb < Gv;
        float2* sm = smem + (size_t)sq * wf::seq_words<S::L>();
        const float* xa = rawI + (va ? ga : 0) * row_stride(nin);
        const float* xb = rawI + (vb ? gb : 0) * row_stride(nin);
        float2 v[E];
        auto src = [&](int i) { return make_float2(va ? xa[i] : 0.0f, vb ? xb[i] : 0.0f); };
        if (a.dir == 0) derivative<S, 0>(v, t, sm, A, a.f, src);
        else derivative<S, 1>(v, t, sm, A, a.f, src);
        float* oa = rawO + (va ? ga : 0) * row_stride(nout);
        float* ob = rawO + (vb ? gb : 0) * row_stride(nout);
        const int off = a.dir == 0 ? 0 : A.lo;
#pragma unroll
        for (int e = 0; e < E; ++e) {
            const int i = t + T * e - off;
            if (i >= 0 && i < nout) {
                if (va) oa[i] = a.accumulate ? oa[i] + v[e].x : v[e].x;
                if (vb) ob[i] = a.accumulate ? ob[i] + v[e].y : v[e].y;
            }
        }
    }
    PSTD_SYNCCTA();
    tile_store(a.out, nout, A, o, i0, Gv, rawO, tid, nthr);
}

}  // namespace wk
}  // namespace pstd
