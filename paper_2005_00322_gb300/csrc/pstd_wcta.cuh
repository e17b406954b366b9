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

#include <type_traits>

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

// Asynchronous global -> shared copies (cp.async): every copy of a CTA is in
// flight at once, and no register holds the data on the way.
PSTD_HD void async_copy16(void* sdst, const void* gsrc) {
#ifdef __CUDA_ARCH__
    const unsigned s = (unsigned)__cvta_generic_to_shared(sdst);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(s), "l"(gsrc) : "memory");
#else
    const float4* a = (const float4*)gsrc;
    *(float4*)sdst = *a;
#endif
}
PSTD_HD void async_copy4(void* sdst, const void* gsrc) {
#ifdef __CUDA_ARCH__
    const unsigned s = (unsigned)__cvta_generic_to_shared(sdst);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(s), "l"(gsrc) : "memory");
#else
    *(float*)sdst = *(const float*)gsrc;
#endif
}
// Programmatic dependent launch: a pass launched with the programmatic-
// serialisation attribute may start while the previous pass drains; it loads
// its constant tables first and waits here before touching any field.
PSTD_HD void pdl_wait() {
#ifdef __CUDA_ARCH__
    asm volatile("griddepcontrol.wait;\n" ::: "memory");
#endif
}
// Let the next pass be scheduled (called once this CTA's work is done).
PSTD_HD void pdl_trigger() {
#ifdef __CUDA_ARCH__
    asm volatile("griddepcontrol.launch_dependents;\n" ::: "memory");
#endif
}

// Wait for this thread's copies; a CTA barrier must follow before others read.
PSTD_HD void async_wait_all() {
#ifdef __CUDA_ARCH__
    asm volatile("cp.async.wait_all;\n" ::: "memory");
#endif
}

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

// Table access of one derivative.  The throughput schedules read the
// (shared-memory staged) tables directly; the latency schedules first copy
// the lane's slice of every table into registers, so that all table loads of
// a derivative are in flight together with the line loads.
// f0 / f1: coefficient tables of direction 0 (p -> u) and 1 (u -> p).
template <class S>
struct TablesDirect {
    const float2* tw;
    const float2* f0;
    const float2* f1;
    const float2* shift;
    int t;
    PSTD_HD float2 twid(int i) const { return tw[i * S::T + t]; }
    template <int W>
    PSTD_HD float2 coef(int e) const { return (W ? f1 : f0)[t + S::T * e]; }
    PSTD_HD float2 sh(int e) const { return shift[t + S::T * e]; }
};
template <class S>
struct TablesInRegs {
    const float2* tw;
    const float2* f0;
    const float2* f1;
    const float2* shift;
    int t;
    float2 rtw[wf::tw_per_lane<S>() > 0 ? wf::tw_per_lane<S>() : 1];
    float2 rf0[S::E], rf1[S::E], rsh[S::E];
    PSTD_HD void load(bool group2) {
#pragma unroll
        for (int i = 0; i < wf::tw_per_lane<S>(); ++i) rtw[i] = tw[i * S::T + t];
#pragma unroll
        for (int e = 0; e < S::E; ++e) {
            rf0[e] = f0 ? f0[t + S::T * e] : make_float2(0.0f, 0.0f);
            rf1[e] = f1 ? f1[t + S::T * e] : make_float2(0.0f, 0.0f);
            rsh[e] = group2 ? shift[t + S::T * e] : make_float2(1.0f, 0.0f);
        }
    }
    PSTD_HD float2 twid(int i) const { return rtw[i]; }
    template <int W>
    PSTD_HD float2 coef(int e) const { return W ? rf1[e] : rf0[e]; }
    PSTD_HD float2 sh(int e) const { return rsh[e]; }
};

template <class S, bool INV, int p = 0, class Tab>
PSTD_HD void fft(float2 (&v)[S::E], int t, float2* sm, const Tab& tab) {
    wf::pass_compute<S, p, INV>(v, [&](int i) { return tab.twid(i); });
    if constexpr (p + 1 < S::P) {
        wf::pass_scatter<S, p>(v, t, sm);
        seq_sync<S>();
        wf::gather<S>(v, t, sm);
        seq_sync<S>();
        fft<S, INV, p + 1>(v, t, sm, tab);
    }
}

// One staggered derivative of a line pair.  `src(i)` returns the pair's
// stored input at index i; on return v[e] holds the pair's output at
// extension position t + T e.  All lanes of the sequence must call it.
template <class S, int DIR, class Tab, class Src>
PSTD_HD void derivative(float2 (&v)[S::E], int t, float2* sm, const WAxis& A, const Tab& tab,
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
        if (A.group2) val = cmul(val, tab.sh(e));
        v[e] = val;
    }
    seq_sync<S>();   // the source may be this sequence's buffer
    fft<S, false>(v, t, sm, tab);
#pragma unroll
    for (int e = 0; e < E; ++e) v[e] = cmul(v[e], tab.template coef<DIR>(e));
    fft<S, true>(v, t, sm, tab);
    if (A.group2) {
#pragma unroll
        for (int e = 0; e < E; ++e) v[e] = cmulc(v[e], tab.sh(e));
    }
}

// Tables of one derivative for schedule S (registers for the latency
// schedules, direct access otherwise).
template <class S>
using TablesOf = typename std::conditional<S::V >= 1, TablesInRegs<S>, TablesDirect<S>>::type;

template <class S>
PSTD_HD TablesOf<S> tables(const WAxis& A, const float2* f0, const float2* f1, int t) {
    TablesOf<S> tb;
    tb.tw = A.tw;
    tb.f0 = f0;
    tb.f1 = f1;
    tb.shift = A.shift;
    tb.t = t;
    if constexpr (S::V >= 1) tb.load(A.group2 != 0);
    return tb;
}

// Lane geometry of a CTA: sequence (within the CTA) and lane within it.
template <class S>
PSTD_HD void lane_of(int tid, int& seq, int& t) {
    seq = tid / S::T;
    t = tid - seq * S::T;
}

// Copy the axis tables into shared memory at `dst` (CTA-cooperative, 16-byte
// cp.async chunks) and point A / f1 / f2 at the copies; returns the first free
// word.  Table lengths are even (the host pads the pass twiddles), so every
// chunk holds two complex words.  The caller waits (async_wait_all) and
// places a CTA barrier before the tables are read.
template <class S>
PSTD_HD float2* stage_tables(WAxis& A, const float2*& f1, const float2*& f2, float2* dst, int tid,
                             int nthr) {
    if constexpr (S::V >= 1) return dst;   // latency schedules keep tables in registers
    constexpr int ntw = (wf::tw_total<S>() + 1) & ~1;
    constexpr int L = S::L;
    float2* p = dst;
    for (int i = 2 * tid; i < ntw; i += 2 * nthr) async_copy16(p + i, A.tw + i);
    A.tw = p;
    p += ntw;
    if (A.group2) {
        for (int i = 2 * tid; i < L; i += 2 * nthr) async_copy16(p + i, A.shift + i);
        A.shift = p;
        p += L;
    }
    for (int i = 2 * tid; i < L; i += 2 * nthr) async_copy16(p + i, f1 + i);
    f1 = p;
    p += L;
    if (f2) {
        for (int i = 2 * tid; i < L; i += 2 * nthr) async_copy16(p + i, f2 + i);
        f2 = p;
        p += L;
    }
    return p;
}

// ---- contiguous layout ------------------------------------------------------
template <class S>
PSTD_HD void step_contig(const WStep& a, int64_t block, float2* smem, int tid, int nthr) {
    constexpr int T = S::T, E = S::E;
    int sq, t;
    lane_of<S>(tid, sq, t);
    WAxis A = a.ax;
    const float2* fP = a.fP;
    const float2* fU = a.fU;
    float2* bufs = stage_tables<S>(A, fP, fU, smem, tid, nthr);
    const auto tab = tables<S>(A, fP, fU, t);
    pdl_wait();
    const int64_t seq = block * A.seqs + sq;
    const int64_t la = 2 * seq, lb = 2 * seq + 1;
    const bool va = la < A.nlines, vb = lb < A.nlines;
    float2* sm = bufs + (size_t)sq * wf::seq_words<S::L>();
    const int N = A.N, lp = A.lp;
    // prefetch u^{n-1/2} and the accumulator at this lane's output positions
    float* ua = a.u + (va ? la : 0) * N;
    float* ub = a.u + (vb ? lb : 0) * N;
    const float* ia = a.acc_in + (va ? la : 0) * lp;
    const float* ib = a.acc_in + (vb ? lb : 0) * lp;
    float2 uo[E], ao[E];
#pragma unroll
    for (int e = 0; e < E; ++e) {
        const int m = t + T * e;
        const int i = m - A.lo;
        uo[e] = make_float2(va && m < N ? ua[m] : 0.0f, vb && m < N ? ub[m] : 0.0f);
        const bool ok = i >= 0 && i < lp;
        ao[e] = make_float2(va && ok ? ia[i] : 0.0f, vb && ok ? ib[i] : 0.0f);
    }
    async_wait_all();
    PSTD_SYNCCTA();
    const float* pa = a.p + (va ? la : 0) * lp;
    const float* pb = a.p + (vb ? lb : 0) * lp;
    float2 v[E];
    derivative<S, 0>(v, t, sm, A, tab, [&](int i) {
        return make_float2(va ? pa[i] : 0.0f, vb ? pb[i] : 0.0f);
    });
    // u^{n+1/2} = u^{n-1/2} + f_P(p^n); the pair goes to the buffer for f_U
    seq_sync<S>();
#pragma unroll
    for (int e = 0; e < E; ++e) {
        const int m = t + T * e;
        if (m < N) {
            const float2 w = cadd(uo[e], v[e]);
            if (va) ua[m] = w.x;
            if (vb) ub[m] = w.y;
            sm[m] = w;
        }
    }
    seq_sync<S>();
    derivative<S, 1>(v, t, sm, A, tab, [&](int m) { return sm[m]; });
    float* oa = a.acc_out + (va ? la : 0) * lp;
    float* ob = a.acc_out + (vb ? lb : 0) * lp;
#pragma unroll
    for (int e = 0; e < E; ++e) {
        const int i = t + T * e - A.lo;
        if (i >= 0 && i < lp) {
            if (va) oa[i] = ao[e].x + v[e].x;
            if (vb) ob[i] = ao[e].y + v[e].y;
        }
    }
    pdl_trigger();
}

template <class S>
PSTD_HD void grad_contig(const WGrad& a, int64_t block, float2* smem, int tid, int nthr) {
    constexpr int T = S::T, E = S::E;
    int sq, t;
    lane_of<S>(tid, sq, t);
    WAxis A = a.ax;
    const float2* f = a.f;
    const float2* none = nullptr;
    float2* bufs = stage_tables<S>(A, f, none, smem, tid, nthr);
    const auto tab = tables<S>(A, a.dir == 0 ? f : nullptr, a.dir == 0 ? nullptr : f, t);
    async_wait_all();
    PSTD_SYNCCTA();
    pdl_wait();
    const int64_t seq = block * A.seqs + sq;
    const int64_t la = 2 * seq, lb = 2 * seq + 1;
    const bool va = la < A.nlines, vb = lb < A.nlines;
    float2* sm = bufs + (size_t)sq * wf::seq_words<S::L>();
    const int nin = a.dir == 0 ? A.lp : A.N;
    const int nout = a.dir == 0 ? A.N : A.lp;
    const float* xa = a.in + (va ? la : 0) * nin;
    const float* xb = a.in + (vb ? lb : 0) * nin;
    float2 v[E];
    auto src = [&](int i) { return make_float2(va ? xa[i] : 0.0f, vb ? xb[i] : 0.0f); };
    if (a.dir == 0) derivative<S, 0>(v, t, sm, A, tab, src);
    else derivative<S, 1>(v, t, sm, A, tab, src);
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

// G is a power of two: item idx is (position idx >> log2 G, line idx & (G-1)).
PSTD_HD int log2_pow2(int G) {
    int s = 0;
    while ((1 << s) < G) ++s;
    return s;
}

PSTD_HD void tile_load(const float* f, int len, const WAxis& A, int64_t o, int64_t i0, int Gv,
                       float* raw, int tid, int nthr) {
    const int rs = row_stride(len);
    const int gs = log2_pow2(A.G), gm = A.G - 1;
    const float* base = f + o * (int64_t)len * A.inner + i0;
    const int total = len << gs;
    for (int idx = tid; idx < total; idx += nthr) {
        const int pos = idx >> gs, g = idx & gm;
        if (g < Gv) async_copy4(&raw[g * rs + pos], &base[(int64_t)pos * A.inner + g]);
    }
}

PSTD_HD void tile_store(float* f, int len, const WAxis& A, int64_t o, int64_t i0, int Gv,
                        const float* raw, int tid, int nthr) {
    const int rs = row_stride(len);
    const int gs = log2_pow2(A.G), gm = A.G - 1;
    float* base = f + o * (int64_t)len * A.inner + i0;
    const int total = len << gs;
    for (int idx = tid; idx < total; idx += nthr) {
        const int pos = idx >> gs, g = idx & gm;
        if (g < Gv) base[(int64_t)pos * A.inner + g] = raw[g * rs + pos];
    }
}

// shared memory of a strided step tile (without the staged tables), in floats
PSTD_HD size_t strided_step_floats(const WAxis& A, int seq_words, bool separate_acc) {
    const size_t fft = (size_t)A.seqs * seq_words * 2;
    const size_t p = (size_t)A.G * row_stride(A.lp);
    const size_t u = (size_t)A.G * row_stride(A.N);
    return fft + p + u + (separate_acc ? p : 0);
}

template <class S>
PSTD_HD void step_strided(const WStep& a, int64_t block, float2* smem0, int tid, int nthr) {
    constexpr int T = S::T, E = S::E;
    WAxis A = a.ax;
    const float2* fP = a.fP;
    const float2* fU = a.fU;
    float2* smem = stage_tables<S>(A, fP, fU, smem0, tid, nthr);
    int sq, t;
    lane_of<S>(tid, sq, t);
    const auto tab = tables<S>(A, fP, fU, t);
    int64_t o, i0;
    int Gv;
    tile_of(A, block, o, i0, Gv);
    const int N = A.N, lp = A.lp;
    const bool sep = a.acc_in != a.p;
    float* rawP = (float*)(smem + (size_t)A.seqs * wf::seq_words<S::L>());
    float* rawU = rawP + (size_t)A.G * row_stride(lp);
    float* rawA = sep ? rawU + (size_t)A.G * row_stride(N) : rawP;
    pdl_wait();
    tile_load(a.p, lp, A, o, i0, Gv, rawP, tid, nthr);
    tile_load(a.u, N, A, o, i0, Gv, rawU, tid, nthr);
    if (sep) tile_load(a.acc_in, lp, A, o, i0, Gv, rawA, tid, nthr);
    async_wait_all();
    PSTD_SYNCCTA();
    if (sq < A.seqs) {
        const int ga = 2 * sq, gb = 2 * sq + 1;
        const bool va = ga < Gv, vb = gb < Gv;
        float2* sm = smem + (size_t)sq * wf::seq_words<S::L>();
        const float* pa = rawP + (va ? ga : 0) * row_stride(lp);
        const float* pb = rawP + (vb ? gb : 0) * row_stride(lp);
        float2 v[E];
        derivative<S, 0>(v, t, sm, A, tab, [&](int i) {
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
        derivative<S, 1>(v, t, sm, A, tab, [&](int m) {
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
    pdl_trigger();
}

template <class S>
PSTD_HD void grad_strided(const WGrad& a, int64_t block, float2* smem0, int tid, int nthr) {
    constexpr int T = S::T, E = S::E;
    WAxis A = a.ax;
    const float2* f = a.f;
    const float2* none = nullptr;
    float2* smem = stage_tables<S>(A, f, none, smem0, tid, nthr);
    int sq, t;
    lane_of<S>(tid, sq, t);
    const auto tab = tables<S>(A, a.dir == 0 ? f : nullptr, a.dir == 0 ? nullptr : f, t);
    int64_t o, i0;
    int Gv;
    tile_of(A, block, o, i0, Gv);
    const int nin = a.dir == 0 ? A.lp : A.N;
    const int nout = a.dir == 0 ? A.N : A.lp;
    float* rawI = (float*)(smem + (size_t)A.seqs * wf::seq_words<S::L>());
    float* rawO = rawI + (size_t)A.G * row_stride(nin);
    pdl_wait();
    tile_load(a.in, nin, A, o, i0, Gv, rawI, tid, nthr);
    if (a.accumulate) tile_load(a.out, nout, A, o, i0, Gv, rawO, tid, nthr);
    async_wait_all();
    PSTD_SYNCCTA();
    if (sq < A.seqs) {
        const int ga = 2 * sq, gb = 2 * sq + 1;
        const bool va = ga < Gv, vb = gb < Gv;
        float2* sm = smem + (size_t)sq * wf::seq_words<S::L>();
        const float* xa = rawI + (va ? ga : 0) * row_stride(nin);
        const float* xb = rawI + (vb ? gb : 0) * row_stride(nin);
        float2 v[E];
        auto src = [&](int i) { return make_float2(va ? xa[i] : 0.0f, vb ? xb[i] : 0.0f); };
        if (a.dir == 0) derivative<S, 0>(v, t, sm, A, tab, src);
        else derivative<S, 1>(v, t, sm, A, tab, src);
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
