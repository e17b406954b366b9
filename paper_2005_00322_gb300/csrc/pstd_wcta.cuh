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
    const float2* sym;       // per bin: factor on the stored bin of the velocity spectrum (see spec_slot)
    float* ph;               // velocity spectrum of the missing partner of an unpaired line
                             // (N floats each: contiguous 1, strided one per outer block), or null
};

// One leapfrog pass of an axis.  The velocity u_a is held as its spectrum:
// the FFT of its (pre-twiddled) symmetric-periodic extension divided by L,
// i.e. T2 u in bin form, one stored value per velocity sample (spec_slot).
// The pass transforms p forward, updates the spectrum with the p -> u
// coefficients, and transforms the u -> p coefficients times the spectrum
// back onto the nodes: one forward and one inverse FFT per line pair.
struct WStep {
    WAxis ax;
    const float2* fP;        // -(dt/rho0) derivative coefficients, p -> u
    const float2* fU;        // L times the -(dt rho0 c0^2) derivative coefficients, u -> p
    const float* p;
    float* u;
    const float* acc_in;
    float* acc_out;
};

struct WGrad {
    WAxis ax;
    int dir;                 // 0: p -> u, 1: u -> p, 2: u -> its spectrum, 3: spectrum -> u,
                             // 4: p -> p (the second-order form's composed operator)
    const float2* f;
    const float* in;
    float* out;
    int accumulate;
    float scale;             // dir 2: 1 / L
    float* pout = nullptr;   // dir 4: also write in + (the new out) here (may be `in`)
};

// A line with no partner (odd line count) still has a complex spectrum:
// the partner's half of its 2N reals lives in WAxis::ph (the "phantom"
// partner line), read and written like a real partner's velocity slots.

// Stored slot of bin k (0 <= k < L) of a velocity line-pair spectrum, and
// whether bin k is the slot's owner (the bin whose value the slot holds).
// The extension of u is mirrored about the right wall with sign sR_u, so the
// packed spectrum obeys, for group I, U[L-k] = sR_u w^k U[k] (w = e^{-2 pi i/L}),
// which forces U[0] = 0 (sR_u = -1) or U[N] = 0 (sR_u = +1); for group II
// (pre-twiddled) U[L-1-k] = sR_u e^{i pi (L-1)/L} w^k U[k].  So N bins carry
// the line pair, stored as N complex values = the pair's 2N real samples:
// slot k < N holds bin k, except that slot 0 holds bin N when bin 0 vanishes.
// A periodic axis (L == N) stores every bin.  Non-owner bins are the slot's
// value times WAxis::sym[k] (0 for a vanishing bin).
PSTD_HD int spec_slot(const WAxis& A, int k, bool& owner) {
    const int N = A.N, L = A.L;
    if (L == N) {
        owner = true;
        return k;
    }
    if (A.group2) {
        owner = k < N;
        return k < N ? k : L - 1 - k;
    }
    if (k < N) {
        owner = k > 0 || A.sR_u > 0.0f;
        return k;
    }
    owner = k == N && A.sR_u < 0.0f;
    return k == N ? 0 : L - k;
}

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
    const float2* sy;
    int t;
    PSTD_HD float2 twid(int i) const { return tw[i * S::T + t]; }
    template <int W>
    PSTD_HD float2 coef(int e) const { return (W ? f1 : f0)[t + S::T * e]; }
    PSTD_HD float2 sh(int e) const { return shift[t + S::T * e]; }
    PSTD_HD float2 sym(int e) const { return sy[t + S::T * e]; }
};
template <class S>
struct TablesInRegs {
    const float2* tw;
    const float2* f0;
    const float2* f1;
    const float2* shift;
    const float2* sy;
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
    // symmetry factors are needed for half the bins once per pass: read them
    // from the (L1-cached, global) table rather than holding them in registers
    PSTD_HD float2 sym(int e) const { return sy[t + S::T * e]; }
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

// Schedules whose lanes hold at most 8 elements keep their tables in
// registers (except V = 4 and 5, which trade them for occupancy); the others
// stage them in shared memory, except V = 5, which reads them from global
// memory (L1-cached) where they are.
template <class S>
constexpr bool reg_tables() {
    return S::V >= 1 && S::V != 4 && S::V != 5 && S::E <= 8;
}
template <class S>
constexpr bool staged_tables() {
    return !reg_tables<S>() && S::V != 5;
}

// Schedules 3, 4 and 5 serve only walled axes, L = 2 N: fixing N and L in
// the pass's copy of the axis turns the index logic of the extension and of
// the spectrum slots (bin k = t + T e against N) into compile-time branches
// on e.
template <class S>
PSTD_HD void fix_extent(WAxis& A) {
    if constexpr (S::V >= 3) {
        A.L = S::L;
        A.N = S::L / 2;
    }
}

// Tables of one derivative for schedule S (registers for the latency
// schedules, direct access otherwise).
template <class S>
using TablesOf = typename std::conditional<reg_tables<S>(), TablesInRegs<S>, TablesDirect<S>>::type;

template <class S>
PSTD_HD TablesOf<S> tables(const WAxis& A, const float2* f0, const float2* f1, int t) {
    TablesOf<S> tb;
    tb.tw = A.tw;
    tb.f0 = f0;
    tb.f1 = f1;
    tb.shift = A.shift;
    tb.sy = A.sym;
    tb.t = t;
    if constexpr (reg_tables<S>()) tb.load(A.group2 != 0);
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
    if constexpr (!staged_tables<S>()) return dst;   // tables in registers or read in place
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
    if (f1) {
        for (int i = 2 * tid; i < L; i += 2 * nthr) async_copy16(p + i, f1 + i);
        f1 = p;
        p += L;
    }
    if (A.sym) {
        for (int i = 2 * tid; i < L; i += 2 * nthr) async_copy16(p + i, A.sym + i);
        A.sym = p;
        p += L;
    }
    if (f2) {
        for (int i = 2 * tid; i < L; i += 2 * nthr) async_copy16(p + i, f2 + i);
        f2 = p;
        p += L;
    }
    return p;
}

// Load the pressure pair's symmetric-periodic extension at this lane's
// positions t + T e (pre-twiddled for group II).
template <class S, class Tab, class Src>
PSTD_HD void load_p_ext(float2 (&v)[S::E], int t, const WAxis& A, const Tab& tab, Src&& src) {
#pragma unroll
    for (int e = 0; e < S::E; ++e) {
        const int j = t + S::T * e;
        const bool mirror = j > A.N;
        const int i = (mirror ? 2 * A.N - j : j) - A.lo;
        float2 val = (i >= 0 && i < A.lp) ? src(i) : make_float2(0.0f, 0.0f);
        if (mirror) val = cscale(val, A.sR_p);
        if (A.group2) val = cmul(val, tab.sh(e));
        v[e] = val;
    }
}

// The velocity spectrum at this lane's bins t + T e, from the stored slots.
template <class S, class Tab, class Ld>
PSTD_HD void load_spectrum(float2 (&w)[S::E], int t, const WAxis& A, const Tab& tab, Ld&& ld) {
#pragma unroll
    for (int e = 0; e < S::E; ++e) {
        bool own;
        const int s = spec_slot(A, t + S::T * e, own);
        w[e] = own ? ld(s) : cmul(tab.sym(e), ld(s));
    }
}

// Second half of a pass on a line pair in registers.  On entry v holds the
// pressure spectrum V and w the velocity spectrum at this lane's bins; the
// spectrum is updated, w += fP V (stored back through `st` for the owner
// bins), and the inverse FFT of fU w leaves the pressure contribution at
// extension positions t + T e in v.
template <class S, class Tab, class St>
PSTD_HD void update_and_inverse(float2 (&v)[S::E], const float2 (&w)[S::E], int t, float2* sm, const WAxis& A,
                                const Tab& tab, St&& st) {
#pragma unroll
    for (int e = 0; e < S::E; ++e) {
        const float2 wn = cadd(w[e], cmul(v[e], tab.template coef<0>(e)));
        bool own;
        const int s = spec_slot(A, t + S::T * e, own);
        if (own) st(s, wn);
        v[e] = cmul(wn, tab.template coef<1>(e));
    }
    fft<S, true>(v, t, sm, tab);
    if (A.group2) {
#pragma unroll
        for (int e = 0; e < S::E; ++e) v[e] = cmulc(v[e], tab.sh(e));
    }
}

// ---- contiguous layout ------------------------------------------------------
// Shared memory of a contiguous step pass beyond its FFT buffers: each
// sequence's two velocity-spectrum lines and two accumulator lines, staged
// by the lean form (floats).
PSTD_HD size_t contig_stage_floats(const WAxis& A) { return (size_t)A.seqs * (2 * A.N + 2 * A.lp); }

template <class S>
PSTD_HD void step_contig(const WStep& a, int64_t block, float2* smem, int tid, int nthr) {
    constexpr int T = S::T, E = S::E;
    // Lean form (the 3-D lengths, L <= 768): nothing is held in registers
    // across the forward FFT, so that the pass fits 128 registers and 4 CTAs
    // per SM; instead the spectrum slots and the accumulator are copied into
    // shared memory (cp.async) while the forward FFT runs.  The 2-D length
    // 1024 is latency-bound and prefetches the slots, the symmetry factors and
    // the accumulator into registers with the tables.
    constexpr bool lean = S::V >= 1 && S::L <= 768;
    int sq, t;
    lane_of<S>(tid, sq, t);
    WAxis A = a.ax;
    fix_extent<S>(A);
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
    const bool vbu = vb || (va && A.ph);     // the spectrum's second line: partner or phantom
    float* ua = a.u + (va ? la : 0) * N;
    float* ub = vb ? a.u + lb * N : (vbu ? A.ph : a.u);
    const float* ia = a.acc_in + (va ? la : 0) * lp;
    const float* ib = a.acc_in + (vb ? lb : 0) * lp;
    auto slot = [&](int s) { return make_float2(va ? ua[s] : 0.0f, vbu ? ub[s] : 0.0f); };
    auto acc = [&](int e) {
        const int i = t + T * e - A.lo;
        const bool ok = i >= 0 && i < lp;
        return make_float2(va && ok ? ia[i] : 0.0f, vb && ok ? ib[i] : 0.0f);
    };
    float2 w[E], ao[E], sy[E];
    if constexpr (!lean) {
        // prefetch this lane's spectrum slots and accumulator
#pragma unroll
        for (int e = 0; e < E; ++e) {
            bool own;
            const int s = spec_slot(A, t + T * e, own);
            w[e] = slot(s);
            // latency schedules: the symmetry factor (a global table) is
            // fetched with the slots, off the critical path
            if constexpr (reg_tables<S>()) sy[e] = own ? make_float2(1.0f, 0.0f) : A.sym[t + T * e];
            ao[e] = acc(e);
        }
    }
    async_wait_all();
    PSTD_SYNCCTA();
    // lean form: this sequence's spectrum lines [a | b] and accumulator lines
    // [a | b], copied now and read after the forward FFT
    float* su = (float*)(bufs + (size_t)A.seqs * wf::seq_words<S::L>()) + (size_t)sq * (2 * N + 2 * lp);
    float* sa = su + 2 * N;
    if constexpr (lean) {
        for (int i = t; i < N; i += T) {
            if (va) async_copy4(&su[i], &ua[i]);
            if (vbu) async_copy4(&su[N + i], &ub[i]);
        }
        for (int i = t; i < lp; i += T) {
            if (va) async_copy4(&sa[i], &ia[i]);
            if (vb) async_copy4(&sa[lp + i], &ib[i]);
        }
    }
    if constexpr (!lean) {
        // staged tables are readable from here on: non-owner bins from their slot
#pragma unroll
        for (int e = 0; e < E; ++e) {
            bool own;
            spec_slot(A, t + T * e, own);
            if (!own) w[e] = cmul(reg_tables<S>() ? sy[e] : tab.sym(e), w[e]);
        }
    }
    const float* pa = a.p + (va ? la : 0) * lp;
    const float* pb = a.p + (vb ? lb : 0) * lp;
    float2 v[E];
    load_p_ext<S>(v, t, A, tab, [&](int i) { return make_float2(va ? pa[i] : 0.0f, vb ? pb[i] : 0.0f); });
    fft<S, false>(v, t, sm, tab);
    if constexpr (lean) {
        async_wait_all();
        seq_sync<S>();   // every lane's copies are visible to the sequence
        load_spectrum<S>(w, t, A, tab,
                         [&](int s) { return make_float2(va ? su[s] : 0.0f, vbu ? su[N + s] : 0.0f); });
    }
    // (the slots are read from the staged copy (lean form) or were prefetched
    // before the forward FFT, whose exchange barriers ordered those reads
    // before the owner writes; a one-lane sequence has no other reader)
    update_and_inverse<S>(v, w, t, sm, A, tab, [&](int s, float2 x) {
        if (va) ua[s] = x.x;
        if (vbu) ub[s] = x.y;
    });
    float* oa = a.acc_out + (va ? la : 0) * lp;
    float* ob = a.acc_out + (vb ? lb : 0) * lp;
#pragma unroll
    for (int e = 0; e < E; ++e) {
        const int i = t + T * e - A.lo;
        if (i >= 0 && i < lp) {
            const float2 c = lean ? make_float2(va ? sa[i] : 0.0f, vb ? sa[lp + i] : 0.0f) : ao[e];
            if (va) oa[i] = c.x + v[e].x;
            if (vb) ob[i] = c.y + v[e].y;
        }
    }
    pdl_trigger();
}

// Velocity <-> its spectrum (WGrad dir 2 / 3), one line pair in registers;
// `ld(i)` reads the pair's stored input at index i and `st(i, x)` writes its
// output.  In place is allowed: every read precedes the FFT's barriers.
template <class S, class Tab, class Ld, class St>
PSTD_HD void spec_convert(int dir, float scale, int t, float2* sm, const WAxis& A, const Tab& tab, Ld&& ld,
                          St&& st) {
    constexpr int T = S::T, E = S::E;
    const int N = A.N;
    float2 v[E];
    if (dir == 2) {
#pragma unroll
        for (int e = 0; e < E; ++e) {
            const int j = t + T * e;
            const bool mirror = j >= N;
            float2 val = ld(mirror ? 2 * N - 1 - j : j);
            if (mirror) val = cscale(val, A.sR_u);
            if (A.group2) val = cmul(val, tab.sh(e));
            v[e] = val;
        }
        seq_sync<S>();
        fft<S, false>(v, t, sm, tab);
#pragma unroll
        for (int e = 0; e < E; ++e) {
            bool own;
            const int s = spec_slot(A, t + T * e, own);
            if (own) st(s, cscale(v[e], scale));
        }
    } else {
        load_spectrum<S>(v, t, A, tab, ld);
        seq_sync<S>();
        fft<S, true>(v, t, sm, tab);
#pragma unroll
        for (int e = 0; e < E; ++e) {
            const int m = t + T * e;
            if (m < N) st(m, A.group2 ? cmulc(v[e], tab.sh(e)) : v[e]);
        }
    }
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
    const bool from_p = a.dir == 0 || a.dir == 4;   // input on the pressure nodes
    const auto tab = tables<S>(A, from_p ? f : nullptr, from_p ? nullptr : f, t);
    async_wait_all();
    PSTD_SYNCCTA();
    pdl_wait();
    const int64_t seq = block * A.seqs + sq;
    const int64_t la = 2 * seq, lb = 2 * seq + 1;
    const bool va = la < A.nlines, vb = lb < A.nlines;
    float2* sm = bufs + (size_t)sq * wf::seq_words<S::L>();
    if (a.dir == 2 || a.dir == 3) {
        // spectrum side of an unpaired line: the phantom partner
        const bool ph = !vb && va && A.ph;
        const bool rb = vb || (ph && a.dir == 3), wb = vb || (ph && a.dir == 2);
        const float* xa = a.in + (va ? la : 0) * A.N;
        const float* xb = vb ? a.in + lb * A.N : (ph ? A.ph : a.in);
        float* oa = a.out + (va ? la : 0) * A.N;
        float* ob = vb ? a.out + lb * A.N : (ph ? A.ph : a.out);
        spec_convert<S>(a.dir, a.scale, t, sm, A, tab,
                        [&](int i) { return make_float2(va ? xa[i] : 0.0f, rb ? xb[i] : 0.0f); },
                        [&](int i, float2 x) {
                            if (va) oa[i] = x.x;
                            if (wb) ob[i] = x.y;
                        });
        return;
    }
    const int nin = from_p ? A.lp : A.N;
    const int nout = a.dir == 0 ? A.N : A.lp;
    const float* xa = a.in + (va ? la : 0) * nin;
    const float* xb = a.in + (vb ? lb : 0) * nin;
    float2 v[E];
    auto src = [&](int i) { return make_float2(va ? xa[i] : 0.0f, vb ? xb[i] : 0.0f); };
    if (from_p) derivative<S, 0>(v, t, sm, A, tab, src);
    else derivative<S, 1>(v, t, sm, A, tab, src);
    float* oa = a.out + (va ? la : 0) * nout;
    float* ob = a.out + (vb ? lb : 0) * nout;
    const int off = a.dir == 0 ? 0 : A.lo;
    // dir 4 with pout: the sequence's reads of `in` all precede the FFT's
    // barriers, so pout may be `in` (each node belongs to one line)
    float* qa = a.pout ? a.pout + (va ? la : 0) * nin : nullptr;
    float* qb = a.pout ? a.pout + (vb ? lb : 0) * nin : nullptr;
#pragma unroll
    for (int e = 0; e < E; ++e) {
        const int i = t + T * e - off;
        if (i >= 0 && i < nout) {
            if (va) {
                const float y = a.accumulate ? oa[i] + v[e].x : v[e].x;
                oa[i] = y;
                if (qa) qa[i] = xa[i] + y;
            }
            if (vb) {
                const float y = a.accumulate ? ob[i] + v[e].y : v[e].y;
                ob[i] = y;
                if (qb) qb[i] = xb[i] + y;
            }
        }
    }
    pdl_trigger();
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

// Row stride in shared memory of a tile of G lines of `len` words each: odd.
// (A stride of 32 / G (mod 32) words would put the 32 words of a warp's
// staging copies on distinct banks, but measured slower on 256^3: 0.602
// against 0.570 ms per step.)
PSTD_HD int row_stride(int len, int G) {
    (void)G;
    return len | 1;
}

// G is a power of two: item idx is (position idx >> log2 G, line idx & (G-1)).
PSTD_HD int log2_pow2(int G) {
    int s = 0;
    while ((1 << s) < G) ++s;
    return s;
}

// Item idx of a tile is (position idx >> log2 G, line idx & (G-1)), so
// consecutive threads cover the G adjacent lines of one position.  When the
// CTA's thread count is a multiple of G (every schedule with two or more
// lanes per sequence) each thread keeps one line and walks the positions with
// fixed increments; otherwise (one lane per sequence, G > threads) the items
// are enumerated directly.
PSTD_HD void tile_load(const float* f, int len, const WAxis& A, int64_t o, int64_t i0, int Gv,
                       float* raw, int tid, int nthr) {
    const int rs = row_stride(len, A.G);
    const int gs = log2_pow2(A.G), gm = A.G - 1;
    const float* base = f + o * (int64_t)len * A.inner + i0;
    if ((nthr & gm) == 0) {
        const int g = tid & gm, step = nthr >> gs;
        if (g >= Gv) return;
        int pos = tid >> gs;
        const float* src = base + (int64_t)pos * A.inner + g;
        float* dst = raw + g * rs + pos;
        const int64_t gstep = (int64_t)step * A.inner;
        for (; pos < len; pos += step, src += gstep, dst += step) async_copy4(dst, src);
        return;
    }
    const int total = len << gs;
    for (int idx = tid; idx < total; idx += nthr) {
        const int pos = idx >> gs, g = idx & gm;
        if (g < Gv) async_copy4(&raw[g * rs + pos], &base[(int64_t)pos * A.inner + g]);
    }
}

PSTD_HD void tile_store(float* f, int len, const WAxis& A, int64_t o, int64_t i0, int Gv,
                        const float* raw, int tid, int nthr) {
    const int rs = row_stride(len, A.G);
    const int gs = log2_pow2(A.G), gm = A.G - 1;
    float* base = f + o * (int64_t)len * A.inner + i0;
    if ((nthr & gm) == 0) {
        const int g = tid & gm, step = nthr >> gs;
        if (g >= Gv) return;
        int pos = tid >> gs;
        float* dst = base + (int64_t)pos * A.inner + g;
        const float* src = raw + g * rs + pos;
        const int64_t gstep = (int64_t)step * A.inner;
        for (; pos < len; pos += step, dst += gstep, src += step) *dst = *src;
        return;
    }
    const int total = len << gs;
    for (int idx = tid; idx < total; idx += nthr) {
        const int pos = idx >> gs, g = idx & gm;
        if (g < Gv) base[(int64_t)pos * A.inner + g] = raw[g * rs + pos];
    }
}

// shared memory of a strided step tile (without the staged tables), in floats
PSTD_HD size_t strided_step_floats(const WAxis& A, int seq_words, bool separate_acc) {
    const size_t fft = (size_t)A.seqs * seq_words * 2;
    const size_t p = (size_t)A.G * row_stride(A.lp, A.G);
    const size_t u = (size_t)A.G * row_stride(A.N, A.G);
    return fft + p + u + (separate_acc ? p : 0);
}

template <class S>
PSTD_HD void step_strided(const WStep& a, int64_t block, float2* smem0, int tid, int nthr) {
    constexpr int T = S::T, E = S::E;
    WAxis A = a.ax;
    fix_extent<S>(A);
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
    float* rawU = rawP + (size_t)A.G * row_stride(lp, A.G);
    float* rawA = sep ? rawU + (size_t)A.G * row_stride(N, A.G) : rawP;
    pdl_wait();
    tile_load(a.p, lp, A, o, i0, Gv, rawP, tid, nthr);
    tile_load(a.u, N, A, o, i0, Gv, rawU, tid, nthr);
    if (sep) tile_load(a.acc_in, lp, A, o, i0, Gv, rawA, tid, nthr);
    // an odd tile's last line pairs with the phantom row Gv (< G)
    const bool phrow = A.ph && (Gv & 1);
    if (phrow)
        for (int m = tid; m < N; m += nthr) rawU[Gv * row_stride(N, A.G) + m] = A.ph[o * N + m];
    async_wait_all();
    PSTD_SYNCCTA();
    if (sq < A.seqs) {
        const int ga = 2 * sq, gb = 2 * sq + 1;
        const bool va = ga < Gv, vb = gb < Gv;
        const bool vbu = vb || (phrow && gb == Gv);
        float2* sm = smem + (size_t)sq * wf::seq_words<S::L>();
        const float* pa = rawP + (va ? ga : 0) * row_stride(lp, A.G);
        const float* pb = rawP + (vb ? gb : 0) * row_stride(lp, A.G);
        float* ua = rawU + (va ? ga : 0) * row_stride(N, A.G);
        float* ub = rawU + (vbu ? gb : 0) * row_stride(N, A.G);
        float2 v[E];
        load_p_ext<S>(v, t, A, tab, [&](int i) { return make_float2(va ? pa[i] : 0.0f, vb ? pb[i] : 0.0f); });
        fft<S, false>(v, t, sm, tab);
        // the spectrum slots are read from the tile only now, so that they do
        // not occupy registers during the forward FFT
        float2 w[E];
        load_spectrum<S>(w, t, A, tab, [&](int s) { return make_float2(va ? ua[s] : 0.0f, vbu ? ub[s] : 0.0f); });
        seq_sync<S>();   // every lane has read its slots before any owner writes
        update_and_inverse<S>(v, w, t, sm, A, tab, [&](int s, float2 x) {
            if (va) ua[s] = x.x;
            if (vbu) ub[s] = x.y;
        });
        float* aa = rawA + (va ? ga : 0) * row_stride(lp, A.G);
        float* ab = rawA + (vb ? gb : 0) * row_stride(lp, A.G);
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
    if (phrow)
        for (int m = tid; m < N; m += nthr) A.ph[o * N + m] = rawU[Gv * row_stride(N, A.G) + m];
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
    const bool from_p = a.dir == 0 || a.dir == 4;   // input on the pressure nodes
    const auto tab = tables<S>(A, from_p ? f : nullptr, from_p ? nullptr : f, t);
    int64_t o, i0;
    int Gv;
    tile_of(A, block, o, i0, Gv);
    const int nin = from_p ? A.lp : A.N;
    const int nout = a.dir == 0 || a.dir == 2 || a.dir == 3 ? A.N : A.lp;
    float* rawI = (float*)(smem + (size_t)A.seqs * wf::seq_words<S::L>());
    float* rawO = rawI + (size_t)A.G * row_stride(nin, A.G);
    pdl_wait();
    tile_load(a.in, nin, A, o, i0, Gv, rawI, tid, nthr);
    if (a.accumulate) tile_load(a.out, nout, A, o, i0, Gv, rawO, tid, nthr);
    async_wait_all();
    PSTD_SYNCCTA();
    if (a.dir == 2 || a.dir == 3) {
        // in place through the tile: rawO is a separate buffer of the same
        // shape.  An odd tile's last line pairs with the phantom row Gv: read
        // from WAxis::ph (dir 3) or written to it (dir 2).
        const bool phrow = A.ph && (Gv & 1);
        if (phrow && a.dir == 3) {
            for (int m = tid; m < A.N; m += nthr) rawI[Gv * row_stride(nin, A.G) + m] = A.ph[o * A.N + m];
            PSTD_SYNCCTA();
        }
        if (sq < A.seqs) {
            const int ga = 2 * sq, gb = 2 * sq + 1;
            const bool va = ga < Gv, vb = gb < Gv;
            const bool ph = phrow && gb == Gv;
            const bool rb = vb || (ph && a.dir == 3), wb = vb || (ph && a.dir == 2);
            float2* sm = smem + (size_t)sq * wf::seq_words<S::L>();
            const float* xa = rawI + (va ? ga : 0) * row_stride(nin, A.G);
            const float* xb = rawI + (rb ? gb : 0) * row_stride(nin, A.G);
            float* oa = rawO + (va ? ga : 0) * row_stride(nout, A.G);
            float* ob = rawO + (wb ? gb : 0) * row_stride(nout, A.G);
            spec_convert<S>(a.dir, a.scale, t, sm, A, tab,
                            [&](int i) { return make_float2(va ? xa[i] : 0.0f, rb ? xb[i] : 0.0f); },
                            [&](int i, float2 x) {
                                if (va) oa[i] = x.x;
                                if (wb) ob[i] = x.y;
                            });
        }
        PSTD_SYNCCTA();
        tile_store(a.out, nout, A, o, i0, Gv, rawO, tid, nthr);
        if (phrow && a.dir == 2)
            for (int m = tid; m < A.N; m += nthr) A.ph[o * A.N + m] = rawO[Gv * row_stride(nout, A.G) + m];
        return;
    }
    if (sq < A.seqs) {
        const int ga = 2 * sq, gb = 2 * sq + 1;
        const bool va = ga < Gv, vb = gb < Gv;
        float2* sm = smem + (size_t)sq * wf::seq_words<S::L>();
        const float* xa = rawI + (va ? ga : 0) * row_stride(nin, A.G);
        const float* xb = rawI + (vb ? gb : 0) * row_stride(nin, A.G);
        float2 v[E];
        auto src = [&](int i) { return make_float2(va ? xa[i] : 0.0f, vb ? xb[i] : 0.0f); };
        if (from_p) derivative<S, 0>(v, t, sm, A, tab, src);
        else derivative<S, 1>(v, t, sm, A, tab, src);
        float* oa = rawO + (va ? ga : 0) * row_stride(nout, A.G);
        float* ob = rawO + (vb ? gb : 0) * row_stride(nout, A.G);
        // dir 4 with pout: the input rows become in + out in place (this
        // sequence's reads of them precede the FFT's barriers)
        float* ia = rawI + (va ? ga : 0) * row_stride(nin, A.G);
        float* ib = rawI + (vb ? gb : 0) * row_stride(nin, A.G);
        const int off = a.dir == 0 ? 0 : A.lo;
#pragma unroll
        for (int e = 0; e < E; ++e) {
            const int i = t + T * e - off;
            if (i >= 0 && i < nout) {
                if (va) {
                    const float y = a.accumulate ? oa[i] + v[e].x : v[e].x;
                    oa[i] = y;
                    if (a.pout) ia[i] += y;
                }
                if (vb) {
                    const float y = a.accumulate ? ob[i] + v[e].y : v[e].y;
                    ob[i] = y;
                    if (a.pout) ib[i] += y;
                }
            }
        }
    }
    PSTD_SYNCCTA();
    tile_store(a.out, nout, A, o, i0, Gv, rawO, tid, nthr);
    if (a.pout) tile_store(a.pout, nin, A, o, i0, Gv, rawI, tid, nthr);
    pdl_trigger();
}

}  // namespace wk
}  // namespace pstd
