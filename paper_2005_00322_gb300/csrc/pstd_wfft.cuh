// pstd_wfft.cuh -- register-resident complex FFTs owned by T lanes of a warp.
//
// A sequence of length L is held by T = L / E lanes, lane t holding the E
// elements x[t + T e] (e = 0..E-1) in registers.  The FFT is a sequence of
// Stockham autosort passes of radix R (R divides E, so each lane computes
// E / R radix-R butterflies entirely in registers).  Between two passes the
// outputs are scattered through a per-sequence shared-memory buffer and
// gathered back into the layout x[t + T e]; the last pass's outputs already
// land in that layout, so an FFT of P passes needs P - 1 exchanges and no
// block-level barrier.  The radix-R DFTs are fully unrolled decimation-in-
// frequency recursions whose twiddles are compile-time constants; the
// inter-pass twiddles come from a per-pass table laid out [b][k-1][t] so that
// a warp's loads are contiguous.
//
// Constants: cos/sin of 2 pi k / R are evaluated at compile time from their
// Taylor series in double precision (this file's own evaluation) and rounded
// once to float.
#pragma once

#include <utility>

#include "pstd_ops.cuh"

namespace pstd {
namespace wf {

constexpr double kPi = 3.141592653589793238462643383279502884;

constexpr double taylor_sin(double x) {
    double term = x, sum = x;
    for (int n = 1; n < 40; ++n) {
        term *= -x * x / ((2.0 * n) * (2.0 * n + 1.0));
        sum += term;
    }
    return sum;
}
constexpr double taylor_cos(double x) {
    double term = 1.0, sum = 1.0;
    for (int n = 1; n < 40; ++n) {
        term *= -x * x / ((2.0 * n - 1.0) * (2.0 * n));
        sum += term;
    }
    return sum;
}
// angle 2 pi k / R reduced to (-pi, pi]
constexpr double unit_angle(int k, int R) {
    const int kk = ((k % R) + R) % R;
    return 2 * kk > R ? 2.0 * kPi * (double)(kk - R) / R : 2.0 * kPi * (double)kk / R;
}
template <int R, int K>
struct Unit {  // exp(+2 pi i K / R)
    static constexpr float c = (float)taylor_cos(unit_angle(K, R));
    static constexpr float s = (float)taylor_sin(unit_angle(K, R));
};

// ---- radix-R DFT in registers, natural order in and out ----------------------
// forward: y_k = sum_n a_n exp(-2 pi i n k / R); inverse: exp(+...)
template <int R, bool INV>
struct Dft;

template <int R, bool INV, int K>
PSTD_HD void dif_bfly(float2* a) {
    constexpr int H = R / 2;
    const float2 x = a[K], y = a[K + H];
    a[K] = cadd(x, y);
    const float2 d = csub(x, y);
    if constexpr (K == 0) {
        a[K + H] = d;
    } else if constexpr (4 * K == R) {
        a[K + H] = INV ? make_float2(-d.y, d.x) : make_float2(d.y, -d.x);
    } else {
        constexpr float c = Unit<R, K>::c;
        constexpr float s = INV ? Unit<R, K>::s : -Unit<R, K>::s;
        a[K + H] = make_float2(d.x * c - d.y * s, d.x * s + d.y * c);
    }
}
template <int R, bool INV, int... K>
PSTD_HD void dif_stage(float2* a, std::integer_sequence<int, K...>) {
    (dif_bfly<R, INV, K>(a), ...);
}

template <int R, bool INV>
struct Dft {
    static PSTD_HD void run(float2* a) {
        constexpr float sg = INV ? 1.0f : -1.0f;
        if constexpr (R == 1) {
        } else if constexpr (R == 2) {
            dft2(a);
        } else if constexpr (R == 3) {
            dft3(a, sg);
        } else if constexpr (R == 4) {
            dft4(a, sg);
        } else if constexpr (R == 5) {
            dft5(a, sg);
        } else if constexpr (R == 8) {
            dft8(a, sg);
        } else {
            static_assert(R % 2 == 0, "radix must be 2^k, 3 or 5");
            constexpr int H = R / 2;
            dif_stage<R, INV>(a, std::make_integer_sequence<int, H>{});
            Dft<H, INV>::run(a);
            Dft<H, INV>::run(a + H);
            float2 tmp[R];
#pragma unroll
            for (int m = 0; m < H; ++m) {
                tmp[2 * m] = a[m];
                tmp[2 * m + 1] = a[H + m];
            }
#pragma unroll
            for (int i = 0; i < R; ++i) a[i] = tmp[i];
        }
    }
};

// ---- schedules -------------------------------------------------------------
// Sched<L, V>: lanes per sequence T and the radix of each pass (all divide E).
// V = 0 (throughput): many elements per lane, few passes, for axes with many
// lines.  V = 1 (latency): 8 elements per lane spread over up to 128 lanes,
// for axes with too few lines to fill the GPU, where one sequence's latency
// sets the pass time.  V = 4: the radices of V = 1 with the tables read from
// shared memory instead of registers (fewer registers, more resident CTAs).
// V = 5: the same with the tables read from global memory through L1, so
// that neither registers nor shared memory hold them.  A sequence wider than a warp exchanges through a CTA
// barrier.
template <int L, int V = 0>
struct Sched;
#define PSTD_SCHED(LL, VV, TT, ...)                            \
    template <>                                                \
    struct Sched<LL, VV> {                                     \
        static constexpr int L = LL, V = VV, T = TT, E = LL / TT; \
        static constexpr int R[] = {__VA_ARGS__};              \
        static constexpr int P = sizeof(R) / sizeof(int);      \
    };
PSTD_SCHED(2, 0, 1, 2)
PSTD_SCHED(4, 0, 1, 4)
PSTD_SCHED(8, 0, 1, 8)
PSTD_SCHED(16, 0, 1, 16)
PSTD_SCHED(32, 0, 1, 32)
PSTD_SCHED(64, 0, 4, 16, 4)
PSTD_SCHED(128, 0, 8, 16, 8)
PSTD_SCHED(256, 0, 16, 16, 16)
PSTD_SCHED(512, 0, 16, 32, 16)
PSTD_SCHED(1024, 0, 32, 32, 32)
PSTD_SCHED(96, 0, 4, 8, 4, 3)
PSTD_SCHED(192, 0, 8, 8, 8, 3)
PSTD_SCHED(384, 0, 16, 8, 8, 2, 3)
PSTD_SCHED(768, 0, 32, 8, 8, 4, 3)
PSTD_SCHED(256, 1, 32, 8, 8, 4)
PSTD_SCHED(512, 1, 64, 8, 8, 8)
PSTD_SCHED(1024, 1, 128, 8, 8, 8, 2)
PSTD_SCHED(1024, 2, 64, 16, 16, 4)
PSTD_SCHED(768, 1, 64, 4, 4, 4, 4, 3)
PSTD_SCHED(1024, 3, 256, 4, 4, 4, 4, 4)
PSTD_SCHED(512, 3, 128, 4, 4, 4, 4, 2)
PSTD_SCHED(256, 4, 32, 8, 8, 4)
PSTD_SCHED(512, 4, 64, 8, 8, 8)
PSTD_SCHED(256, 5, 32, 8, 8, 4)
PSTD_SCHED(512, 5, 64, 8, 8, 8)
PSTD_SCHED(768, 4, 64, 4, 4, 4, 4, 3)
#undef PSTD_SCHED

// Ns before pass p (product of earlier radices)
template <class S, int p>
constexpr int span_before() {
    int ns = 1;
    for (int i = 0; i < p; ++i) ns *= S::R[i];
    return ns;
}
// entries of pass p's twiddle table: max(1, Ns / T) * (R - 1) * T  (0 for Ns = 1)
template <class S, int p>
constexpr int tw_entries() {
    constexpr int ns = span_before<S, p>();
    if (ns == 1) return 0;
    constexpr int bm = ns / S::T > 1 ? ns / S::T : 1;
    return bm * (S::R[p] - 1) * S::T;
}
template <class S, int p>
constexpr int tw_offset() {
    int off = 0;
    if constexpr (p > 0) off = tw_offset<S, p - 1>() + tw_entries<S, p - 1>();
    return off;
}
template <class S>
constexpr int tw_total() {
    return tw_offset<S, S::P - 1>() + tw_entries<S, S::P - 1>();
}

// padded shared-memory index: one spare slot per 32 complex words
PSTD_HD int pad(int i) { return i + (i >> 5); }
template <int L>
constexpr int seq_words() { return L + L / 32 + 1; }

// Butterflies of pass p for lane t (in registers, outputs in place).  The
// inter-pass twiddles come from `tw(i)`: entry i of this lane's slice of the
// pass tables, i = tw_offset<S, p>() / T + bm (R - 1) + (k - 1).
template <class S, int p, bool INV, class Tw>
PSTD_HD void pass_compute(float2 (&v)[S::E], Tw&& tw) {
    constexpr int E = S::E, T = S::T, R = S::R[p], B = E / R;
    constexpr int Ns = span_before<S, p>();
    constexpr int base = tw_offset<S, p>() / T;
#pragma unroll
    for (int b = 0; b < B; ++b) {
        float2 a[R];
#pragma unroll
        for (int k = 0; k < R; ++k) a[k] = v[b + k * B];
        if constexpr (Ns > 1) {
            constexpr int BM = Ns / T > 1 ? Ns / T : 1;
            const int bm = b % BM;
#pragma unroll
            for (int k = 1; k < R; ++k) {
                float2 w = tw(base + bm * (R - 1) + (k - 1));
                if (INV) w.y = -w.y;
                a[k] = cmul(a[k], w);
            }
        }
        Dft<R, INV>::run(a);
#pragma unroll
        for (int k = 0; k < R; ++k) v[b + k * B] = a[k];
    }
}

// Entries of one lane's slice of the pass tables (tw_total is a multiple of T).
template <class S>
constexpr int tw_per_lane() { return tw_total<S>() / S::T; }

// Scatter pass p's outputs (not the last pass) into the sequence buffer.
template <class S, int p>
PSTD_HD void pass_scatter(const float2 (&v)[S::E], int t, float2* sm) {
    constexpr int E = S::E, T = S::T, R = S::R[p], B = E / R;
    constexpr int Ns = span_before<S, p>();
#pragma unroll
    for (int b = 0; b < B; ++b) {
        const int j = t + T * b;
        const int jm = j % Ns;
        const int idxD = (j - jm) * R + jm;
#pragma unroll
        for (int k = 0; k < R; ++k) sm[pad(idxD + k * Ns)] = v[b + k * B];
    }
}

// Gather the natural layout x[t + T e] from the sequence buffer.
template <class S>
PSTD_HD void gather(float2 (&v)[S::E], int t, const float2* sm) {
#pragma unroll
    for (int e = 0; e < S::E; ++e) v[e] = sm[pad(t + S::T * e)];
}

// Host: fill the pass twiddle tables of schedule S (FP64 angles, rounded once).
// tw_total<S>() entries; entry for (pass p, bm, k, t) is
// exp(-2 pi i jm k / (Ns R)) with jm = (t + T bm) mod Ns.
template <class S, class F>
void fill_pass_twiddles(F&& put) {
    int Ns = 1, off = 0;
    for (int p = 0; p < S::P; ++p) {
        const int R = S::R[p];
        if (Ns > 1) {
            const int BM = Ns / S::T > 1 ? Ns / S::T : 1;
            for (int bm = 0; bm < BM; ++bm)
                for (int k = 1; k < R; ++k)
                    for (int t = 0; t < S::T; ++t) {
                        const int jm = (t + S::T * bm) % Ns;
                        const long m = (long)jm * k;          // angle 2 pi m / (Ns R)
                        put(off + (bm * (R - 1) + (k - 1)) * S::T + t, m, (long)Ns * R);
                    }
            off += BM * (R - 1) * S::T;
        }
        Ns *= R;
    }
}

}  // namespace wf
}  // namespace pstd
