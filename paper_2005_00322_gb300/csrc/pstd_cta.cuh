// pstd_cta.cuh -- CTA programs of the axis passes.
//
// A CTA owns G lines of one axis.  Two programs exist:
//
//  * cta_step: the fused per-axis leapfrog of Eq. (dtt_pstd_solution),
//        u_a  <- u_a + f_P(p^n)                 (f_P = -(dt/rho0) D_p, folded)
//        acc_out <- acc_in + f_U(u_a^{new})     (f_U = -(dt rho0 c0^2) D_u)
//    reading each p line once, updating the u_a line once, and reusing the
//    updated u_a line from shared memory for the second derivative.  acc is
//    the running pressure sum over axes (p^n for the first axis processed,
//    the scratch accumulator in between, p^{n+1} for the last).
//  * cta_grad: out <- (accumulate ? out : 0) + f(in), one derivative (or,
//        for the second-order form, the composed operator on the pressure
//        nodes, optionally followed by pout <- in + out).
//
// Line l of an axis with stride `inner` (the product of the later extents)
// starts at (l / inner) * len * inner + (l % inner) in a field with `len`
// entries along the axis.  Loads and stores walk the line index fastest when
// inner > 1 (adjacent lines are adjacent in memory) and the position along
// the line fastest when inner == 1, so that a warp touches contiguous words.
#pragma once

#include "pstd_ops.cuh"

#ifdef __CUDA_ARCH__
#define PSTD_SYNC() __syncthreads()
#else
#define PSTD_SYNC() \
    do {            \
    } while (0)
#endif

namespace pstd {

struct StepArgs {
    LineOp opP;             // pressure -> u_a, scaled by -dt/rho0
    LineOp opU;             // u_a -> pressure, scaled by -dt rho0 c0^2
    int64_t nlines;         // lines along this axis
    int64_t inner;          // stride of the axis in elements
    int G;                  // lines per CTA
    int rs;                 // floats per staged line in shared memory
    const float* p;         // p^n
    float* u;               // u_a (read and written)
    const float* acc_in;    // p^n or the scratch accumulator
    float* acc_out;         // the scratch accumulator or p^{n+1}
};

struct GradArgs {
    LineOp op;
    int64_t nlines, inner;
    int G, rs;
    const float* in;
    float* out;
    int accumulate;
    float* pout = nullptr;  // input and output on one grid: also write in + (the new out)
                            // here (may be `in`: each entry belongs to one line)
};

// A batch of plans run as one cooperative kernel on the generic CTA program:
// pass k of a step (k = 0 the last axis of each member) is, over all members,
// prefix[k][members] work items (line groups), member m owning items
// prefix[k][m] .. prefix[k][m + 1] - 1 with its pass mem[m * 3 + k].
struct StepPersistArgs {
    const StepArgs* mem;       // [members][3], device memory
    const int64_t* prefix;     // [3][members + 1], device memory
    int members;
    int npass;                 // passes per step: the most axes of any member
    int64_t nsteps;
};

PSTD_HD int64_t line_base(int64_t l, int64_t inner, int len) {
    return (l / inner) * (int64_t)len * inner + (l % inner);
}

// (g, i) of work item t for Gv lines of `len` entries
PSTD_HD void item(int t, int Gv, int len, int64_t inner, int& g, int& i) {
    if (inner == 1) {
        g = t / len;
        i = t - g * len;
    } else {
        i = t / Gv;
        g = t - i * Gv;
    }
}

PSTD_HD void phase_load(const float* field, int len, int64_t l0, int Gv, int64_t inner,
                        float* raw, int rs, int tid, int nthr) {
    const int total = Gv * len;
    for (int t = tid; t < total; t += nthr) {
        int g, i;
        item(t, Gv, len, inner, g, i);
        const int64_t b = line_base(l0 + g, inner, len);
        raw[(size_t)g * rs + i] = field[b + (int64_t)i * inner];
    }
}

// Forward FFT, multiply, inverse FFT (or the dense product); returns the
// buffer that holds the result.  All threads of the CTA must call it.
PSTD_HD const float2* run_op(const LineOp& op, const float* raw, int rs, int G, float2* A,
                             float2* B, int tid, int nthr) {
    if (op.kind == 1) {
        phase_dense(op, raw, rs, G, A, tid, nthr);
        PSTD_SYNC();
        return A;
    }
    const int nseq = (G + 1) / 2;
    phase_extend(op, raw, rs, G, A, tid, nthr);
    PSTD_SYNC();
    float2* src = A;
    float2* dst = B;
    int Ns = 1;
    for (int p = 0; p < op.fft.npass; ++p) {
        fft_pass(op.fft, p, Ns, src, dst, nseq, -1.0f, tid, nthr);
        PSTD_SYNC();
        float2* t = src;
        src = dst;
        dst = t;
    }
    phase_multiply(op, src, G, tid, nthr);
    PSTD_SYNC();
    Ns = 1;
    for (int p = 0; p < op.fft.npass; ++p) {
        fft_pass(op.fft, p, Ns, src, dst, nseq, +1.0f, tid, nthr);
        PSTD_SYNC();
        float2* t = src;
        src = dst;
        dst = t;
    }
    return src;
}

PSTD_HD size_t cta_smem_bytes(int G, int L, int rs) {
    const int nseq = (G + 1) / 2;
    return (size_t)2 * nseq * L * sizeof(float2) + (size_t)G * rs * sizeof(float);
}

PSTD_HD void cta_step(const StepArgs& a, int64_t block, void* smem, int tid, int nthr) {
    const int L = a.opP.seqlen;
    const int nseq = (a.G + 1) / 2;
    float2* A = (float2*)smem;
    float2* B = A + (size_t)nseq * L;
    float* raw = (float*)(B + (size_t)nseq * L);
    const int64_t l0 = block * a.G;
    if (l0 >= a.nlines) return;
    const int Gv = (int)((a.nlines - l0) < a.G ? (a.nlines - l0) : a.G);

    phase_load(a.p, a.opP.nin, l0, Gv, a.inner, raw, a.rs, tid, nthr);
    PSTD_SYNC();
    const float2* y = run_op(a.opP, raw, a.rs, Gv, A, B, tid, nthr);

    // u_a^{n+1/2} = u_a^{n-1/2} + f_P(p^n); keep the new line for f_U
    {
        const int len = a.opP.nout;
        const int total = Gv * len;
        for (int t = tid; t < total; t += nthr) {
            int g, i;
            item(t, Gv, len, a.inner, g, i);
            const int64_t idx = line_base(l0 + g, a.inner, len) + (int64_t)i * a.inner;
            const float v = a.u[idx] + op_value(a.opP, y, g, i);
            a.u[idx] = v;
            raw[(size_t)g * a.rs + i] = v;
        }
    }
    PSTD_SYNC();
    y = run_op(a.opU, raw, a.rs, Gv, A, B, tid, nthr);

    // acc_out = acc_in + f_U(u_a^{n+1/2})
    {
        const int len = a.opU.nout;
        const int total = Gv * len;
        for (int t = tid; t < total; t += nthr) {
            int g, i;
            item(t, Gv, len, a.inner, g, i);
            const int64_t idx = line_base(l0 + g, a.inner, len) + (int64_t)i * a.inner;
            a.acc_out[idx] = a.acc_in[idx] + op_value(a.opU, y, g, i);
        }
    }
}

PSTD_HD void cta_grad(const GradArgs& a, int64_t block, void* smem, int tid, int nthr) {
    const int L = a.op.seqlen;
    const int nseq = (a.G + 1) / 2;
    float2* A = (float2*)smem;
    float2* B = A + (size_t)nseq * L;
    float* raw = (float*)(B + (size_t)nseq * L);
    const int64_t l0 = block * a.G;
    if (l0 >= a.nlines) return;
    const int Gv = (int)((a.nlines - l0) < a.G ? (a.nlines - l0) : a.G);

    phase_load(a.in, a.op.nin, l0, Gv, a.inner, raw, a.rs, tid, nthr);
    PSTD_SYNC();
    const float2* y = run_op(a.op, raw, a.rs, Gv, A, B, tid, nthr);
    const int len = a.op.nout;
    const int total = Gv * len;
    for (int t = tid; t < total; t += nthr) {
        int g, i;
        item(t, Gv, len, a.inner, g, i);
        const int64_t idx = line_base(l0 + g, a.inner, len) + (int64_t)i * a.inner;
        const float v = op_value(a.op, y, g, i);
        const float r = a.accumulate ? a.out[idx] + v : v;
        a.out[idx] = r;
        if (a.pout) a.pout[idx] = a.in[idx] + r;
    }
}

}  // namespace pstd
