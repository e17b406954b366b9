// pstd_tc16.cu -- split-precision dense form of the axis pass with BF16
// operands on the 5th-generation tensor cores (tcgen05.mma kind::f16, FP32
// accumulators in tensor memory, operator tiles fed by TMA).
//
// Each staggered derivative of an axis is a dense FP64-built operator D
// (Section 3.2: the transforms, k-multiply and inverse of Table 2 as one
// matrix, the time-step factors folded in) applied to every line:
//     Y[line, m] = Cin[line, m] + sum_k D[m, k] X[line, k].
//
// Exact three-way split (the error-free splitting of Ozaki, Ogita, Oishi and
// Rump, "Error-free transformations of matrix multiplication by using fast
// routines of matrix multiplication", Numer. Algorithms 59, 2012, with BF16
// slices).  Within one 64-wide k chunk every operator row m gets a power of
// two 2^E > max_k |D[m, k]| and every line gets 2^F > max_k |X[line, k]|;
// each value is cut into three BF16 slices on the grids 2^(E-8), 2^(E-16),
// 2^(E-24):
//     D = Dh + Dm + Dl,  |Dh| <= 2^8,  |Dm|, |Dl| <= 2^7  (in units of their grid)
// (the field: exactly, since an FP32 value has 24 significant bits; the
// operator: to 2^-25 of the row's chunk maximum).  The products kept are
//     L0 = Dh Xh                          (grid 2^(E+F-16))
//     L1 = Dh Xm + Dm Xh                  (grid 2^(E+F-24))
//     L2 = Dh Xl + Dm Xm + Dl Xh          (grid 2^(E+F-32))
// (dropped: Dm Xl + Dl Xm + Dl Xl, below 2^-25 of |D||X|).  Over 64 values
// of k, L0 is an integer below 2^22 on its grid, so the tensor core sums it
// exactly whatever its internal rounding: the main product carries no
// accumulation error.  (A running FP32 sum inside the tensor core is
// truncated, biased toward zero; over thousands of steps such a bias of the
// operator shifts the discrete frequencies into phase drift.)  L1 + L2 are
// 2^-8 of the result and run in one accumulator over all k.  Each chunk's L0
// starts from zero in one of two tensor-memory accumulators, which the
// epilogue warps add into FP32 registers while the next chunk runs.
//
// A CTA computes a 128-row output tile (MMA M) for 128 lines (MMA N):
//   warp 0     TMA producer: the chunk's three operator slices, one 3-D box of
//              64 k x 128 rows x 3 slices, 128-byte swizzle;
//   warp 1     allocates tensor memory; one thread issues the 6 MMAs of each
//              16-wide k step and commits them to the stage's and the
//              accumulator's mbarriers;
//   warps 2-5  load the field lines of the next chunk into registers, split
//              them and store the three slices in the MMA's K-major
//              128-byte-swizzled layout;
//   warps 6-9  epilogue: promote each chunk's L0, add L1 + L2 at the end,
//              write Y = Cin + sum (through shared memory on strided axes so
//              that the stores are coalesced).
// Two stages of 96 KB.  Every wait is bounded: a wait that gives up sets
// *status and a shared abort flag that ends every other wait, the MMAs and
// TMA loads in flight are waited for (bounded), and tensor memory is freed.
#include "pstd_tc16.h"

#include <cuda_bf16.h>

#include <cmath>
#include <cstring>

namespace pstd {

namespace {

constexpr int BM = 128;                        // output rows per tile (MMA M)
constexpr int NL = 128;                        // lines per tile (MMA N)
constexpr int BK = 64;                         // k per chunk: one 128-byte swizzle row of BF16
constexpr int STAGES = 2;
constexpr uint32_t PLANE = BM * BK * 2;        // one BF16 slice of one tile: 16 KB
constexpr uint32_t STAGE_BYTES = 6 * PLANE;    // operator Dh Dm Dl, field Xh Xm Xl
constexpr size_t SMEM = STAGES * STAGE_BYTES + 1024;
constexpr int THREADS = 320;
constexpr uint32_t TMEM_COLS = 512;            // L0[0] at 0, L0[1] at 128, L1+L2 at 256
constexpr long long kWaitLimit = 1 << 22;

// Instruction descriptor of kind::f16: D FP32, A and B BF16, both K-major.
constexpr uint32_t kIdesc = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(NL >> 3) << 17) |
                            ((uint32_t)(BM >> 4) << 24);

#ifdef __CUDA_ARCH__
__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(bar), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint32_t bar) {
    asm volatile("{\n .reg .b64 st;\n mbarrier.arrive.shared::cta.b64 st, [%0];\n}\n" ::"r"(bar) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes) {
    asm volatile("{\n .reg .b64 st;\n mbarrier.arrive.expect_tx.shared::cta.b64 st, [%0], %1;\n}\n" ::"r"(bar),
                 "r"(bytes)
                 : "memory");
}
__device__ __forceinline__ bool mbar_try(uint32_t bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(bar), "r"(parity)
        : "memory");
    return ok != 0;
}
// Bounded wait for the phase of `parity`; false once the shared abort flag is
// set (by this or another thread) or the limit is reached (which sets it).
__device__ __forceinline__ bool wait_bar(uint32_t bar, uint32_t parity, volatile int* abort_flag, int* status) {
    for (long long i = 0; i < kWaitLimit; ++i) {
        if (mbar_try(bar, parity)) return true;
        if (*abort_flag) return false;
    }
    *abort_flag = 1;
    if (status) atomicExch(status, 1);
    return false;
}
// Bounded wait that ignores the abort flag (teardown: copies and MMAs in flight).
__device__ __forceinline__ void drain_bar(uint32_t bar, uint32_t parity, int* status) {
    for (long long i = 0; i < kWaitLimit; ++i)
        if (mbar_try(bar, parity)) return;
    if (status) atomicExch(status, 1);
}

// K-major operand tile with 128-byte swizzle: rows of 128 bytes, 8-row groups
// 1024 bytes apart (SBO); the leading offset is unused for this layout.
__device__ __forceinline__ uint64_t desc_sw128(uint32_t addr) {
    uint64_t d = (uint64_t)((addr & 0x3FFFFu) >> 4);
    d |= (uint64_t)1 << 16;
    d |= (uint64_t)(1024u >> 4) << 32;
    d |= (uint64_t)1 << 46;            // descriptor version of the tcgen05 family
    d |= (uint64_t)2 << 61;            // 128-byte swizzle
    return d;
}

__device__ __forceinline__ void mma_bf16(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t acc) {
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
        " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(d_tmem),
        "l"(a), "l"(b), "r"(kIdesc), "r"(acc)
        : "memory");
}
__device__ __forceinline__ void mma_commit(uint32_t bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(bar)
                 : "memory");
}

// 32 consecutive accumulator columns of this warp's 32 lanes.
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, float (&v)[32]) {
    uint32_t r[32];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
        "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];\n"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
          "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]),
          "=r"(r[23]), "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]),
          "=r"(r[30]), "=r"(r[31])
        : "r"(taddr)
        : "memory");
    asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::: "memory");
#pragma unroll
    for (int j = 0; j < 32; ++j) v[j] = __uint_as_float(r[j]);
}

// Rounding constants 1.5 * 2^(E+15), 1.5 * 2^(E+7), 1.5 * 2^(E-1): adding and
// subtracting one rounds (to nearest even) to the grid 2^(E-8), 2^(E-16),
// 2^(E-24) of a value below 2^E.
struct Grids {
    float c0, c1, c2;
};
__device__ __forceinline__ Grids grids_for(float mx) {
    int E = (int)((__float_as_uint(mx) >> 23) & 0xFFu) - 126;   // 2^E > mx
    E = E < -100 ? -100 : (E > 100 ? 100 : E);
    Grids g;
    g.c0 = __uint_as_float(((uint32_t)(E + 142) << 23) | 0x400000u);
    g.c1 = __uint_as_float(((uint32_t)(E + 134) << 23) | 0x400000u);
    g.c2 = __uint_as_float(((uint32_t)(E + 126) << 23) | 0x400000u);
    return g;
}
// x = h + m + l exactly (|x| < 2^E), each on its grid; the adds and subtracts
// are the _rn intrinsics so that nothing contracts or reassociates them.
__device__ __forceinline__ void split3(float x, const Grids& g, float& h, float& m, float& l) {
    h = __fsub_rn(__fadd_rn(x, g.c0), g.c0);
    const float r1 = __fsub_rn(x, h);
    m = __fsub_rn(__fadd_rn(r1, g.c1), g.c1);
    const float r2 = __fsub_rn(r1, m);
    l = __fsub_rn(__fadd_rn(r2, g.c2), g.c2);
}
__device__ __forceinline__ uint32_t pack_bf16(float lo, float hi) {
    const __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);
    return *reinterpret_cast<const uint32_t*>(&v);
}
#endif

__global__ void __launch_bounds__(THREADS, 1) k_tc16(const __grid_constant__ CUtensorMap map, const Tc16Gemm g) {
#ifdef __CUDA_ARCH__
    extern __shared__ uint8_t tc16_raw[];
    __shared__ __align__(8) uint64_t bars[11];
    __shared__ uint32_t tmem_slot;
    __shared__ int abort_flag;
    uint8_t* sm = (uint8_t*)(((uintptr_t)tc16_raw + 1023) & ~(uintptr_t)1023);
    const uint32_t sbase = smem_u32(sm);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int mt = (int)(blockIdx.x % (unsigned)g.MT);
    const int64_t l0 = (int64_t)(blockIdx.x / (unsigned)g.MT) * NL;
    const int nc = g.KC;
    volatile int* abortp = &abort_flag;
    // barriers: tma_full[2], cvt_full[2], empty[2], acc_full[2], acc_empty[2], final
    auto bar = [&](int i) { return smem_u32(&bars[i]); };
    const int TMA_FULL = 0, CVT_FULL = 2, EMPTY = 4, ACC_FULL = 6, ACC_EMPTY = 8, FINAL = 10;

    if (tid == 0) {
        abort_flag = 0;
        for (int s = 0; s < 2; ++s) {
            mbar_init(bar(TMA_FULL + s), 1);
            mbar_init(bar(CVT_FULL + s), 4);
            mbar_init(bar(EMPTY + s), 1);
            mbar_init(bar(ACC_FULL + s), 1);
            mbar_init(bar(ACC_EMPTY + s), 4);
        }
        mbar_init(bar(FINAL), 1);
        asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
        asm volatile("prefetch.tensormap [%0];\n" ::"l"((uint64_t)&map) : "memory");
    }
    if (warp == 1) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(
                         smem_u32(&tmem_slot)),
                     "r"(TMEM_COLS)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n" ::: "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
    const uint32_t tmem = tmem_slot;

    if (warp == 0) {
        // ---- TMA producer: the operator's three slices of each chunk ----
        if (lane == 0) {
            int issued[2] = {0, 0};
            for (int c = 0; c < nc; ++c) {
                const int s = c & 1, n = c >> 1;
                if (c >= 2 && !wait_bar(bar(EMPTY + s), (uint32_t)((n - 1) & 1), abortp, g.status)) break;
                mbar_expect_tx(bar(TMA_FULL + s), 3 * PLANE);
                asm volatile(
                    "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
                    " [%0], [%1, {%3, %4, %5}], [%2];\n" ::"r"(sbase + (uint32_t)s * STAGE_BYTES),
                    "l"((uint64_t)&map), "r"(bar(TMA_FULL + s)), "r"(c * BK), "r"(mt * BM), "r"(0)
                    : "memory");
                issued[s] = n + 1;
            }
            // copies still in flight land before the CTA ends
            for (int s = 0; s < 2; ++s)
                if (issued[s] > 0) drain_bar(bar(TMA_FULL + s), (uint32_t)((issued[s] - 1) & 1), g.status);
        }
    } else if (warp == 1) {
        // ---- MMA issuer ----
        if (lane == 0) {
            const uint32_t X = tmem + 256u;
            for (int c = 0; c < nc; ++c) {
                const int s = c & 1, n = c >> 1;
                bool ok = wait_bar(bar(TMA_FULL + s), (uint32_t)(n & 1), abortp, g.status) &&
                          wait_bar(bar(CVT_FULL + s), (uint32_t)(n & 1), abortp, g.status);
                if (ok && c >= 2) ok = wait_bar(bar(ACC_EMPTY + s), (uint32_t)((n - 1) & 1), abortp, g.status);
                if (!ok) break;
                asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
                const uint32_t st = sbase + (uint32_t)s * STAGE_BYTES;
                const uint32_t L0 = tmem + (uint32_t)s * 128u;
#pragma unroll
                for (int ks = 0; ks < BK / 16; ++ks) {
                    const uint32_t o = (uint32_t)ks * 32u;
                    const uint64_t dh = desc_sw128(st + o), dm = desc_sw128(st + PLANE + o),
                                   dl = desc_sw128(st + 2 * PLANE + o);
                    const uint64_t xh = desc_sw128(st + 3 * PLANE + o), xm = desc_sw128(st + 4 * PLANE + o),
                                   xl = desc_sw128(st + 5 * PLANE + o);
                    mma_bf16(X, dh, xm, (c > 0 || ks > 0) ? 1u : 0u);
                    mma_bf16(X, dm, xh, 1u);
                    mma_bf16(X, dh, xl, 1u);
                    mma_bf16(X, dm, xm, 1u);
                    mma_bf16(X, dl, xh, 1u);
                    mma_bf16(L0, dh, xh, ks > 0 ? 1u : 0u);
                }
                mma_commit(bar(EMPTY + s));
                mma_commit(bar(ACC_FULL + s));
            }
            // every MMA issued has completed before tensor memory is freed
            mma_commit(bar(FINAL));
            drain_bar(bar(FINAL), 0u, g.status);
        }
    } else if (warp < 6) {
        // ---- field loaders and splitters (128 threads) ----
        const int cw = warp - 2, t = tid - 64;
        float v[64];
        if (g.inner > 1) {
            // thread t owns line l0 + t; consecutive lines are consecutive words
            const int64_t l = l0 + t;
            const bool valid = l < g.nlines;
            const float* xp = g.X;
            if (valid) xp += (l / g.inner) * (int64_t)g.K * g.inner + (l % g.inner);
            auto load = [&](int c) {
#pragma unroll
                for (int j = 0; j < 64; ++j) {
                    const int k = c * BK + j;
                    v[j] = (valid && k < g.K) ? __ldg(xp + (int64_t)k * g.inner) : 0.0f;
                }
            };
            load(0);
            for (int c = 0; c < nc; ++c) {
                const int s = c & 1, n = c >> 1;
                bool ok = true;
                if (c >= 2) ok = wait_bar(bar(EMPTY + s), (uint32_t)((n - 1) & 1), abortp, g.status);
                if (!__all_sync(0xFFFFFFFFu, ok)) break;
                float mx = 0.0f;
#pragma unroll
                for (int j = 0; j < 64; ++j) mx = fmaxf(mx, fabsf(v[j]));
                const Grids gr = grids_for(mx);
                uint8_t* row = sm + (size_t)s * STAGE_BYTES + 3 * PLANE + (size_t)t * 128;
#pragma unroll
                for (int q = 0; q < 8; ++q) {
                    uint32_t w[3][4];
#pragma unroll
                    for (int e = 0; e < 4; ++e) {
                        float h0, m0, s0, h1, m1, s1;
                        split3(v[8 * q + 2 * e], gr, h0, m0, s0);
                        split3(v[8 * q + 2 * e + 1], gr, h1, m1, s1);
                        w[0][e] = pack_bf16(h0, h1);
                        w[1][e] = pack_bf16(m0, m1);
                        w[2][e] = pack_bf16(s0, s1);
                    }
                    const uint32_t off = (uint32_t)((q ^ (t & 7)) << 4);
#pragma unroll
                    for (int p = 0; p < 3; ++p)
                        *reinterpret_cast<uint4*>(row + (size_t)p * PLANE + off) =
                            make_uint4(w[p][0], w[p][1], w[p][2], w[p][3]);
                }
                asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
                __syncwarp();
                if (lane == 0) mbar_arrive(bar(CVT_FULL + s));
                if (c + 1 < nc) load(c + 1);
            }
        } else {
            // contiguous lines: warp cw owns rows 32 cw .. 32 cw + 31, lane t
            // holds k = 2 t, 2 t + 1 of each
            auto load = [&](int c) {
                const int k = c * BK + 2 * lane;
#pragma unroll
                for (int j = 0; j < 32; ++j) {
                    const int64_t l = l0 + 32 * cw + j;
                    const bool valid = l < g.nlines;
                    const float* xp = g.X + (valid ? l * (int64_t)g.K : 0);
                    v[2 * j] = (valid && k < g.K) ? __ldg(xp + k) : 0.0f;
                    v[2 * j + 1] = (valid && k + 1 < g.K) ? __ldg(xp + k + 1) : 0.0f;
                }
            };
            load(0);
            for (int c = 0; c < nc; ++c) {
                const int s = c & 1, n = c >> 1;
                bool ok = true;
                if (c >= 2) ok = wait_bar(bar(EMPTY + s), (uint32_t)((n - 1) & 1), abortp, g.status);
                if (!__all_sync(0xFFFFFFFFu, ok)) break;
                uint8_t* planes = sm + (size_t)s * STAGE_BYTES + 3 * PLANE;
#pragma unroll
                for (int j = 0; j < 32; ++j) {
                    float mx = fmaxf(fabsf(v[2 * j]), fabsf(v[2 * j + 1]));
#pragma unroll
                    for (int o = 16; o > 0; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xFFFFFFFFu, mx, o));
                    const Grids gr = grids_for(mx);
                    float h0, m0, s0, h1, m1, s1;
                    split3(v[2 * j], gr, h0, m0, s0);
                    split3(v[2 * j + 1], gr, h1, m1, s1);
                    const int r = 32 * cw + j;
                    const size_t off = (size_t)r * 128 + (size_t)((((lane >> 2) ^ (r & 7)) << 4) + (lane & 3) * 4);
                    *reinterpret_cast<uint32_t*>(planes + off) = pack_bf16(h0, h1);
                    *reinterpret_cast<uint32_t*>(planes + PLANE + off) = pack_bf16(m0, m1);
                    *reinterpret_cast<uint32_t*>(planes + 2 * PLANE + off) = pack_bf16(s0, s1);
                }
                asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
                __syncwarp();
                if (lane == 0) mbar_arrive(bar(CVT_FULL + s));
                if (c + 1 < nc) load(c + 1);
            }
        }
    } else {
        // ---- epilogue (128 threads): lane quarter q of tensor memory ----
        const int q = warp & 3;
        const uint32_t lrow = (uint32_t)(32 * q) << 16;
        float acc[NL];
#pragma unroll
        for (int j = 0; j < NL; ++j) acc[j] = 0.0f;
        bool ok = true;
        for (int c = 0; c < nc && ok; ++c) {
            const int s = c & 1, n = c >> 1;
            ok = __all_sync(0xFFFFFFFFu, wait_bar(bar(ACC_FULL + s), (uint32_t)(n & 1), abortp, g.status));
            if (!ok) break;
            asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
#pragma unroll
            for (int cc = 0; cc < NL / 32; ++cc) {
                float r[32];
                tmem_ld32(tmem + lrow + (uint32_t)s * 128u + (uint32_t)(32 * cc), r);
#pragma unroll
                for (int j = 0; j < 32; ++j) acc[32 * cc + j] += r[j];
            }
            asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
            __syncwarp();
            if (lane == 0) mbar_arrive(bar(ACC_EMPTY + s));
        }
        if (ok) {
            // L1 + L2, complete with the last chunk's commit
#pragma unroll
            for (int cc = 0; cc < NL / 32; ++cc) {
                float r[32];
                tmem_ld32(tmem + lrow + 256u + (uint32_t)(32 * cc), r);
#pragma unroll
                for (int j = 0; j < 32; ++j) acc[32 * cc + j] += r[j];
            }
            const int mrow = mt * BM + 32 * q;
            if (g.inner == 1) {
                const int m = mrow + lane;
                if (m < g.Mout) {
#pragma unroll
                    for (int j = 0; j < NL; ++j) {
                        const int64_t l = l0 + j;
                        if (l < g.nlines) {
                            const int64_t at = l * g.Mout + m;
                            g.Y[at] = g.Cin[at] + acc[j];
                        }
                    }
                }
            } else {
                // transpose through this warp's 32 x 129 words (the stages are
                // idle: every copy and MMA has completed)
                float* T = reinterpret_cast<float*>(sm) + (size_t)(warp - 6) * 32 * (NL + 1);
#pragma unroll
                for (int j = 0; j < NL; ++j) T[lane * (NL + 1) + j] = acc[j];
                __syncwarp();
                int64_t ob[NL / 32];
                bool ov[NL / 32];
#pragma unroll
                for (int jj = 0; jj < NL / 32; ++jj) {
                    const int64_t l = l0 + lane + 32 * jj;
                    ov[jj] = l < g.nlines;
                    ob[jj] = ov[jj] ? (l / g.inner) * (int64_t)g.Mout * g.inner + (l % g.inner) : 0;
                }
                for (int rr = 0; rr < 32; ++rr) {
                    const int m = mrow + rr;
                    if (m >= g.Mout) break;
#pragma unroll
                    for (int jj = 0; jj < NL / 32; ++jj)
                        if (ov[jj]) {
                            const int64_t at = ob[jj] + (int64_t)m * g.inner;
                            g.Y[at] = g.Cin[at] + T[rr * (NL + 1) + lane + 32 * jj];
                        }
                }
            }
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
    if (warp == 1)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(tmem), "r"(TMEM_COLS)
                     : "memory");
#endif
}

typedef CUresult (*EncodeTiled)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiled encoder() {
    static EncodeTiled fn = nullptr;
    static bool tried = false;
    if (!tried) {
        tried = true;
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = (EncodeTiled)p;
    }
    return fn;
}

// BF16 bits of a value with at most 8 significant bits (exact).
uint16_t bf16_exact(double x) {
    const float f = (float)x;
    uint32_t u;
    std::memcpy(&u, &f, 4);
    return (uint16_t)(u >> 16);
}

}  // namespace

int tc16_operator(const std::vector<double>& D, int Mout, int K, uint16_t** planes, CUtensorMap* map) {
    const int Mpad = (Mout + BM - 1) / BM * BM, Kpad = (K + BK - 1) / BK * BK;
    const size_t P = (size_t)Mpad * Kpad;
    std::vector<uint16_t> h(3 * P, 0);
    for (int m = 0; m < Mout; ++m)
        for (int k0 = 0; k0 < K; k0 += BK) {
            const int k1 = k0 + BK < K ? k0 + BK : K;
            double mx = 0;
            for (int k = k0; k < k1; ++k) mx = std::fmax(mx, std::fabs(D[(size_t)m * K + k]));
            if (mx == 0) continue;
            int E;
            std::frexp(mx, &E);                        // 2^E > mx
            const double g0 = std::ldexp(1.0, E - 8), g1 = std::ldexp(1.0, E - 16), g2 = std::ldexp(1.0, E - 24);
            for (int k = k0; k < k1; ++k) {
                const double x = D[(size_t)m * K + k];
                const double a = std::nearbyint(x / g0) * g0;
                const double r1 = x - a;
                const double b = std::nearbyint(r1 / g1) * g1;
                const double c = std::nearbyint((r1 - b) / g2) * g2;
                const size_t at = (size_t)m * Kpad + k;
                h[at] = bf16_exact(a);
                h[P + at] = bf16_exact(b);
                h[2 * P + at] = bf16_exact(c);
            }
        }
    cudaError_t e = cudaMalloc((void**)planes, h.size() * sizeof(uint16_t));
    if (e != cudaSuccess) return (int)e;
    e = cudaMemcpy(*planes, h.data(), h.size() * sizeof(uint16_t), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) return (int)e;
    EncodeTiled enc = encoder();
    if (!enc) return -1;
    const cuuint64_t dims[3] = {(cuuint64_t)Kpad, (cuuint64_t)Mpad, 3};
    const cuuint64_t strides[2] = {(cuuint64_t)Kpad * 2, (cuuint64_t)P * 2};
    const cuuint32_t box[3] = {(cuuint32_t)BK, (cuuint32_t)BM, 3};
    const cuuint32_t estr[3] = {1, 1, 1};
    const CUresult r = enc(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 3, *planes, dims, strides, box, estr,
                           CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                           CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS ? 0 : -1;
}

cudaError_t tc16_set_smem() {
    return cudaFuncSetAttribute(k_tc16, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)SMEM);
}

size_t tc16_smem_bytes() { return SMEM; }

cudaError_t tc16_launch(const CUtensorMap& map, const Tc16Gemm& g, cudaStream_t st) {
    const int64_t tiles = (g.nlines + NL - 1) / NL;
    if (tiles * g.MT > 0x7FFFFFFF) return cudaErrorInvalidValue;
    k_tc16<<<(unsigned)(tiles * g.MT), THREADS, SMEM, st>>>(map, g);
    return cudaGetLastError();
}

}  // namespace pstd
