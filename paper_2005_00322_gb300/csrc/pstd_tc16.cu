// pstd_tc16.cu -- split-precision dense form of the axis pass with BF16
// operands on the 5th-generation tensor cores (tcgen05.mma kind::f16, FP32
// accumulators in tensor memory, operator tiles fed by TMA).
//
// Each staggered derivative of an axis is a dense FP64-built operator D
// (Section 3.2: the transforms, k-multiply and inverse of Table 2 as one
// matrix, the time-step factors folded in) applied to every line:
//     Y[line, m] = Cin[line, m] + sum_k D[m, k] X[line, k].
//
// Split into BF16 slices after Ozaki, Ogita, Oishi and Rump ("Error-free
// transformations of matrix multiplication by using fast routines of matrix
// multiplication", Numer. Algorithms 59, 2012).  k runs in blocks of 32; in
// block p every operator row m has a power of two 2^E > max |D[m, k]| and
// every line one 2^F > max |X[line, k]| (over the block), and each value is
// cut into three BF16 slices on the grids 2^(E-8), 2^(E-16), 2^(E-24):
//     D = Dh + Dm + Dl   (to 2^-25 of the block's row maximum),
//     X = Xh + Xm + Xl   (exactly, FP32 having 24 significant bits),
// with |Dh|, |Xh| <= 2^8 and |Dm|, |Dl|, |Xm|, |Xl| <= 2^7 on their grids.
// Per block the main product L0 = Dh Xh is an integer below 2^21 on the grid
// 2^(E+F-16): the tensor core sums it exactly, whatever its internal rounding
// (a running FP32 sum inside the tensor core is truncated toward zero, and
// for a smooth field, whose derivative's terms cancel, such a bias would
// shrink the low modes' frequencies and grow into phase drift).  Each block's
// L0 starts from zero in one of two tensor-memory accumulators and is added
// (FP32, round to nearest) into a running sum S kept in tensor memory by the
// epilogue warps while the next block runs.  The products 2^-8 and 2^-16
// below, Dh Xm + Dm Xh + Dh Xl + Dm Xm + Dl Xh, run in one accumulator X over
// the whole k range (their truncation is 2^-8 smaller); Dm Xl, Dl Xm and
// Dl Xl (2^-23 and below) are dropped.  Y = Cin + (S + X).
//
// Persistent kernel, one CTA per SM, walking (line tile, output tile) pairs:
// a tile is 128 output rows (MMA M) x 128 lines (MMA N); the MMAs run on
// 16-wide k chunks.
//   warp 0      TMA producer: the chunk's three operator slices, one 3-D box of
//               16 k x 128 rows x 3 slices, 32-byte swizzle;
//   warp 1      allocates tensor memory; one thread issues the 6 MMAs of each
//               chunk and commits them to the stage's mbarrier and, at the
//               end of a block, to the block's accumulator mbarrier;
//   warps 2-5   converters: copy the field's 32-wide blocks into a 4-deep
//               ring in shared memory (cp.async, three blocks in flight), then
//               per block find each line's maximum, split and store the three
//               slices in the MMA's K-major 32-byte-swizzled layout;
//   warps 6-9   epilogue: add each block's L0 into S; at the end of a tile move
//               S + X into a shared output tile (which frees tensor memory for
//               the next tile) and write Y = Cin + S + X with coalesced accesses.
// Every wait is bounded: a wait that gives up sets *status and a shared abort
// flag that ends every other wait, the MMAs and copies in flight are waited
// for (bounded), and tensor memory is freed.
#include "pstd_tc16.h"

#include <cuda_bf16.h>

#include <cmath>
#include <cstring>

namespace pstd {

namespace {

constexpr int BM = 128;                        // output rows per tile (MMA M)
constexpr int NL = 128;                        // lines per tile (MMA N)
constexpr int BK = 16;                         // k per MMA chunk: one 32-byte swizzle row of BF16
constexpr int KB = 32;                         // k per scale block (two chunks)
constexpr int STAGES = 3;
constexpr int RING = 4;                        // raw field blocks in shared memory
constexpr uint32_t PLANE = BM * BK * 2;        // one BF16 slice of one chunk: 4 KB
constexpr uint32_t STAGE_BYTES = 6 * PLANE;    // operator Dh Dm Dl, field Xh Xm Xl
constexpr int RAW_LD = KB + 1;                 // contiguous layout: [line][k], padded
constexpr uint32_t RAW_BYTES = NL * RAW_LD * 4;
constexpr int OB_LD = NL + 1;                  // output tile row (padded)
constexpr uint32_t OB_BYTES = BM * OB_LD * 4;
constexpr size_t SMEM = STAGES * STAGE_BYTES + RING * RAW_BYTES + OB_BYTES + 1024;
constexpr int THREADS = 320;
constexpr uint32_t TMEM_COLS = 512;            // L0[0] 0, L0[1] 128, X 256, S 384
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
// Warp-uniform bounded wait.
__device__ __forceinline__ bool warp_wait(uint32_t bar, uint32_t parity, volatile int* abort_flag, int* status) {
    return __all_sync(0xFFFFFFFFu, wait_bar(bar, parity, abort_flag, status));
}
// Barrier among the 128 threads of one warp group (id 1..3; 0 is
// __syncthreads), returning the AND of `v` over the group so that every warp
// of the group takes the same branch after it.
__device__ __forceinline__ bool group_and(int id, bool v) {
    uint32_t r;
    asm volatile(
        "{\n .reg .pred p, q;\n setp.ne.u32 q, %1, 0;\n bar.red.and.pred p, %2, 128, q;\n"
        " selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(r)
        : "r"((uint32_t)v), "r"(id)
        : "memory");
    return r != 0;
}
__device__ __forceinline__ void group_sync(int id) { asm volatile("bar.sync %0, 128;\n" ::"r"(id) : "memory"); }

// 4-byte asynchronous copy global -> shared; `n` = 0 stores a zero.
__device__ __forceinline__ void cp4(uint32_t dst, const float* src, int n) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;\n" ::"r"(dst), "l"(src), "r"(n) : "memory");
}
__device__ __forceinline__ void cp_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_wait() { asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory"); }

// K-major operand tile with 32-byte swizzle: rows of 32 bytes, 8-row groups
// 256 bytes apart (SBO); the leading offset is unused for this layout.
__device__ __forceinline__ uint64_t desc_sw32(uint32_t addr) {
    uint64_t d = (uint64_t)((addr & 0x3FFFFu) >> 4);
    d |= (uint64_t)1 << 16;
    d |= (uint64_t)(256u >> 4) << 32;
    d |= (uint64_t)1 << 46;            // descriptor version of the tcgen05 family
    d |= (uint64_t)6 << 61;            // 32-byte swizzle
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

#define TC16_R32 "{%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}"
// 32 consecutive accumulator columns of this warp's 32 lanes (no wait).
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, uint32_t (&r)[32]) {
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x32.b32 " TC16_R32 ", [%32];\n"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
                   "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
                   "=r"(r[14]), "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]),
                   "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]),
                   "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
                 : "r"(taddr)
                 : "memory");
}
__device__ __forceinline__ void tmem_st32(uint32_t taddr, const uint32_t (&r)[32]) {
    asm volatile("tcgen05.st.sync.aligned.32x32b.x32.b32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,"
                 "%14,%15,%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31,%32};\n" ::"r"(taddr),
                 "r"(r[0]), "r"(r[1]), "r"(r[2]), "r"(r[3]), "r"(r[4]), "r"(r[5]), "r"(r[6]), "r"(r[7]),
                 "r"(r[8]), "r"(r[9]), "r"(r[10]), "r"(r[11]), "r"(r[12]), "r"(r[13]), "r"(r[14]), "r"(r[15]),
                 "r"(r[16]), "r"(r[17]), "r"(r[18]), "r"(r[19]), "r"(r[20]), "r"(r[21]), "r"(r[22]), "r"(r[23]),
                 "r"(r[24]), "r"(r[25]), "r"(r[26]), "r"(r[27]), "r"(r[28]), "r"(r[29]), "r"(r[30]), "r"(r[31])
                 : "memory");
}

// Rounding constants 1.5 * 2^(E+15), 1.5 * 2^(E+7), 1.5 * 2^(E-1): adding
// and subtracting one rounds (to nearest even) to the grid 2^(E-8),
// 2^(E-16), 2^(E-24) of a value below 2^E.
struct Grids {
    float c0, c1, c2;
};
__device__ __forceinline__ Grids grids_for(float mx) {
    int E = (int)((__float_as_uint(mx) >> 23) & 0xFFu) - 126;   // 2^E > mx
    E = E < -90 ? -90 : (E > 90 ? 90 : E);
    const int e0 = E + 15 + 127;
    Grids g;
    g.c0 = __uint_as_float(((uint32_t)e0 << 23) | 0x400000u);
    g.c1 = __uint_as_float(((uint32_t)(e0 - 8) << 23) | 0x400000u);
    g.c2 = __uint_as_float(((uint32_t)(e0 - 16) << 23) | 0x400000u);
    return g;
}
// x = h + m + l, each on its grid; the adds and subtracts are the _rn
// intrinsics so that nothing contracts or reassociates them.
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
    __shared__ __align__(8) uint64_t bars[3 * STAGES + 6];
    __shared__ uint32_t tmem_slot;
    __shared__ int abort_flag;
    uint8_t* sm = (uint8_t*)(((uintptr_t)tc16_raw + 1023) & ~(uintptr_t)1023);
    float* RAW = reinterpret_cast<float*>(sm + STAGES * STAGE_BYTES);
    float* OB = reinterpret_cast<float*>(sm + STAGES * STAGE_BYTES + RING * RAW_BYTES);
    const uint32_t sbase = smem_u32(sm);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int nc = g.KC;                        // 16-wide chunks per tile
    const int nb = (nc + 1) / 2;                // 32-wide blocks per tile
    const int64_t ntiles = ((g.nlines + NL - 1) / NL) * g.MT;
    volatile int* abortp = &abort_flag;
    auto bar = [&](int i) { return smem_u32(&bars[i]); };
    // tma_full[S], cvt_full[S], empty[S], blk_full[2], blk_empty[2], acc_empty, final
    const int TMA_FULL = 0, CVT_FULL = STAGES, EMPTY = 2 * STAGES, BLK_FULL = 3 * STAGES,
              BLK_EMPTY = BLK_FULL + 2, ACC_EMPTY = BLK_FULL + 4, FINAL = BLK_FULL + 5;
    auto tile_of = [&](int64_t j, int& mt, int64_t& l0) {
        const int64_t tix = (int64_t)blockIdx.x + j * gridDim.x;
        mt = (int)(tix % g.MT);
        l0 = (tix / g.MT) * NL;
    };
    const int64_t my_tiles = (int64_t)blockIdx.x < ntiles ? (ntiles - 1 - blockIdx.x) / gridDim.x + 1 : 0;

    if (tid == 0) {
        abort_flag = 0;
        for (int s = 0; s < STAGES; ++s) {
            mbar_init(bar(TMA_FULL + s), 1);
            mbar_init(bar(CVT_FULL + s), 4);
            mbar_init(bar(EMPTY + s), 1);
        }
        for (int b = 0; b < 2; ++b) {
            mbar_init(bar(BLK_FULL + b), 1);
            mbar_init(bar(BLK_EMPTY + b), 4);
        }
        mbar_init(bar(ACC_EMPTY), 4);
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
            int issued[STAGES] = {};
            int64_t gc = 0;                 // chunk count over this CTA's tiles
            bool ok = true;
            for (int64_t j = 0; j < my_tiles && ok; ++j) {
                int mt;
                int64_t l0;
                tile_of(j, mt, l0);
                for (int c = 0; c < nc; ++c, ++gc) {
                    const int s = (int)(gc % STAGES);
                    const int64_t n = gc / STAGES;
                    if (gc >= STAGES && !wait_bar(bar(EMPTY + s), (uint32_t)((n - 1) & 1), abortp, g.status)) {
                        ok = false;
                        break;
                    }
                    mbar_expect_tx(bar(TMA_FULL + s), 3 * PLANE);
                    asm volatile(
                        "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
                        " [%0], [%1, {%3, %4, %5}], [%2];\n" ::"r"(sbase + (uint32_t)s * STAGE_BYTES),
                        "l"((uint64_t)&map), "r"(bar(TMA_FULL + s)), "r"(c * BK), "r"(mt * BM), "r"(0)
                        : "memory");
                    issued[s] = (int)(n + 1);
                }
            }
            // copies still in flight land before the CTA ends
            for (int s = 0; s < STAGES; ++s)
                if (issued[s] > 0) drain_bar(bar(TMA_FULL + s), (uint32_t)((issued[s] - 1) & 1), g.status);
        }
    } else if (warp == 1) {
        // ---- MMA issuer ----
        if (lane == 0) {
            const uint32_t X = tmem + 256u;
            int64_t gc = 0, gb = 0;         // chunks and blocks over this CTA's tiles
            bool ok = true;
            for (int64_t j = 0; j < my_tiles && ok; ++j) {
                // the epilogue has moved the previous tile's X and S out
                if (j > 0 && !wait_bar(bar(ACC_EMPTY), (uint32_t)((j - 1) & 1), abortp, g.status)) break;
                for (int c = 0; c < nc; ++c, ++gc) {
                    const int s = (int)(gc % STAGES);
                    const int64_t n = gc / STAGES;
                    const int slot = (int)(gb & 1);
                    ok = wait_bar(bar(TMA_FULL + s), (uint32_t)(n & 1), abortp, g.status) &&
                         wait_bar(bar(CVT_FULL + s), (uint32_t)(n & 1), abortp, g.status);
                    // the first chunk of a block reuses the L0 slot of block gb - 2
                    if (ok && (c & 1) == 0 && gb >= 2)
                        ok = wait_bar(bar(BLK_EMPTY + slot), (uint32_t)(((gb >> 1) - 1) & 1), abortp, g.status);
                    if (!ok) break;
                    asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
                    const uint32_t st = sbase + (uint32_t)s * STAGE_BYTES;
                    const uint64_t dh = desc_sw32(st), dm = desc_sw32(st + PLANE), dl = desc_sw32(st + 2 * PLANE);
                    const uint32_t f = st + 3 * PLANE;
                    const uint64_t xh = desc_sw32(f), xm = desc_sw32(f + PLANE), xl = desc_sw32(f + 2 * PLANE);
                    const uint32_t L0 = tmem + (uint32_t)slot * 128u;
                    const uint32_t xacc = c > 0 ? 1u : 0u;
                    mma_bf16(X, dh, xm, xacc);
                    mma_bf16(X, dm, xh, 1u);
                    mma_bf16(X, dh, xl, 1u);
                    mma_bf16(X, dm, xm, 1u);
                    mma_bf16(X, dl, xh, 1u);
                    mma_bf16(L0, dh, xh, (c & 1) ? 1u : 0u);
                    mma_commit(bar(EMPTY + s));
                    if ((c & 1) == 1 || c == nc - 1) {
                        mma_commit(bar(BLK_FULL + slot));
                        ++gb;
                    }
                }
            }
            // every MMA issued has completed before tensor memory is freed
            mma_commit(bar(FINAL));
            drain_bar(bar(FINAL), 0u, g.status);
        }
    } else if (warp < 6) {
        // ---- converters (128 threads): thread t owns line l0 + t of each tile ----
        const int cw = warp - 2, t = tid - 64;
        // copies of block p of tile j into ring slot (total block count) % RING
        auto issue_block = [&](int64_t j, int p, int slot) {
            int mt;
            int64_t l0;
            tile_of(j, mt, l0);
            float* raw = RAW + (size_t)slot * (RAW_BYTES / 4);
            const int k0 = p * KB;
            if (g.inner > 1) {
                // raw[k][line]: thread t copies its own line
                const int64_t l = l0 + t;
                const bool valid = l < g.nlines;
                const float* xp = g.X + (valid ? (l / g.inner) * (int64_t)g.K * g.inner + (l % g.inner) : 0);
#pragma unroll 8
                for (int k = 0; k < KB; ++k) {
                    const bool in = valid && k0 + k < g.K;
                    cp4(smem_u32(raw + k * NL + t), in ? xp + (int64_t)(k0 + k) * g.inner : g.X, in ? 4 : 0);
                }
            } else {
                // raw[line][k] (padded rows): warp cw copies its 32 lines, lane = k
#pragma unroll 8
                for (int jj = 0; jj < 32; ++jj) {
                    const int r = 32 * cw + jj;
                    const int64_t l = l0 + r;
                    const bool in = l < g.nlines && k0 + lane < g.K;
                    cp4(smem_u32(raw + r * RAW_LD + lane), in ? g.X + l * (int64_t)g.K + k0 + lane : g.X, in ? 4 : 0);
                }
            }
        };
        // the blocks in order over this CTA's tiles: (tile, block) of index q
        int64_t qj = 0;
        int qp = 0;
        auto next_q = [&]() {
            if (++qp == nb) {
                qp = 0;
                ++qj;
            }
        };
        // fill the ring: RING - 1 blocks ahead
        int64_t issued = 0;
        for (int i = 0; i < RING - 1; ++i) {
            if (qj < my_tiles) {
                issue_block(qj, qp, (int)(issued % RING));
                next_q();
            }
            cp_commit();
            ++issued;
        }
        int64_t gc = 0, done = 0;
        bool ok = true;
        for (int64_t j = 0; j < my_tiles && ok; ++j) {
            for (int p = 0; p < nb && ok; ++p, ++done) {
                // block `done` has landed (this thread's copies; __syncwarp for
                // the contiguous layout, whose rows the warp copied together)
                cp_wait<RING - 2>();
                __syncwarp();
                const float* raw = RAW + (size_t)(done % RING) * (RAW_BYTES / 4);
                float v[KB];
#pragma unroll
                for (int k = 0; k < KB; ++k) v[k] = g.inner > 1 ? raw[k * NL + t] : raw[t * RAW_LD + k];
                __syncwarp();
                // refill the slot just read
                if (qj < my_tiles) {
                    issue_block(qj, qp, (int)(issued % RING));
                    next_q();
                }
                cp_commit();
                ++issued;
                float mx = 0.0f;
#pragma unroll
                for (int k = 0; k < KB; ++k) mx = fmaxf(mx, fabsf(v[k]));
                const Grids gr = grids_for(mx);
                for (int h2 = 0; h2 < 2; ++h2) {
                    if (2 * p + h2 >= nc) break;
                    const int s = (int)(gc % STAGES);
                    bool w = true;
                    if (gc >= STAGES)
                        w = wait_bar(bar(EMPTY + s), (uint32_t)((gc / STAGES - 1) & 1), abortp, g.status);
                    if (!__all_sync(0xFFFFFFFFu, w)) {
                        ok = false;
                        break;
                    }
                    uint8_t* row = sm + (size_t)s * STAGE_BYTES + 3 * PLANE + (size_t)t * 32;
#pragma unroll
                    for (int qq = 0; qq < 2; ++qq) {
                        uint32_t w3[3][4];
#pragma unroll
                        for (int e = 0; e < 4; ++e) {
                            float h0, m0, s0, h1, m1, s1;
                            const int k = 16 * h2 + 8 * qq + 2 * e;
                            split3(v[k], gr, h0, m0, s0);
                            split3(v[k + 1], gr, h1, m1, s1);
                            w3[0][e] = pack_bf16(h0, h1);
                            w3[1][e] = pack_bf16(m0, m1);
                            w3[2][e] = pack_bf16(s0, s1);
                        }
                        const uint32_t off = (uint32_t)((qq ^ ((t >> 2) & 1)) << 4);
#pragma unroll
                        for (int pl = 0; pl < 3; ++pl)
                            *reinterpret_cast<uint4*>(row + (size_t)pl * PLANE + off) =
                                make_uint4(w3[pl][0], w3[pl][1], w3[pl][2], w3[pl][3]);
                    }
                    asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
                    __syncwarp();
                    if (lane == 0) mbar_arrive(bar(CVT_FULL + s));
                    ++gc;
                }
            }
        }
        cp_wait<0>();     // no copy outlives the CTA
    } else {
        // ---- epilogue (128 threads): lane quarter q of tensor memory ----
        const int q = warp & 3, ew = warp - 6;
        const uint32_t lrow = (uint32_t)(32 * q) << 16;
        const uint32_t X = tmem + lrow + 256u, S = tmem + lrow + 384u;
        int64_t gb = 0;
        for (int64_t j = 0; j < my_tiles; ++j) {
            int mt;
            int64_t l0;
            tile_of(j, mt, l0);
            bool ok = true;
            // S = sum of the blocks' L0, each added as soon as it completes
            for (int p = 0; p < nb; ++p, ++gb) {
                const int slot = (int)(gb & 1);
                ok = warp_wait(bar(BLK_FULL + slot), (uint32_t)((gb >> 1) & 1), abortp, g.status);
                if (!ok) break;
                asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
                const uint32_t L0 = tmem + lrow + (uint32_t)slot * 128u;
                for (int pc = 0; pc < NL / 32; ++pc) {
                    uint32_t a[32], b[32];
                    tmem_ld32(L0 + (uint32_t)(32 * pc), a);
                    if (p > 0) tmem_ld32(S + (uint32_t)(32 * pc), b);
                    asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::: "memory");
                    if (p > 0)
#pragma unroll
                        for (int jj = 0; jj < 32; ++jj)
                            a[jj] = __float_as_uint(__uint_as_float(a[jj]) + __uint_as_float(b[jj]));
                    tmem_st32(S + (uint32_t)(32 * pc), a);
                }
                asm volatile("tcgen05.wait::st.sync.aligned;\n" ::: "memory");
                asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
                __syncwarp();
                if (lane == 0) mbar_arrive(bar(BLK_EMPTY + slot));
            }
            // the last block's commit covered every MMA of the tile (X too);
            // all four warps leave together if one gave up
            if (!group_and(1, ok)) break;
            asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
            // S + X of this thread's row into the output tile: [line][row] on
            // contiguous axes, [row][line] on strided ones
            const int r = 32 * q + lane;
            for (int pc = 0; pc < NL / 32; ++pc) {
                uint32_t a[32], b[32];
                tmem_ld32(S + (uint32_t)(32 * pc), a);
                tmem_ld32(X + (uint32_t)(32 * pc), b);
                asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::: "memory");
#pragma unroll
                for (int jj = 0; jj < 32; ++jj) {
                    const float val = __uint_as_float(a[jj]) + __uint_as_float(b[jj]);
                    if (g.inner == 1) OB[(32 * pc + jj) * OB_LD + r] = val;
                    else OB[r * OB_LD + 32 * pc + jj] = val;
                }
            }
            // X and S are free for the next tile
            asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
            __syncwarp();
            if (lane == 0) mbar_arrive(bar(ACC_EMPTY));
            group_sync(1);
            // Y = Cin + sum, coalesced: contiguous axes walk lines (the rows of
            // the tile are consecutive words), strided axes walk rows.  Each
            // warp takes every fourth line (row) in batches of 16, so that 64
            // loads of Cin per lane are in flight at once.
            constexpr int WB = 16;
            if (g.inner == 1) {
                for (int b0 = 0; b0 < NL / 4; b0 += WB) {
                    float cin[WB][4];
#pragma unroll
                    for (int u = 0; u < WB; ++u) {
                        const int64_t lg = l0 + ew + 4 * (b0 + u);
#pragma unroll
                        for (int i = 0; i < 4; ++i) {
                            const int m = mt * BM + 32 * i + lane;
                            cin[u][i] = (lg < g.nlines && m < g.Mout) ? g.Cin[lg * g.Mout + m] : 0.0f;
                        }
                    }
#pragma unroll
                    for (int u = 0; u < WB; ++u) {
                        const int ll = ew + 4 * (b0 + u);
                        const int64_t lg = l0 + ll;
#pragma unroll
                        for (int i = 0; i < 4; ++i) {
                            const int m = mt * BM + 32 * i + lane;
                            if (lg < g.nlines && m < g.Mout)
                                g.Y[lg * g.Mout + m] = cin[u][i] + OB[ll * OB_LD + 32 * i + lane];
                        }
                    }
                }
            } else {
                int64_t ob[4];
                bool ov[4];
#pragma unroll
                for (int i = 0; i < 4; ++i) {
                    const int64_t lg = l0 + 32 * i + lane;
                    ov[i] = lg < g.nlines;
                    ob[i] = ov[i] ? (lg / g.inner) * (int64_t)g.Mout * g.inner + (lg % g.inner) : 0;
                }
                for (int b0 = 0; b0 < BM / 4; b0 += WB) {
                    float cin[WB][4];
#pragma unroll
                    for (int u = 0; u < WB; ++u) {
                        const int m = mt * BM + ew + 4 * (b0 + u);
#pragma unroll
                        for (int i = 0; i < 4; ++i)
                            cin[u][i] = (ov[i] && m < g.Mout) ? g.Cin[ob[i] + (int64_t)m * g.inner] : 0.0f;
                    }
#pragma unroll
                    for (int u = 0; u < WB; ++u) {
                        const int rr = ew + 4 * (b0 + u);
                        const int m = mt * BM + rr;
#pragma unroll
                        for (int i = 0; i < 4; ++i)
                            if (ov[i] && m < g.Mout)
                                g.Y[ob[i] + (int64_t)m * g.inner] = cin[u][i] + OB[rr * OB_LD + 32 * i + lane];
                    }
                }
            }
            group_sync(1);      // the output tile is read before the next one overwrites it
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
    const int Mpad = (Mout + BM - 1) / BM * BM, Kpad = (K + KB - 1) / KB * KB;
    const size_t P = (size_t)Mpad * Kpad;
    std::vector<uint16_t> h(3 * P, 0);
    for (int m = 0; m < Mout; ++m)
        for (int k0 = 0; k0 < K; k0 += KB) {
            const int k1 = k0 + KB < K ? k0 + KB : K;
            double mx = 0;
            for (int k = k0; k < k1; ++k) mx = std::fmax(mx, std::fabs(D[(size_t)m * K + k]));
            if (mx == 0) continue;
            int E;
            std::frexp(mx, &E);                        // 2^E > mx
            for (int k = k0; k < k1; ++k) {
                double r = D[(size_t)m * K + k];
                for (int p = 0; p < 3; ++p) {
                    const double gp = std::ldexp(1.0, E - 8 - 8 * p);
                    const double a = std::nearbyint(r / gp) * gp;
                    h[(size_t)p * P + (size_t)m * Kpad + k] = bf16_exact(a);
                    r -= a;
                }
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
                           CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_32B,
                           CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS ? 0 : -1;
}

int tc16_chunks(int K) { return (K + KB - 1) / KB * (KB / BK); }

cudaError_t tc16_set_smem() {
    return cudaFuncSetAttribute(k_tc16, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)SMEM);
}

size_t tc16_smem_bytes() { return SMEM; }

cudaError_t tc16_launch(const CUtensorMap& map, const Tc16Gemm& g, cudaStream_t st) {
    static thread_local int dev_cached = -1, nsm = 0;
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev != dev_cached) {
        e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
        if (e != cudaSuccess) return e;
        dev_cached = dev;
    }
    const int64_t tiles = (g.nlines + NL - 1) / NL * g.MT;
    const int64_t grid = tiles < nsm ? tiles : nsm;      // persistent: at most one CTA per SM
    if (grid <= 0) return cudaSuccess;
    k_tc16<<<(unsigned)grid, THREADS, SMEM, st>>>(map, g);
    return cudaGetLastError();
}

}  // namespace pstd
