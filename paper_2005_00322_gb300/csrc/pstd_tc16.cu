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
// Fields are read and written by TMA: the plan keeps p, the velocities and
// the accumulator in its own copies whose last dimension is padded to a
// multiple of 4 floats, so that every tensor map stride is a multiple of 16
// bytes.  Lines and rows beyond a field's extent read as zeros and are not
// written (the tensor maps carry the true extents).
//
// Persistent kernel, one CTA per SM, walking (line tile, output tile) pairs:
// a tile is 128 output rows (MMA M) x 128 lines (MMA N); the MMAs run on
// 16-wide k chunks.
//   warp 0      producer: the chunk's three operator slices, one contiguous
//               12 KB bulk copy (the host stores the operator tiled and
//               swizzled exactly as the MMA reads it);
//   warp 1      allocates tensor memory; one thread issues the 6 MMAs of each
//               chunk and commits them to the stage's mbarrier and, at the
//               end of a block, to the block's accumulator mbarrier;
//   warps 2-5   converters: the field's 32-wide blocks arrive by TMA in a
//               4-deep ring (three in flight); per block each thread finds its
//               line's maximum, splits the values and stores the three slices
//               in the MMA's K-major 32-byte-swizzled layout;
//   warps 6-9   epilogue: the tile's Cin arrives by TMA in a shared output
//               tile while the blocks run; each block's L0 is added into S;
//               at the end S + X is added into the output tile (which frees
//               tensor memory for the next tile) and a TMA store writes Y.
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
constexpr int STAGES = 4;
constexpr int RING = 3;                        // field blocks in shared memory (two in flight)
constexpr uint32_t PLANE = BM * BK * 2;        // one BF16 slice of one chunk: 4 KB
constexpr uint32_t STAGE_BYTES = 6 * PLANE;    // operator Dh Dm Dl, field Xh Xm Xl
constexpr uint32_t RAW_BYTES = NL * KB * 4;    // one FP32 field block: 16 KB
constexpr uint32_t OB_BYTES = BM * NL * 4;     // the output tile: 64 KB
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

// Contiguous bulk copy (16-byte aligned, size a multiple of 16) into this
// CTA's shared memory, completing on an mbarrier.
__device__ __forceinline__ void bulk_load(uint32_t dst, const void* src, uint32_t bytes, uint32_t bar) {
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];\n" ::"r"(dst),
                 "l"((uint64_t)src), "r"(bytes), "r"(bar)
                 : "memory");
}
// TMA tile loads into this CTA's shared memory, completing on an mbarrier.
__device__ __forceinline__ void tma_load2(uint32_t dst, const CUtensorMap* m, uint32_t bar, int c0, int c1) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%3, %4}], [%2];\n" ::"r"(
            dst),
        "l"((uint64_t)m), "r"(bar), "r"(c0), "r"(c1)
        : "memory");
}
__device__ __forceinline__ void tma_load3(uint32_t dst, const CUtensorMap* m, uint32_t bar, int c0, int c1, int c2) {
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%3, %4, %5}], "
        "[%2];\n" ::"r"(dst),
        "l"((uint64_t)m), "r"(bar), "r"(c0), "r"(c1), "r"(c2)
        : "memory");
}
// TMA tile stores from shared memory (bulk async group of this thread).
__device__ __forceinline__ void tma_store2(const CUtensorMap* m, uint32_t src, int c0, int c1) {
    asm volatile("cp.async.bulk.tensor.2d.global.shared::cta.tile.bulk_group [%0, {%2, %3}], [%1];\n" ::"l"(
                     (uint64_t)m),
                 "r"(src), "r"(c0), "r"(c1)
                 : "memory");
}
__device__ __forceinline__ void tma_store3(const CUtensorMap* m, uint32_t src, int c0, int c1, int c2) {
    asm volatile("cp.async.bulk.tensor.3d.global.shared::cta.tile.bulk_group [%0, {%2, %3, %4}], [%1];\n" ::"l"(
                     (uint64_t)m),
                 "r"(src), "r"(c0), "r"(c1), "r"(c2)
                 : "memory");
}

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

__global__ void __launch_bounds__(THREADS, 1)
    k_tc16(const __grid_constant__ CUtensorMap mx, const __grid_constant__ CUtensorMap mcin,
           const __grid_constant__ CUtensorMap my, const Tc16Gemm g) {
#ifdef __CUDA_ARCH__
    extern __shared__ uint8_t tc16_raw[];
    __shared__ __align__(8) uint64_t bars[3 * STAGES + RING + 7];
    __shared__ uint32_t tmem_slot;
    __shared__ int abort_flag;
    uint8_t* sm = (uint8_t*)(((uintptr_t)tc16_raw + 1023) & ~(uintptr_t)1023);
    uint8_t* RAW = sm + STAGES * STAGE_BYTES;
    float* OB = reinterpret_cast<float*>(sm + STAGES * STAGE_BYTES + RING * RAW_BYTES);
    const uint32_t sbase = smem_u32(sm);
    const uint32_t rbase = sbase + STAGES * STAGE_BYTES, obase = rbase + RING * RAW_BYTES;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int nc = g.KC;                        // 16-wide chunks per tile
    const int nb = (nc + 1) / 2;                // 32-wide blocks per tile
    const int64_t ntiles = g.tiles * g.MT;
    volatile int* abortp = &abort_flag;
    auto bar = [&](int i) { return smem_u32(&bars[i]); };
    // tma_full[S], cvt_full[S], empty[S], raw_full[RING], blk_full[2],
    // blk_empty[2], acc_empty, cin_full, final
    const int TMA_FULL = 0, CVT_FULL = STAGES, EMPTY = 2 * STAGES, RAW_FULL = 3 * STAGES,
              BLK_FULL = RAW_FULL + RING, BLK_EMPTY = BLK_FULL + 2, ACC_EMPTY = BLK_FULL + 4,
              CIN_FULL = BLK_FULL + 5, FINAL = BLK_FULL + 6;
    // the j-th tile of this CTA: output tile mt, line tile lt -> TMA
    // coordinates of its lines (contiguous axis: row l0; strided: inner i0 of
    // outer block o)
    struct TileAt {
        int mt, l0, i0, o;
    };
    auto tile_of = [&](int64_t j) {
        const int64_t tix = (int64_t)blockIdx.x + j * gridDim.x;
        TileAt t;
        t.mt = (int)(tix % g.MT);
        const int64_t lt = tix / g.MT;
        if (g.contiguous) {
            t.l0 = (int)(lt * NL);
            t.i0 = t.o = 0;
        } else {
            t.o = (int)(lt / g.tpo);
            t.i0 = (int)((lt % g.tpo) * NL);
            t.l0 = 0;
        }
        return t;
    };
    const int64_t my_tiles = (int64_t)blockIdx.x < ntiles ? (ntiles - 1 - blockIdx.x) / gridDim.x + 1 : 0;

    if (tid == 0) {
        abort_flag = 0;
        for (int s = 0; s < STAGES; ++s) {
            mbar_init(bar(TMA_FULL + s), 1);
            mbar_init(bar(CVT_FULL + s), 4);
            mbar_init(bar(EMPTY + s), 1);
        }
        for (int r = 0; r < RING; ++r) mbar_init(bar(RAW_FULL + r), 1);
        for (int b = 0; b < 2; ++b) {
            mbar_init(bar(BLK_FULL + b), 1);
            mbar_init(bar(BLK_EMPTY + b), 4);
        }
        mbar_init(bar(ACC_EMPTY), 4);
        mbar_init(bar(CIN_FULL), 1);
        mbar_init(bar(FINAL), 1);
        asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
        asm volatile("prefetch.tensormap [%0];\n" ::"l"((uint64_t)&mx) : "memory");
        asm volatile("prefetch.tensormap [%0];\n" ::"l"((uint64_t)&mcin) : "memory");
        asm volatile("prefetch.tensormap [%0];\n" ::"l"((uint64_t)&my) : "memory");
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
                const TileAt t = tile_of(j);
                for (int c = 0; c < nc; ++c, ++gc) {
                    const int s = (int)(gc % STAGES);
                    const int64_t n = gc / STAGES;
                    if (gc >= STAGES && !wait_bar(bar(EMPTY + s), (uint32_t)((n - 1) & 1), abortp, g.status)) {
                        ok = false;
                        break;
                    }
                    mbar_expect_tx(bar(TMA_FULL + s), 3 * PLANE);
                    bulk_load(sbase + (uint32_t)s * STAGE_BYTES, g.op + ((size_t)t.mt * nc + c) * (3 * PLANE),
                              3 * PLANE, bar(TMA_FULL + s));
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
        // ---- converters (128 threads): thread t owns line t of each tile ----
        const int t = tid - 64;
        // the blocks in order over this CTA's tiles: (tile, block) of index q
        int64_t qj = 0;
        int qp = 0;
        auto issue_next = [&](int slot) {       // thread 0: the next block into `slot`
            if (qj >= my_tiles) return false;
            const TileAt tl = tile_of(qj);
            const uint32_t dst = rbase + (uint32_t)slot * RAW_BYTES;
            mbar_expect_tx(bar(RAW_FULL + slot), RAW_BYTES);
            if (g.contiguous) tma_load2(dst, &mx, bar(RAW_FULL + slot), qp * KB, tl.l0);
            else tma_load3(dst, &mx, bar(RAW_FULL + slot), tl.i0, qp * KB, tl.o);
            if (++qp == nb) {
                qp = 0;
                ++qj;
            }
            return true;
        };
        int64_t inflight = 0;                   // blocks issued (thread 0)
        if (t == 0)
            for (int i = 0; i < RING - 1; ++i)
                if (issue_next((int)(inflight % RING))) ++inflight;
        // The four converter warps meet at a named barrier once per block, so
        // none of them leaves the loop early: after a failed wait (`live`
        // false) they keep iterating without work, every later wait failing
        // at once on the abort flag.
        int64_t gc = 0, q = 0, waited = 0;
        bool live = true;
        for (int64_t j = 0; j < my_tiles; ++j) {
            for (int p = 0; p < nb; ++p, ++q) {
                const int slot = (int)(q % RING);
                live = live && warp_wait(bar(RAW_FULL + slot), (uint32_t)((q / RING) & 1), abortp, g.status);
                if (live) waited = q + 1;
                // this thread's line of the block: [line][32 k] rows of 128 bytes
                // with 128-byte swizzle (contiguous axis), [32 k][line] (strided)
                const uint8_t* raw = RAW + (size_t)slot * RAW_BYTES;
                float v[KB];
                if (g.contiguous) {
#pragma unroll
                    for (int c = 0; c < 8; ++c) {
                        const float4 w4 = *reinterpret_cast<const float4*>(raw + (size_t)t * 128 +
                                                                           (size_t)((c ^ (t & 7)) << 4));
                        v[4 * c] = w4.x;
                        v[4 * c + 1] = w4.y;
                        v[4 * c + 2] = w4.z;
                        v[4 * c + 3] = w4.w;
                    }
                } else {
#pragma unroll
                    for (int k = 0; k < KB; ++k) v[k] = reinterpret_cast<const float*>(raw)[k * NL + t];
                }
                // every converter has read the slot: thread 0 refills it
                group_sync(2);
                if (t == 0 && live && issue_next((int)(inflight % RING))) ++inflight;
                float mx = 0.0f;
#pragma unroll
                for (int k = 0; k < KB; ++k) mx = fmaxf(mx, fabsf(v[k]));
                const Grids gr = grids_for(mx);
                for (int h2 = 0; h2 < 2; ++h2, ++gc) {
                    const int s = (int)(gc % STAGES);
                    if (gc >= STAGES)
                        live = live && warp_wait(bar(EMPTY + s), (uint32_t)((gc / STAGES - 1) & 1), abortp,
                                                 g.status);
                    if (!live) continue;
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
                }
            }
        }
        // the field copies still in flight land before the CTA ends
        if (t == 0)
            for (int64_t b = waited; b < inflight; ++b)
                drain_bar(bar(RAW_FULL + (int)(b % RING)), (uint32_t)((b / RING) & 1), g.status);
    } else {
        // ---- epilogue (128 threads): lane quarter q of tensor memory ----
        const int qd = warp & 3, et = tid - 192;
        const uint32_t lrow = (uint32_t)(32 * qd) << 16;
        const uint32_t X = tmem + lrow + 256u, S = tmem + lrow + 384u;
        const int r = 32 * qd + lane;           // this thread's output row of the tile
        int64_t gb = 0;
        bool cin_pending = false;
        for (int64_t j = 0; j < my_tiles; ++j) {
            const TileAt t = tile_of(j);
            // the tile's Cin into the output tile, once the previous tile's
            // store has read it
            if (et == 0) {
                asm volatile("cp.async.bulk.wait_group.read 0;\n" ::: "memory");
                mbar_expect_tx(bar(CIN_FULL), OB_BYTES);
                if (g.contiguous) {
                    tma_load2(obase, &mcin, bar(CIN_FULL), t.mt * BM, t.l0);
                } else {
                    for (int c = 0; c < 4; ++c)
                        tma_load3(obase + (uint32_t)c * (OB_BYTES / 4), &mcin, bar(CIN_FULL), t.i0 + 32 * c,
                                  t.mt * BM, t.o);
                }
                cin_pending = true;
            }
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
            if (ok) ok = warp_wait(bar(CIN_FULL), (uint32_t)(j & 1), abortp, g.status);
            // all four warps leave together if one gave up
            if (!group_and(1, ok)) break;
            cin_pending = false;
            asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
            // output tile += S + X: [line][row] (contiguous axis, rows of 512
            // bytes) or four [row][32 lines] blocks with 128-byte swizzle
            for (int pc = 0; pc < NL / 32; ++pc) {
                uint32_t a[32], b[32];
                tmem_ld32(S + (uint32_t)(32 * pc), a);
                tmem_ld32(X + (uint32_t)(32 * pc), b);
                asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::: "memory");
                if (g.contiguous) {
#pragma unroll
                    for (int jj = 0; jj < 32; ++jj) {
                        float* o = OB + (size_t)(32 * pc + jj) * BM + r;
                        *o += __uint_as_float(a[jj]) + __uint_as_float(b[jj]);
                    }
                } else {
                    uint8_t* blk = reinterpret_cast<uint8_t*>(OB) + (size_t)pc * (OB_BYTES / 4) + (size_t)r * 128;
#pragma unroll
                    for (int c = 0; c < 8; ++c) {
                        float4* o = reinterpret_cast<float4*>(blk + (size_t)((c ^ (r & 7)) << 4));
                        float4 w4 = *o;
                        w4.x += __uint_as_float(a[4 * c]) + __uint_as_float(b[4 * c]);
                        w4.y += __uint_as_float(a[4 * c + 1]) + __uint_as_float(b[4 * c + 1]);
                        w4.z += __uint_as_float(a[4 * c + 2]) + __uint_as_float(b[4 * c + 2]);
                        w4.w += __uint_as_float(a[4 * c + 3]) + __uint_as_float(b[4 * c + 3]);
                        *o = w4;
                    }
                }
            }
            // X and S are free for the next tile
            asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
            __syncwarp();
            if (lane == 0) mbar_arrive(bar(ACC_EMPTY));
            // the output tile's writes reach the TMA (async proxy), then Y
            asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
            group_sync(1);
            if (et == 0) {
                if (g.contiguous) {
                    tma_store2(&my, obase, t.mt * BM, t.l0);
                } else {
                    for (int c = 0; c < 4; ++c)
                        tma_store3(&my, obase + (uint32_t)c * (OB_BYTES / 4), t.i0 + 32 * c, t.mt * BM, t.o);
                }
                asm volatile("cp.async.bulk.commit_group;\n" ::: "memory");
            }
        }
        if (et == 0) {
            // every store has completed, and no Cin load is left in flight
            asm volatile("cp.async.bulk.wait_group 0;\n" ::: "memory");
            if (cin_pending) drain_bar(bar(CIN_FULL), (uint32_t)((my_tiles - 1) & 1), g.status);
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

int tc16_operator(const std::vector<double>& D, int Mout, int K, uint16_t** planes) {
    const int MT = (Mout + BM - 1) / BM, KC = tc16_chunks(K);
    // per (row, 32-wide k block): E with 2^E > the block's maximum, then three
    // slices on the grids 2^(E-8), 2^(E-16), 2^(E-24)
    std::vector<uint16_t> h((size_t)MT * KC * 3 * PLANE / 2, 0);
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
                // the chunk's 12 KB as the MMA reads it: [slice][row][32 bytes],
                // each row's 16-byte halves swapped when bit 2 of the row is set
                const int mt = m / BM, rr = m % BM, kc = k / BK, kk = k % BK;
                const size_t blk = ((size_t)mt * KC + kc) * (3 * PLANE);
                const size_t in = (size_t)rr * 32 + (size_t)(((kk >> 3) ^ ((rr >> 2) & 1)) << 4) + (size_t)(kk & 7) * 2;
                for (int p = 0; p < 3; ++p) {
                    const double gp = std::ldexp(1.0, E - 8 - 8 * p);
                    const double a = std::nearbyint(r / gp) * gp;
                    h[(blk + (size_t)p * PLANE + in) / 2] = bf16_exact(a);
                    r -= a;
                }
            }
        }
    cudaError_t e = cudaMalloc((void**)planes, h.size() * sizeof(uint16_t));
    if (e != cudaSuccess) return (int)e;
    e = cudaMemcpy(*planes, h.data(), h.size() * sizeof(uint16_t), cudaMemcpyHostToDevice);
    return (int)e;
}

int tc16_chunks(int K) { return (K + KB - 1) / KB * (KB / BK); }

cudaError_t tc16_set_smem() {
    return cudaFuncSetAttribute(k_tc16, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)SMEM);
}

size_t tc16_smem_bytes() { return SMEM; }

int tc16_field_map(float* base, int contiguous, int64_t len, int64_t lines_or_inner, int64_t outer, int64_t pitch,
                   int ymap, CUtensorMap* map) {
    EncodeTiled enc = encoder();
    if (!enc) return -1;
    CUresult r;
    const cuuint32_t e2[2] = {1, 1}, e3[3] = {1, 1, 1};
    if (contiguous) {
        // rows of `len` values, `pitch` apart; X: 32 k x 128 lines with
        // 128-byte swizzle; Y: 128 rows x 128 lines
        const cuuint64_t dims[2] = {(cuuint64_t)len, (cuuint64_t)lines_or_inner};
        const cuuint64_t strides[1] = {(cuuint64_t)pitch * 4};
        const cuuint32_t box[2] = {ymap ? (cuuint32_t)BM : (cuuint32_t)KB, (cuuint32_t)NL};
        r = enc(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, base, dims, strides, box, e2, CU_TENSOR_MAP_INTERLEAVE_NONE,
                ymap ? CU_TENSOR_MAP_SWIZZLE_NONE : CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    } else {
        // (inner, position along the axis, outer); X: 128 lines x 32 k;
        // Y: 32 lines x 128 rows with 128-byte swizzle (four per tile)
        const cuuint64_t dims[3] = {(cuuint64_t)lines_or_inner, (cuuint64_t)len, (cuuint64_t)outer};
        const cuuint64_t strides[2] = {(cuuint64_t)lines_or_inner * 4, (cuuint64_t)(len * lines_or_inner) * 4};
        const cuuint32_t box[3] = {ymap ? 32u : (cuuint32_t)NL, ymap ? (cuuint32_t)BM : (cuuint32_t)KB, 1};
        r = enc(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, base, dims, strides, box, e3, CU_TENSOR_MAP_INTERLEAVE_NONE,
                ymap ? CU_TENSOR_MAP_SWIZZLE_128B : CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    }
    return r == CUDA_SUCCESS ? 0 : -1;
}

cudaError_t tc16_launch(const CUtensorMap& mx, const CUtensorMap& mcin, const CUtensorMap& my, const Tc16Gemm& g,
                        cudaStream_t st) {
    static thread_local int dev_cached = -1, nsm = 0;
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev != dev_cached) {
        e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
        if (e != cudaSuccess) return e;
        dev_cached = dev;
    }
    const int64_t tiles = g.tiles * g.MT;
    const int64_t grid = tiles < nsm ? tiles : nsm;      // persistent: at most one CTA per SM
    if (grid <= 0) return cudaSuccess;
    k_tc16<<<(unsigned)grid, THREADS, SMEM, st>>>(mx, mcin, my, g);
    return cudaGetLastError();
}

}  // namespace pstd
