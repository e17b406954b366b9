// pstd_tc.cu -- the learned operator's strided batched GEMM on the 5th-generation
// tensor cores (tcgen05, kind::tf32, accumulators in tensor memory).
//
// One CTA of 128 threads computes a 128 x 64 tile of C[b] = alpha A[b] B[b] +
// beta C[b] (same descriptor and strides as pstd_nn_gemm):
//   * the k dimension runs in slices of 16; the 128
//     threads stage A's 128-row and B's 64-row slice (B read as N x K) into
//     shared memory in the canonical K-major layout without swizzle (8-row x
//     16-byte core matrices, K-adjacent core matrices 128 bytes apart),
//     rounding to TF32, in two buffers: slice s+1 is staged while the tensor
//     cores run slice s;
//   * one thread issues the K = 8 MMAs of a slice into a 128-lane x 64-column
//     FP32 accumulator in tensor memory and commits them to the buffer's
//     mbarrier;
//   * after the last slice every warp reads its 32 accumulator lanes
//     (tcgen05.ld) and applies alpha / beta.
// Every wait on the mbarrier is bounded: a wait that gives up sets *status,
// waits once more (bounded) for the MMAs in flight, frees the tensor memory
// and ends the CTA.
#include <cuda_runtime.h>
#include <stdint.h>

#include "pstd.h"

namespace {

constexpr int BM = 128, BN = 64;
constexpr uint32_t LBO = 128;          // bytes between K-adjacent core matrices
constexpr uint32_t TMEM_COLS = 64;      // plain: one 128 x 64 FP32 accumulator
constexpr uint32_t TMEM_COLS_SPLIT = 128; // split: two, one per k slice in turn
constexpr long long kWaitLimit = 1 << 22;

// k slice per stage: 16 (two stages of 24 KB for the plain kernel, of 48 KB
// with the split form's hi and lo copies); 8-row groups are 4 core matrices
// of 128 bytes apart.
template <bool SPLIT>
struct Tile {
    static constexpr int BK = 16;
    static constexpr uint32_t SBO = (uint32_t)BK * 4u * 8u;
    static constexpr int A_WORDS = BM * BK, B_WORDS = BN * BK;
    // one stage: A (hi [, lo]) then B (hi [, lo]); two stages
    static constexpr int STAGE_WORDS = (SPLIT ? 2 : 1) * (A_WORDS + B_WORDS);
    static constexpr size_t SMEM = 2u * STAGE_WORDS * 4u;
};

// Byte offset of element (row r, k) of a staged slice.
template <bool SPLIT>
__host__ __device__ __forceinline__ uint32_t canon(int r, int k) {
    return (uint32_t)(r >> 3) * Tile<SPLIT>::SBO + (uint32_t)(k >> 2) * LBO + (uint32_t)(r & 7) * 16u +
           (uint32_t)(k & 3) * 4u;
}

// Instruction descriptor of kind::tf32: D FP32, A and B TF32, both K-major.
__host__ __device__ constexpr uint32_t idesc_tf32(int M, int N) {
    return (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

#ifdef __CUDA_ARCH__
__device__ __forceinline__ uint32_t smem_addr(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

// Shared-memory matrix descriptor: K-major, no swizzle.
template <bool SPLIT>
__device__ __forceinline__ uint64_t sdesc(uint32_t addr) {
    uint64_t d = (uint64_t)((addr >> 4) & 0x3FFFu);
    d |= (uint64_t)((LBO >> 4) & 0x3FFFu) << 16;
    d |= (uint64_t)((Tile<SPLIT>::SBO >> 4) & 0x3FFFu) << 32;
    d |= (uint64_t)1 << 46;            // descriptor version of the tcgen05 family
    return d;
}

__device__ __forceinline__ float to_tf32(float x) {
    uint32_t r;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
    return __uint_as_float(r);
}

__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t phase, long long limit) {
    for (long long i = 0; i < limit; ++i) {
        uint32_t done;
        asm volatile(
            "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
            : "=r"(done)
            : "r"(bar), "r"(phase)
            : "memory");
        if (done) return true;
    }
    return false;
}

__device__ __forceinline__ void mma_tf32(uint32_t tmem, uint64_t ad, uint64_t bd, uint32_t idesc, uint32_t acc) {
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
        " tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem),
        "l"(ad), "l"(bd), "r"(idesc), "r"(acc)
        : "memory");
}
#endif

// C[b] = alpha A[b] B[b] + beta C[b].  SPLIT: A = Ah + Al and B = Bh + Bl with
// TF32 parts (Bl from B_lo, else split on the fly), summed as Ah Bh + Ah Bl +
// Al Bh: about 22 significant bits per operand.
template <bool SPLIT>
__global__ void __launch_bounds__(128) k_tc_gemm(pstd_gemm_desc d, const float* B_lo, int* status) {
#ifdef __CUDA_ARCH__
    using TL = Tile<SPLIT>;
    constexpr int BK = TL::BK;
    constexpr uint32_t NCOLS = SPLIT ? TMEM_COLS_SPLIT : TMEM_COLS;
    extern __shared__ __align__(1024) float tsm[];
    __shared__ __align__(8) uint64_t bar[2];
    __shared__ uint32_t tmem_slot;
    __shared__ int all_ok;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int64_t nb2 = d.batch2 > 1 ? d.batch2 : 1;
    const int64_t b1 = blockIdx.z / nb2, b2 = blockIdx.z - b1 * nb2;
    const int K = (nb2 > 1 && b2 == nb2 - 1) ? d.K_last : d.K;
    const int m0 = blockIdx.y * BM, n0 = blockIdx.x * BN;
    const float* A = d.A + b1 * d.sAb + b2 * d.sAb2;
    const float* B = d.B + b1 * d.sBb + b2 * d.sBb2;
    const float* Bl = B_lo ? B_lo + b1 * d.sBb + b2 * d.sBb2 : nullptr;
    float* C = d.C + b1 * d.sCb + b2 * d.sCb2;
    const bool a_kfast = d.sAk == 1 && d.sAm != 1;
    const bool b_kfast = d.sBk == 1 && d.sBn != 1;

    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(smem_addr(&tmem_slot)),
                     "r"(NCOLS)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n" ::: "memory");
    }
    if (tid == 0) {
        all_ok = 1;
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(smem_addr(&bar[0])) : "memory");
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(smem_addr(&bar[1])) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
    const uint32_t tmem = tmem_slot;
    const uint32_t idesc = idesc_tf32(BM, BN);

    // stage slice s (k0 = s BK) into buffer b: every load of this thread is
    // issued into registers first, then converted and stored, so that the
    // loads are in flight together
    auto stage = [&](int s, int b) {
        float* Ah = tsm + (size_t)b * TL::STAGE_WORDS;
        float* Al = Ah + TL::A_WORDS;
        float* Bh = SPLIT ? Al + TL::A_WORDS : Al;
        float* Blo = Bh + TL::B_WORDS;
        const int k0 = s * BK;
        constexpr int NA = BM * BK / 128, NB = BN * BK / 128;
        float va[NA], vb[NB], vl[SPLIT ? NB : 1];
#pragma unroll
        for (int i = 0; i < NA; ++i) {
            const int idx = tid + 128 * i;
            const int r = a_kfast ? idx / BK : idx & (BM - 1);
            const int kk = a_kfast ? idx % BK : idx >> 7;
            const int m = m0 + r, k = k0 + kk;
            va[i] = (m < d.M && k < K) ? __ldg(&A[m * d.sAm + k * d.sAk]) : 0.0f;
        }
#pragma unroll
        for (int i = 0; i < NB; ++i) {
            const int idx = tid + 128 * i;
            const int r = b_kfast ? idx / BK : idx & (BN - 1);
            const int kk = b_kfast ? idx % BK : idx >> 6;
            const int n = n0 + r, k = k0 + kk;
            const bool in = n < d.N && k < K;
            vb[i] = in ? __ldg(&B[k * d.sBk + n * d.sBn]) : 0.0f;
            if constexpr (SPLIT) vl[i] = (in && Bl) ? __ldg(&Bl[k * d.sBk + n * d.sBn]) : 0.0f;
        }
#pragma unroll
        for (int i = 0; i < NA; ++i) {
            const int idx = tid + 128 * i;
            const int r = a_kfast ? idx / BK : idx & (BM - 1);
            const int kk = a_kfast ? idx % BK : idx >> 7;
            const float h = to_tf32(va[i]);
            const uint32_t o = canon<SPLIT>(r, kk) >> 2;
            Ah[o] = h;
            if constexpr (SPLIT) Al[o] = to_tf32(va[i] - h);
        }
#pragma unroll
        for (int i = 0; i < NB; ++i) {
            const int idx = tid + 128 * i;
            const int r = b_kfast ? idx / BK : idx & (BN - 1);
            const int kk = b_kfast ? idx % BK : idx >> 6;
            const float h = to_tf32(vb[i]);
            const uint32_t o = canon<SPLIT>(r, kk) >> 2;
            Bh[o] = h;
            if constexpr (SPLIT) Blo[o] = to_tf32(Bl ? vl[i] : vb[i] - h);
        }
        // make the staged slices visible to the tensor cores' (async) proxy
        asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
    };
    // the MMAs of slice s on buffer b, committed to bar[b]
    auto issue = [&](int s, int b) {
        const uint32_t base = smem_addr(tsm + (size_t)b * TL::STAGE_WORDS);
        const uint32_t ah = base, al = base + TL::A_WORDS * 4u;
        const uint32_t bh = SPLIT ? al + TL::A_WORDS * 4u : al, bl = bh + TL::B_WORDS * 4u;
        asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
        for (int ks = 0; ks < BK / 8; ++ks) {
            const uint32_t off = (uint32_t)ks * 2u * LBO;
            if constexpr (SPLIT) {
                // each slice starts from zero in its own accumulator; the
                // threads add it into FP32 registers (no long in-MMA sums)
                const uint32_t dst = tmem + (uint32_t)(s & 1) * TMEM_COLS;
                mma_tf32(dst, sdesc<SPLIT>(ah + off), sdesc<SPLIT>(bl + off), idesc, ks > 0 ? 1u : 0u);
                mma_tf32(dst, sdesc<SPLIT>(al + off), sdesc<SPLIT>(bh + off), idesc, 1u);
                mma_tf32(dst, sdesc<SPLIT>(ah + off), sdesc<SPLIT>(bh + off), idesc, 1u);
            } else {
                mma_tf32(tmem, sdesc<SPLIT>(ah + off), sdesc<SPLIT>(bh + off), idesc, (s > 0 || ks > 0) ? 1u : 0u);
            }
        }
        asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(
                         smem_addr(&bar[b]))
                     : "memory");
    };

    // split: this thread's row of the FP32 sum over slices
    float racc[SPLIT ? BN : 1];
    if constexpr (SPLIT)
#pragma unroll
        for (int j = 0; j < BN; ++j) racc[j] = 0.0f;
    // add the (completed) accumulator of slice s into racc
    auto promote = [&](int s) {
        if constexpr (SPLIT) {
            asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
            const uint32_t base = tmem + ((uint32_t)(32 * warp) << 16) + (uint32_t)(s & 1) * TMEM_COLS;
#pragma unroll
            for (int c = 0; c < BN; c += 16) {
                uint32_t r[16];
                asm volatile(
                    "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, "
                    "[%16];\n"
                    : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
                      "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]),
                      "=r"(r[15])
                    : "r"(base + (uint32_t)c)
                    : "memory");
                asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::: "memory");
#pragma unroll
                for (int j = 0; j < 16; ++j) racc[c + j] += __uint_as_float(r[j]);
            }
            asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
        }
    };

    // two buffers: slice s+1 is staged while the MMAs of slice s run
    const int ns = (K + BK - 1) / BK;
    uint32_t ph[2] = {0u, 0u};
    int pending[2] = {0, 0};
    if (ns > 0) stage(0, 0);
    __syncthreads();
    for (int s = 0; s < ns; ++s) {
        const int b = s & 1;
        if (tid == 0) issue(s, b);
        pending[b] = 1;
        if (s + 1 < ns) {
            if (pending[b ^ 1]) {    // buffer b^1 was read by slice s-1's MMAs
                if (tid == 0 && !mbar_wait(smem_addr(&bar[b ^ 1]), ph[b ^ 1], kWaitLimit)) {
                    all_ok = 0;
                    if (status) atomicExch(status, 1);
                }
                ph[b ^ 1] ^= 1u;
                pending[b ^ 1] = 0;
                __syncthreads();
                if (!all_ok) break;
                promote(s - 1);      // slice s-1's accumulator is complete
            }
            stage(s + 1, b ^ 1);
        }
        __syncthreads();
    }
    // wait for every slice still in flight (once more, bounded, after a failure)
    if (tid == 0)
        for (int b = 0; b < 2; ++b)
            if (pending[b] && !mbar_wait(smem_addr(&bar[b]), ph[b], kWaitLimit)) {
                all_ok = 0;
                if (status) atomicExch(status, 1);
            }
    __syncthreads();
    if (all_ok) {
        // the last one or two slices (in slice order)
        if (ns >= 2 && pending[(ns - 2) & 1]) promote(ns - 2);
        if (ns >= 1) promote(ns - 1);
    }
    asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
    if (all_ok) {
        const int row = m0 + 32 * warp + lane;
        if constexpr (SPLIT) {
            if (row < d.M) {
#pragma unroll
                for (int j = 0; j < BN; ++j) {
                    const int n = n0 + j;
                    if (n >= d.N) continue;
                    float* cp = &C[row * d.sCm + n * d.sCn];
                    *cp = d.beta != 0.0f ? d.alpha * racc[j] + d.beta * *cp : d.alpha * racc[j];
                }
            }
        }
        for (int c = 0; c < (SPLIT ? 0 : BN); c += 16) {
            uint32_t r[16];
            const uint32_t taddr = tmem + ((uint32_t)(32 * warp) << 16) + (uint32_t)c;
            asm volatile(
                "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, "
                "[%16];\n"
                : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
                  "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]),
                  "=r"(r[15])
                : "r"(taddr)
                : "memory");
            asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::: "memory");
            if (row < d.M) {
#pragma unroll
                for (int j = 0; j < 16; ++j) {
                    const int n = n0 + c + j;
                    if (n >= d.N) continue;
                    const float acc = K > 0 ? __uint_as_float(r[j]) : 0.0f;
                    float* cp = &C[row * d.sCm + n * d.sCn];
                    *cp = d.beta != 0.0f ? d.alpha * acc + d.beta * *cp : d.alpha * acc;
                }
            }
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
    __syncthreads();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(tmem), "r"(NCOLS) : "memory");
#endif
}

int check_desc(const pstd_gemm_desc* d) {
    if (!d || d->batch < 1 || d->M < 0 || d->N < 0 || d->K < 0 || !d->C) return PSTD_EINVAL;
    if (d->K > 0 && (!d->A || !d->B)) return PSTD_EINVAL;
    const int64_t nb2 = d->batch2 > 1 ? d->batch2 : 1;
    if (nb2 > 1 && (d->K_last < 0 || d->K_last > d->K || (d->K_last > 0 && (!d->A || !d->B)))) return PSTD_EINVAL;
    if (d->batch * nb2 > 65535 || (d->M + BM - 1) / BM > 65535) return PSTD_EINVAL;
    return PSTD_OK;
}

template <bool SPLIT>
int launch_tc(const pstd_gemm_desc* d, const float* B_lo, int* status, cudaStream_t st) {
    int rc = check_desc(d);
    if (rc != PSTD_OK) return rc;
    if (d->M == 0 || d->N == 0) return PSTD_OK;
    static thread_local int configured_dev = -1;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return PSTD_ECUDA;
    if (configured_dev != dev) {
        // 48 KB of dynamic shared memory (two stages)
        if (cudaFuncSetAttribute(k_tc_gemm<SPLIT>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)Tile<SPLIT>::SMEM) != cudaSuccess)
            return PSTD_ECUDA;
        configured_dev = dev;
    }
    const int64_t nb2 = d->batch2 > 1 ? d->batch2 : 1;
    const dim3 grid((unsigned)((d->N + BN - 1) / BN), (unsigned)((d->M + BM - 1) / BM), (unsigned)(d->batch * nb2));
    k_tc_gemm<SPLIT><<<grid, 128, Tile<SPLIT>::SMEM, st>>>(*d, B_lo, status);
    return cudaGetLastError() == cudaSuccess ? PSTD_OK : PSTD_ECUDA;
}

}  // namespace

extern "C" int pstd_nn_gemm_tf32(const pstd_gemm_desc* d, int* status, void* stream) {
    return launch_tc<false>(d, nullptr, status, (cudaStream_t)stream);
}

// The split-precision dense form's GEMM (pstd_internal.h).
int pstd_internal_tc_gemm_split(const pstd_gemm_desc* d, const float* B_lo, int* status, cudaStream_t st) {
    return launch_tc<true>(d, B_lo, status, st);
}
