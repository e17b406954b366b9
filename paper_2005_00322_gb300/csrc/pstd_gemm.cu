// pstd_gemm.cu -- split-precision dense form of the axis pass (tensor cores).
//
// Each staggered derivative of an axis is a dense matrix applied to every line:
// D_p (N x lp, p -> u) and D_u (lp x N, u -> p), built in FP64 on the host
// with the time-step factors folded in.  A CTA owns G lines and computes
//     u_new = u + D_p p           (GEMM 1, M = N,  K = lp, N_gemm = G)
//     acc_out = acc_in + D_u u_new (GEMM 2, M = lp, K = N)
// with FP16 split products on the tensor cores: D / s_D = Dh + 2^-11 Dl and
// each line x / s_x = xh + 2^-11 xl (s_x = max |x| of the line), FP16 each
// (the low parts are stored multiplied by 2^11 so that they stay FP16
// normals: every entry keeps ~22 significant bits, not only the largest), and
// D x ~ s_D s_x (Dh xh + 2^-11 (Dh xl + Dl xh)) with the two sums in separate
// FP32 accumulators (the dropped 2^-22 Dl xl term is below FP32 rounding of
// the result).  A systematic error in D shifts the discrete frequencies and
// grows into phase drift over thousands of steps, hence the care.  The MMA is mma.sync m16n8k16 (FP16 in,
// FP32 accumulate); A fragments come from a fragment-ordered copy of D in
// global memory (one 16-byte load per lane), B fragments from the lines in
// shared memory, [line][k] with a padded row.
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "pstd_gemm.h"

namespace pstd {

namespace {

// Operand type traits of the FP16 operands (low parts x 2^11).
template <class T>
struct Split;
template <>
struct Split<__half> {
    static constexpr float kLo = 2048.0f;
    __device__ static __half cvt(float x) { return __float2half_rn(x); }
    __device__ static float back(__half h) { return __half2float(h); }
    __device__ static void mma(float (&c)[4], const uint4& a, uint32_t b0, uint32_t b1) {
        asm volatile(
            "mma.sync.aligned.m16n8k16.row.col.f32.f16.f16.f32 "
            "{%0, %1, %2, %3}, {%4, %5, %6, %7}, {%8, %9}, {%0, %1, %2, %3};\n"
            : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
            : "r"(a.x), "r"(a.y), "r"(a.z), "r"(a.w), "r"(b0), "r"(b1));
    }
};

template <class T>
__device__ __forceinline__ void split_store(T* hi, T* lo, float x) {
    const T h = Split<T>::cvt(x);
    *hi = h;
    *lo = Split<T>::cvt((x - Split<T>::back(h)) * Split<T>::kLo);
}

// Element (line n, position k) of a tile of G lines.
struct TileAddr {
    int64_t base;      // address of (n = 0, k = 0)
    int64_t stride;    // between positions along the axis
    int64_t nstride;   // between lines
};

__device__ __forceinline__ TileAddr tile_addr(const GemmAxis& A, int64_t block, int len, int& Gv) {
    TileAddr t;
    if (A.inner == 1) {
        const int64_t l0 = block * A.G;
        const int64_t left = A.nlines - l0;
        Gv = (int)(left < A.G ? left : A.G);
        t.base = l0 * len;
        t.stride = 1;
        t.nstride = len;
    } else {
        const int64_t per = (A.inner + A.G - 1) / A.G;
        const int64_t o = block / per;
        const int64_t i0 = (block - o * per) * A.G;
        const int64_t left = A.inner - i0;
        Gv = (int)(left < A.G ? left : A.G);
        t.base = o * (int64_t)len * A.inner + i0;
        t.stride = A.inner;
        t.nstride = 1;
    }
    return t;
}

// Load G lines of `len` words into hi/lo rows of width `kp` (zero padded),
// scaled per line by 1 / max|x|; smax[n] receives max|x| as bits.
template <class T>
__device__ void load_split(const float* f, const TileAddr& t, int len, int Gv, int G, int kp, int ldb,
                           T* bh, T* bl, unsigned* smax) {
    const int tid = threadIdx.x, nthr = blockDim.x;
    const int total = G * kp;
    const bool contig = t.nstride != 1;
    for (int idx = tid; idx < total; idx += nthr) {
        int n, k;
        if (contig) { n = idx / kp; k = idx - n * kp; }
        else { k = idx / G; n = idx - k * G; }
        const float v = (n < Gv && k < len) ? f[t.base + n * t.nstride + k * t.stride] : 0.0f;
        atomicMax(&smax[n], __float_as_uint(fabsf(v)));
    }
    __syncthreads();
    for (int idx = tid; idx < total; idx += nthr) {
        int n, k;
        if (contig) { n = idx / kp; k = idx - n * kp; }
        else { k = idx / G; n = idx - k * G; }
        const float v = (n < Gv && k < len) ? f[t.base + n * t.nstride + k * t.stride] : 0.0f;
        const float m = __uint_as_float(smax[n]);
        const float x = m > 0.0f ? v / m : 0.0f;
        split_store(&bh[n * ldb + k], &bl[n * ldb + k], x);
    }
}

// acc[nt][4] += Ah B_h and acc2[nt][4] += Ah B_l + Al B_h over all k tiles.
// The main product of each 16-wide k tile starts from zero inside the MMA and
// is added to acc with an FP32 add: the tensor core's internal accumulation
// is not round-to-nearest, and letting it carry the running sum over many k
// tiles biases the result toward zero, a systematic error that would grow
// into phase drift.  The 2^-11-scaled cross terms are too small for that to
// matter.
template <class T>
__device__ __forceinline__ void gemm_tile(float (&acc)[8][4], float (&acc2)[8][4], const uint4* Ah,
                                          const uint4* Al, int mt,
                                          int KT, const T* bh, const T* bl, int ldb, int ntiles,
                                          int lane) {
    const int gid = lane >> 2, tig = lane & 3;
    // the operator fragments of k tile kt + 1 are loaded while the MMAs of
    // tile kt run, so that the L2 latency overlaps tensor-core work (a
    // distance of two tiles measured no faster)
    uint4 ah = __ldg(&Ah[(size_t)mt * KT * 32 + lane]);
    uint4 al = __ldg(&Al[(size_t)mt * KT * 32 + lane]);
    for (int kt = 0; kt < KT; ++kt) {
        uint4 ah_next = ah, al_next = al;
        if (kt + 1 < KT) {
            ah_next = __ldg(&Ah[((size_t)mt * KT + kt + 1) * 32 + lane]);
            al_next = __ldg(&Al[((size_t)mt * KT + kt + 1) * 32 + lane]);
        }
#pragma unroll
        for (int nt = 0; nt < 8; ++nt) {
            if (nt >= ntiles) break;
            const int n = nt * 8 + gid;
            const int k = kt * 16 + 2 * tig;
            const uint32_t bh0 = *(const uint32_t*)&bh[n * ldb + k];
            const uint32_t bh1 = *(const uint32_t*)&bh[n * ldb + k + 8];
            const uint32_t bl0 = *(const uint32_t*)&bl[n * ldb + k];
            const uint32_t bl1 = *(const uint32_t*)&bl[n * ldb + k + 8];
            float t[4] = {0.0f, 0.0f, 0.0f, 0.0f};
            Split<T>::mma(t, ah, bh0, bh1);
            acc[nt][0] += t[0];
            acc[nt][1] += t[1];
            acc[nt][2] += t[2];
            acc[nt][3] += t[3];
            Split<T>::mma(acc2[nt], ah, bl0, bl1);
            Split<T>::mma(acc2[nt], al, bh0, bh1);
        }
        ah = ah_next;
        al = al_next;
    }
}

}  // namespace

template <class T>
__global__ void __launch_bounds__(256) k_gemm_step(GemmStep a) {
    constexpr float kLoScale = Split<T>::kLo;
    extern __shared__ float4 gsm4[];
    const GemmAxis& A = a.ax;
    const int G = A.G;
    const int kp1 = A.KT1 * 16, kp2 = A.KT2 * 16;
    const int ld1 = kp1 + 8, ld2 = kp2 + 8;     // padded rows: conflict-free B loads
    const size_t rows = (size_t)G * (ld1 > ld2 ? ld1 : ld2);
    // [hi rows | lo rows] of GEMM 1's lines, later reused for GEMM 2's lines
    T* bh = (T*)gsm4;
    T* bl = bh + rows;
    float* un = (float*)(bl + rows);            // u_new, [G][N], FP32
    unsigned* smax1 = (unsigned*)(un + (size_t)G * A.N);
    unsigned* smax2 = smax1 + G;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nwarp = blockDim.x >> 5;
    const int gid = lane >> 2, tig = lane & 3;
    for (int i = tid; i < 2 * G; i += blockDim.x) smax1[i] = 0u;
    __syncthreads();

    int Gv;
    const TileAddr tp = tile_addr(A, blockIdx.x, A.lp, Gv);
    const TileAddr tu = tile_addr(A, blockIdx.x, A.N, Gv);
    load_split(a.p, tp, A.lp, Gv, G, kp1, ld1, bh, bl, smax1);
    __syncthreads();
    const int ntiles = (Gv + 7) / 8;

    // GEMM 1: u_new = u + s1 * smax1[n] * (D_p p~), written to u and to un
    float acc[8][4], acc2[8][4];
    for (int mt = warp; mt < A.MT1; mt += nwarp) {
#pragma unroll
        for (int nt = 0; nt < 8; ++nt)
#pragma unroll
            for (int c = 0; c < 4; ++c) acc[nt][c] = acc2[nt][c] = 0.0f;
        gemm_tile(acc, acc2, A.A1h, A.A1l, mt, A.KT1, bh, bl, ld1, ntiles, lane);
#pragma unroll
        for (int nt = 0; nt < 8; ++nt) {
            if (nt >= ntiles) break;
#pragma unroll
            for (int c = 0; c < 4; ++c) {
                const int m = mt * 16 + gid + (c >= 2 ? 8 : 0);
                const int n = nt * 8 + 2 * tig + (c & 1);
                if (m < A.N && n < Gv) {
                    const int64_t at = tu.base + n * tu.nstride + m * tu.stride;
                    const float y = acc[nt][c] + acc2[nt][c] * (1.0f / kLoScale);
                    const float v = a.u[at] + y * A.s1 * __uint_as_float(smax1[n]);
                    a.u[at] = v;
                    un[n * A.N + m] = v;
                    atomicMax(&smax2[n], __float_as_uint(fabsf(v)));
                }
            }
        }
    }
    __syncthreads();
    // u_new rows -> hi / lo, scaled per line (over GEMM 1's rows)
    for (int idx = tid; idx < G * kp2; idx += blockDim.x) {
        const int n = idx / kp2, k = idx - n * kp2;
        float x = 0.0f;
        if (n < Gv && k < A.N) {
            const float m = __uint_as_float(smax2[n]);
            x = m > 0.0f ? un[n * A.N + k] / m : 0.0f;
        }
        split_store(&bh[n * ld2 + k], &bl[n * ld2 + k], x);
    }
    __syncthreads();

    // GEMM 2: acc_out = acc_in + s2 * smax2[n] * (D_u u~)
    for (int mt = warp; mt < A.MT2; mt += nwarp) {
#pragma unroll
        for (int nt = 0; nt < 8; ++nt)
#pragma unroll
            for (int c = 0; c < 4; ++c) acc[nt][c] = acc2[nt][c] = 0.0f;
        gemm_tile(acc, acc2, A.A2h, A.A2l, mt, A.KT2, bh, bl, ld2, ntiles, lane);
#pragma unroll
        for (int nt = 0; nt < 8; ++nt) {
            if (nt >= ntiles) break;
#pragma unroll
            for (int c = 0; c < 4; ++c) {
                const int i = mt * 16 + gid + (c >= 2 ? 8 : 0);
                const int n = nt * 8 + 2 * tig + (c & 1);
                if (i < A.lp && n < Gv) {
                    const int64_t at = tp.base + n * tp.nstride + i * tp.stride;
                    const float z = acc[nt][c] + acc2[nt][c] * (1.0f / kLoScale);
                    a.acc_out[at] = a.acc_in[at] + z * A.s2 * __uint_as_float(smax2[n]);
                }
            }
        }
    }
}

cudaError_t launch_gemm_step(unsigned grid, size_t smem, cudaStream_t st, const GemmStep& a) {
    k_gemm_step<__half><<<grid, 256, smem, st>>>(a);
    return cudaGetLastError();
}

cudaError_t gemm_set_smem(int bytes) {
    return cudaFuncSetAttribute(k_gemm_step<__half>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
}

size_t gemm_smem_bytes(int G, int KT1, int KT2, int N) {
    const int ld = (KT1 > KT2 ? KT1 : KT2) * 16 + 8;
    return (size_t)2 * G * ld * sizeof(__half) + (size_t)G * N * sizeof(float) + (size_t)2 * G * sizeof(unsigned);
}

}  // namespace pstd
