// pstd_nn.cu -- kernels of the learned spectral operator (forward, backward, Adam).
//
// The network works in the wall-respecting sine/cosine basis of each axis
// (the truncated T1 of Table 2), so every operation is one of:
//   * a strided batched GEMM  C[b] = alpha A[b] B[b] + beta C[b]  with
//     arbitrary element strides (the per-axis transforms, the per-mode channel
//     mixing, the pointwise channel mixing and all their adjoints);
//   * per-channel elementwise work (lift, bias + ReLU, projection) and their
//     gradients, and per-channel reductions;
//   * an Adam update.
// The GEMM tiles 64 x 64 outputs per CTA (4 x 4 per thread) over 16-wide k
// slices staged in shared memory, FP32 throughout.
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <cmath>
#include <vector>

#include "pstd.h"

namespace {

// One CTA of 256 threads computes a BM x BN tile of C[b] (TM x TN per
// thread) over 16-wide k slices staged in shared memory.  Tile shapes:
// 64 x 64 for square-ish products, 256 x 16 / 16 x 256 for the tall or wide
// products with a mode count (16) on one side, 16 x 16 for the small per-line
// transforms.
template <int BM, int BN, int TM, int TN>
__global__ void __launch_bounds__(256) k_sgemm(pstd_gemm_desc d) {
    static_assert((BM / TM) * (BN / TN) == 256, "256 threads");
    constexpr int LA = 16 * BM / 256, LB = 16 * BN / 256;
    static_assert(LA >= 1 && LB >= 1, "tile too small");
    __shared__ float As[16][BM + 4];
    __shared__ float Bs[16][BN + 4];
    const int tid = threadIdx.x;
    const int tx = tid % (BN / TN), ty = tid / (BN / TN);
    const int64_t nb2 = d.batch2 > 1 ? d.batch2 : 1;
    const int64_t b1 = blockIdx.z / nb2, b2 = blockIdx.z - b1 * nb2;
    const int K = (nb2 > 1 && b2 == nb2 - 1) ? d.K_last : d.K;
    const int m0 = blockIdx.y * BM, n0 = blockIdx.x * BN;
    const float* A = d.A + b1 * d.sAb + b2 * d.sAb2;
    const float* B = d.B + b1 * d.sBb + b2 * d.sBb2;
    float* C = d.C + b1 * d.sCb + b2 * d.sCb2;
    const bool a_kfast = d.sAk == 1 && d.sAm != 1;
    const bool b_kfast = d.sBk == 1 && d.sBn != 1;
    // This thread's slots in the staged k slice (consecutive threads walk the
    // operand's unit-stride index, so the global loads coalesce).
    int akk[LA], amm[LA], bkk[LB], bnn[LB];
#pragma unroll
    for (int i = 0; i < LA; ++i) {
        const int idx = tid + i * 256;
        akk[i] = a_kfast ? (idx & 15) : (idx / BM);
        amm[i] = a_kfast ? (idx >> 4) : (idx % BM);
    }
#pragma unroll
    for (int i = 0; i < LB; ++i) {
        const int idx = tid + i * 256;
        bkk[i] = b_kfast ? (idx & 15) : (idx / BN);
        bnn[i] = b_kfast ? (idx >> 4) : (idx % BN);
    }
    float ra[LA], rb[LB];
    auto fetch = [&](int k0) {
#pragma unroll
        for (int i = 0; i < LA; ++i) {
            const int m = m0 + amm[i], k = k0 + akk[i];
            ra[i] = (m < d.M && k < K) ? A[m * d.sAm + k * d.sAk] : 0.0f;
        }
#pragma unroll
        for (int i = 0; i < LB; ++i) {
            const int n = n0 + bnn[i], k = k0 + bkk[i];
            rb[i] = (n < d.N && k < K) ? B[k * d.sBk + n * d.sBn] : 0.0f;
        }
    };
    float acc[TM][TN] = {};
    if (K > 0) fetch(0);
    for (int k0 = 0; k0 < K; k0 += 16) {
#pragma unroll
        for (int i = 0; i < LA; ++i) As[akk[i]][amm[i]] = ra[i];
#pragma unroll
        for (int i = 0; i < LB; ++i) Bs[bkk[i]][bnn[i]] = rb[i];
        __syncthreads();
        if (k0 + 16 < K) fetch(k0 + 16);      // next slice in flight during this one's FMAs
#pragma unroll
        for (int kk = 0; kk < 16; ++kk) {
            float a[TM], bb[TN];
#pragma unroll
            for (int i = 0; i < TM; ++i) a[i] = As[kk][ty * TM + i];
#pragma unroll
            for (int j = 0; j < TN; ++j) bb[j] = Bs[kk][tx * TN + j];
#pragma unroll
            for (int i = 0; i < TM; ++i)
#pragma unroll
                for (int j = 0; j < TN; ++j) acc[i][j] = fmaf(a[i], bb[j], acc[i][j]);
        }
        __syncthreads();
    }
#pragma unroll
    for (int i = 0; i < TM; ++i) {
        const int m = m0 + ty * TM + i;
        if (m >= d.M) continue;
#pragma unroll
        for (int j = 0; j < TN; ++j) {
            const int n = n0 + tx * TN + j;
            if (n >= d.N) continue;
            float* c = &C[m * d.sCm + n * d.sCn];
            *c = d.beta != 0.0f ? d.alpha * acc[i][j] + d.beta * *c : d.alpha * acc[i][j];
        }
    }
}

// Row kernels: blockIdx.y is the row r = b C + c of a [B][C][P] tensor and
// the x blocks stride over its P points (no per-element index division).

// y[b, c, i] = act(x[b, c, i] + bias[c]) (act: 0 identity, 1 relu)
__global__ void k_bias_act(const float* x, const float* bias, float* y, int C, int64_t P, int act) {
    const int64_t r = blockIdx.y;
    const float bv = bias ? bias[r % C] : 0.0f;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < P; i += (int64_t)gridDim.x * blockDim.x) {
        const float v = x[r * P + i] + bv;
        y[r * P + i] = act == 1 ? fmaxf(v, 0.0f) : v;
    }
}

// dx = dy * (pre > 0)  (relu) or dy (identity), in place allowed
__global__ void k_act_bwd(const float* dy, const float* pre, float* dx, int64_t n, int act) {
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < n;
         t += (int64_t)gridDim.x * blockDim.x)
        dx[t] = (act == 1 && pre[t] <= 0.0f) ? 0.0f : dy[t];
}

// v[b, c, i] = w[c] p[b, i] + bias[c]
__global__ void k_lift(const float* p, const float* w, const float* bias, float* v, int C, int64_t P) {
    const int64_t r = blockIdx.y, b = r / C;
    const int c = (int)(r - b * C);
    const float wc = w[c], bc = bias[c];
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < P; i += (int64_t)gridDim.x * blockDim.x)
        v[r * P + i] = fmaf(wc, p[b * P + i], bc);
}

// out[b, i] = sum_c w[c] v[b, c, i] + bias  (blockIdx.y = b)
__global__ void k_proj(const float* v, const float* w, const float* bias, float* out, int C, int64_t P) {
    const int64_t b = blockIdx.y;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < P; i += (int64_t)gridDim.x * blockDim.x) {
        float acc = bias[0];
        for (int c = 0; c < C; ++c) acc = fmaf(w[c], v[(b * C + c) * P + i], acc);
        out[b * P + i] = acc;
    }
}

// dv[b, c, i] = w[c] dout[b, i]
__global__ void k_proj_bwd(const float* dout, const float* w, float* dv, int C, int64_t P) {
    const int64_t r = blockIdx.y, b = r / C;
    const float wc = w[r - b * C];
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < P; i += (int64_t)gridDim.x * blockDim.x)
        dv[r * P + i] = wc * dout[b * P + i];
}

// g[c] = sum_{b, i} x[b, c, i] * (y ? y[b, c or -, i] : 1); y indexed [b, i] when ybc == 0
__global__ void k_chan_dot(const float* x, const float* y, int ybc, float* g, int64_t B, int C, int64_t P) {
    const int c = blockIdx.x;
    double acc = 0.0;
    for (int64_t b = 0; b < B; ++b) {
        const float* xr = x + (b * C + c) * P;
        const float* yr = y ? (ybc ? y + (b * C + c) * P : y + b * P) : nullptr;
        for (int64_t i = threadIdx.x; i < P; i += blockDim.x)
            acc += (double)xr[i] * (yr ? (double)yr[i] : 1.0);
    }
    __shared__ double red[256];
    red[threadIdx.x] = acc;
    __syncthreads();
    for (int s = blockDim.x / 2; s > 0; s >>= 1) {
        if ((int)threadIdx.x < s) red[threadIdx.x] += red[threadIdx.x + s];
        __syncthreads();
    }
    if (threadIdx.x == 0) g[c] = (float)red[0];
}

// out[j] = sum_b x[b, j]   (sum over the leading dimension)
__global__ void k_sum_lead(const float* x, float* out, int64_t B, int64_t n) {
    for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < n; j += (int64_t)gridDim.x * blockDim.x) {
        double acc = 0.0;
        for (int64_t b = 0; b < B; ++b) acc += x[b * n + j];
        out[j] = (float)acc;
    }
}

// Adam (Kingma & Ba) with bias correction; step t >= 1
__global__ void k_adam(float* w, const float* g, float* m, float* v, int64_t n, float lr, float b1, float b2,
                       float eps, float c1, float c2) {
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < n; t += (int64_t)gridDim.x * blockDim.x) {
        const float gg = g[t];
        const float mm = b1 * m[t] + (1.0f - b1) * gg;
        const float vv = b2 * v[t] + (1.0f - b2) * gg * gg;
        m[t] = mm;
        v[t] = vv;
        w[t] -= lr * (mm / c1) / (sqrtf(vv / c2) + eps);
    }
}

// Block-wide FP64 sum of one value per thread (blockDim.x a power of two <= 1024).
__device__ double block_sum(double v) {
    __shared__ double red[1024];
    red[threadIdx.x] = v;
    __syncthreads();
    for (int s = blockDim.x / 2; s > 0; s >>= 1) {
        if ((int)threadIdx.x < s) red[threadIdx.x] += red[threadIdx.x + s];
        __syncthreads();
    }
    const double r = red[0];
    __syncthreads();
    return r;
}

// Mean squared error of out against target (one CTA): loss[0] = mean (out - t)^2,
// dout = (2 / n) (out - t).
__global__ void k_mse(const float* out, const float* target, float* dout, float* loss, int64_t n) {
    double acc = 0.0;
    const float s = 2.0f / (float)n;
    for (int64_t t = threadIdx.x; t < n; t += blockDim.x) {
        const float df = out[t] - target[t];
        acc += (double)df * (double)df;
        if (dout) dout[t] = s * df;
    }
    const double tot = block_sum(acc);
    if (threadIdx.x == 0) loss[0] = (float)(tot / (double)n);
}

// Per sample b (one CTA each): err[b] = ||a_b - r_b||_2 / ||r_b||_2.
__global__ void k_rel_err(const float* a, const float* r, float* err, int64_t P) {
    const int64_t b = blockIdx.x;
    double num = 0.0, den = 0.0;
    for (int64_t t = threadIdx.x; t < P; t += blockDim.x) {
        const double x = a[b * P + t], y = r[b * P + t];
        num += (x - y) * (x - y);
        den += y * y;
    }
    num = block_sum(num);
    den = block_sum(den);
    if (threadIdx.x == 0) err[b] = den > 0.0 ? (float)sqrt(num / den) : (float)sqrt(num);
}

// dst = src rounded to the nearest bfloat16 (ties to even), kept in FP32 storage.
__global__ void k_round_bf16(const float* src, float* dst, int64_t n) {
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < n; t += (int64_t)gridDim.x * blockDim.x)
        dst[t] = __bfloat162float(__float2bfloat16_rn(src[t]));
}

// rms[b] = sqrt(mean_i x[b, i]^2) (one CTA per sample, FP64 sum)
__global__ void k_row_rms(const float* x, float* rms, int64_t P) {
    const int64_t b = blockIdx.x;
    double acc = 0.0;
    for (int64_t i = threadIdx.x; i < P; i += blockDim.x) acc += (double)x[b * P + i] * x[b * P + i];
    acc = block_sum(acc);
    if (threadIdx.x == 0) rms[b] = (float)sqrt(acc / (double)P);
}

// y[b, i] = x[b, i] / s[b] (mode 0, s[b] == 0 gives 0) or x[b, i] * s[b] (mode 1)
__global__ void k_row_scale(const float* x, const float* sc, float* y, int64_t P, int mode) {
    const int64_t b = blockIdx.y;
    const float f = mode == 1 ? sc[b] : (sc[b] > 0.0f ? 1.0f / sc[b] : 0.0f);
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < P; i += (int64_t)gridDim.x * blockDim.x)
        y[b * P + i] = x[b * P + i] * f;
}

dim3 row_grid(int64_t rows, int64_t P) {
    int64_t bx = (P + 255) / 256;
    return dim3((unsigned)(bx < 64 ? (bx > 0 ? bx : 1) : 64), (unsigned)rows);
}

unsigned blocks_for(int64_t n) {
    int64_t b = (n + 255) / 256;
    return (unsigned)(b < 152 * 32 ? (b > 0 ? b : 1) : 152 * 32);
}

int cuda_rc(cudaError_t e) { return e == cudaSuccess ? PSTD_OK : PSTD_ECUDA; }

}  // namespace

extern "C" {

int pstd_nn_gemm(const pstd_gemm_desc* d, void* stream) {
    if (!d || d->batch < 1 || d->M < 0 || d->N < 0 || d->K < 0 || !d->C) return PSTD_EINVAL;
    if (d->K > 0 && (!d->A || !d->B)) return PSTD_EINVAL;
    if (d->M == 0 || d->N == 0) return PSTD_OK;
    const int64_t nb2 = d->batch2 > 1 ? d->batch2 : 1;
    if (nb2 > 1 && (d->K_last < 0 || d->K_last > d->K || (d->K_last > 0 && (!d->A || !d->B)))) return PSTD_EINVAL;
    if (d->batch * nb2 > 65535 || (d->M + 255) / 256 > 65535) return PSTD_EINVAL;
    // the tile shape that computes the fewest padded outputs (ties: 64 x 64)
    static const int shapes[4][2] = {{64, 64}, {256, 16}, {16, 256}, {16, 16}};
    int best = 0;
    int64_t best_cost = -1;
    for (int t = 0; t < 4; ++t) {
        const int64_t bm = shapes[t][0], bn = shapes[t][1];
        const int64_t gm = (d->M + bm - 1) / bm;
        if (gm > 65535) continue;
        // padded outputs, plus a charge for the extra operand traffic of thin tiles
        const int64_t cost = gm * bm * ((d->N + bn - 1) / bn) * bn * (t == 3 ? 2 : 1);
        if (best_cost < 0 || cost < best_cost) { best_cost = cost; best = t; }
    }
    const cudaStream_t st = (cudaStream_t)stream;
    const unsigned gz = (unsigned)(d->batch * nb2);
    const int bm = shapes[best][0], bn = shapes[best][1];
    const dim3 grid((unsigned)((d->N + bn - 1) / bn), (unsigned)((d->M + bm - 1) / bm), gz);
    switch (best) {
        case 0: k_sgemm<64, 64, 4, 4><<<grid, 256, 0, st>>>(*d); break;
        case 1: k_sgemm<256, 16, 4, 4><<<grid, 256, 0, st>>>(*d); break;
        case 2: k_sgemm<16, 256, 4, 4><<<grid, 256, 0, st>>>(*d); break;
        default: k_sgemm<16, 16, 1, 1><<<grid, 256, 0, st>>>(*d); break;
    }
    return cuda_rc(cudaGetLastError());
}

int pstd_nn_bias_act(const float* x, const float* bias, float* y, int64_t B, int C, int64_t P, int act,
                     void* stream) {
    if (!x || !y || B < 0 || C < 1 || P < 0 || B * C > 65535 || (act != 0 && act != 1)) return PSTD_EINVAL;
    if (B == 0 || P == 0) return PSTD_OK;
    k_bias_act<<<row_grid(B * C, P), 256, 0, (cudaStream_t)stream>>>(x, bias, y, C, P, act);
    return cuda_rc(cudaGetLastError());
}

int pstd_nn_act_bwd(const float* dy, const float* pre, float* dx, int64_t n, int act, void* stream) {
    if (!dy || !dx || (act == 1 && !pre) || n < 0) return PSTD_EINVAL;
    k_act_bwd<<<blocks_for(n), 256, 0, (cudaStream_t)stream>>>(dy, pre, dx, n, act);
    return cuda_rc(cudaGetLastError());
}

int pstd_nn_lift(const float* p, const float* w, const float* bias, float* v, int64_t B, int C, int64_t P,
                 void* stream) {
    if (!p || !w || !bias || !v || C < 1 || B < 0 || P < 0 || B * C > 65535) return PSTD_EINVAL;
    if (B == 0 || P == 0) return PSTD_OK;
    k_lift<<<row_grid(B * C, P), 256, 0, (cudaStream_t)stream>>>(p, w, bias, v, C, P);
    return cuda_rc(cudaGetLastError());
}

int pstd_nn_proj(const float* v, const float* w, const float* bias, float* out, int64_t B, int C, int64_t P,
                 void* stream) {
    if (!v || !w || !bias || !out || C < 1 || B < 0 || P < 0 || B > 65535) return PSTD_EINVAL;
    if (B == 0 || P == 0) return PSTD_OK;
    k_proj<<<row_grid(B, P), 256, 0, (cudaStream_t)stream>>>(v, w, bias, out, C, P);
    return cuda_rc(cudaGetLastError());
}

int pstd_nn_proj_bwd(const float* dout, const float* w, float* dv, int64_t B, int C, int64_t P, void* stream) {
    if (!dout || !w || !dv || C < 1 || B < 0 || P < 0 || B * C > 65535) return PSTD_EINVAL;
    if (B == 0 || P == 0) return PSTD_OK;
    k_proj_bwd<<<row_grid(B * C, P), 256, 0, (cudaStream_t)stream>>>(dout, w, dv, C, P);
    return cuda_rc(cudaGetLastError());
}

int pstd_nn_chan_dot(const float* x, const float* y, int y_has_channels, float* g, int64_t B, int C, int64_t P,
                     void* stream) {
    if (!x || !g || C < 1 || B < 0 || P < 0 || C > 0x7fffffff) return PSTD_EINVAL;
    k_chan_dot<<<C, 256, 0, (cudaStream_t)stream>>>(x, y, y_has_channels, g, B, C, P);
    return cuda_rc(cudaGetLastError());
}

int pstd_nn_sum_lead(const float* x, float* out, int64_t B, int64_t n, void* stream) {
    if (!x || !out || B < 1 || n < 0) return PSTD_EINVAL;
    k_sum_lead<<<blocks_for(n), 256, 0, (cudaStream_t)stream>>>(x, out, B, n);
    return cuda_rc(cudaGetLastError());
}

int pstd_nn_adam(float* w, const float* g, float* m, float* v, int64_t n, float lr, float beta1, float beta2,
                 float eps, int64_t step, void* stream) {
    if (!w || !g || !m || !v || step < 1) return PSTD_EINVAL;
    const float c1 = 1.0f - powf(beta1, (float)step), c2 = 1.0f - powf(beta2, (float)step);
    k_adam<<<blocks_for(n), 256, 0, (cudaStream_t)stream>>>(w, g, m, v, n, lr, beta1, beta2, eps, c1, c2);
    return cuda_rc(cudaGetLastError());
}

int pstd_nn_mse(const float* out, const float* target, float* dout, float* loss, int64_t n, void* stream) {
    if (!out || !target || !loss || n < 1) return PSTD_EINVAL;
    k_mse<<<1, 1024, 0, (cudaStream_t)stream>>>(out, target, dout, loss, n);
    return cuda_rc(cudaGetLastError());
}

int pstd_nn_rel_err(const float* a, const float* ref, float* err, int64_t B, int64_t P, void* stream) {
    if (!a || !ref || !err || B < 1 || B > 0x7fffffff || P < 1) return PSTD_EINVAL;
    k_rel_err<<<(unsigned)B, 256, 0, (cudaStream_t)stream>>>(a, ref, err, P);
    return cuda_rc(cudaGetLastError());
}

int pstd_nn_round_bf16(const float* src, float* dst, int64_t n, void* stream) {
    if (!src || !dst || n < 0) return PSTD_EINVAL;
    k_round_bf16<<<blocks_for(n), 256, 0, (cudaStream_t)stream>>>(src, dst, n);
    return cuda_rc(cudaGetLastError());
}

int pstd_nn_row_rms(const float* x, float* rms, int64_t B, int64_t P, void* stream) {
    if (!x || !rms || B < 1 || B > 0x7fffffff || P < 1) return PSTD_EINVAL;
    k_row_rms<<<(unsigned)B, 256, 0, (cudaStream_t)stream>>>(x, rms, P);
    return cuda_rc(cudaGetLastError());
}

int pstd_nn_row_scale(const float* x, const float* s, float* y, int64_t B, int64_t P, int mode, void* stream) {
    if (!x || !s || !y || B < 0 || B > 65535 || P < 0 || (mode != 0 && mode != 1)) return PSTD_EINVAL;
    if (B == 0 || P == 0) return PSTD_OK;
    k_row_scale<<<row_grid(B, P), 256, 0, (cudaStream_t)stream>>>(x, s, y, P, mode);
    return cuda_rc(cudaGetLastError());
}

// The first K wall-respecting modes of one axis (Table 2, transform T1 of the
// wall pair), from their mode functions on the stored pressure nodes x_j:
//   NN  cos(pi k j / N)        j = 0..N     (T1 = C1)
//   ND  cos(pi (k+1/2) j / N)  j = 0..N-1   (T1 = C3)
//   DN  sin(pi (k+1/2) j / N)  j = 1..N     (T1 = S3)
//   DD  sin(pi (k+1) j / N)    j = 1..N-1   (T1 = S1)
// The unnormalised forward transform is T[k][j] = 2 w_j phi_k(x_j), with
// w_j = 1/2 on a stored wall node and 1 elsewhere (trapezoid weights); its
// inverse (Eq. inverse_transforms, implied period M = 2N for every pair) is
// I[j][k] = (1/M) 2 v_k phi_k(x_j) with v_k = 1/2 for the wall-constant
// modes (k = 0 and k = N of NN) and 1 elsewhere.  Built in FP64, rounded once.
int pstd_sno_basis(int ncells, int bc_left, int bc_right, int K, float* T, float* I) {
    if (ncells < 2 || K < 1 || !T || !I) return PSTD_EINVAL;
    if ((bc_left != PSTD_NEUMANN && bc_left != PSTD_DIRICHLET) ||
        (bc_right != PSTD_NEUMANN && bc_right != PSTD_DIRICHLET))
        return PSTD_EINVAL;
    const int N = ncells;
    const int lo = bc_left == PSTD_DIRICHLET ? 1 : 0;
    const int hi = bc_right == PSTD_DIRICHLET ? N - 1 : N;
    const int lp = hi - lo + 1;
    if (K > lp) return PSTD_EINVAL;
    const bool cosine = bc_left == PSTD_NEUMANN;
    const double shift = bc_left == bc_right ? (cosine ? 0.0 : 1.0) : 0.5;
    const double M = 2.0 * N;
    for (int k = 0; k < K; ++k) {
        const double kap = M_PI * (k + shift) / N;
        const double vk = (cosine && bc_right == PSTD_NEUMANN && (k == 0 || k == N)) ? 0.5 : 1.0;
        for (int jj = 0; jj < lp; ++jj) {
            const int j = jj + lo;
            const double phi = cosine ? std::cos(kap * j) : std::sin(kap * j);
            const double wj = ((j == 0 && bc_left == PSTD_NEUMANN) || (j == N && bc_right == PSTD_NEUMANN)) ? 0.5 : 1.0;
            T[(size_t)k * lp + jj] = (float)(2.0 * wj * phi);
            I[(size_t)jj * K + k] = (float)(2.0 * vk * phi / M);
        }
    }
    return PSTD_OK;
}

}  // extern "C"
