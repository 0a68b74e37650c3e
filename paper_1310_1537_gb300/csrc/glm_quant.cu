// Reduced-precision storage of X: FP32 -> BF16 (round to nearest even) and
// FP32 -> FP8 E4M3 with one power-of-two scale per column. The conversions
// use the hardware's round-to-nearest-even (saturating for E4M3) converts.
#include <cuda_fp8.h>

#include "glm_internal.cuh"

namespace glm {

__global__ void quant_bf16_kernel(const float *__restrict__ X32, int ld32, uint16_t *__restrict__ Xq,
                                  int ld, int P, int64_t N)
{
    const int64_t total = N * (int64_t)ld;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t n = i / ld;
        const int j = (int)(i - n * ld);
        const float v = j < P ? X32[n * ld32 + j] : 0.0f;
        __nv_bfloat16 b = __float2bfloat16_rn(v);
        Xq[i] = *reinterpret_cast<uint16_t *>(&b);
    }
}

// Column maxima of |x| as FP32 bit patterns (non-negative floats order like
// their bit patterns, so an unsigned atomicMax is exact).
__global__ void col_amax_kernel(const float *__restrict__ X32, int ld32, int P, int64_t N,
                                int rows_per_block, unsigned *__restrict__ amax_bits)
{
    const int j = blockIdx.y * blockDim.x + threadIdx.x;
    if (j >= P)
        return;
    const int64_t r0 = (int64_t)blockIdx.x * rows_per_block;
    const int64_t r1 = (r0 + rows_per_block) < N ? (r0 + rows_per_block) : N;
    float m = 0.0f;
    for (int64_t n = r0; n < r1; ++n)
        m = fmaxf(m, fabsf(X32[n * ld32 + j]));
    atomicMax(&amax_bits[j], __float_as_uint(m));
}

// s_j = the smallest power of two with 448 * s_j >= amax_j (1 for a zero
// column), kept >= 2^-126. All comparisons are exact.
__global__ void col_scale_kernel(const unsigned *__restrict__ amax_bits, int P,
                                 float *__restrict__ scale)
{
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= P)
        return;
    const float amax = __uint_as_float(amax_bits[j]);
    float s = 1.0f;
    if (amax > 0.0f) {
        int e = ilogbf(amax) - 9;
        for (int it = 0; it < 320 && ldexpf(448.0f, e) < amax; ++it)
            ++e;
        if (e < -126)
            e = -126;
        s = ldexpf(1.0f, e);
    }
    scale[j] = s;
}

__global__ void quant_fp8_kernel(const float *__restrict__ X32, int ld32, uint8_t *__restrict__ Xq,
                                 int ld, int P, int64_t N, const float *__restrict__ scale)
{
    const int64_t total = N * (int64_t)ld;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t n = i / ld;
        const int j = (int)(i - n * ld);
        uint8_t q = 0;
        if (j < P) {
            // division by a power of two: exact wherever the E4M3 result is non-zero
            const float v = X32[n * ld32 + j] / scale[j];
            q = (uint8_t)__nv_cvt_float_to_fp8(v, __NV_SATFINITE, __NV_E4M3);
        }
        Xq[i] = q;
    }
}

glm_status_t launch_quantize(glm_ctx *h, const float *X32, int ld32, void *Xq, float *x_scale,
                             cudaStream_t s)
{
    const int64_t N = h->d.n_rows;
    const int P = h->d.p;
    const int ld = h->d.ld;
    const int64_t total = N * (int64_t)ld;
    const int threads = 256;
    int64_t want = (total + threads - 1) / threads;
    const int blocks = (int)(want < (int64_t)h->sm_count * 16 ? (want > 0 ? want : 1)
                                                             : (int64_t)h->sm_count * 16);
    if (h->d.xtype == GLM_X_BF16) {
        if (N > 0)
            quant_bf16_kernel<<<blocks, threads, 0, s>>>(X32, ld32, static_cast<uint16_t *>(Xq), ld,
                                                          P, N);
        return cudaGetLastError() == cudaSuccess ? GLM_OK : GLM_ERR_CUDA;
    }
    unsigned *amax = reinterpret_cast<unsigned *>(h->scratch);
    if (cudaMemsetAsync(amax, 0, (size_t)P * 4, s) != cudaSuccess)
        return GLM_ERR_CUDA;
    if (N > 0) {
        const int rpb = 2048;
        dim3 g((unsigned)((N + rpb - 1) / rpb), (unsigned)((P + threads - 1) / threads));
        col_amax_kernel<<<g, threads, 0, s>>>(X32, ld32, P, N, rpb, amax);
    }
    col_scale_kernel<<<(P + threads - 1) / threads, threads, 0, s>>>(amax, P, x_scale);
    if (N > 0)
        quant_fp8_kernel<<<blocks, threads, 0, s>>>(X32, ld32, static_cast<uint8_t *>(Xq), ld, P, N,
                                                     x_scale);
    return cudaGetLastError() == cudaSuccess ? GLM_OK : GLM_ERR_CUDA;
}

}  // namespace glm
