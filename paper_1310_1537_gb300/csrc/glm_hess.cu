// Log-posterior, gradient and Hessian of Bayesian logistic regression in one
// pass over X (the §4.2 derivatives taken one order further, as §5.2
// proposes for Newton-type and Riemannian samplers):
//   f = sum_n [y_n eta_n - log(1 + e^eta_n)] + log N(beta | 0, s^2 I)
//   g = X^T (y - mu) - beta / s^2
//   H = -X^T diag(mu (1 - mu)) X - I / s^2,       mu = 1 / (1 + e^-eta)
// for one coefficient vector, P <= 64, X FP32 row-major.
//
// Persistent CTAs (three per SM) take 64-row tiles round-robin; a tile
// arrives by one bulk copy into a 3-slot ring. Per tile: phase A, four
// threads per row, forms eta, w = mu (1 - mu), r = y - mu and the
// log-likelihood term; phase B1, thread j < P, adds sum_n r_n x_nj to its g_j;
// phase B2, one thread per (8 x 4 block of the upper triangle of X^T W X,
// group of every third row) adds sum_n (x_n,i..i+7) (w_n x_n,j..j+3)^T over
// its rows to 32 register accumulators (three 16-byte shared loads per 32
// FMAs); the remaining threads do phase B1, g_j += sum_n r_n x_nj. At the end
// the three row groups' sums are added in a fixed order through shared
// memory, the CTA's sums are written once as partials and a second kernel
// adds them in a fixed order in FP64 (deterministic), adds the prior and
// fills the symmetric H.
#include <cmath>
#include <cstring>
#include <new>

#include "glm_internal.cuh"

struct glm_hess {
    int64_t n_rows;
    int p, ld, device, sm_count, grid;
    double prior_sigma;
    void *ws;
    double *part_f;            // grid
    float *part_g;             // grid x 64
    float *part_h;             // grid x kHessMaxBlocks x 32
    unsigned *status;
};

namespace glm {

constexpr int kHessRows = 64;             // rows per tile
constexpr int kHessThreads = 256;
constexpr int kHessStages = 3;
constexpr int kHessMaxP = 64;
// 8 x 4 blocks (I, J) with J >= 2I: sum over I of (P/4 - 2I) = 72 at P = 64
constexpr int kHessMaxBlocks = 72;
constexpr int kHessBlockElems = 32;
constexpr int kHessRowGroups = 3;                            // B2 thread groups
constexpr int kHessB2Threads = kHessMaxBlocks * kHessRowGroups;   // 216
constexpr int kHessB1Threads = kHessThreads - kHessB2Threads;     // 40

// block index -> (I, J) of an 8 x 4 block covering the upper triangle
__host__ __device__ inline bool hess_block(int t, int PB, int &I, int &J)
{
    for (I = 0; 2 * I < PB; ++I) {
        const int cnt = PB - 2 * I;
        if (t < cnt) {
            J = 2 * I + t;
            return true;
        }
        t -= cnt;
    }
    return false;
}

// bytes of the ring region: 3 tiles plus 8 floats of slack, at least the
// two row groups' block sums handed over at the end
__host__ __device__ inline int hess_ring_bytes(int ld)
{
    const int ring = kHessStages * kHessRows * ld * 4 + 32;
    const int xch = 2 * kHessMaxBlocks * kHessBlockElems * 4;
    return ring > xch ? ring : xch;
}

__host__ __device__ inline int hess_nblocks(int PB)
{
    int nb = 0;
    for (int I = 0; 2 * I < PB; ++I)
        nb += PB - 2 * I;
    return nb;
}

struct HessParams {
    const float *X;
    const uint8_t *y;
    const float *beta;
    int64_t N;
    int P, ld;
    double *part_f;
    float *part_g;
    float *part_h;
    unsigned *status;
};

__global__ void __launch_bounds__(kHessThreads, 3) hess_kernel(HessParams p)
{
    extern __shared__ __align__(128) uint8_t smem_raw[];
    uint8_t *smem = smem_raw + ((128u - (ptx::smem_u32(smem_raw) & 127u)) & 127u);
    const int tid = threadIdx.x, lane = tid & 31;
    const int P = p.P, ld = p.ld;
    const int PB = (P + 3) / 4;                          // 4-column blocks
    const int NB = hess_nblocks(PB);                     // 8 x 4 blocks over the upper triangle
    float *ring = reinterpret_cast<float *>(smem);       // [stages][64][ld] + 8 floats of slack
    float *bs = reinterpret_cast<float *>(smem + hess_ring_bytes(ld));             // beta [64]
    float *ws = bs + kHessMaxP;                          // w [64]
    float *rs = ws + kHessRows;                          // r [64]
    double *red = reinterpret_cast<double *>(rs + kHessRows);                 // [8]
    uint64_t *bars = reinterpret_cast<uint64_t *>(red + 8);                    // [stages]
    __shared__ int s_ok;

    const int64_t ntiles = (p.N + kHessRows - 1) / kHessRows;
    const int b = blockIdx.x, G = gridDim.x;
    const int nt = (int)(ntiles > b ? (ntiles - b + G - 1) / G : 0);

    for (int j = tid; j < kHessMaxP; j += kHessThreads)
        bs[j] = j < P ? p.beta[j] : 0.0f;
    if (tid == 0) {
        for (int s = 0; s < kHessStages; ++s)
            ptx::mbar_init(&bars[s], 1);
        ptx::fence_mbar_init();
        s_ok = 1;
    }
    __syncthreads();
    auto issue = [&](int i) {                             // tile i of this CTA into slot i % stages
        const int64_t row0 = (int64_t)(b + (int64_t)i * G) * kHessRows;
        const int rows = (int)((p.N - row0) < kHessRows ? (p.N - row0) : kHessRows);
        uint64_t *bar = &bars[i % kHessStages];
        ptx::mbar_arrive_expect_tx(bar, (unsigned)(rows * ld * 4));
        ptx::bulk_g2s(ring + (size_t)(i % kHessStages) * kHessRows * ld, p.X + row0 * ld,
                      (unsigned)(rows * ld * 4), bar, ptx::policy_evict_first());
    };
    if (tid == 0)
        for (int i = 0; i < nt && i < kHessStages; ++i)
            issue(i);

    // this thread's H block (rows 8 bi .. 8 bi + 7, columns 4 bj .. 4 bj + 3)
    // and row group; threads from kHessB2Threads on do phase B1
    const int blk = tid % kHessMaxBlocks;
    const int rgrp = tid / kHessMaxBlocks;
    const bool b2 = tid < kHessB2Threads && blk < NB;
    int bi = 0, bj = 0;
    if (b2)
        hess_block(blk, PB, bi, bj);
    float hacc[kHessBlockElems];
#pragma unroll
    for (int e = 0; e < kHessBlockElems; ++e)
        hacc[e] = 0.0f;
    float gacc[(kHessMaxP + kHessB1Threads - 1) / kHessB1Threads];
#pragma unroll
    for (int q = 0; q < (kHessMaxP + kHessB1Threads - 1) / kHessB1Threads; ++q)
        gacc[q] = 0.0f;
    float facc = 0.0f;
    const int arow = tid >> 2, aq = tid & 3;             // phase A: row, quarter

    for (int i = 0; i < nt; ++i) {
        const int s = i % kHessStages;
        const int64_t row0 = (int64_t)(b + (int64_t)i * G) * kHessRows;
        const int rows = (int)((p.N - row0) < kHessRows ? (p.N - row0) : kHessRows);
        if (!ptx::mbar_wait_bounded(&bars[s], (unsigned)(i / kHessStages) & 1u, kSpinLimit)) {
            if (lane == 0) {
                atomicOr(p.status, kDevTimeout);
                s_ok = 0;
            }
        }
        float *xt = ring + (size_t)s * kHessRows * ld;
        // rows beyond N in a partial tile: zero them (they then add nothing)
        if (rows < kHessRows) {
            for (int q = rows * ld + tid; q < kHessRows * ld; q += kHessThreads)
                xt[q] = 0.0f;
            ptx::fence_proxy_async_smem();                  // before any later copy into the slot
        }
        __syncthreads();
        // ---- phase A: eta, w, r, ell (4 threads per row) ---------------------------
        // thread aq takes the row's 16-byte chunks aq, aq + 4, aq + 8, aq + 12,
        // in an order rotated by the row, so that the two rows of each 8-lane
        // shared-memory access use different bank groups
        {
            const float *xr = xt + arow * ld;
            float pa = 0.0f;
#pragma unroll
            for (int cc = 0; cc < 4; ++cc) {
                const int c = 4 * (aq + 4 * ((cc + arow) & 3));     // first column of the chunk
                if (c >= ld)
                    continue;
                const float4 xv = *reinterpret_cast<const float4 *>(xr + c);
                pa = fmaf(xv.x, bs[c], pa);
                pa = fmaf(xv.y, bs[c + 1], pa);
                pa = fmaf(xv.z, bs[c + 2], pa);
                pa = fmaf(xv.w, bs[c + 3], pa);
            }
            pa += __shfl_xor_sync(0xFFFFFFFFu, pa, 1);
            pa += __shfl_xor_sync(0xFFFFFFFFu, pa, 2);
            if (aq == 0) {
                float w = 0.0f, r = 0.0f;
                if (arow < rows) {
                    const float eta = pa;
                    const float yv = (float)p.y[row0 + arow];
                    const float e = __expf(-fabsf(eta));
                    const float d = 1.0f + e;
                    const float inv = __fdividef(1.0f, d);
                    const float mu = eta >= 0.0f ? inv : e * inv;       // logistic
                    w = e * inv * inv;                                  // mu (1 - mu)
                    r = yv - mu;
                    facc += fmaf(yv, eta, -fmaxf(eta, 0.0f)) - __logf(d);
                }
                ws[arow] = w;
                rs[arow] = r;
            }
        }
        __syncthreads();
        // ---- phase B1: g_j += sum_n r_n x_nj --------------------------------------
        if (tid >= kHessB2Threads) {
#pragma unroll
            for (int q = 0; q < (kHessMaxP + kHessB1Threads - 1) / kHessB1Threads; ++q) {
                const int j = tid - kHessB2Threads + q * kHessB1Threads;
                if (j < P) {
                    float t = 0.0f;
#pragma unroll 8
                    for (int n = 0; n < kHessRows; ++n)
                        t = fmaf(rs[n], xt[n * ld + j], t);
                    gacc[q] += t;
                }
            }
        }
        // ---- phase B2: H block += sum_n (x_n,i) (w_n x_n,j)^T ---------------------
        if (b2) {
            const float *xi = xt + 8 * bi;   // may read past column P (into the next row or the
            const float *xj = xt + 4 * bj;   // ring's slack): those entries are never combined
#pragma unroll 2
            for (int n = rgrp; n < kHessRows; n += kHessRowGroups) {
                const float4 a0 = *reinterpret_cast<const float4 *>(xi + n * ld);
                const float4 a1 = *reinterpret_cast<const float4 *>(xi + n * ld + 4);
                const float4 c4 = *reinterpret_cast<const float4 *>(xj + n * ld);
                const float wn = ws[n];
                const float a[8] = {a0.x, a0.y, a0.z, a0.w, a1.x, a1.y, a1.z, a1.w};
                const float c[4] = {wn * c4.x, wn * c4.y, wn * c4.z, wn * c4.w};
#pragma unroll
                for (int u = 0; u < 8; ++u)
#pragma unroll
                    for (int v = 0; v < 4; ++v)
                        hacc[4 * u + v] = fmaf(a[u], c[v], hacc[4 * u + v]);
            }
        }
        __syncthreads();                                    // slot s and ws/rs free
        if (tid == 0 && i + kHessStages < nt)
            issue(i + kHessStages);
    }
    // ---- partials of this CTA ---------------------------------------------------
    double fv = (double)facc;
#pragma unroll
    for (int m = 16; m > 0; m >>= 1)
        fv += __shfl_xor_sync(0xFFFFFFFFu, fv, m);
    if (lane == 0)
        red[tid >> 5] = fv;
    __syncthreads();
    if (tid == 0) {
        double t = 0.0;
        for (int w = 0; w < kHessThreads / 32; ++w)
            t += red[w];
        p.part_f[b] = s_ok ? t : __longlong_as_double(0x7FF8000000000000LL);
    }
    if (tid >= kHessB2Threads) {
#pragma unroll
        for (int q = 0; q < (kHessMaxP + kHessB1Threads - 1) / kHessB1Threads; ++q) {
            const int j = tid - kHessB2Threads + q * kHessB1Threads;
            if (j < kHessMaxP)
                p.part_g[(size_t)b * kHessMaxP + j] = j < P ? gacc[q] : 0.0f;
        }
    }
    // row groups 1 and 2 hand their block sums to group 0 through the ring
    // (free now: every copy has landed and been consumed)
    float *xch = ring;                                       // [2][kHessMaxBlocks][32]
    if (b2 && rgrp > 0) {
        float *dst = xch + ((size_t)(rgrp - 1) * kHessMaxBlocks + blk) * kHessBlockElems;
#pragma unroll
        for (int e = 0; e < kHessBlockElems; ++e)
            dst[e] = hacc[e];
    }
    __syncthreads();
    if (b2 && rgrp == 0) {
        const float *s1 = xch + (size_t)blk * kHessBlockElems;
        const float *s2 = xch + ((size_t)kHessMaxBlocks + blk) * kHessBlockElems;
        float *dst = p.part_h + ((size_t)b * kHessMaxBlocks + blk) * kHessBlockElems;
#pragma unroll
        for (int e = 0; e < kHessBlockElems; ++e)
            dst[e] = (hacc[e] + s1[e]) + s2[e];
    }
}

// Fixed-order sums of the CTAs' partials, prior, symmetric H. A block takes
// 32 consecutive output elements; its 8 warps each add a contiguous range of
// CTAs (all loads of a range in flight, coalesced over the elements), then
// warp 0 adds the 8 range sums in order.
constexpr int kHessRedWarps = 8;

__global__ void __launch_bounds__(32 * kHessRedWarps)
    hess_combine_kernel(const double *__restrict__ part_f, const float *__restrict__ part_g,
                        const float *__restrict__ part_h, int parts, int P,
                        const float *__restrict__ beta, double inv_s2, double prior_const,
                        double *__restrict__ f_out, float *__restrict__ g_out,
                        float *__restrict__ H_out)
{
    __shared__ double sum[kHessRedWarps][32];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int PB = (P + 3) / 4;
    const int NB = hess_nblocks(PB);
    const int nel = 1 + P + NB * kHessBlockElems;
    const int e = blockIdx.x * 32 + lane;
    const int per = (parts + kHessRedWarps - 1) / kHessRedWarps;
    const int q0 = warp * per;
    const int q1 = q0 + per < parts ? q0 + per : parts;
    double v = 0.0;
    if (e < nel) {
        for (int qb = q0; qb < q1; qb += 16) {
            double buf[16];
#pragma unroll
            for (int u = 0; u < 16; ++u) {
                const int q = qb + u;
                double t = 0.0;
                if (q < q1) {
                    if (e == 0)
                        t = part_f[q];
                    else if (e <= P)
                        t = (double)part_g[(size_t)q * kHessMaxP + e - 1];
                    else
                        t = (double)part_h[(size_t)q * kHessMaxBlocks * kHessBlockElems + (e - 1 - P)];
                }
                buf[u] = t;
            }
#pragma unroll
            for (int u = 0; u < 16; ++u)
                v += buf[u];
        }
    }
    sum[warp][lane] = v;
    __syncthreads();
    if (warp != 0 || e >= nel)
        return;
    double tot = 0.0;
#pragma unroll
    for (int w = 0; w < kHessRedWarps; ++w)
        tot += sum[w][lane];
    if (e == 0) {
        double bb = 0.0;
        for (int j = 0; j < P; ++j)
            bb += (double)beta[j] * (double)beta[j];
        *f_out = tot - 0.5 * inv_s2 * bb - prior_const;
    } else if (e <= P) {
        const int j = e - 1;
        g_out[j] = (float)tot - beta[j] * (float)inv_s2;
    } else {
        const int k = e - 1 - P;
        const int blk = k / kHessBlockElems, u = (k % kHessBlockElems) >> 2, v2 = k & 3;
        int I = 0, J = 0;
        hess_block(blk, PB, I, J);
        const int i = 8 * I + u, j = 4 * J + v2;
        if (i >= P || j >= P || j < i)
            return;                                         // outside P, or mirrored from j >= i
        const float hv = -(float)tot - (i == j ? (float)inv_s2 : 0.0f);
        H_out[(size_t)i * P + j] = hv;
        H_out[(size_t)j * P + i] = hv;
    }
}

}  // namespace glm

using namespace glm;

static int hess_smem_bytes(int ld)
{
    return hess_ring_bytes(ld) + (kHessMaxP + 2 * kHessRows) * 4 + 8 * 8 + kHessStages * 8 + 128;
}

extern "C" {

glm_status_t glm_hess_create(int64_t n_rows, int32_t p, int32_t ld, double prior_sigma, int32_t device,
                             glm_hess_t *out)
{
    if (!out)
        return GLM_ERR_INVALID_ARG;
    *out = nullptr;
    if (n_rows < 0 || p < 1 || p > kHessMaxP || ld < p || ld > kHessMaxP || (ld & 3) ||
        !(prior_sigma > 0.0) || !std::isfinite(prior_sigma) || device < 0)
        return GLM_ERR_INVALID_ARG;
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev == 0) {
        cudaGetLastError();
        return GLM_ERR_NO_DEVICE;
    }
    if (device >= ndev || cudaSetDevice(device) != cudaSuccess)
        return GLM_ERR_INVALID_ARG;
    int major = 0, minor = 0, sms = 0;
    cudaDeviceGetAttribute(&major, cudaDevAttrComputeCapabilityMajor, device);
    cudaDeviceGetAttribute(&minor, cudaDevAttrComputeCapabilityMinor, device);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device);
    if (major != 10 || minor != 3)
        return GLM_ERR_NO_DEVICE;
    glm_hess *h = new (std::nothrow) glm_hess;
    if (!h)
        return GLM_ERR_OOM;
    std::memset(h, 0, sizeof(*h));
    h->n_rows = n_rows;
    h->p = p;
    h->ld = ld;
    h->device = device;
    h->sm_count = sms;
    h->grid = 3 * sms;
    h->prior_sigma = prior_sigma;
    const size_t fb = (size_t)h->grid * 8, gb = (size_t)h->grid * kHessMaxP * 4,
                 hb = (size_t)h->grid * kHessMaxBlocks * kHessBlockElems * 4;
    if (cudaMalloc(&h->ws, fb + gb + hb + 256) != cudaSuccess) {
        cudaGetLastError();
        delete h;
        return GLM_ERR_OOM;
    }
    uint8_t *base = static_cast<uint8_t *>(h->ws);
    h->part_f = reinterpret_cast<double *>(base);
    h->part_g = reinterpret_cast<float *>(base + fb);
    h->part_h = reinterpret_cast<float *>(base + fb + gb);
    h->status = reinterpret_cast<unsigned *>(base + fb + gb + hb);
    if (cudaMemset(h->status, 0, 256) != cudaSuccess) {
        cudaFree(h->ws);
        delete h;
        return GLM_ERR_CUDA;
    }
    *out = h;
    return GLM_OK;
}

glm_status_t glm_hess_destroy(glm_hess_t h)
{
    if (!h)
        return GLM_OK;
    cudaSetDevice(h->device);
    cudaFree(h->ws);
    delete h;
    return GLM_OK;
}

glm_status_t glm_hess_eval(glm_hess_t h, const float *X, const uint8_t *y, const float *beta,
                           double *f_out, float *g_out, float *H_out, glm_stream_t stream)
{
    if (!h || !beta || !f_out || !g_out || !H_out || (h->n_rows > 0 && (!X || !y)) ||
        (reinterpret_cast<uintptr_t>(X) & 15u) || (reinterpret_cast<uintptr_t>(f_out) & 7u))
        return GLM_ERR_INVALID_ARG;
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    HessParams p;
    std::memset(&p, 0, sizeof(p));
    p.X = X;
    p.y = y;
    p.beta = beta;
    p.N = h->n_rows;
    p.P = h->p;
    p.ld = h->ld;
    p.part_f = h->part_f;
    p.part_g = h->part_g;
    p.part_h = h->part_h;
    p.status = h->status;
    const int smem = hess_smem_bytes(h->ld);
    if (cudaFuncSetAttribute(hess_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, smem) != cudaSuccess)
        return GLM_ERR_CUDA;
    hess_kernel<<<h->grid, kHessThreads, smem, st>>>(p);
    const double s2 = h->prior_sigma * h->prior_sigma;
    const int nel = 1 + h->p + hess_nblocks((h->p + 3) / 4) * kHessBlockElems;
    hess_combine_kernel<<<(nel + 31) / 32, 32 * kHessRedWarps, 0, st>>>(
        h->part_f, h->part_g, h->part_h, h->grid, h->p, beta, 1.0 / s2,
        0.5 * h->p * std::log(2.0 * M_PI * s2), f_out, g_out, H_out);
    return cudaGetLastError() == cudaSuccess ? GLM_OK : GLM_ERR_CUDA;
}

glm_status_t glm_hess_sync(glm_hess_t h, glm_stream_t stream)
{
    if (!h)
        return GLM_ERR_INVALID_ARG;
    if (cudaStreamSynchronize(reinterpret_cast<cudaStream_t>(stream)) != cudaSuccess)
        return GLM_ERR_CUDA;
    unsigned st = 0;
    if (cudaMemcpy(&st, h->status, sizeof(st), cudaMemcpyDeviceToHost) != cudaSuccess)
        return GLM_ERR_CUDA;
    if (st) {
        cudaMemset(h->status, 0, sizeof(unsigned));
        return GLM_ERR_TIMEOUT;
    }
    return GLM_OK;
}

}  // extern "C"
