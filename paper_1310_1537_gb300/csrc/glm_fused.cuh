// Fused single-HBM-pass log-posterior + gradient on the CUDA cores.
//
// One persistent CTA per SM owns a contiguous block of rows (the paper's
// partial loop fusion, §3.4.1, with each worker's rows split into chunks that
// stay on chip, §4.2.1 "cache fusion"). Row tiles are streamed from HBM into
// shared memory by the TMA engine (cp.async.bulk, multi-stage ring, mbarrier
// completion) so each byte of X is read from HBM exactly once. From the same
// staged tile the CTA computes
//   phase 1 (LA map + TR map, §3.2): eta_nk = x_n . beta_k by SPLIT threads
//           per row, then ell_nk and the residual r_nk = y_n - logistic(eta_nk)
//           with overflow-free forms; ell is summed per thread in FP32;
//   phase 2 (second LA map, §4.2): g_k += r_nk x_n with each thread owning a
//           16-byte column chunk, accumulated in registers for the whole run.
// Per-CTA partials (f in FP64, g summed over thread groups in FP64) go to the
// workspace once at the end (the one-combine-per-worker reduction of §4.2.2);
// the last CTA to finish (ticket counter) reduces them in a fixed order, adds
// the Gaussian prior, and, in Metropolis mode, takes the FP64 accept decision.
#pragma once

#include <cuda_fp8.h>
#include "glm_internal.cuh"

namespace glm {

// --- storage types ----------------------------------------------------------
struct F32Tag {};
struct BF16Tag {};
struct FP8Tag {};

template <typename Tag>
struct XTraits;

template <>
struct XTraits<F32Tag> {
    static constexpr int EPC = 4;   // elements per 16-byte chunk
    static constexpr int ES = 4;
    __device__ __forceinline__ static void load(const uint8_t *p, float *v)
    {
        float4 a = *reinterpret_cast<const float4 *>(p);
        v[0] = a.x; v[1] = a.y; v[2] = a.z; v[3] = a.w;
    }
};

template <>
struct XTraits<BF16Tag> {
    static constexpr int EPC = 8;
    static constexpr int ES = 2;
    __device__ __forceinline__ static void load(const uint8_t *p, float *v)
    {
        uint4 a = *reinterpret_cast<const uint4 *>(p);
        const uint32_t w[4] = {a.x, a.y, a.z, a.w};
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            v[2 * i] = __uint_as_float(w[i] << 16);
            v[2 * i + 1] = __uint_as_float(w[i] & 0xFFFF0000u);
        }
    }
};

template <>
struct XTraits<FP8Tag> {
    static constexpr int EPC = 16;
    static constexpr int ES = 1;
    __device__ __forceinline__ static void load(const uint8_t *p, float *v)
    {
        uint4 a = *reinterpret_cast<const uint4 *>(p);
        const uint32_t w[4] = {a.x, a.y, a.z, a.w};
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            __half2_raw lo = __nv_cvt_fp8x2_to_halfraw2(
                static_cast<__nv_fp8x2_storage_t>(w[i] & 0xFFFFu), __NV_E4M3);
            __half2_raw hi = __nv_cvt_fp8x2_to_halfraw2(
                static_cast<__nv_fp8x2_storage_t>(w[i] >> 16), __NV_E4M3);
            float2 a2 = __half22float2(*reinterpret_cast<__half2 *>(&lo));
            float2 b2 = __half22float2(*reinterpret_cast<__half2 *>(&hi));
            v[4 * i] = a2.x; v[4 * i + 1] = a2.y; v[4 * i + 2] = b2.x; v[4 * i + 3] = b2.y;
        }
    }
};

// --- shared-memory layout (host and device agree through this function) -----
struct FusedLayout {
    int stage_bytes;
    int tiles_bytes;     // stages * stage_bytes, or the reduction buffer if larger
    int beta_off;        // KC x PCE floats
    int rbuf_off;        // T x KC floats
    int bar_off;         // stages x 8 bytes
    int total;
};

__host__ __device__ inline int round_up(int a, int b) { return (a + b - 1) / b * b; }

__host__ __device__ inline FusedLayout fused_layout(int srow, int ld, int epc, int tile_rows,
                                                    int stages, int kc)
{
    FusedLayout L;
    const int pce = (ld / epc) * epc;        // stored row length in elements
    L.stage_bytes = tile_rows * srow;        // srow: staged row stride in bytes
    const int red_bytes = kFusedThreads * kc * epc * 4;   // >= row groups x KC x used columns
    L.tiles_bytes = round_up(stages * L.stage_bytes > red_bytes ? stages * L.stage_bytes : red_bytes,
                             128);
    L.beta_off = L.tiles_bytes;
    L.rbuf_off = L.beta_off + round_up(kc * pce * 4, 16);
    L.bar_off = L.rbuf_off + round_up(tile_rows * kc * 4, 16);
    L.total = L.bar_off + kMaxStages * 8 + 64 + 128;   // + slack to align the base to 128 B
    return L;
}

// --- the TR map, FP32 --------------------------------------------------------
// ell = -[(1-y) eta + log(1 + exp(-eta))] = y eta - (max(eta,0) + log1p(exp(-|eta|)))
// r   = y - 1/(1 + exp(-eta)), with exp(-|eta|) <= 1 so nothing overflows.
__device__ __forceinline__ void tr_map(float eta, float yv, float &ell, float &r)
{
    float e = expf(-fabsf(eta));
    float sp = fmaxf(eta, 0.0f) + log1pf(e);
    ell = fmaf(yv, eta, -sp);
    float inv = __frcp_rn(1.0f + e);
    float sig = eta >= 0.0f ? inv : e * inv;
    r = yv - sig;
}

// --- the kernel --------------------------------------------------------------
template <typename Tag, int KC, int SPLIT>
__global__ void __launch_bounds__(kFusedThreads, 1)
    fused_logpost_grad_kernel(const __grid_constant__ CUtensorMap xmap, FusedParams p)
{
    using TR = XTraits<Tag>;
    constexpr int NT = kFusedThreads;
    constexpr int RB = NT / SPLIT;         // rows per phase-1 batch
    static_assert(SPLIT == 1 || SPLIT == 2 || SPLIT == 4 || SPLIT == 32, "SPLIT");
    constexpr int EPC = TR::EPC;
    constexpr int ES = TR::ES;

    extern __shared__ __align__(128) uint8_t smem_raw[];
    // tensor copies want 128-byte aligned destinations: align the base
    uint8_t *smem = smem_raw + ((128u - (ptx::smem_u32(smem_raw) & 127u)) & 127u);
    const int P = p.P;
    const int ld = p.ld;
    const int PC = ld / EPC;               // chunks per stored row
    const int PCE = PC * EPC;
    const int PCU = (P + EPC - 1) / EPC;   // chunks that hold used columns
    const int row_bytes = ld * ES;         // row stride in global memory
    const int srow = p.srow;               // row stride of the staged tile
    const int SC = srow / 16;              // staged chunks per row
    const int T = p.tile_rows;             // rows per staged tile, a multiple of RB
    const FusedLayout L = fused_layout(srow, ld, EPC, T, p.stages, KC);
    uint8_t *tiles = smem;
    float *beta_s = reinterpret_cast<float *>(smem + L.beta_off);
    float *rbuf = reinterpret_cast<float *>(smem + L.rbuf_off);
    uint64_t *bars = reinterpret_cast<uint64_t *>(smem + L.bar_off);
    __shared__ double s_red[NT / 32][KC];
    __shared__ int s_flag;
    __shared__ int s_failed;

    const int tid = threadIdx.x;
    const int lane = tid & 31;
    const int warp = tid >> 5;
    const int b = blockIdx.x;
    const int grid = gridDim.x;
    const int stages = p.stages;

    const int64_t r_begin = (p.N * (int64_t)b) / grid;
    const int64_t r_end = (p.N * (int64_t)(b + 1)) / grid;
    const int ntiles = (int)((r_end - r_begin + T - 1) / T);

    if (tid == 0) {
        for (int s = 0; s < stages; ++s)
            ptx::mbar_init(&bars[s], 1);
        ptx::fence_mbar_init();
        s_failed = 0;
    }

    // Phase-1 thread -> (row, split part) mapping.
    // SPLIT <= 4: 8 consecutive lanes take 8 consecutive rows of the same part
    // (a contiguous run of chunks), so a quarter-warp's 16-byte loads fall in
    // distinct bank groups when the staged chunk stride is odd (rows are
    // staged padded to an odd stride whenever the tensor-copy path is on);
    // for an even stride each lane starts its walk at a rotated chunk.
    // SPLIT == 32: one warp per row, lane l takes chunks l, l+32, ...; each
    // step reads 512 contiguous bytes.
    const int i8 = lane & 7;
    int h, row_in_batch, c_lo, c_len, c_step, rot;
    if constexpr (SPLIT == 32) {
        h = lane;
        row_in_batch = warp;
        c_lo = lane;
        c_len = PCU > lane ? (PCU - lane + 31) / 32 : 0;
        c_step = 32;
        rot = 0;
    } else {
        h = (lane >> 3) & (SPLIT - 1);
        const int octet = lane >> 3 >> (SPLIT == 1 ? 0 : (SPLIT == 2 ? 1 : 2));
        row_in_batch = warp * (32 / SPLIT) + octet * 8 + i8;
        const int seg = (PCU + SPLIT - 1) / SPLIT;
        c_lo = h * seg;
        const int c_hi = (c_lo + seg) < PCU ? (c_lo + seg) : PCU;
        c_len = c_hi > c_lo ? c_hi - c_lo : 0;
        c_step = 1;
        rot = ((SC & 1) == 0 && c_len > 0) ? (i8 % c_len) : 0;
    }

    // Phase-2 mapping: thread -> (column chunk, row group).
    const int c2 = tid % PCU;
    const int q2 = tid / PCU;
    const int G2 = NT / PCU;
    const int PCUE = PCU * EPC;            // reduction-buffer row length

    float facc[KC];
    float gacc[KC][EPC];
#pragma unroll
    for (int k = 0; k < KC; ++k) {
        facc[k] = 0.0f;
#pragma unroll
        for (int e = 0; e < EPC; ++e)
            gacc[k][e] = 0.0f;
    }
    bool failed = false;

    // Labels are prefetched one tile ahead into registers (at most
    // kMaxBatches phase-1 batches per tile) so their global-load latency
    // overlaps the previous tile's work.
    constexpr int kMaxBatches = 4;
    float ycur[kMaxBatches], ynext[kMaxBatches];
    auto load_y = [&](int tt, float *dst) {
#pragma unroll
        for (int bi = 0; bi < kMaxBatches; ++bi) {
            dst[bi] = 0.0f;
            if (tt < ntiles && h == 0) {
                const int64_t r0 = r_begin + (int64_t)tt * T;
                const int rws = (int)((r_end - r0) < T ? (r_end - r0) : T);
                const int row = bi * RB + row_in_batch;
                if (row < rws)
                    dst[bi] = (float)__ldg(p.y + r0 + row);
            }
        }
    };
    // Prologue. X and y are never written by the previous launch of a
    // Metropolis chain, so those launches may start streaming them before
    // the programmatic dependency on the previous kernel resolves; every
    // other read waits for it.
    const uint64_t policy = ptx::policy_evict_first();
    // Stage rows [row0, row0 + rows) into ring slot `slot`: one 1-D bulk copy
    // of the dense rows, or ceil(rows / box_rows) 2-D tensor copies that
    // write each row srow bytes apart (the extra chunk is zero fill).
    auto issue_tile = [&](int slot, int64_t row0, int rows) {
        uint8_t *dst = tiles + slot * L.stage_bytes;
        if (p.box_rows == 0) {
            const unsigned bytes = (unsigned)(rows * row_bytes);
            ptx::mbar_arrive_expect_tx(&bars[slot], bytes);
            ptx::bulk_g2s(dst, static_cast<const uint8_t *>(p.X) + row0 * (int64_t)row_bytes,
                          bytes, &bars[slot], policy);
        } else {
            const int br = p.box_rows;
            const int nb = (rows + br - 1) / br;
            ptx::mbar_arrive_expect_tx(&bars[slot], (unsigned)(nb * br * srow));
            for (int j = 0; j < nb; ++j)
                ptx::tensor_g2s_2d(dst + j * br * srow, &xmap, 0, (int)(row0 + j * br),
                                   &bars[slot], policy);
        }
    };
    auto issue_prologue = [&]() {
        if (tid != 0)
            return;
        const int pre = ntiles < stages ? ntiles : stages;
        for (int t = 0; t < pre; ++t) {
            const int64_t row0 = r_begin + (int64_t)t * T;
            const int rows = (int)((r_end - row0) < T ? (r_end - row0) : T);
            issue_tile(t, row0, rows);
        }
    };

    if (p.early_prefetch) {
        issue_prologue();
        load_y(0, ycur);
    }
    ptx::grid_dep_wait();
    if (!p.early_prefetch) {
        issue_prologue();
        load_y(0, ycur);
    }
    // Coefficients (scaled by the FP8 column scales) into shared memory.
    for (int idx = tid; idx < KC * PCE; idx += NT) {
        const int k = idx / PCE;
        const int j = idx - k * PCE;
        float v = 0.0f;
        if (k < p.K && j < P) {
            const int64_t o = (int64_t)k * P + j;
            v = p.rwm ? fmaf(p.step, p.z[o], p.state[o]) : p.beta[o];
            if (p.x_scale)
                v *= p.x_scale[j];
        }
        beta_s[idx] = v;
    }
    __syncthreads();
    ptx::grid_dep_launch_dependents();

    for (int t = 0; t < ntiles; ++t) {
        const int s = t % stages;
        const unsigned parity = (unsigned)(t / stages) & 1u;
        const int64_t row0 = r_begin + (int64_t)t * T;
        const int rows = (int)((r_end - row0) < T ? (r_end - row0) : T);
        load_y(t + 1, ynext);
        const bool ok = ptx::mbar_wait_bounded(&bars[s], parity, kSpinLimit);
        const uint8_t *tile = tiles + s * L.stage_bytes;

        // ---- phase 1: eta, ell, r ------------------------------------------
#pragma unroll
        for (int bi = 0; bi < kMaxBatches; ++bi) {
            const int rb = bi * RB;
            if (rb >= rows)
                break;
            const int my_row = rb + row_in_batch;
            float acc[KC];
#pragma unroll
            for (int k = 0; k < KC; ++k)
                acc[k] = 0.0f;
            const bool valid = my_row < rows;
            const float yv = ycur[bi];
            if (valid) {
                const uint8_t *xr = tile + my_row * srow;
                int cs = rot;
#pragma unroll 4
                for (int it = 0; it < c_len; ++it) {
                    const int c = c_lo + cs * c_step;
                    cs = (cs + 1 == c_len) ? 0 : cs + 1;
                    float xv[EPC];
                    TR::load(xr + c * 16, xv);
#pragma unroll
                    for (int k = 0; k < KC; ++k) {
                        const float *bk = beta_s + k * PCE + c * EPC;
                        float part = 0.0f;
#pragma unroll
                        for (int e = 0; e < EPC; e += 4) {
                            float4 bb = *reinterpret_cast<const float4 *>(bk + e);
                            part = fmaf(xv[e], bb.x, part);
                            part = fmaf(xv[e + 1], bb.y, part);
                            part = fmaf(xv[e + 2], bb.z, part);
                            part = fmaf(xv[e + 3], bb.w, part);
                        }
                        acc[k] += part;
                    }
                }
            }
            if constexpr (SPLIT == 32) {
#pragma unroll
                for (int m = 1; m < 32; m <<= 1)
#pragma unroll
                    for (int k = 0; k < KC; ++k)
                        acc[k] += __shfl_xor_sync(0xFFFFFFFFu, acc[k], m);
            } else {
#pragma unroll
                for (int m = 8; m < 8 * SPLIT; m <<= 1)
#pragma unroll
                    for (int k = 0; k < KC; ++k)
                        acc[k] += __shfl_xor_sync(0xFFFFFFFFu, acc[k], m);
            }
            if (valid && h == 0) {
#pragma unroll
                for (int k = 0; k < KC; ++k) {
                    float ell, r;
                    tr_map(acc[k], yv, ell, r);
                    if (k < p.K)
                        facc[k] += ell;
                    rbuf[my_row * KC + k] = r;
                }
            }
        }
        if (__syncthreads_or(!ok)) {
            // A staged tile never arrived: stop, record it, and let the copies
            // still in flight land (bounded) before the ring is reused.
            failed = true;
            if (tid == 0) {
                atomicOr(p.status, kDevTimeout);
                const int last = (t + stages < ntiles) ? t + stages : ntiles;
                for (int tt = t; tt < last; ++tt)
                    ptx::mbar_wait_bounded(&bars[tt % stages], (unsigned)(tt / stages) & 1u,
                                           kSpinLimit);
            }
            __syncthreads();
            break;
        }

        // ---- phase 2: g += r x over the same tile ----------------------------
        if (q2 < G2) {
            const uint8_t *xc = tile + c2 * 16;
#pragma unroll 4
            for (int i = q2; i < rows; i += G2) {
                float xv[EPC];
                TR::load(xc + i * srow, xv);
                float rk[KC];
                if constexpr (KC % 4 == 0) {
#pragma unroll
                    for (int k = 0; k < KC; k += 4) {
                        float4 r4 = *reinterpret_cast<const float4 *>(rbuf + i * KC + k);
                        rk[k] = r4.x; rk[k + 1] = r4.y; rk[k + 2] = r4.z; rk[k + 3] = r4.w;
                    }
                } else {
#pragma unroll
                    for (int k = 0; k < KC; ++k)
                        rk[k] = rbuf[i * KC + k];
                }
#pragma unroll
                for (int k = 0; k < KC; ++k)
#pragma unroll
                    for (int e = 0; e < EPC; ++e)
                        gacc[k][e] = fmaf(rk[k], xv[e], gacc[k][e]);
            }
        }
        __syncthreads();

        // ---- refill the released stage ---------------------------------------
        if (tid == 0 && t + stages < ntiles) {
            const int64_t nrow0 = r_begin + (int64_t)(t + stages) * T;
            const int nrows = (int)((r_end - nrow0) < T ? (r_end - nrow0) : T);
            issue_tile(s, nrow0, nrows);
        }
#pragma unroll
        for (int bi = 0; bi < kMaxBatches; ++bi)
            ycur[bi] = ynext[bi];
    }

    // ---- per-CTA partials ------------------------------------------------------
    if (failed && tid == 0)
        s_failed = 1;   // block-uniform: every thread left the loop together
    // f: warp sums in FP64, then warps in order.
#pragma unroll
    for (int k = 0; k < KC; ++k) {
        double v = (double)facc[k];
#pragma unroll
        for (int m = 16; m > 0; m >>= 1)
            v += __shfl_xor_sync(0xFFFFFFFFu, v, m);
        if (lane == 0)
            s_red[warp][k] = v;
    }
    // g: every row group's registers into shared memory (the tile ring is idle).
    float *red = reinterpret_cast<float *>(tiles);
    if (q2 < G2) {
#pragma unroll
        for (int k = 0; k < KC; ++k)
#pragma unroll
            for (int e = 0; e < EPC; ++e)
                red[(q2 * KC + k) * PCUE + c2 * EPC + e] = gacc[k][e];
    }
    __syncthreads();
    const bool bad = s_failed != 0;
    // Every CTA adds its partial sums into 128-bit fixed-point accumulators
    // (integer adds are associative, so the totals do not depend on the order
    // in which CTAs arrive: the result is bitwise reproducible).
    for (int idx = tid; idx < p.K * (P + 1); idx += NT) {
        const int k = idx / (P + 1);
        const int j = idx - k * (P + 1);
        double v = 0.0;
        if (j == 0) {
            for (int w = 0; w < NT / 32; ++w)
                v += s_red[w][k];
        } else {
            for (int q = 0; q < G2; ++q)
                v += (double)red[(q * KC + k) * PCUE + (j - 1)];
        }
        fx::add(p.acc + (size_t)idx * fx::kLimbs, bad ? __longlong_as_double(0x7FF8000000000000LL) : v,
                p.acc_flag);
    }

    // ---- last CTA: read the totals, add the prior, accept ----------------------
    __threadfence();
    __syncthreads();
    if (tid == 0) {
        const unsigned prev = atomicAdd(p.ticket, 1u);
        s_flag = (prev == (unsigned)grid - 1u) ? 1 : 0;
    }
    __syncthreads();
    if (!s_flag)
        return;
    __threadfence();

    __shared__ double s_f[KC];
    __shared__ double s_bb[KC];
    __shared__ int s_acc[KC];
    // |beta_k|^2 in FP64, warp k-strided, fixed lane order.
    for (int k = warp; k < p.K; k += NT / 32) {
        double v = 0.0;
        for (int j = lane; j < P; j += 32) {
            const int64_t o = (int64_t)k * P + j;
            const float bj = p.rwm ? fmaf(p.step, p.z[o], p.state[o]) : p.beta[o];
            v += (double)bj * (double)bj;
        }
#pragma unroll
        for (int m = 16; m > 0; m >>= 1)
            v += __shfl_xor_sync(0xFFFFFFFFu, v, m);
        if (lane == 0)
            s_bb[k] = v;
    }
    __syncthreads();
    const bool nan_out = __ldcg(p.acc_flag) != 0u;
    for (int idx = tid; idx < p.K * (P + 1); idx += NT) {
        const int k = idx / (P + 1);
        const int j = idx - k * (P + 1);
        unsigned long long *a = p.acc + (size_t)idx * fx::kLimbs;
        double t = fx::read_and_clear(a);
        if (nan_out)
            t = __longlong_as_double(0x7FF8000000000000LL);
        if (j == 0) {
            const double v0 = t - 0.5 * p.inv_s2 * s_bb[k] - p.prior_const;
            s_f[k] = v0;
            if (p.f_out)
                p.f_out[k] = v0;
        } else {
            const int jj = j - 1;
            const int64_t o = (int64_t)k * P + jj;
            const float bj = p.rwm ? fmaf(p.step, p.z[o], p.state[o]) : p.beta[o];
            const double sc = p.x_scale ? (double)p.x_scale[jj] : 1.0;
            if (p.g_out)
                p.g_out[o] = (float)(sc * t - (double)bj * p.inv_s2);
        }
    }
    __syncthreads();
    if (p.rwm) {
        if (tid < p.K) {
            const int k = tid;
            const double la = s_f[k] - p.f_state[k];
            const int acc = (p.log_u[k] < la) ? 1 : 0;
            s_acc[k] = acc;
            if (acc)
                p.f_state[k] = s_f[k];
            if (p.accept)
                p.accept[k] = (uint8_t)acc;
            if (p.logpost)
                p.logpost[k] = acc ? s_f[k] : p.f_state[k];
        }
        __syncthreads();
        for (int idx = tid; idx < p.K * P; idx += NT) {
            const int k = idx / P;
            float v = p.state[idx];
            if (s_acc[k]) {
                v = fmaf(p.step, p.z[idx], v);
                p.state[idx] = v;
            }
            if (p.samples)
                p.samples[idx] = v;
        }
    }
    if (tid == 0) {
        *p.ticket = 0u;
        *p.acc_flag = 0u;
    }
}

// Host-side launch helper for one storage type.
template <typename Tag>
glm_status_t launch_fused_t(glm_ctx *h, const FusedParams &prm, int kc, cudaStream_t s)
{
    using TR = XTraits<Tag>;
    const FusedLayout L = fused_layout(prm.srow, prm.ld, TR::EPC, prm.tile_rows, prm.stages, kc);
    if (prm.box_rows > 0 && fused_tensor_map(h, prm.X) != GLM_OK)
        return GLM_ERR_CUDA;
    void (*fn)(const CUtensorMap, FusedParams) = nullptr;
#define GLM_PICK(KCV, SP)                                                   \
    if (kc == KCV && h->split == SP)                                        \
        fn = fused_logpost_grad_kernel<Tag, KCV, SP>;
    GLM_PICK(1, 1) GLM_PICK(1, 2) GLM_PICK(1, 4) GLM_PICK(1, 32)
    GLM_PICK(2, 1) GLM_PICK(2, 2) GLM_PICK(2, 4) GLM_PICK(2, 32)
    GLM_PICK(4, 1) GLM_PICK(4, 2) GLM_PICK(4, 4) GLM_PICK(4, 32)
    if constexpr (TR::EPC <= 8) {
        GLM_PICK(8, 1) GLM_PICK(8, 2) GLM_PICK(8, 4) GLM_PICK(8, 32)
    }
#undef GLM_PICK
    if (!fn)
        return GLM_ERR_UNSUPPORTED;
    if (allow_max_dynamic_smem(reinterpret_cast<const void *>(fn)) != cudaSuccess)
        return GLM_ERR_CUDA;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)h->grid);
    cfg.blockDim = dim3(kFusedThreads);
    cfg.dynamicSmemBytes = (size_t)L.total;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = h->use_pdl ? 1 : 0;
    const CUtensorMap *map = reinterpret_cast<const CUtensorMap *>(h->fx_map);
    if (cudaLaunchKernelEx(&cfg, fn, *map, prm) != cudaSuccess)
        return GLM_ERR_CUDA;
    return GLM_OK;
}

}  // namespace glm
