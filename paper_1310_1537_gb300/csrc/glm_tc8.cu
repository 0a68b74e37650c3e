// Batched log-posterior + gradient on the tcgen05 tensor cores with X stored
// as FP8 E4M3, the operands taken by the MMAs in E4M3 (kind::f8f6f4): no
// widening of X on the chip.
//
// With K coefficient vectors the paper's two LA maps (§4.2: X beta, then
// X^t g_f) are N x P x K contractions. One persistent CTA per SM streams
// 128-row tiles of X into shared memory with TMA (128-byte swizzle) and, from
// the same staged tile (§4.2.1 cache fusion),
//   MMA1: D1[128 rows x 256] = X_tile . Bt^t, where Bt holds four E4M3 terms
//         of every coefficient vector, term t of vector k in column 64 t + k;
//   epilogue: thread = tile row. eta_k = 2^-e_k sum_t 16^-t D1[t, k]; the TR
//         map (ell, r); f accumulated per (row, vector); r written as five
//         E4M3 terms in two blocks (below) to the R tiles;
//   MMA2: D2[P x 128] += X_tile^t . [hi | dhi] + X_tile^t . [mid | dlo] and
//         D2[P x 64] += X_tile^t . lo (X read MN-major): columns 0..63 of
//         D2 collect block A, columns 64..127 block B.
// D2 stays in tensor memory for the CTA's whole run;
// g_kj = s_j (2^-8 D2[j, k] + 2^-20 D2[j, 64 + k]).
//
// Precision (FP32 accumulation, FP64 final combine of f): E4M3 keeps 4
// significant bits, so the coefficients s_j beta_kj (s_j the column scale) are
// written as four E4M3 terms, term t scaled by 2^(e_k + 4 t), where 2^e_k
// brings the vector's largest coefficient into [128, 256). Each term has its
// own scale, so coefficients far below the vector's largest stay in E4M3's
// normal range down to 2^-22 of it. The residual r (|r| < 1) needs about 20
// bits where g is a near-cancelling sum (near the mode): v = 2^8 r is rounded
// to FP16 (a16) and a16 split exactly (FP16 differences) into three E4M3
// terms (block A, scale 2^8); the FP32 remainder (v - a16) 2^12 is rounded to
// FP16 and split into two more (block B, scale 2^20).
//
// Warp roles: all ten warps first stage the coefficients and write their
// E4M3 terms into shared memory; then warp 0 issues the TMA loads, warp 1
// owns tensor memory and one of its threads issues the MMAs, and warps 2..9
// run the epilogue. Every wait is bounded.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_fp16.h>
#include <cmath>
#include <cstring>

#include "glm_internal.cuh"
#include "glm_tc_common.cuh"

namespace glm {

namespace {

constexpr int kRows = 128;                  // tile rows = tensor-memory lanes
constexpr int kVec = 64;                    // vectors per launch
constexpr int kBT = 4;                      // E4M3 terms per coefficient
constexpr int kEpiWarps = 8;
constexpr int kThreads = 32 * (2 + kEpiWarps);
constexpr int kT8MaxStages = 6;
constexpr int kMaxNR = 2;                   // R tile buffers
constexpr int kMaxP = 256;
constexpr int kAtom = kRows * 128;          // one 128-column atom of a tile: 16 KB
constexpr int kBetaAtom = kBT * kVec * 128; // coefficient terms for 128 columns: 32 KB
constexpr int kR128 = kRows * 128;          // R tiles [hi | dhi] and [mid | dlo]: 128 rows x 128 B
constexpr int kR64 = kRows * 64;            // R tile lo: 128 rows x 64 B
constexpr int kRbuf = 2 * kR128 + kR64;
constexpr int kTmemCols = 512;
constexpr int kD1Col = 0;                   // 256 columns: (term, vector)
constexpr int kD2Col = 256;                 // block mb at 256 + 128 mb

struct Tc8Params {
    const uint8_t *y;
    const float *beta;          // kk x P, this chunk
    const float *x_scale;       // P column scales
    int64_t N;
    int P;
    int kk;                     // vectors in this chunk (<= 64)
    int PA;                     // 128-column atoms of a tile
    int stages;
    int nr;                     // R tile buffers (1 or 2)
    double *part_f;             // grid x 64
    float *part_g;              // grid x 64 x (PA * 128)
    unsigned *status;
};

struct Tc8Layout {
    int x_stage;
    int b_off;
    int r_off;
    int bar_off;
    int total;                  // including 1 KB alignment slack
};

__host__ __device__ inline Tc8Layout tc8_layout(int PA, int stages, int nr)
{
    Tc8Layout L;
    L.x_stage = PA * kAtom;
    L.b_off = stages * L.x_stage;
    L.r_off = L.b_off + PA * kBetaAtom;
    L.bar_off = L.r_off + nr * kRbuf;
    L.total = L.bar_off + 1024 + 1024;
    return L;
}

// Two E4M3 codes (round to nearest even, saturating) of a0, a1 in bytes 0
// and 1, and their values.
__device__ __forceinline__ uint32_t e4m3_pair(float a0, float a1, float &v0, float &v1)
{
    unsigned short h;
    uint32_t h2;
    asm("cvt.rn.satfinite.e4m3x2.f32 %0, %1, %2;" : "=h"(h) : "f"(a1), "f"(a0));
    asm("cvt.rn.f16x2.e4m3x2 %0, %1;" : "=r"(h2) : "h"(h));
    const __half2 hv = *reinterpret_cast<const __half2 *>(&h2);
    v0 = __low2float(hv);
    v1 = __high2float(hv);
    return (uint32_t)h;
}

// Four values v = 2^8 r (|v| < 256): a16 = fp16(v) split exactly into three
// E4M3 terms (block A: hi, mid, lo), and d = v - a16, exact in FP32, rounded
// to FP16, scaled by 2^12 (exact) and split into two (block B: dhi, dlo). Word t holds term
// t (hi, mid, lo, dhi, dlo) of value i in byte i.
__device__ __forceinline__ void split5(float a0, float a1, float a2, float a3, uint32_t *w)
{
    asm("{\n\t"
        ".reg .b32 h01, h23, d01, d23, b01, b23, k12;\n\t"
        ".reg .b16 e01, e23, x0, x1, x2, x3;\n\t"
        ".reg .f32 f0, f1, f2, f3;\n\t"
        "cvt.rn.f16x2.f32 h01, %6, %5;\n\t"
        "cvt.rn.f16x2.f32 h23, %8, %7;\n\t"
        "mov.b32 {x0, x1}, h01;\n\t"
        "mov.b32 {x2, x3}, h23;\n\t"
        "cvt.f32.f16 f0, x0;\n\t"
        "cvt.f32.f16 f1, x1;\n\t"
        "cvt.f32.f16 f2, x2;\n\t"
        "cvt.f32.f16 f3, x3;\n\t"
        "sub.f32 f0, %5, f0;\n\t"
        "sub.f32 f1, %6, f1;\n\t"
        "sub.f32 f2, %7, f2;\n\t"
        "sub.f32 f3, %8, f3;\n\t"
        "cvt.rn.f16x2.f32 d01, f1, f0;\n\t"
        "cvt.rn.f16x2.f32 d23, f3, f2;\n\t"
        "mov.b32 k12, 0x6C006C00;\n\t"
        "mul.rn.f16x2 d01, d01, k12;\n\t"
        "mul.rn.f16x2 d23, d23, k12;\n\t"
        "cvt.rn.satfinite.e4m3x2.f16x2 e01, h01;\n\t"
        "cvt.rn.satfinite.e4m3x2.f16x2 e23, h23;\n\t"
        "mov.b32 %0, {e01, e23};\n\t"
        "cvt.rn.f16x2.e4m3x2 b01, e01;\n\t"
        "cvt.rn.f16x2.e4m3x2 b23, e23;\n\t"
        "sub.rn.f16x2 h01, h01, b01;\n\t"
        "sub.rn.f16x2 h23, h23, b23;\n\t"
        "cvt.rn.satfinite.e4m3x2.f16x2 e01, h01;\n\t"
        "cvt.rn.satfinite.e4m3x2.f16x2 e23, h23;\n\t"
        "mov.b32 %1, {e01, e23};\n\t"
        "cvt.rn.f16x2.e4m3x2 b01, e01;\n\t"
        "cvt.rn.f16x2.e4m3x2 b23, e23;\n\t"
        "sub.rn.f16x2 h01, h01, b01;\n\t"
        "sub.rn.f16x2 h23, h23, b23;\n\t"
        "cvt.rn.satfinite.e4m3x2.f16x2 e01, h01;\n\t"
        "cvt.rn.satfinite.e4m3x2.f16x2 e23, h23;\n\t"
        "mov.b32 %2, {e01, e23};\n\t"
        "cvt.rn.satfinite.e4m3x2.f16x2 e01, d01;\n\t"
        "cvt.rn.satfinite.e4m3x2.f16x2 e23, d23;\n\t"
        "mov.b32 %3, {e01, e23};\n\t"
        "cvt.rn.f16x2.e4m3x2 b01, e01;\n\t"
        "cvt.rn.f16x2.e4m3x2 b23, e23;\n\t"
        "sub.rn.f16x2 d01, d01, b01;\n\t"
        "sub.rn.f16x2 d23, d23, b23;\n\t"
        "cvt.rn.satfinite.e4m3x2.f16x2 e01, d01;\n\t"
        "cvt.rn.satfinite.e4m3x2.f16x2 e23, d23;\n\t"
        "mov.b32 %4, {e01, e23};\n\t"
        "}"
        : "=r"(w[0]), "=r"(w[1]), "=r"(w[2]), "=r"(w[3]), "=r"(w[4])
        : "f"(a0), "f"(a1), "f"(a2), "f"(a3));
}

// The TR map for one (row, vector) pair with the label folded into signs:
// z = (1 - 2y) eta, ell = -softplus(z), r = y - sigma(eta) = -(1 - 2y) sigma(z).
// Returns 2^8 r; adds ell to facc. ysign = y ? sign bit : 0.
__device__ __forceinline__ float tr_pair(float eta, uint32_t ysign, float &facc)
{
    constexpr float kLog2e = 1.4426950408889634f;
    constexpr float kLn2 = 0.69314718055994531f;
    const float z = __uint_as_float(__float_as_uint(eta) ^ ysign);
    const float e = tc::ex2_approx(-fabsf(eta) * kLog2e);          // exp(-|z|) in (0, 1]
    const float L = tc::lg2_approx(1.0f + e);                      // log2(1 + e)
    facc = fmaf(-kLn2, L, facc) - fmaxf(z, 0.0f);
    const float s8 = tc::ex2_approx(fmaf(fminf(z, 0.0f), kLog2e, 8.0f - L));   // 2^8 sigma(z)
    return __uint_as_float(__float_as_uint(s8) ^ (ysign ^ 0x80000000u));
}

__global__ void __launch_bounds__(kThreads, 1)
    tc8_logpost_grad_kernel(const __grid_constant__ CUtensorMap tmap, Tc8Params p)
{
    constexpr uint32_t ID1 = tc::idesc_make(kRows, kBT * kVec, 0, 0, 0, 0);   // X . Bt^t
    constexpr uint32_t ID2 = tc::idesc_make(kRows, 2 * kVec, 0, 0, 1, 1);     // X^t . [A | B] terms
    constexpr uint32_t ID2L = tc::idesc_make(kRows, kVec, 0, 0, 1, 1);        // X^t . lo

    extern __shared__ uint8_t smem_raw[];
    uint8_t *smem = smem_raw + ((1024u - (ptx::smem_u32(smem_raw) & 1023u)) & 1023u);
    const int PA = p.PA;
    const int S = p.stages;
    const int NR = p.nr;
    const Tc8Layout L = tc8_layout(PA, S, NR);
    uint8_t *xs = smem;
    uint8_t *bs = smem + L.b_off;
    uint8_t *rs = smem + L.r_off;
    uint64_t *bars = reinterpret_cast<uint64_t *>(smem + L.bar_off);
    uint64_t *x_full = bars;                        // [S]
    uint64_t *x_empty = bars + kT8MaxStages;          // [S]
    uint64_t *d1_full = bars + 2 * kT8MaxStages;
    uint64_t *d1_empty = d1_full + 1;
    uint64_t *r_full = d1_empty + 1;                // [NR]
    uint64_t *r_empty = r_full + kMaxNR;            // [NR]
    uint64_t *d2_done = r_empty + kMaxNR;
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(d2_done + 1);
    float *vsc = reinterpret_cast<float *>(smem + L.bar_off + 256);      // [64] 2^-e_k
    float *vsc_inv = reinterpret_cast<float *>(smem + L.bar_off + 512);  // [64] 2^e_k
    double *sf = reinterpret_cast<double *>(smem + L.r_off);             // [4][64], at the end
    __shared__ int s_abort;

    const int tid = threadIdx.x;
    const int warp = tid >> 5;
    const int lane = tid & 31;
    const int grid = gridDim.x;
    const int b = blockIdx.x;
    const int64_t ntiles_all = (p.N + kRows - 1) / kRows;
    const int nt = (int)(ntiles_all > b ? (ntiles_all - b + grid - 1) / grid : 0);

    if (tid == 0) {
        for (int s = 0; s < kT8MaxStages; ++s) {
            ptx::mbar_init(&x_full[s], 1);
            ptx::mbar_init(&x_empty[s], 1);
        }
        ptx::mbar_init(d1_full, 1);
        ptx::mbar_init(d1_empty, kEpiWarps);
        for (int j = 0; j < kMaxNR; ++j) {
            ptx::mbar_init(&r_full[j], kEpiWarps);
            ptx::mbar_init(&r_empty[j], 1);
        }
        ptx::mbar_init(d2_done, 1);
        ptx::fence_mbar_init();
        s_abort = 0;
        asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&tmap)) : "memory");
    }
    if (warp == 1) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                         ptx::smem_u32(tmem_slot)),
                     "r"(kTmemCols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    ptx::grid_dep_wait();

    // ---- coefficient terms into shared memory ---------------------------------------
    // The chunk's coefficients and the column scales are first copied into the
    // (still idle) operand ring and R tile with independent wide loads, so the
    // terms are computed from shared memory, not from chains of global loads.
    const int et = tid - 64;
    float *bst = reinterpret_cast<float *>(xs);            // kk x P (the ring is >= 64 KB)
    float *sst = reinterpret_cast<float *>(rs);            // P
    {
        const int nb = p.kk * p.P;
        if ((reinterpret_cast<uintptr_t>(p.beta) & 15u) == 0 && (nb & 3) == 0) {
            // batches of eight independent 16-byte loads per thread
            const float4 *src = reinterpret_cast<const float4 *>(p.beta);
            float4 *dst = reinterpret_cast<float4 *>(bst);
            const int n4 = nb / 4;
            for (int base = tid; base < n4; base += 8 * kThreads) {
                float4 t[8];
#pragma unroll
                for (int u = 0; u < 8; ++u) {
                    const int idx = base + u * kThreads;
                    t[u] = idx < n4 ? __ldg(src + idx) : make_float4(0.0f, 0.0f, 0.0f, 0.0f);
                }
#pragma unroll
                for (int u = 0; u < 8; ++u) {
                    const int idx = base + u * kThreads;
                    if (idx < n4)
                        dst[idx] = t[u];
                }
            }
        } else {
#pragma unroll 4
            for (int idx = tid; idx < nb; idx += kThreads)
                bst[idx] = __ldg(p.beta + idx);
        }
        for (int idx = tid; idx < p.P; idx += kThreads)
            sst[idx] = __ldg(p.x_scale + idx);
    }
    __syncthreads();
    // e_k: 2^e_k brings max_j |s_j beta_kj| into [128, 256). Warp w of the
    // epilogue group takes vectors w, w + 8, ...
    if (warp >= 2) {
        const int ew = et >> 5;
        for (int k = ew; k < kVec; k += kEpiWarps) {
            float m = 0.0f;
            if (k < p.kk)
                for (int col = lane; col < p.P; col += 32)
                    m = fmaxf(m, fabsf(bst[k * p.P + col] * sst[col]));
#pragma unroll
            for (int o = 16; o > 0; o >>= 1)
                m = fmaxf(m, __shfl_xor_sync(0xFFFFFFFFu, m, o));
            if (lane == 0) {
                int e = 0;
                if (m > 0.0f && m <= 3.0e38f) {
                    int ex;
                    frexpf(m, &ex);             // m in [2^(ex-1), 2^ex)
                    e = 8 - ex;
                    e = e < -100 ? -100 : (e > 100 ? 100 : e);
                }
                vsc_inv[k] = ldexpf(1.0f, e);
                vsc[k] = ldexpf(1.0f, -e);
            }
        }
    }
    __syncthreads();
    {
        // item = (vector k, four consecutive columns): one 32-bit word per term
        // at line 64 t + k of the K-major, 128-byte-swizzled term matrix
        const int ngrp = PA * 32;
        for (int it = tid; it < kVec * ngrp; it += kThreads) {
            const int k = it / ngrp;
            const int col0 = (it - k * ngrp) * 4;
            uint32_t w[kBT] = {0u, 0u, 0u, 0u};
            if (k < p.kk) {
                const float sc = vsc_inv[k];
                float rem[4];
#pragma unroll
                for (int c = 0; c < 4; ++c) {
                    const int col = col0 + c;
                    rem[c] = col < p.P ? bst[k * p.P + col] * sst[col] * sc : 0.0f;
                }
                // term t = E4M3(rem 16^t); rem -= value 16^-t (exact: powers of two)
#pragma unroll
                for (int t = 0; t < kBT; ++t) {
                    const float up = (float)(1 << (4 * t));
                    const float dn = 1.0f / up;
                    float v[4];
                    const uint32_t lo = e4m3_pair(rem[0] * up, rem[1] * up, v[0], v[1]);
                    const uint32_t hi = e4m3_pair(rem[2] * up, rem[3] * up, v[2], v[3]);
                    w[t] = lo | (hi << 16);
#pragma unroll
                    for (int c = 0; c < 4; ++c)
                        rem[c] = fmaf(-v[c], dn, rem[c]);
                }
            }
            const int a = col0 >> 7;
#pragma unroll
            for (int t = 0; t < kBT; ++t) {
                const int n = t * kVec + k;
                const int off = a * kBetaAtom + n * 128 + ((((col0 & 127) >> 4) ^ (n & 7)) << 4) +
                                (col0 & 15);
                *reinterpret_cast<uint32_t *>(bs + off) = w[t];
            }
        }
    }
    // the terms are read by the tensor cores and the ring is refilled by TMA
    // (async proxy) after these generic-proxy accesses
    ptx::fence_proxy_async_smem();
    tc::fence_before();
    __syncthreads();
    tc::fence_after();
    const uint32_t tmem = *tmem_slot;
    ptx::grid_dep_launch_dependents();

    if (warp == 0) {
        // ---- TMA producer (lane 0) ---------------------------------------------------------
        // (Prefetching the tiles beyond the ring into L2 from this warp's
        // lanes was measured 3 % slower: its instructions share the MIO queue
        // with the epilogue.)
        if (lane == 0) {
            const unsigned bytes = (unsigned)(PA * kAtom);
            for (int i = 0; i < nt; ++i) {
                const int s = i % S;
                const int use = i / S;
                if (use > 0 && !ptx::mbar_wait_bounded(&x_empty[s], (unsigned)(use - 1) & 1u, kSpinLimit)) {
                    atomicOr(p.status, kDevTimeout);
                    s_abort = 1;
                    break;
                }
                const int row0 = (int)((int64_t)(b + (int64_t)i * grid) * kRows);
                ptx::mbar_arrive_expect_tx(&x_full[s], bytes);
                for (int a = 0; a < PA; ++a)
                    tc::tma_load_2d(xs + s * L.x_stage + a * kAtom, &tmap, a * 128, row0, &x_full[s]);
            }
        }
    } else if (warp == 1) {
        // ---- MMA issuer -----------------------------------------------------------------
        if (lane == 0) {
            // descriptors built once and stepped by adding address offset / 16
            // (the 14-bit address field; shared addresses stay below 256 KB)
            const uint32_t xs0 = ptx::smem_u32(xs);
            const uint32_t rs0 = ptx::smem_u32(rs);
            const uint64_t dA1 = tc::mdesc(xs0, 16, 1024);                 // X, K-major
            const uint64_t dB1 = tc::mdesc(ptx::smem_u32(bs), 16, 1024);   // terms, K-major
            const uint64_t dA2 = tc::mdesc(xs0, kAtom, 1024);              // X, MN-major
            const uint64_t dR1 = tc::mdesc(rs0, kR128, 1024);              // [hi | dhi], MN-major
            const uint64_t dR2 = tc::mdesc(rs0 + kR128, kR128, 1024);      // [mid | dlo], MN-major
            const uint64_t dR3 = tc::mdesc(rs0 + 2 * kR128, kR64, 512, 4u); // lo, MN-major, 64B
            const int ksteps = (p.P + 31) / 32;
            bool ok = true;
            for (int i = 0; i <= nt && ok; ++i) {
                if (i < nt) {
                    const int s = i % S;
                    ok = ptx::mbar_wait_bounded(&x_full[s], (unsigned)(i / S) & 1u, kSpinLimit);
                    if (ok && i >= 1)
                        ok = ptx::mbar_wait_bounded(d1_empty, (unsigned)(i - 1) & 1u, kSpinLimit);
                    if (!ok)
                        break;
                    tc::fence_after();
                    const uint64_t a0 = dA1 + (uint64_t)((s * L.x_stage) >> 4);
                    for (int c = 0; c < ksteps; ++c) {
                        const uint32_t xo = (uint32_t)((c >> 2) * kAtom + (c & 3) * 32);
                        const uint32_t bo = (uint32_t)((c >> 2) * kBetaAtom + (c & 3) * 32);
                        tc::mma_f8(tmem + kD1Col, a0 + (xo >> 4), dB1 + (bo >> 4), ID1,
                                   c > 0 ? 1u : 0u);
                    }
                    tc::commit(d1_full);
                }
                if (i >= 1) {
                    const int j = i - 1;
                    const int sj = j % S;
                    const int rj = j % NR;
                    ok = ptx::mbar_wait_bounded(&r_full[rj], (unsigned)(j / NR) & 1u, kSpinLimit);
                    if (!ok)
                        break;
                    tc::fence_after();
                    const uint64_t a2 = dA2 + (uint64_t)((sj * L.x_stage) >> 4);
                    const uint64_t rstep = (uint64_t)((rj * kRbuf) >> 4);
                    for (int mb = 0; mb < PA; ++mb) {
                        const uint32_t dt = tmem + kD2Col + mb * 128;
#pragma unroll
                        for (int ks = 0; ks < kRows / 32; ++ks) {      // 32 rows each
                            const uint64_t am = a2 + (uint64_t)((mb * kAtom + ks * 4096) >> 4);
                            const uint64_t r128 = rstep + (uint64_t)((ks * 4096) >> 4);
                            tc::mma_f8(dt, am, dR1 + r128, ID2, (j > 0 || ks > 0) ? 1u : 0u);
                            tc::mma_f8(dt, am, dR2 + r128, ID2, 1u);
                            tc::mma_f8(dt, am, dR3 + rstep + (uint64_t)((ks * 2048) >> 4), ID2L, 1u);
                        }
                    }
                    tc::commit(&x_empty[sj]);
                    tc::commit(&r_empty[rj]);
                }
            }
            if (!ok) {
                atomicOr(p.status, kDevTimeout);
                s_abort = 1;
            }
            if (nt > 0)
                tc::commit(d2_done);
        }
    } else {
        // ---- epilogue: thread = tile row, 32 vectors --------------------------------------
        // Per tile: eta of the 32 vectors from tensor memory, then the TR map and
        // the residual terms in batches of 8. Rows past N arrive as zeros
        // (TMA fill): they add nothing to g and exactly -ln 2 to each f
        // accumulator (eta = 0), which is taken back at the end.
        constexpr float kLn2 = 0.69314718055994531f;
        const int q = warp & 3;                     // tensor-memory lane quarter
        const int c = (warp - 2) >> 2;              // vectors 32c .. 32c + 31
        const int rl = q * 32 + lane;               // tile row
        const uint32_t tq = tmem + ((uint32_t)(q * 32) << 16);
        float facc[32];
#pragma unroll
        for (int j = 0; j < 32; ++j)
            facc[j] = 0.0f;
        int n_pad = 0;                              // rows of this thread past N
        auto label = [&](int i) -> int {
            if (i >= nt)
                return -1;
            const int64_t row = (int64_t)(b + (int64_t)i * grid) * kRows + rl;
            return row < p.N ? (int)__ldg(p.y + row) : -1;
        };
        auto load_batch = [&](int h, float (*v)[8]) {
#pragma unroll
            for (int t = 0; t < kBT; ++t)
                tc::tmem_ld<8>(tq + kD1Col + t * kVec + 32 * c + 8 * h, v[t]);
        };
        int ycur = label(0);
        bool ok = true;
        for (int i = 0; i < nt; ++i) {
            const int ynext = label(i + 1);
            if (!ptx::mbar_wait_bounded(d1_full, (unsigned)i & 1u, kSpinLimit)) {
                ok = false;
                break;
            }
            tc::fence_after();
            n_pad += ycur < 0 ? 1 : 0;
            const uint32_t ysign = ycur == 1 ? 0x80000000u : 0u;
            const int rb = i % NR;
            uint8_t *rbuf = rs + rb * kRbuf;
            // eta for all 32 vectors first (four batches, the loads of batch h + 1
            // in flight while batch h is combined), then D1 is released so the
            // next tile's MMA1 overlaps the TR map below
            float eta[32];
            {
                float va[kBT][8], vb[kBT][8];
                load_batch(0, va);
                tc::tmem_wait_ld();
#pragma unroll
                for (int h = 0; h < 4; ++h) {
                    float (*cur)[8] = (h & 1) ? vb : va;
                    float (*nxt)[8] = (h & 1) ? va : vb;
                    if (h < 3)
                        load_batch(h + 1, nxt);
                    const float4 s0 = *reinterpret_cast<const float4 *>(vsc + 32 * c + 8 * h);
                    const float4 s1 = *reinterpret_cast<const float4 *>(vsc + 32 * c + 8 * h + 4);
                    const float sv[8] = {s0.x, s0.y, s0.z, s0.w, s1.x, s1.y, s1.z, s1.w};
#pragma unroll
                    for (int j = 0; j < 8; ++j) {
                        float es = fmaf(cur[3][j], 0.0625f, cur[2][j]);
                        es = fmaf(es, 0.0625f, cur[1][j]);
                        es = fmaf(es, 0.0625f, cur[0][j]);
                        eta[8 * h + j] = es * sv[j];
                    }
                    if (h < 3)
                        tc::tmem_wait_ld();
                }
            }
            tc::fence_before();
            __syncwarp();
            if (lane == 0)
                ptx::mbar_arrive(d1_empty);
            uint32_t w[5][8];
#pragma unroll
            for (int h = 0; h < 4; ++h) {              // vectors 32c + 8h .. + 7
                float r8[8];
#pragma unroll
                for (int j = 0; j < 8; ++j)
                    r8[j] = tr_pair(eta[8 * h + j], ysign, facc[8 * h + j]);
                uint32_t wa[5], wb[5];
                split5(r8[0], r8[1], r8[2], r8[3], wa);
                split5(r8[4], r8[5], r8[6], r8[7], wb);
#pragma unroll
                for (int t = 0; t < 5; ++t) {
                    w[t][2 * h] = wa[t];
                    w[t][2 * h + 1] = wb[t];
                }
            }
            // R tile, written last: with one buffer the previous tile's MMA2
            // (issued when that tile's epilogue ended) has to have read it,
            // and by now it has had the whole TR map to do so
            if (i >= NR && !ptx::mbar_wait_bounded(&r_empty[rb], (unsigned)(i / NR - 1) & 1u, kSpinLimit))
                ok = false;
            // [hi | dhi] and [mid | dlo] are 128-byte rows with 16-byte chunks
            // permuted by row & 7, lo 64-byte rows with chunks permuted by
            // (row >> 1) & 3; chunk 2c + half holds vectors 32c + 16 half ..
#pragma unroll
            for (int half = 0; half < 2; ++half) {
                const uint32_t ch = (uint32_t)(2 * c + half);
                const uint32_t sw = (uint32_t)(rl & 7);
                const uint32_t ca = (ch ^ sw) << 4;
                const uint32_t cb = ((4u + ch) ^ sw) << 4;
                const int o = 4 * half;
                *reinterpret_cast<uint4 *>(rbuf + rl * 128 + ca) =
                    make_uint4(w[0][o], w[0][o + 1], w[0][o + 2], w[0][o + 3]);
                *reinterpret_cast<uint4 *>(rbuf + rl * 128 + cb) =
                    make_uint4(w[3][o], w[3][o + 1], w[3][o + 2], w[3][o + 3]);
                *reinterpret_cast<uint4 *>(rbuf + kR128 + rl * 128 + ca) =
                    make_uint4(w[1][o], w[1][o + 1], w[1][o + 2], w[1][o + 3]);
                *reinterpret_cast<uint4 *>(rbuf + kR128 + rl * 128 + cb) =
                    make_uint4(w[4][o], w[4][o + 1], w[4][o + 2], w[4][o + 3]);
                *reinterpret_cast<uint4 *>(rbuf + 2 * kR128 + rl * 64 +
                                           ((ch ^ ((uint32_t)(rl >> 1) & 3u)) << 4)) =
                    make_uint4(w[2][o], w[2][o + 1], w[2][o + 2], w[2][o + 3]);
            }
            if (!ok)
                break;
            ptx::fence_proxy_async_smem();
            __syncwarp();
            if (lane == 0)
                ptx::mbar_arrive(&r_full[rb]);
            ycur = ynext;
        }
        if (!ok) {
            atomicOr(p.status, kDevTimeout);
            s_abort = 1;
        }
        const int PP = PA * 128;
        const bool have = nt > 0 && ok && ptx::mbar_wait_bounded(d2_done, 0u, kSpinLimit);
        if (nt > 0 && !have) {
            atomicOr(p.status, kDevTimeout);
            s_abort = 1;
        }
        tc::fence_after();
        // f partial: the warp's 32 rows (the R tiles are free: every MMA has
        // completed), then the four lane quarters in order
        const float pad = (float)n_pad * kLn2;
        // (FP32 across the 32 lanes: each lane holds a sum of about 50 terms, and
        // FP64 arithmetic is slow on this part; FP64 from the quarter sums on)
#pragma unroll
        for (int j = 0; j < 32; ++j) {
            float v = facc[j] + pad;
#pragma unroll
            for (int o = 16; o > 0; o >>= 1)
                v += __shfl_xor_sync(0xFFFFFFFFu, v, o);
            if (lane == 0)
                sf[q * kVec + 32 * c + j] = (double)v;
        }
        asm volatile("bar.sync 1, %0;" ::"r"(kEpiWarps * 32) : "memory");
        if (et < p.kk) {
            const double tot = ((sf[et] + sf[kVec + et]) + sf[2 * kVec + et]) + sf[3 * kVec + et];
            p.part_f[(size_t)b * kVec + et] =
                s_abort ? __longlong_as_double(0x7FF8000000000000LL) : tot;
        }
        // g partial: lanes of D2 block mb are columns of X; this warp's 32
        // vectors, 16 at a time
        for (int mb = 0; mb < PA; ++mb) {
            const int pcol = mb * 128 + q * 32 + lane;
#pragma unroll
            for (int half = 0; half < 2; ++half) {
                float g0[16], g1[16];
                const int k0 = 32 * c + 16 * half;
                if (have) {
                    tc::tmem_ld<16>(tq + kD2Col + mb * 128 + k0, g0);
                    tc::tmem_ld<16>(tq + kD2Col + mb * 128 + kVec + k0, g1);
                    tc::tmem_wait_ld();
                }
#pragma unroll
                for (int j = 0; j < 16; ++j) {
                    const int k = k0 + j;
                    if (k < p.kk)
                        p.part_g[((size_t)b * kVec + k) * PP + pcol] =
                            have ? fmaf(g1[j], 1.0f / 1048576.0f, g0[j] * (1.0f / 256.0f)) : 0.0f;
                }
            }
        }
    }
    tc::fence_before();
    __syncthreads();
    tc::fence_after();
    if (warp == 1)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                     "r"(kTmemCols)
                     : "memory");
}

}  // namespace

// Fixed-order combine of the per-CTA partials (defined with the BF16 pass).
__global__ void tc_reduce_kernel(const double *__restrict__ part_f, const float *__restrict__ part_g,
                                 int parts, int KB, int PP, int P, int kk, int nf,
                                 const float *__restrict__ beta, const float *__restrict__ x_scale,
                                 double inv_s2, double prior_const, double *__restrict__ f_out,
                                 float *__restrict__ g_out);
constexpr int kTc8RedWarps = 8;

bool tc8_supported(int p) { return p <= kMaxP; }

// Operand-tile stages and R buffers that fit: two R buffers with at least
// four stages, else one buffer and the deepest ring (P = 256: three stages).
static bool tc8_stages(int PA, int *stages, int *nr)
{
    for (int st = kT8MaxStages; st >= 4; --st)
        if (tc8_layout(PA, st, 2).total <= kSmemDynamicBudget) {
            *stages = st;
            *nr = 2;
            return true;
        }
    for (int st = kT8MaxStages; st >= 3; --st)
        if (tc8_layout(PA, st, 1).total <= kSmemDynamicBudget) {
            *stages = st;
            *nr = 1;
            return true;
        }
    return false;
}

// The E4M3 rows as bytes, 128-column boxes of 128 rows with the 128-byte
// swizzle: each box lands as one K-major operand atom.
static glm_status_t tc8_tensor_map(glm_ctx *h, const void *X)
{
    if (h->tc_map_ptr == X)
        return GLM_OK;
    PFN_cuTensorMapEncodeTiled_v12000 encode = tensor_map_encoder();
    if (!encode)
        return GLM_ERR_CUDA;
    CUtensorMap *map = reinterpret_cast<CUtensorMap *>(h->tc_map);
    const cuuint64_t dims[2] = {(cuuint64_t)h->d.ld, (cuuint64_t)h->d.n_rows};
    const cuuint64_t strides[1] = {(cuuint64_t)h->d.ld};
    const cuuint32_t box[2] = {128, (cuuint32_t)kRows};
    const cuuint32_t estr[2] = {1, 1};
    CUresult r = encode(map, CU_TENSOR_MAP_DATA_TYPE_UINT8, 2, const_cast<void *>(X), dims,
                        strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                        CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                        CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS)
        return GLM_ERR_CUDA;
    h->tc_map_ptr = X;
    return GLM_OK;
}

glm_status_t launch_tc8(glm_ctx *h, const void *X, const float *x_scale, const uint8_t *y,
                        const float *beta, int K, double *f_out, float *g_out, cudaStream_t s)
{
    if (!h->tc_part_f || h->d.n_rows > ((int64_t)1 << 31) - kRows || h->d.p > kMaxP)
        return GLM_ERR_UNSUPPORTED;
    glm_status_t st = tc8_tensor_map(h, X);
    if (st != GLM_OK)
        return st;
    const int P = h->d.p;
    const int PA = (P + 127) / 128;
    int stages = 0, nr = 0;
    if (!tc8_stages(PA, &stages, &nr))
        return GLM_ERR_UNSUPPORTED;
    const double s2 = h->d.prior_sigma * h->d.prior_sigma;
    const bool prior = !(h->d.flags & GLM_FLAG_NO_PRIOR);
    const CUtensorMap *map = reinterpret_cast<const CUtensorMap *>(h->tc_map);
    const Tc8Layout L = tc8_layout(PA, stages, nr);
    if (allow_max_dynamic_smem(reinterpret_cast<const void *>(&tc8_logpost_grad_kernel)) !=
        cudaSuccess)
        return GLM_ERR_CUDA;
    // the partial layout shared with the combine kernel: 128-column blocks
    const int PP = ((P + 127) / 128) * 128;
    for (int k0 = 0; k0 < K; k0 += kVec) {
        const int kk = (K - k0) < kVec ? (K - k0) : kVec;
        Tc8Params prm;
        std::memset(&prm, 0, sizeof(prm));
        prm.y = y;
        prm.beta = beta + (size_t)k0 * P;
        prm.x_scale = x_scale;
        prm.N = h->d.n_rows;
        prm.P = P;
        prm.kk = kk;
        prm.PA = PA;
        prm.stages = stages;
        prm.nr = nr;
        prm.part_f = h->tc_part_f;
        prm.part_g = h->tc_part_g;
        prm.status = h->status;
        cudaLaunchConfig_t cfg = {};
        cfg.gridDim = dim3((unsigned)h->sm_count);
        cfg.blockDim = dim3(kThreads);
        cfg.dynamicSmemBytes = (size_t)L.total;
        cfg.stream = s;
        cudaLaunchAttribute attr[1];
        attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
        attr[0].val.programmaticStreamSerializationAllowed = 1;
        cfg.attrs = attr;
        cfg.numAttrs = 1;
        if (cudaLaunchKernelEx(&cfg, tc8_logpost_grad_kernel, *map, prm) != cudaSuccess)
            return GLM_ERR_CUDA;
        const int ng = kk * ((P + 127) / 128);
        const int nf = (kk + kTc8RedWarps - 1) / kTc8RedWarps;
        cudaLaunchConfig_t rc = {};
        rc.gridDim = dim3((unsigned)(ng + nf));
        rc.blockDim = dim3(32 * kTc8RedWarps);
        rc.stream = s;
        rc.attrs = attr;
        rc.numAttrs = 1;
        if (cudaLaunchKernelEx(&rc, tc_reduce_kernel, (const double *)h->tc_part_f,
                               (const float *)h->tc_part_g, h->sm_count, kVec, PP, P, kk, nf,
                               beta + (size_t)k0 * P, x_scale, prior ? 1.0 / s2 : 0.0,
                               prior ? 0.5 * (double)P * std::log(2.0 * M_PI * s2) : 0.0,
                               f_out + k0, g_out + (size_t)k0 * P) != cudaSuccess)
            return GLM_ERR_CUDA;
    }
    return GLM_OK;
}

}  // namespace glm
