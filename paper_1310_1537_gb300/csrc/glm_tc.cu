// Batched log-posterior + gradient on the tcgen05 tensor cores.
//
// With K coefficient vectors the two LA maps of the paper's gradient routine
// (§4.2: X beta, then X^t g_f) become real contractions, N x P x K each. One
// persistent CTA per SM streams 128-row tiles of X (BF16) into shared memory
// with TMA (128B swizzle, 2-4 stages) and, from the same staged tile,
//   MMA1: D1[128 lanes x 128 rows] = B1 . X_tile^T, with A = B1 in tensor
//         memory (lanes in groups of 16: lane 16g + v holds the bf16 hi part
//         of beta for vector 16q + 8g + v of lane quarter q, the lo part
//         eight lanes further) and B = the tile, K-major;
//   epilogue (16 warps): 16x256b tensor-memory loads give each thread the hi
//         and lo partial sums of its (row, vector) pairs, which add to eta;
//         the TR map (labels folded in as a sign) gives ell and r; f is
//         accumulated per thread, and r is split into bf16 hi + lo and
//         written transposed (lane = vector and term, rows contiguous) into
//         the residual tile in shared memory;
//   MMA2: D2^t[128 lanes x P] += R^t . X_tile, with A = the residual tile
//         (K-major) and B = the X tile read MN-major, N = the tile's columns.
// D2^t stays in tensor memory for the CTA's whole run: the gradient never
// leaves the SM until the end, when the hi and lo lanes are added. Splitting
// beta and r into two bf16 terms keeps about 16 significant bits, so the
// results match the FP32 path to ~1e-5 while X stays in 2-byte storage.
// Per-CTA partials are combined by a second kernel in a fixed order
// (deterministic).
//
// FP8 E4M3 storage has its own pass (glm_tc8.cu), which takes the E4M3
// operands directly.
//
// Warp roles: warp 0 issues TMA loads, warp 1 allocates tensor memory and one
// of its threads issues the MMAs, warps 2..17 first write beta into tensor
// memory and then run the epilogue. Every wait is bounded.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_fp16.h>
#include <cmath>
#include <cstdlib>
#include <cstring>

#include "glm_internal.cuh"
#include "glm_tc_common.cuh"

namespace glm {

constexpr int kTcRows = 128;
constexpr int kTcEpiWarps = 16;
constexpr int kTcEpiGroups = kTcEpiWarps / 4;       // warps per tensor-memory lane quarter
constexpr int kTcEpiCols = 128 / kTcEpiGroups;      // D1 columns (tile rows) per warp
constexpr int kTcThreads = 32 * (2 + kTcEpiWarps);
constexpr int kTcMaxStages = 4;
constexpr int kTcMaxP = 256;
constexpr int kTcMaxKB = 64;
constexpr int kTcTmemCols = 512;

struct TcParams {
    const uint8_t *y;
    const float *beta;          // kk x P, this chunk
    int64_t N;
    int P;
    int kk;                     // vectors in this chunk (<= KB)
    int PA;                     // 64-column atoms of the tile
    int MB;                     // 128-column blocks of P (row stride of part_g)
    int stages;
    int y_al4;                  // y is 4-byte aligned: labels read as words
    double *part_f;             // grid x 64
    float *part_g;              // grid x 64 x (MB*128)
    unsigned *status;
};

namespace tc {

// kind::f16 instruction descriptor: D f32, A and B both bf16 (ab_type 1) or
// both f16 (ab_type 0), M=128, N=n.
__host__ __device__ constexpr uint32_t idesc_f16kind(int n, int a_mn, int b_mn, uint32_t ab_type)
{
    return (1u << 4) | (ab_type << 7) | (ab_type << 10) | ((uint32_t)a_mn << 15) |
           ((uint32_t)b_mn << 16) | ((uint32_t)(n >> 3) << 17) | ((uint32_t)(kTcRows >> 4) << 24);
}

// TR map on the hardware base-2 exponential and logarithm, overflow-free:
// with e = exp(-|z|) and L = log2(1 + e),
//   softplus(z) = max(z, 0) + L ln 2,
//   sigma(z) = exp(min(z, 0)) / (1 + e) = 2^(min(z, 0) log2(e) - L),
// so the logistic needs one more exponential and no reciprocal or select.
// TR map with the label folded into a sign: z = (1 - 2y) eta, so that
// ell = -softplus(z) and r = y - sigma(eta) = (2y - 1) sigma(z); ysh holds the
// label in its sign bit. Adds ell to facc and returns r.
__device__ __forceinline__ float tr_r(float eta, uint32_t ysh, float &facc)
{
    constexpr float kLog2e = 1.4426950408889634f;
    constexpr float kLn2 = 0.69314718055994531f;
    const float z = __uint_as_float(__float_as_uint(eta) ^ (ysh & 0x80000000u));
    const float e = ex2_approx(-fabsf(z) * kLog2e);       // exp(-|z|) in (0, 1]
    const float L = lg2_approx(1.0f + e);
    facc -= fmaxf(z, 0.0f);
    facc = fmaf(-kLn2, L, facc);
    const float sg = ex2_approx(fmaf(fminf(z, 0.0f), kLog2e, -L));   // sigma(z)
    return __uint_as_float(__float_as_uint(sg) ^ (~ysh & 0x80000000u));
}

// Residuals of two consecutive rows split into BF16 terms hi = round(r),
// lo = round(r - hi): the hi terms packed in one word and the lo terms in
// another (row a in the low half).
__device__ __forceinline__ void split_pair(float ra, float rb, uint32_t &hw, uint32_t &lw)
{
    const float ha = __bfloat162float(__float2bfloat16_rn(ra));
    const float hb = __bfloat162float(__float2bfloat16_rn(rb));
    __nv_bfloat162 h = __floats2bfloat162_rn(ha, hb);
    __nv_bfloat162 l = __floats2bfloat162_rn(ra - ha, rb - hb);
    hw = *reinterpret_cast<uint32_t *>(&h);
    lw = *reinterpret_cast<uint32_t *>(&l);
}

__device__ __forceinline__ uint32_t pack_bf16(float a, float b)
{
    __nv_bfloat162 v = __floats2bfloat162_rn(a, b);
    return *reinterpret_cast<uint32_t *>(&v);
}

// Two-term split of v in BF16: hi = round(v), lo = v - hi (rounded when packed).
__device__ __forceinline__ void split2(float v, float &hi, float &lo)
{
    hi = __bfloat162float(__float2bfloat16_rn(v));
    lo = v - hi;
}

}  // namespace tc

// Shared-memory layout of the tensor-core kernel (1024-byte aligned parts).
struct TcLayout {
    int x_stage;    // PA * 16 KB (bf16 / f16 operand tile, 128B swizzle)
    int x_off;
    int r_off;      // residual tile R^t: 2 atoms of (128 lanes x 128 B), K-major
    int bar_off;    // barriers, tensor-memory slot, per-vector scales
    int sf_off;     // 4 x 64 doubles (inside the residual tile, used after the last MMA)
    int total;      // including 1 KB alignment slack
};

__host__ __device__ inline TcLayout tc_layout(int PA, int stages)
{
    TcLayout L;
    L.x_stage = PA * 16384;
    L.x_off = 0;
    L.r_off = stages * L.x_stage;
    L.bar_off = L.r_off + 2 * 16384;
    L.sf_off = L.r_off;
    L.total = L.bar_off + 512 + 1024;
    return L;
}

// Tensor-memory columns: beta (A operand of MMA1) at 0, D1 at 128, D2 block
// mb at 256 + 128 mb.
constexpr int kTcB1Col = 0;
constexpr int kTcD1Col = 128;
constexpr int kTcD2Col = 256;

__global__ void __launch_bounds__(kTcThreads, 1)
    tc_logpost_grad_kernel(const __grid_constant__ CUtensorMap tmap, TcParams p)
{
    constexpr uint32_t AB = 1u;
    constexpr uint32_t ID1 = tc::idesc_f16kind(128, 0, 0, AB);
    const uint32_t ID2 = tc::idesc_f16kind(p.PA * 64, 0, 1, AB);   // N = the tile's columns

    extern __shared__ uint8_t smem_raw[];
    uint8_t *smem = smem_raw + ((1024u - (ptx::smem_u32(smem_raw) & 1023u)) & 1023u);
    const int PA = p.PA;
    const int MB = p.MB;
    const int stages = p.stages;
    const TcLayout L = tc_layout(PA, stages);
    uint8_t *xs = smem + L.x_off;
    uint8_t *rb = smem + L.r_off;
    uint64_t *bars = reinterpret_cast<uint64_t *>(smem + L.bar_off);
    uint64_t *x_full = bars;                    // [stages]
    uint64_t *x_empty = bars + kTcMaxStages;    // [stages]
    uint64_t *d1_full = bars + 2 * kTcMaxStages;
    uint64_t *d1_empty = d1_full + 1;
    uint64_t *r_full = d1_empty + 1;
    uint64_t *r_empty = r_full + 1;
    uint64_t *d2_done = r_empty + 1;
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(d2_done + 1);
    double *sf = reinterpret_cast<double *>(smem + L.sf_off);
    __shared__ int s_abort;

    const int tid = threadIdx.x;
    const int warp = tid >> 5;
    const int lane = tid & 31;
    const int grid = gridDim.x;
    const int b = blockIdx.x;
    const int64_t ntiles_all = (p.N + kTcRows - 1) / kTcRows;
    const int nt = (int)(ntiles_all > b ? (ntiles_all - b + grid - 1) / grid : 0);

    if (tid == 0) {
        for (int s = 0; s < kTcMaxStages; ++s) {
            ptx::mbar_init(&x_full[s], 1);
            ptx::mbar_init(&x_empty[s], 1);
        }
        ptx::mbar_init(d1_full, 1);
        ptx::mbar_init(d1_empty, kTcEpiWarps);
        ptx::mbar_init(r_full, kTcEpiWarps);
        ptx::mbar_init(r_empty, 1);
        ptx::mbar_init(d2_done, 1);
        ptx::fence_mbar_init();
        s_abort = 0;
        asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&tmap)) : "memory");
    }
    if (warp == 1) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                         ptx::smem_u32(tmem_slot)),
                     "r"(kTcTmemCols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    ptx::grid_dep_wait();
    tc::fence_before();
    __syncthreads();
    tc::fence_after();
    const uint32_t tmem = *tmem_slot;

    // beta into tensor memory, two columns of beta per 32-bit cell. Lanes go
    // in groups of 16: in lane quarter q, group g holds vectors
    // k = 16q + 8g + v (v = 0..7), the hi term of beta_k in lane 16g + v and
    // the lo term eight lanes further. A 16x256b tensor-memory load then gives
    // each epilogue thread both partial sums of one (row, vector) pair, so
    // they add in registers with no exchange between lanes.
    constexpr int EPI0 = 2;                         // first epilogue warp
    // All 16 epilogue warps fill it: warp (q, hh) writes the 32-column blocks
    // cb = 32 hh, 32 (hh + 4), ... of lane quarter q, so each thread has one
    // batch of loads in flight (a thread's 64 columns are contiguous: 16-byte
    // loads when the rows allow them).
    if (warp >= EPI0) {
        const int q = warp & 3;
        const int hh = (warp - EPI0) >> 2;
        const int k = 16 * q + 8 * (lane >> 4) + (lane & 7);
        const int part = (lane >> 3) & 1;
        const bool kin = k < p.kk;
        const float *brow = p.beta + (size_t)(kin ? k : 0) * p.P;
        const bool vec = kin && (p.P & 3) == 0 && (reinterpret_cast<uintptr_t>(p.beta) & 15u) == 0;
        for (int cb = 32 * hh; cb < PA * 32; cb += 32 * kTcEpiGroups) {
            float v[64];
            if (vec) {
#pragma unroll
                for (int u = 0; u < 16; ++u) {
                    const int col = 2 * cb + 4 * u;
                    float4 t = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
                    if (col < p.P)
                        t = __ldg(reinterpret_cast<const float4 *>(brow + col));
                    v[4 * u] = t.x;
                    v[4 * u + 1] = t.y;
                    v[4 * u + 2] = t.z;
                    v[4 * u + 3] = t.w;
                }
            } else {
#pragma unroll
                for (int e = 0; e < 64; ++e) {
                    const int col = 2 * cb + e;
                    v[e] = (kin && col < p.P) ? __ldg(brow + col) : 0.0f;
                }
            }
            uint32_t r[32];
#pragma unroll
            for (int j = 0; j < 32; ++j) {
                float h0, l0, h1, l1;
                tc::split2(v[2 * j], h0, l0);
                tc::split2(v[2 * j + 1], h1, l1);
                r[j] = part ? tc::pack_bf16(l0, l1) : tc::pack_bf16(h0, h1);
            }
            tc::tmem_st32(tmem + ((uint32_t)(q * 32) << 16) + kTcB1Col + cb, r);
        }
        tc::tmem_wait_st();
    }
    tc::fence_before();
    __syncthreads();
    tc::fence_after();
    ptx::grid_dep_launch_dependents();
    if (warp < 2) {
      if (warp == 0) {
        // ---- TMA producer ------------------------------------------------------------
        if (lane == 0) {
            const unsigned bytes = (unsigned)(PA * 16384);
            for (int i = 0; i < nt; ++i) {
                const int s = i % stages;
                const int use = i / stages;
                if (use > 0 && !ptx::mbar_wait_bounded(&x_empty[s], (unsigned)(use - 1) & 1u, kSpinLimit)) {
                    atomicOr(p.status, kDevTimeout);
                    s_abort = 1;
                    break;
                }
                const int row0 = (int)((int64_t)(b + (int64_t)i * grid) * kTcRows);
                ptx::mbar_arrive_expect_tx(&x_full[s], bytes);
                for (int a = 0; a < PA; ++a)
                    tc::tma_load_2d(xs + s * L.x_stage + a * 16384, &tmap, a * 64, row0, &x_full[s]);
            }
        }
      } else if (warp == 1) {
        // ---- MMA issuer ----------------------------------------------------------------
        if (lane == 0) {
            // descriptors are built once and stepped by adding the address
            // offset / 16 (the low 14-bit field; shared addresses stay below
            // 256 KB, so no carry): one thread issues every MMA, and its
            // per-MMA work bounds the issue rate
            const uint64_t bk0 = tc::mdesc(ptx::smem_u32(xs), 16, 1024);       // X, K-major
            const uint64_t xm0 = tc::mdesc(ptx::smem_u32(xs), 16384, 1024);    // X, MN-major
            const uint64_t rt0 = tc::mdesc(ptx::smem_u32(rb), 16, 1024);       // R^t, K-major
            const uint64_t stage_step = (uint64_t)(L.x_stage >> 4);
            bool ok = true;
            for (int i = 0; i <= nt && ok; ++i) {
                if (i < nt) {
                    const int s = i % stages;
                    ok = ptx::mbar_wait_bounded(&x_full[s], (unsigned)(i / stages) & 1u, kSpinLimit);
                    if (ok && i >= 1)
                        ok = ptx::mbar_wait_bounded(d1_empty, (unsigned)(i - 1) & 1u, kSpinLimit);
                    if (!ok)
                        break;
                    tc::fence_after();
                    const uint64_t bks = bk0 + (uint64_t)s * stage_step;
                    for (int a = 0; a < PA; ++a) {
                        const uint64_t bda = bks + (uint64_t)(a * (16384 >> 4));
                        const uint32_t aa = tmem + kTcB1Col + a * 32;
#pragma unroll
                        for (int sub = 0; sub < 4; ++sub)     // 16 columns: 32 bytes, 8 cells
                            tc::mma_ta(tmem + kTcD1Col, aa + 8 * sub, bda + 2 * sub, ID1,
                                       (a | sub) ? 1u : 0u);
                    }
                    tc::commit(d1_full);
                }
                if (i >= 1) {
                    const int j = i - 1;
                    const int sj = j % stages;
                    ok = ptx::mbar_wait_bounded(r_full, (unsigned)j & 1u, kSpinLimit);
                    if (!ok)
                        break;
                    tc::fence_after();
                    // D2^t[(vector, term) x P] += R^t . X over the tile's rows,
                    // 16 rows per MMA (R^t atom ks / 4, 32 bytes per step;
                    // X rows 16 ks: 2 KB per step)
                    const uint64_t xb = xm0 + (uint64_t)sj * stage_step;
#pragma unroll
                    for (int ks = 0; ks < kTcRows / 16; ++ks)
                        tc::mma(tmem + kTcD2Col,
                                rt0 + (uint64_t)((ks >> 2) * (16384 >> 4) + (ks & 3) * 2),
                                xb + (uint64_t)(ks * 128), ID2, (j > 0 || ks > 0) ? 1u : 0u);
                    tc::commit(&x_empty[sj]);
                    tc::commit(r_empty);
                }
            }
            if (!ok) {
                atomicOr(p.status, kDevTimeout);
                s_abort = 1;
            }
            if (nt > 0)
                tc::commit(d2_done);
        }
      }
    } else {
        // ---- epilogue ---------------------------------------------------------------------
        // Warp (q, hh): lane quarter q (vectors 16q .. 16q + 15) and tile rows
        // CW hh .. CW hh + 31. Thread (tq, tr) = (lane / 4, lane % 4) takes the
        // vectors k = 16q + tq and k + 8 on the rows CW hh + 8m + 2tr + j
        // (m = 0..3, j = 0, 1): 16 (row, vector) pairs per tile, each read as
        // its hi and lo partial sums by two 16x256b loads.
        constexpr int CW = kTcEpiCols;
        const int q = warp & 3;
        const int hh = (warp - EPI0) >> 2;
        const int tq = lane >> 2;
        const int tr = lane & 3;
        const int kq = 16 * q + tq;
        const int row_t = CW * hh + 2 * tr;     // this thread's first row in the tile
        // the label of row row_t + 8m + j is byte 2(tr & 1) + j of word m below;
        // shifted so that its low bit is the sign bit
        const uint32_t sh0 = 31u - 16u * (uint32_t)(tr & 1);
        const uint32_t sh1 = sh0 - 8u;
        // R^t tile stores (the A operand of MMA2, K-major: each (vector, term)
        // lane n holds its 128 rows contiguous, two 64-row atoms of 128 B
        // rows with the 128B swizzle of 16-byte chunks by n & 7 = tq). The
        // thread's rows row_t + 8m + {0, 1} of vector 16q + 8g + tq are one
        // word per term, in lane n = 32q + 16g + 8 term + tq: chunk
        // (4 (hh & 1) + m) ^ tq, word tr. Conflict-free across the warp.
        const uint32_t rt_base = (uint32_t)((hh >> 1) * 16384 + (32 * q + tq) * 128 + 4 * tr);
        float facc0 = 0.0f, facc1 = 0.0f;
        uint32_t yw[4], yn[4];
        auto load_y = [&](int i, uint32_t *dst) {
#pragma unroll
            for (int m = 0; m < 4; ++m)
                dst[m] = 0u;
            if (i >= nt)
                return;
            const int64_t t0 = (int64_t)(b + (int64_t)i * grid) * kTcRows;
            const int64_t r0 = t0 + CW * hh + 4 * (tr >> 1);     // word m: rows r0 + 8m ..
            if (p.y_al4 && t0 + kTcRows <= p.N) {
                const uint32_t *yp = reinterpret_cast<const uint32_t *>(p.y + r0);
#pragma unroll
                for (int m = 0; m < 4; ++m)
                    dst[m] = __ldg(yp + 2 * m);
            } else {
                for (int m = 0; m < 4; ++m)
                    for (int c = 0; c < 4; ++c)
                        if (r0 + 8 * m + c < p.N)
                            dst[m] |= (uint32_t)__ldg(p.y + r0 + 8 * m + c) << (8 * c);
            }
        };
        load_y(0, yw);
        bool ok = true;
        for (int i = 0; i < nt; ++i) {
            load_y(i + 1, yn);
            if (!ptx::mbar_wait_bounded(d1_full, (unsigned)i & 1u, kSpinLimit)) {
                ok = false;
                break;
            }
            tc::fence_after();
            float v0[16], v1[16];
            const uint32_t ta = tmem + ((uint32_t)(q * 32) << 16) + kTcD1Col + CW * hh;
            tc::tmem_ld16x256_x4(ta, v0);
            tc::tmem_ld16x256_x4(ta + (16u << 16), v1);
            tc::tmem_wait_ld();
            tc::fence_before();
            __syncwarp();
            if (lane == 0)
                ptx::mbar_arrive(d1_empty);
            const int64_t left = p.N - (int64_t)(b + (int64_t)i * grid) * kTcRows;
            uint32_t wh[2][4], wl[2][4];        // hi and lo terms of rows (2j pair) per (g, m)
            if (left >= kTcRows) {
#pragma unroll
                for (int m = 0; m < 4; ++m) {
                    const uint32_t y0 = yw[m] << sh0, y1 = yw[m] << sh1;
                    const float a0 = tc::tr_r(v0[4 * m] + v0[4 * m + 2], y0, facc0);
                    const float a1 = tc::tr_r(v0[4 * m + 1] + v0[4 * m + 3], y1, facc0);
                    const float b0 = tc::tr_r(v1[4 * m] + v1[4 * m + 2], y0, facc1);
                    const float b1 = tc::tr_r(v1[4 * m + 1] + v1[4 * m + 3], y1, facc1);
                    tc::split_pair(a0, a1, wh[0][m], wl[0][m]);
                    tc::split_pair(b0, b1, wh[1][m], wl[1][m]);
                }
            } else {
#pragma unroll
                for (int m = 0; m < 4; ++m) {
                    const uint32_t y0 = yw[m] << sh0, y1 = yw[m] << sh1;
                    const bool in0 = row_t + 8 * m < left, in1 = row_t + 8 * m + 1 < left;
                    float f00 = 0.0f, f01 = 0.0f, f10 = 0.0f, f11 = 0.0f;
                    float a0 = tc::tr_r(v0[4 * m] + v0[4 * m + 2], y0, f00);
                    float a1 = tc::tr_r(v0[4 * m + 1] + v0[4 * m + 3], y1, f01);
                    float b0 = tc::tr_r(v1[4 * m] + v1[4 * m + 2], y0, f10);
                    float b1 = tc::tr_r(v1[4 * m + 1] + v1[4 * m + 3], y1, f11);
                    a0 = in0 ? a0 : 0.0f;
                    b0 = in0 ? b0 : 0.0f;
                    a1 = in1 ? a1 : 0.0f;
                    b1 = in1 ? b1 : 0.0f;
                    facc0 += (in0 ? f00 : 0.0f) + (in1 ? f01 : 0.0f);
                    facc1 += (in0 ? f10 : 0.0f) + (in1 ? f11 : 0.0f);
                    tc::split_pair(a0, a1, wh[0][m], wl[0][m]);
                    tc::split_pair(b0, b1, wh[1][m], wl[1][m]);
                }
            }
            if (i >= 1 && !ptx::mbar_wait_bounded(r_empty, (unsigned)(i - 1) & 1u, kSpinLimit)) {
                ok = false;
                break;
            }
#pragma unroll
            for (int m = 0; m < 4; ++m) {
                const uint32_t sw = ((uint32_t)((4 * (hh & 1) + m) ^ tq)) << 4;
#pragma unroll
                for (int g = 0; g < 2; ++g) {
                    uint8_t *dst = rb + rt_base + (uint32_t)(16 * g * 128) + sw;
                    *reinterpret_cast<uint32_t *>(dst) = wh[g][m];              // term hi: lane + 0
                    *reinterpret_cast<uint32_t *>(dst + 8 * 128) = wl[g][m];    // term lo: lane + 8
                }
            }
            ptx::fence_proxy_async_smem();
            __syncwarp();
            if (lane == 0)
                ptx::mbar_arrive(r_full);
#pragma unroll
            for (int m = 0; m < 4; ++m)
                yw[m] = yn[m];
        }
        if (!ok) {
            atomicOr(p.status, kDevTimeout);
            s_abort = 1;
        }
        const int PP = MB * 128;
        const bool have = nt > 0 && ok && ptx::mbar_wait_bounded(d2_done, 0u, kSpinLimit);
        if (nt > 0 && !have) {
            atomicOr(p.status, kDevTimeout);
            s_abort = 1;
        }
        tc::fence_after();
        // g partial: D2^t lanes as beta's (hi of vector 16q + 8g + v in lane
        // 16g + v of quarter q, lo eight lanes further), columns = columns of
        // X; warp hh takes the 32-column chunks c = hh, hh + 4, and a
        // 16x256b load gives each thread both terms of its (vector, column)
        // pairs
        const int ncol = PA * 64;
        for (int c = hh; 32 * c < ncol; c += kTcEpiGroups) {
            float ga[16], gb[16];
            if (have) {
                const uint32_t tg = tmem + ((uint32_t)(q * 32) << 16) + kTcD2Col + 32 * c;
                tc::tmem_ld16x256_x4(tg, ga);
                tc::tmem_ld16x256_x4(tg + (16u << 16), gb);
                tc::tmem_wait_ld();
            }
#pragma unroll
            for (int g = 0; g < 2; ++g) {
                const int kv = kq + 8 * g;
                if (kv >= p.kk)
                    continue;
                const float *v = g ? gb : ga;
                float *dst = p.part_g + ((size_t)b * 64 + kv) * PP + 32 * c + 2 * tr;
#pragma unroll
                for (int i2 = 0; i2 < 4; ++i2) {
                    float2 o;
                    o.x = have ? v[4 * i2] + v[4 * i2 + 2] : 0.0f;
                    o.y = have ? v[4 * i2 + 1] + v[4 * i2 + 3] : 0.0f;
                    *reinterpret_cast<float2 *>(dst + 8 * i2) = o;
                }
            }
        }
        // f partial: the four lanes of a vector, then the row groups in order
        double f0 = (double)facc0, f1 = (double)facc1;
        f0 += __shfl_xor_sync(0xFFFFFFFFu, f0, 1);
        f1 += __shfl_xor_sync(0xFFFFFFFFu, f1, 1);
        f0 += __shfl_xor_sync(0xFFFFFFFFu, f0, 2);
        f1 += __shfl_xor_sync(0xFFFFFFFFu, f1, 2);
        asm volatile("bar.sync 1, %0;" ::"r"(kTcEpiWarps * 32) : "memory");
        if (tr == 0) {
            sf[hh * 64 + kq] = f0;
            sf[hh * 64 + kq + 8] = f1;
        }
        asm volatile("bar.sync 1, %0;" ::"r"(kTcEpiWarps * 32) : "memory");
        const int et = tid - 32 * EPI0;
        if (et < p.kk) {
            double tot = 0.0;
            for (int g2 = 0; g2 < kTcEpiGroups; ++g2)
                tot += sf[g2 * 64 + et];
            p.part_f[(size_t)b * 64 + et] = s_abort ? __longlong_as_double(0x7FF8000000000000LL) : tot;
        }
    }
    tc::fence_before();
    __syncthreads();
    tc::fence_after();
    if (warp == 1)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                     "r"(kTcTmemCols)
                     : "memory");
}

// Fixed-order combine of the per-CTA partials, plus the Gaussian prior.
// The first nf blocks take f: one warp per vector, lanes over CTAs (FP64)
// and over columns of beta (FP32), finished by a butterfly. The other blocks
// take g: a block takes 128 consecutive columns of one vector, lane l
// columns 4l .. 4l + 3 (16-byte loads; the partial rows are padded to a
// multiple of 128 columns), its 8 warps each add a contiguous range of CTAs
// with all loads of the range in flight, then warp 0 adds the 8 range sums in
// order. FP32 sums: FP64 throughput is low on this part, and the partials
// are FP32 tensor-memory sums already.
constexpr int kTcRedWarps = 8;

__global__ void __launch_bounds__(32 * kTcRedWarps)
    tc_reduce_kernel(const double *__restrict__ part_f, const float *__restrict__ part_g, int parts,
                     int KB, int PP, int P, int kk, int nf, const float *__restrict__ beta,
                     const float *__restrict__ x_scale, double inv_s2, double prior_const,
                     double *__restrict__ f_out, float *__restrict__ g_out)
{
    ptx::grid_dep_wait();
    const int warp = threadIdx.x >> 5;
    const int lane = threadIdx.x & 31;
    if ((int)blockIdx.x < nf) {
        const int k = (int)blockIdx.x * kTcRedWarps + warp;
        if (k >= kk)
            return;
        double v = 0.0;
        for (int c = lane; c < parts; c += 32)
            v += part_f[(size_t)c * KB + k];
        float bb = 0.0f;
        for (int t = lane; t < P; t += 32) {
            const float bt = beta[(size_t)k * P + t];
            bb = fmaf(bt, bt, bb);
        }
#pragma unroll
        for (int m = 16; m > 0; m >>= 1) {
            v += __shfl_xor_sync(0xFFFFFFFFu, v, m);
            bb += __shfl_xor_sync(0xFFFFFFFFu, bb, m);
        }
        if (lane == 0)
            f_out[k] = v - 0.5 * inv_s2 * (double)bb - prior_const;
        return;
    }
    __shared__ float4 part_sum[kTcRedWarps][32];
    const int gblk = (int)blockIdx.x - nf;
    const int cpk = (P + 127) / 128;                   // column blocks per vector
    const int k = gblk / cpk;
    const int jj = (gblk - k * cpk) * 128 + 4 * lane;
    const int per = (parts + kTcRedWarps - 1) / kTcRedWarps;
    const int c0 = warp * per;
    const int c1 = (c0 + per) < parts ? (c0 + per) : parts;
    float4 v = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
    if (jj < P) {
        const float *src = part_g + (size_t)k * PP + jj;
        const size_t stride = (size_t)KB * PP;
        for (int cb = c0; cb < c1; cb += 16) {
            float4 buf[16];
#pragma unroll
            for (int u = 0; u < 16; ++u)
                buf[u] = (cb + u < c1) ? __ldg(reinterpret_cast<const float4 *>(src + (size_t)(cb + u) * stride))
                                       : make_float4(0.0f, 0.0f, 0.0f, 0.0f);
#pragma unroll
            for (int u = 0; u < 16; ++u) {
                v.x += buf[u].x;
                v.y += buf[u].y;
                v.z += buf[u].z;
                v.w += buf[u].w;
            }
        }
    }
    part_sum[warp][lane] = v;
    __syncthreads();
    if (warp != 0 || jj >= P)
        return;
    float t[4] = {0.0f, 0.0f, 0.0f, 0.0f};
#pragma unroll
    for (int w = 0; w < kTcRedWarps; ++w) {
        const float4 q = part_sum[w][lane];
        t[0] += q.x;
        t[1] += q.y;
        t[2] += q.z;
        t[3] += q.w;
    }
#pragma unroll
    for (int e = 0; e < 4; ++e) {
        const int col = jj + e;
        if (col < P) {
            const float sc = x_scale ? x_scale[col] : 1.0f;
            g_out[(size_t)k * P + col] = fmaf(sc, t[e], -beta[(size_t)k * P + col] * (float)inv_s2);
        }
    }
}

// ---------------------------------------------------------------------------

bool tc_supported(const glm_ctx *h)
{
    return (h->d.xtype == GLM_X_BF16 || h->d.xtype == GLM_X_FP8E4M3) && h->d.p <= kTcMaxP &&
           h->d.k_max >= 16;
}

// Operand-tile stages that fit (4 down to 2). Returns false if nothing fits.
static bool tc_stages(int PA, int *stages)
{
    for (int st = kTcMaxStages; st >= 2; --st) {
        if (tc_layout(PA, st).total <= kSmemDynamicBudget) {
            *stages = st;
            return true;
        }
    }
    return false;
}

// BF16: 64-column boxes with the 128B swizzle, loaded straight into the MMA
// layout.
static glm_status_t tc_tensor_map(glm_ctx *h, const void *X)
{
    if (h->tc_map_ptr == X)
        return GLM_OK;
    PFN_cuTensorMapEncodeTiled_v12000 encode = tensor_map_encoder();
    if (!encode)
        return GLM_ERR_CUDA;
    CUtensorMap *map = reinterpret_cast<CUtensorMap *>(h->tc_map);
    const cuuint32_t estr[2] = {1, 1};
    CUresult r;
    const cuuint64_t dims[2] = {(cuuint64_t)h->d.ld, (cuuint64_t)h->d.n_rows};
    const cuuint64_t strides[1] = {(cuuint64_t)h->d.ld * 2};
    const cuuint32_t box[2] = {64, (cuuint32_t)kTcRows};
    r = encode(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void *>(X), dims, strides,
               box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
               CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS)
        return GLM_ERR_CUDA;
    h->tc_map_ptr = X;
    return GLM_OK;
}

size_t tc_workspace_bytes(const glm_ctx *h)
{
    const int MB = (h->d.p + 127) / 128;
    return (size_t)h->sm_count * kTcMaxKB * 8 + (size_t)h->sm_count * kTcMaxKB * MB * 128 * 4 + 256;
}

glm_status_t launch_tc8(glm_ctx *h, const void *X, const float *x_scale, const uint8_t *y,
                        const float *beta, int K, double *f_out, float *g_out, cudaStream_t s);

glm_status_t launch_tc(glm_ctx *h, const void *X, const float *x_scale, const uint8_t *y,
                       const float *beta, int K, double *f_out, float *g_out, cudaStream_t s)
{
    if (h->d.xtype == GLM_X_FP8E4M3)
        return launch_tc8(h, X, x_scale, y, beta, K, f_out, g_out, s);
    if (!h->tc_part_f || h->d.n_rows > ((int64_t)1 << 31) - kTcRows)
        return GLM_ERR_UNSUPPORTED;
    glm_status_t st = tc_tensor_map(h, X);
    if (st != GLM_OK)
        return st;
    const int P = h->d.p;
    const int PA = (P + 63) / 64;
    const int MB = (P + 127) / 128;
    const double s2 = h->d.prior_sigma * h->d.prior_sigma;
    const bool prior = !(h->d.flags & GLM_FLAG_NO_PRIOR);
    const CUtensorMap *map = reinterpret_cast<const CUtensorMap *>(h->tc_map);
    int stages = 0;
    if (!tc_stages(PA, &stages))
        return GLM_ERR_UNSUPPORTED;
    for (int k0 = 0; k0 < K; k0 += kTcMaxKB) {
        const int kk = (K - k0) < kTcMaxKB ? (K - k0) : kTcMaxKB;
        const int KB = kTcMaxKB;
        TcParams prm;
        std::memset(&prm, 0, sizeof(prm));
        prm.y = y;
        prm.y_al4 = (reinterpret_cast<uintptr_t>(y) & 3u) == 0 ? 1 : 0;
        prm.beta = beta + (size_t)k0 * P;
        prm.N = h->d.n_rows;
        prm.P = P;
        prm.kk = kk;
        prm.PA = PA;
        prm.MB = MB;
        prm.stages = stages;
        prm.part_f = h->tc_part_f;
        prm.part_g = h->tc_part_g;
        prm.status = h->status;
        auto fn = &tc_logpost_grad_kernel;
        const TcLayout L = tc_layout(PA, prm.stages);
        if (allow_max_dynamic_smem(reinterpret_cast<const void *>(fn)) != cudaSuccess)
            return GLM_ERR_CUDA;
        cudaLaunchConfig_t cfg = {};
        cfg.gridDim = dim3((unsigned)h->sm_count);
        cfg.blockDim = dim3(kTcThreads);
        cfg.dynamicSmemBytes = (size_t)L.total;
        cfg.stream = s;
        cudaLaunchAttribute attr[1];
        attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
        attr[0].val.programmaticStreamSerializationAllowed = 1;
        cfg.attrs = attr;
        cfg.numAttrs = 1;
        if (cudaLaunchKernelEx(&cfg, fn, *map, prm) != cudaSuccess)
            return GLM_ERR_CUDA;
        const int ng = kk * ((P + 127) / 128);
        const int nf = (kk + kTcRedWarps - 1) / kTcRedWarps;
        cudaLaunchConfig_t rc = {};
        rc.gridDim = dim3((unsigned)(ng + nf));
        rc.blockDim = dim3(32 * kTcRedWarps);
        rc.stream = s;
        rc.attrs = attr;
        rc.numAttrs = 1;
        if (cudaLaunchKernelEx(&rc, tc_reduce_kernel, (const double *)h->tc_part_f,
                               (const float *)h->tc_part_g, h->sm_count, KB, MB * 128, P, kk, nf,
                               beta + (size_t)k0 * P, x_scale, prior ? 1.0 / s2 : 0.0,
                               prior ? 0.5 * (double)P * std::log(2.0 * M_PI * s2) : 0.0, f_out + k0,
                               g_out + (size_t)k0 * P) != cudaSuccess)
            return GLM_ERR_CUDA;
    }
    return GLM_OK;
}

}  // namespace glm
