// Log-posterior, gradient and Hessian of Bayesian logistic regression in one
// pass over X (the §4.2 derivatives taken one order further, as §5.2
// proposes for Newton-type and Riemannian samplers):
//   f = sum_n [y_n eta_n - log(1 + e^eta_n)] + log N(beta | 0, s^2 I)
//   g = X^T (y - mu) - beta / s^2
//   H = -X^T diag(w) X - I / s^2,   mu = 1 / (1 + e^-eta),  w = mu (1 - mu)
// for one coefficient vector, P <= 64, X FP32 row-major.
//
// X^T diag(w) X is a P x P x N contraction and runs on the tcgen05 tensor
// cores. One persistent CTA per SM streams 128-row tiles of X into shared
// memory with TMA (128-byte swizzle, a two-tile ring). Eight converter warps (thread = one row and 32
// columns) form eta (a partial dot product per half row, exchanged through
// shared memory), w, r = y - mu and the log-likelihood term, add r x_n to
// their gradient registers, and write two BF16 operand tiles split into
// hi + lo terms (hi = bf16(v), lo = bf16(v - hi), about 16 significant bits):
//   A = [ (w x)_hi | (w x)_lo ],  B = [ x_hi | x_lo ]   (128 rows x 128 columns)
// One thread issues D[128 x 128] += A^T B (kind::f16, both operands MN-major,
// K = 16 rows per MMA); D stays in tensor memory for the CTA's whole run and
// X^T W X = D00 + D01 + D10 + D11 (its four 64 x 64 blocks). The operand tiles
// are double-buffered so that the converters fill one while the MMAs read the
// other. At the end each CTA writes its f, g and 64 x 64 partials and a second
// kernel adds them in a fixed order (deterministic), adds the prior and writes
// the upper triangle mirrored (H exactly symmetric). Every wait is bounded.
#include <cmath>
#include <cstring>
#include <new>

#include "glm_internal.cuh"
#include "glm_tc_common.cuh"

struct glm_hess {
    int64_t n_rows;
    int p, ld, device, sm_count, grid;
    double prior_sigma;
    void *ws;
    double *part_f;            // grid
    float *part_g;             // grid x 64
    float *part_h;             // grid x 64 x 64
    unsigned *status;
    alignas(64) unsigned char map[128];   // CUtensorMap of the last X seen
    const void *map_ptr;
};

namespace glm {

constexpr int kHRows = 128;                 // rows per tile
constexpr int kHMaxP = 64;
constexpr int kHConv = 8;                   // converter warps
constexpr int kHThreads = 32 * (2 + kHConv);
constexpr int kHStages = 2;                 // X ring (32 KB tiles)
constexpr int kHXTile = kHRows * kHMaxP * 4;
constexpr int kHAtom = kHRows * 128;        // one 128-byte-wide operand atom (64 bf16)
constexpr int kHOpBuf = 4 * kHAtom;         // A (two atoms) and B (two atoms)
constexpr int kHTmemCols = 128;

struct HessLayout {
    int x_off, ab_off, ep_off, bar_off, total;
};

__host__ __device__ inline HessLayout hess_layout()
{
    HessLayout L;
    L.x_off = 0;
    L.ab_off = kHStages * kHXTile;
    L.ep_off = L.ab_off + 2 * kHOpBuf;                  // eta halves: [2][2][128] floats
    L.bar_off = L.ep_off + 2 * 2 * kHRows * 4;
    L.total = L.bar_off + 256 + 256 + 1024;             // barriers, f sums, alignment
    return L;
}

struct HessParams {
    const uint8_t *y;
    const float *beta;
    int64_t N;
    int P;
    double *part_f;
    float *part_g;
    float *part_h;
    unsigned *status;
};

// v as bf16 hi + lo terms, two values at a time: bf16x2 words of (a0, a1).
__device__ __forceinline__ void split_bf16x2(float a0, float a1, uint32_t &hi, uint32_t &lo)
{
    asm("cvt.rn.bf16x2.f32 %0, %1, %2;" : "=r"(hi) : "f"(a1), "f"(a0));
    const float h0 = __uint_as_float(hi << 16);
    const float h1 = __uint_as_float(hi & 0xFFFF0000u);
    asm("cvt.rn.bf16x2.f32 %0, %1, %2;" : "=r"(lo) : "f"(a1 - h1), "f"(a0 - h0));
}

__global__ void __launch_bounds__(kHThreads, 1)
    hess_tc_kernel(const __grid_constant__ CUtensorMap tmap, HessParams p)
{
    constexpr uint32_t IDH = tc::idesc_make(kHRows, 128, 1, 1, 1, 1);   // bf16, both MN-major

    extern __shared__ uint8_t smem_raw[];
    uint8_t *smem = smem_raw + ((1024u - (ptx::smem_u32(smem_raw) & 1023u)) & 1023u);
    const HessLayout L = hess_layout();
    uint8_t *xs = smem + L.x_off;
    uint8_t *ab = smem + L.ab_off;
    float *ep = reinterpret_cast<float *>(smem + L.ep_off);
    uint64_t *bars = reinterpret_cast<uint64_t *>(smem + L.bar_off);
    uint64_t *x_full = bars;                    // [2]
    uint64_t *x_empty = bars + 2;               // [2]
    uint64_t *ab_full = bars + 4;               // [2]
    uint64_t *ab_empty = bars + 6;              // [2]
    uint64_t *d_done = bars + 8;
    uint64_t *ep_bar = bars + 9;                // [2] eta halves written, by tile parity
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(bars + 11);
    float *sfq = reinterpret_cast<float *>(smem + L.bar_off + 256);   // [4] f per row quarter
    __shared__ int s_abort;

    const int tid = threadIdx.x;
    const int warp = tid >> 5;
    const int lane = tid & 31;
    const int grid = gridDim.x;
    const int b = blockIdx.x;
    const int64_t ntiles_all = (p.N + kHRows - 1) / kHRows;
    const int nt = (int)(ntiles_all > b ? (ntiles_all - b + grid - 1) / grid : 0);

    if (tid == 0) {
        for (int s = 0; s < 2; ++s) {
            ptx::mbar_init(&x_full[s], 1);
            ptx::mbar_init(&x_empty[s], kHConv);
            ptx::mbar_init(&ab_full[s], kHConv);
            ptx::mbar_init(&ab_empty[s], 1);
        }
        ptx::mbar_init(d_done, 1);
        ptx::mbar_init(&ep_bar[0], kHConv);
        ptx::mbar_init(&ep_bar[1], kHConv);
        ptx::fence_mbar_init();
        s_abort = 0;
        if (p.N > 0)        // with no rows the tensor map is not encoded and never used
            asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&tmap)) : "memory");
    }
    if (warp == 1) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                         ptx::smem_u32(tmem_slot)),
                     "r"(kHTmemCols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    ptx::grid_dep_wait();
    tc::fence_before();
    __syncthreads();
    tc::fence_after();
    const uint32_t tmem = *tmem_slot;
    ptx::grid_dep_launch_dependents();

    if (warp == 0) {
        // ---- TMA producer (lane 0) ---------------------------------------------------------
        // (Prefetching the tiles beyond the ring into L2 from this warp's
        // lanes was measured 1 % slower.)
        if (lane == 0) {
            for (int i = 0; i < nt; ++i) {
                const int s = i % kHStages;
                const int use = i / kHStages;
                if (use > 0 && !ptx::mbar_wait_bounded(&x_empty[s], (unsigned)(use - 1) & 1u, kSpinLimit)) {
                    atomicOr(p.status, kDevTimeout);
                    s_abort = 1;
                    break;
                }
                const int row0 = (int)((int64_t)(b + (int64_t)i * grid) * kHRows);
                ptx::mbar_arrive_expect_tx(&x_full[s], (unsigned)kHXTile);
                tc::tma_load_2d(xs + s * kHXTile, &tmap, 0, row0, &x_full[s]);
                tc::tma_load_2d(xs + s * kHXTile + kHAtom, &tmap, 32, row0, &x_full[s]);
            }
        }
    } else if (warp == 1) {
        // ---- MMA issuer: D += A^T B over the tile's 128 rows, 16 per MMA ----------------
        if (lane == 0) {
            const uint32_t ab0 = ptx::smem_u32(ab);
            const uint64_t dA = tc::mdesc(ab0, kHAtom, 1024);                 // [wx_hi | wx_lo]
            const uint64_t dB = tc::mdesc(ab0 + 2 * kHAtom, kHAtom, 1024);    // [x_hi | x_lo]
            bool ok = true;
            for (int i = 0; i < nt && ok; ++i) {
                const int s = i & 1;
                ok = ptx::mbar_wait_bounded(&ab_full[s], (unsigned)(i >> 1) & 1u, kSpinLimit);
                if (!ok)
                    break;
                tc::fence_after();
                const uint64_t step = (uint64_t)((s * kHOpBuf) >> 4);
#pragma unroll
                for (int ks = 0; ks < kHRows / 16; ++ks)      // 16 rows = 2 KB of each atom
                    tc::mma(tmem, dA + step + (uint64_t)(ks * 128), dB + step + (uint64_t)(ks * 128),
                            IDH, (i > 0 || ks > 0) ? 1u : 0u);
                tc::commit(&ab_empty[s]);
            }
            if (!ok) {
                atomicOr(p.status, kDevTimeout);
                s_abort = 1;
            }
            if (nt > 0)
                tc::commit(d_done);
        }
    } else {
        // ---- converters: thread = one row of each tile and 32 of its columns ---------------
        constexpr float kLog2e = 1.4426950408889634f;
        constexpr float kLn2 = 0.69314718055994531f;
        const int e = warp - 2;                     // 0 .. 7
        const int et = tid - 64;
        const int rq = e & 3;                       // tile rows 32 rq .. 32 rq + 31
        const int hf = e >> 2;                      // columns 32 hf .. 32 hf + 31
        const int r = rq * 32 + lane;
        float bt[32], gacc[32];
#pragma unroll
        for (int j = 0; j < 32; ++j) {
            const int col = 32 * hf + j;
            bt[j] = col < p.P ? __ldg(p.beta + col) : 0.0f;
            gacc[j] = 0.0f;
        }
        float facc = 0.0f;
        bool ok = true;
        // labels one tile ahead
        auto label = [&](int i) -> int {
            const int64_t rw = (int64_t)(b + (int64_t)i * grid) * kHRows + r;
            return (i < nt && rw < p.N) ? (int)__ldg(p.y + rw) : 0;
        };
        int ynext = label(0);
        for (int i = 0; i < nt; ++i) {
            const int s = i % kHStages;
            const int64_t row = (int64_t)(b + (int64_t)i * grid) * kHRows + r;
            const bool valid = row < p.N;
            const int yl = ynext;
            ynext = label(i + 1);
            if (!ptx::mbar_wait_bounded(&x_full[s], (unsigned)(i / kHStages) & 1u, kSpinLimit)) {
                ok = false;
                break;
            }
            // the row's 32 columns: 16-byte chunks permuted by row & 7 (TMA swizzle);
            // rows past N arrive as zeros
            const uint8_t *xrow = xs + s * kHXTile + hf * kHAtom + r * 128;
            float x[32];
#pragma unroll
            for (int c = 0; c < 8; ++c) {
                const float4 v = *reinterpret_cast<const float4 *>(xrow + ((c ^ (r & 7)) << 4));
                x[4 * c] = v.x;
                x[4 * c + 1] = v.y;
                x[4 * c + 2] = v.z;
                x[4 * c + 3] = v.w;
            }
            if (32 * hf + 32 > p.P) {               // padding columns (any value) count as 0
#pragma unroll
                for (int j = 0; j < 32; ++j)
                    x[j] = 32 * hf + j < p.P ? x[j] : 0.0f;
            }
            // four independent chains (a shorter dependency than one of 32)
            float pc[4] = {0.0f, 0.0f, 0.0f, 0.0f};
#pragma unroll
            for (int j = 0; j < 32; ++j)
                pc[j & 3] = fmaf(x[j], bt[j], pc[j & 3]);
            const float part = (pc[0] + pc[1]) + (pc[2] + pc[3]);
            // exchange the half-row sums (buffer and barrier by tile parity: no
            // warp can be two tiles ahead, as every tile needs all eight)
            float *epb = ep + (i & 1) * 2 * kHRows;
            epb[hf * kHRows + r] = part;
            __syncwarp();
            if (lane == 0)
                ptx::mbar_arrive(&ep_bar[i & 1]);
            if (!ptx::mbar_wait_bounded(&ep_bar[i & 1], (unsigned)(i >> 1) & 1u, kSpinLimit)) {
                ok = false;
                break;
            }
            const float eta = epb[r] + epb[kHRows + r];
            __syncwarp();
            if (lane == 0)
                ptx::mbar_arrive(&x_empty[s]);              // the tile is in registers
            // TR map with the label folded into signs (z = (1 - 2y) eta):
            // ell = -softplus(z), mu = sigma(eta), w = mu (1 - mu), r = y - mu = +-sigma(z)
            const uint32_t ysign = yl == 1 ? 0x80000000u : 0u;
            const float z = __uint_as_float(__float_as_uint(eta) ^ ysign);
            const float ee = tc::ex2_approx(-fabsf(eta) * kLog2e);    // e^-|eta|
            const float lg = tc::lg2_approx(1.0f + ee);               // log2(1 + e^-|eta|)
            const float ru = tc::ex2_approx(-lg);                     // 1 / (1 + e^-|eta|)
            const float w = ee * ru * ru;
            const float sz = z >= 0.0f ? ru : ee * ru;                // sigma(z)
            const float rr = yl == 1 ? sz : -sz;
            if (valid && hf == 0)
                facc -= fmaf(lg, kLn2, fmaxf(z, 0.0f));
#pragma unroll
            for (int j = 0; j < 32; ++j)
                gacc[j] = fmaf(rr, x[j], gacc[j]);
            const int ob = i & 1;
            if (i >= 2 && !ptx::mbar_wait_bounded(&ab_empty[ob], (unsigned)((i >> 1) - 1) & 1u, kSpinLimit)) {
                ok = false;
                break;
            }
            // operand rows: A = [(w x)_hi | (w x)_lo], B = [x_hi | x_lo], each a
            // 128-byte-wide atom of 64 bf16 per row, 16-byte chunks permuted by row & 7
            uint8_t *abuf = ab + ob * kHOpBuf;
            const uint32_t sw = (uint32_t)(r & 7);
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                uint32_t wh[4], wl[4], xh[4], xl[4];
#pragma unroll
                for (int m = 0; m < 4; ++m) {
                    const float a0 = x[8 * q + 2 * m], a1 = x[8 * q + 2 * m + 1];
                    split_bf16x2(w * a0, w * a1, wh[m], wl[m]);
                    split_bf16x2(a0, a1, xh[m], xl[m]);
                }
                const uint32_t off = (uint32_t)(r * 128) + ((((uint32_t)(4 * hf + q)) ^ sw) << 4);
                *reinterpret_cast<uint4 *>(abuf + off) = make_uint4(wh[0], wh[1], wh[2], wh[3]);
                *reinterpret_cast<uint4 *>(abuf + kHAtom + off) = make_uint4(wl[0], wl[1], wl[2], wl[3]);
                *reinterpret_cast<uint4 *>(abuf + 2 * kHAtom + off) = make_uint4(xh[0], xh[1], xh[2], xh[3]);
                *reinterpret_cast<uint4 *>(abuf + 3 * kHAtom + off) = make_uint4(xl[0], xl[1], xl[2], xl[3]);
            }
            ptx::fence_proxy_async_smem();
            __syncwarp();
            if (lane == 0)
                ptx::mbar_arrive(&ab_full[ob]);
        }
        if (!ok) {
            atomicOr(p.status, kDevTimeout);
            s_abort = 1;
        }
        const bool have = nt > 0 && ok && ptx::mbar_wait_bounded(d_done, 0u, kSpinLimit);
        if (nt > 0 && !have) {
            atomicOr(p.status, kDevTimeout);
            s_abort = 1;
        }
        tc::fence_after();
        // the ring is free now (every tile read, every MMA done): sums go there
        float *hx = reinterpret_cast<float *>(xs);                  // [128][65]
        float *gs = reinterpret_cast<float *>(xs + 40 * 1024);      // [8][32]
        // f: the row quarters' sums (FP32 over 32 lanes, FP64 from here on)
        float fv = facc;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1)
            fv += __shfl_xor_sync(0xFFFFFFFFu, fv, o);
        if (hf == 0 && lane == 0)
            sfq[rq] = fv;
        // g: each column over the warp's 32 rows
#pragma unroll
        for (int j = 0; j < 32; ++j) {
            float v = gacc[j];
#pragma unroll
            for (int o = 16; o > 0; o >>= 1)
                v += __shfl_xor_sync(0xFFFFFFFFu, v, o);
            if (lane == 0)
                gs[e * 32 + j] = v;
        }
        // D rows (tensor-memory lanes) 32 lq .. 32 lq + 31, one warp per lane quarter:
        // T[m][j] = D[m][j] + D[m][64 + j]
        if (e < 4) {
            const int lq = warp & 3;
            const int m = lq * 32 + lane;
            const uint32_t ta = tmem + ((uint32_t)(lq * 32) << 16);
#pragma unroll
            for (int j0 = 0; j0 < 64; j0 += 16) {
                float d0[16], d1[16];
                if (have) {
                    tc::tmem_ld<16>(ta + j0, d0);
                    tc::tmem_ld<16>(ta + 64 + j0, d1);
                    tc::tmem_wait_ld();
                }
#pragma unroll
                for (int j = 0; j < 16; ++j)
                    hx[m * 65 + j0 + j] = have ? d0[j] + d1[j] : 0.0f;
            }
        }
        asm volatile("bar.sync 1, %0;" ::"r"(kHConv * 32) : "memory");
        // (X^T W X)_ij = T[i][j] + T[64 + i][j], in a fixed order
        for (int idx = et; idx < kHMaxP * kHMaxP; idx += kHConv * 32) {
            const int i2 = idx >> 6, j2 = idx & 63;
            p.part_h[(size_t)b * kHMaxP * kHMaxP + idx] = hx[i2 * 65 + j2] + hx[(64 + i2) * 65 + j2];
        }
        if (et < kHMaxP) {
            const int h2 = et >> 5, j = et & 31;
            p.part_g[(size_t)b * kHMaxP + et] =
                ((gs[(4 * h2) * 32 + j] + gs[(4 * h2 + 1) * 32 + j]) + gs[(4 * h2 + 2) * 32 + j]) +
                gs[(4 * h2 + 3) * 32 + j];
        }
        if (et == 0)
            p.part_f[b] = s_abort ? __longlong_as_double(0x7FF8000000000000LL)
                                  : (((double)sfq[0] + (double)sfq[1]) + (double)sfq[2]) + (double)sfq[3];
    }
    tc::fence_before();
    __syncthreads();
    tc::fence_after();
    if (warp == 1)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                     "r"(kHTmemCols)
                     : "memory");
}

// Fixed-order combine of the per-CTA partials, plus the Gaussian prior: one
// thread per output element (f, g_j, H_ij with i <= j); its block's 8 warps
// each add a contiguous range of CTAs with all loads of a range in flight,
// then warp 0 adds the 8 range sums in order. H_ij is written to both
// triangles (exactly symmetric).
constexpr int kHessRedWarps = 16;

// Fixed-order combine of the per-CTA partials: a block takes 32 outputs (f,
// an entry of g, or an upper-triangle entry of H), each of its warps adds a
// contiguous range of CTAs (all loads of a range in flight) and warp 0 adds
// the warps' sums in order. g and H are summed in FP32 (152 partials: a
// relative rounding error of order 1e-6; this part's FP64 pipe made the FP64
// version 4x slower), f in FP64.
__global__ void __launch_bounds__(32 * kHessRedWarps)
    hess_combine_kernel(const double *__restrict__ part_f, const float *__restrict__ part_g,
                        const float *__restrict__ part_h, int parts, int P,
                        const float *__restrict__ beta, double inv_s2, double prior_const,
                        double *__restrict__ f_out, float *__restrict__ g_out,
                        float *__restrict__ H_out)
{
    ptx::grid_dep_wait();
    __shared__ float sum[kHessRedWarps][32];
    __shared__ double fsum[kHessRedWarps];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int nel = 1 + kHMaxP + kHMaxP * kHMaxP;
    const int e = blockIdx.x * 32 + lane;
    int i = 0, j = 0;
    bool want = e < nel;
    if (want && e > kHMaxP) {
        i = (e - 1 - kHMaxP) >> 6;
        j = (e - 1 - kHMaxP) & 63;
        want = i < P && j < P && j >= i;
    } else if (want && e >= 1) {
        want = e - 1 < P;
    }
    const int per = (parts + kHessRedWarps - 1) / kHessRedWarps;
    const int q0 = warp * per;
    const int q1 = q0 + per < parts ? q0 + per : parts;
    float v = 0.0f;
    if (want && e > 0) {
        const float *src = e <= kHMaxP ? part_g + (e - 1) : part_h + (e - 1 - kHMaxP);
        const size_t stride = e <= kHMaxP ? (size_t)kHMaxP : (size_t)kHMaxP * kHMaxP;
        for (int qb = q0; qb < q1; qb += 16) {
            float buf[16];
#pragma unroll
            for (int u = 0; u < 16; ++u)
                buf[u] = qb + u < q1 ? __ldg(src + (size_t)(qb + u) * stride) : 0.0f;
#pragma unroll
            for (int u = 0; u < 16; ++u)
                v += buf[u];
        }
    }
    if (blockIdx.x == 0 && lane == 0) {             // f: this warp's CTA range in FP64
        double fv = 0.0;
        for (int q = q0; q < q1; ++q)
            fv += part_f[q];
        fsum[warp] = fv;
    }
    sum[warp][lane] = v;
    __syncthreads();
    if (warp != 0)
        return;
    float tot = 0.0f;
#pragma unroll
    for (int w = 0; w < kHessRedWarps; ++w)
        tot += sum[w][lane];
    if (blockIdx.x == 0) {
        // ||beta||^2 across the warp (P <= 64), then f
        float bb = 0.0f;
        for (int t = lane; t < P; t += 32)
            bb = fmaf(beta[t], beta[t], bb);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1)
            bb += __shfl_xor_sync(0xFFFFFFFFu, bb, o);
        if (lane == 0) {
            double ft = 0.0;
            for (int w = 0; w < kHessRedWarps; ++w)
                ft += fsum[w];
            *f_out = ft - 0.5 * inv_s2 * (double)bb - prior_const;
        }
    }
    if (!want || e == 0)
        return;
    if (e <= kHMaxP) {
        g_out[e - 1] = tot - beta[e - 1] * (float)inv_s2;
    } else {
        const float hv = -tot - (i == j ? (float)inv_s2 : 0.0f);
        H_out[(size_t)i * P + j] = hv;
        H_out[(size_t)j * P + i] = hv;
    }
}

}  // namespace glm

using namespace glm;

// X as FP32 rows: 32-column boxes of 128 rows with the 128-byte swizzle; the
// second box starts at column 32 (columns past ld read as zeros).
static glm_status_t hess_tensor_map(glm_hess *h, const void *X)
{
    if (h->map_ptr == X)
        return GLM_OK;
    PFN_cuTensorMapEncodeTiled_v12000 encode = tensor_map_encoder();
    if (!encode)
        return GLM_ERR_CUDA;
    const cuuint64_t dims[2] = {(cuuint64_t)h->ld, (cuuint64_t)h->n_rows};
    const cuuint64_t strides[1] = {(cuuint64_t)h->ld * 4};
    const cuuint32_t box[2] = {32, (cuuint32_t)kHRows};
    const cuuint32_t estr[2] = {1, 1};
    CUresult r = encode(reinterpret_cast<CUtensorMap *>(h->map), CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2,
                        const_cast<void *>(X), dims, strides, box, estr,
                        CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                        CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS)
        return GLM_ERR_CUDA;
    h->map_ptr = X;
    return GLM_OK;
}

extern "C" {

glm_status_t glm_hess_create(int64_t n_rows, int32_t p, int32_t ld, double prior_sigma, int32_t device,
                             glm_hess_t *out)
{
    if (!out)
        return GLM_ERR_INVALID_ARG;
    *out = nullptr;
    if (n_rows < 0 || p < 1 || p > kHMaxP || ld < p || ld > kHMaxP || (ld & 3) ||
        !(prior_sigma > 0.0) || !std::isfinite(prior_sigma) || device < 0)
        return GLM_ERR_INVALID_ARG;
    if (n_rows > ((int64_t)1 << 31) - kHRows)
        return GLM_ERR_UNSUPPORTED;
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
    h->grid = sms;
    h->prior_sigma = prior_sigma;
    const size_t fb = (size_t)h->grid * 8, gb = (size_t)h->grid * kHMaxP * 4,
                 hb = (size_t)h->grid * kHMaxP * kHMaxP * 4;
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
    cudaDeviceSynchronize();
    cudaFree(h->ws);
    delete h;
    return GLM_OK;
}

glm_status_t glm_hess_eval(glm_hess_t h, const float *X, const uint8_t *y, const float *beta,
                           double *f_out, float *g_out, float *H_out, glm_stream_t stream)
{
    if (!h || !beta || !f_out || !g_out || !H_out || (h->n_rows > 0 && (!X || !y)) ||
        (reinterpret_cast<uintptr_t>(X) & 15u) || (reinterpret_cast<uintptr_t>(f_out) & 7u) ||
        (reinterpret_cast<uintptr_t>(beta) & 3u) || (reinterpret_cast<uintptr_t>(g_out) & 3u) ||
        (reinterpret_cast<uintptr_t>(H_out) & 3u))
        return GLM_ERR_INVALID_ARG;
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    if (h->n_rows > 0) {
        glm_status_t gs = hess_tensor_map(h, X);
        if (gs != GLM_OK)
            return gs;
    }                   // with no rows no tile is loaded and the map is never read
    HessParams p;
    std::memset(&p, 0, sizeof(p));
    p.y = y;
    p.beta = beta;
    p.N = h->n_rows;
    p.P = h->p;
    p.part_f = h->part_f;
    p.part_g = h->part_g;
    p.part_h = h->part_h;
    p.status = h->status;
    const HessLayout L = hess_layout();
    if (allow_max_dynamic_smem(reinterpret_cast<const void *>(&hess_tc_kernel)) != cudaSuccess)
        return GLM_ERR_CUDA;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)h->grid);
    cfg.blockDim = dim3(kHThreads);
    cfg.dynamicSmemBytes = (size_t)L.total;
    cfg.stream = st;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    const CUtensorMap *map = reinterpret_cast<const CUtensorMap *>(h->map);
    if (cudaLaunchKernelEx(&cfg, hess_tc_kernel, *map, p) != cudaSuccess)
        return GLM_ERR_CUDA;
    const double s2 = h->prior_sigma * h->prior_sigma;
    const int nel = 1 + kHMaxP + kHMaxP * kHMaxP;
    cudaLaunchConfig_t rc = {};
    rc.gridDim = dim3((unsigned)((nel + 31) / 32));
    rc.blockDim = dim3(32 * kHessRedWarps);
    rc.stream = st;
    rc.attrs = attr;
    rc.numAttrs = 1;
    if (cudaLaunchKernelEx(&rc, hess_combine_kernel, (const double *)h->part_f,
                           (const float *)h->part_g, (const float *)h->part_h, h->grid, h->p, beta,
                           1.0 / s2, 0.5 * h->p * std::log(2.0 * M_PI * s2), f_out, g_out,
                           H_out) != cudaSuccess)
        return GLM_ERR_CUDA;
    return GLM_OK;
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
