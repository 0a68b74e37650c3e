// Grouped (hierarchical-Bayes) log-posterior + gradient, §4.1: group m owns
// rows [off[m], off[m+1]) and its own coefficient vector beta_m, with prior
// N(mu, tau^2 I). All groups are evaluated by one persistent launch.
//
// The rows [off[0], off[G]) are split evenly over every warp of the grid (the
// paper's fine-grained mapping of §4.1: parallelism inside a group, not one
// worker per group, which balances groups of 20 to 50,000 rows). Each warp
// streams its rows once through its own ring of TMA slots (32 rows per slot,
// mbarrier completion, no block-wide barrier in the loop):
//   phase 1: lane l takes row l of the slot, finds the row's group, computes
//            eta = x . beta_group and the TR map (ell, r) in FP32;
//   phase 2: lanes own (row slot, 16-byte column chunk) pairs and accumulate
//            g += r x for the current group in registers.
// When a group ends (or the warp's rows end), a group that lies wholly in
// the warp's rows is finished from registers (prior added, f and g written);
// a group shared with neighbouring warps gets the warp's f and g sums in its
// 128-bit fixed-point accumulators, and its completion counter tells the last
// contributing warp (the number of warps covering a group follows from the
// even row split) to add the prior and write f and g. Integer accumulation
// makes the result independent of arrival order: bitwise reproducible.
//
// The kernel has a compile-time instance for rows of eight 16-byte chunks
// (row stride, chunk rotation and lane mapping constant). A second kernel,
// for at most 32 used columns, keeps each row, the group's coefficients and
// the gradient sums in registers. glm_autotune_grouped times both over
// warps per CTA, rows per slot, ring slots and CTAs per SM;
// glm_grouped_set_shape sets one of those shapes directly.
#include <cmath>
#include <cstdlib>
#include <cstring>

#include "glm_fused.cuh"

namespace glm {

constexpr int kGroupedMaxThreads = 512;
constexpr int kGroupedRows = 32;          // rows per slot = lanes per warp

__device__ __forceinline__ double warp_sum_f64(double v)
{
#pragma unroll
    for (int m = 16; m > 0; m >>= 1)
        v += __shfl_xor_sync(0xFFFFFFFFu, v, m);
    return v;
}

// Warp-cooperative: write f_g and g_g from the group's totals (read from the
// accumulators, which are cleared, or zero for an empty group) plus the prior.
__device__ void group_finalize(const GroupedParams &p, int g, bool from_acc, int lane)
{
    const int P = p.P;
    const bool nan_out = from_acc && (__ldcg(p.gflag + g) != 0u);
    double dd = 0.0;
    for (int j = lane; j < P; j += 32) {
        const double d = (double)p.beta[(size_t)g * P + j] - (double)p.mu[j];
        dd += d * d;
    }
    dd = warp_sum_f64(dd);
    for (int j = lane; j <= P; j += 32) {
        double t = 0.0;
        if (from_acc)
            t = fx::read_and_clear(p.acc + ((size_t)g * (P + 1) + j) * fx::kLimbs);
        if (nan_out)
            t = __longlong_as_double(0x7FF8000000000000LL);
        if (j == 0) {
            p.f_out[g] = t - 0.5 * p.inv_t2 * dd - p.prior_const;
        } else {
            const int jj = j - 1;
            const double sc = p.x_scale ? (double)p.x_scale[jj] : 1.0;
            const double d = (double)p.beta[(size_t)g * P + jj] - (double)p.mu[jj];
            p.g_out[(size_t)g * P + jj] = (float)(sc * t - d * p.inv_t2);
        }
    }
    if (lane == 0 && from_acc) {
        p.gflag[g] = 0u;
        p.gticket[g] = 0u;
    }
}

// PCX > 0: rows of exactly PCX 16-byte chunks, all of them holding used
// columns (ld * element size = 16 PCX, ceil(P / EPC) = PCX), so that the row
// stride, the chunk rotation and the lane mapping are compile-time constants;
// PCX = 0 takes them from the parameters.
template <typename Tag, int PCX>
__global__ void __launch_bounds__(kGroupedMaxThreads, 1) grouped_logpost_grad_kernel(GroupedParams p)
{
    using TR = XTraits<Tag>;
    constexpr int EPC = TR::EPC;
    constexpr int ES = TR::ES;
    constexpr unsigned FULL = 0xFFFFFFFFu;
    constexpr int CR = kGroupedRows;
    static_assert((PCX & (PCX - 1)) == 0, "PCX is 0 or a power of two");
    constexpr int kU1 = PCX ? PCX : 4;

    extern __shared__ __align__(128) uint8_t smem[];
    const int tid = threadIdx.x;
    const int lane = tid & 31;
    const int warp = tid >> 5;
    const int NW = blockDim.x >> 5;
    const int b = blockIdx.x;
    const int grid = gridDim.x;
    const int P = p.P;
    const int ld = p.ld;
    const int PC = PCX ? PCX : ld / EPC;
    const int PCU = PCX ? PCX : (P + EPC - 1) / EPC;
    const int row_bytes = PCX ? 16 * PCX : ld * ES;
    const int G = p.G;
    const int stages = p.stages;
    const int slot_bytes = CR * row_bytes;
    const int ring_bytes = (stages * slot_bytes + 127) / 128 * 128;
    uint8_t *ring = smem + warp * ring_bytes;
    uint64_t *bars = reinterpret_cast<uint64_t *>(smem + NW * ring_bytes) + warp * stages;
    const int64_t *off = p.off;

    ptx::grid_dep_wait();
    // Every CTA checks the offsets itself (non-decreasing, within [0, N]); a
    // malformed list gives NaN results instead of out-of-range reads.
    bool ok = true;
    for (int g = tid; g < G; g += blockDim.x)
        if (off[g] > off[g + 1])
            ok = false;
    if (tid == 0 && (off[0] < 0 || off[G] > p.N))
        ok = false;
    if (__syncthreads_or(!ok)) {
        for (int i = b * blockDim.x + tid; i < G * (P + 1); i += grid * blockDim.x) {
            const int g = i / (P + 1);
            const int j = i - g * (P + 1);
            const double nanv = __longlong_as_double(0x7FF8000000000000LL);
            if (j == 0)
                p.f_out[g] = nanv;
            else
                p.g_out[(size_t)g * P + j - 1] = (float)nanv;
        }
        return;
    }
    ptx::grid_dep_launch_dependents();

    const int Wall = grid * NW;
    const int gw = b * NW + warp;
    // Empty groups: the prior alone.
    for (int g = gw; g < G; g += Wall)
        if (off[g] == off[g + 1])
            group_finalize(p, g, false, lane);

    // Rows split over W = min(warps, rows) warps, so every working warp has at
    // least one row and a group's rows meet consecutive warps only.
    const int64_t r_lo = off[0];
    const int64_t R = off[G] - r_lo;
    const int W = (int)(R < (int64_t)Wall ? R : (int64_t)Wall);
    const int64_t wr0 = gw < W ? r_lo + (R * gw) / W : r_lo;
    const int64_t wr1 = gw < W ? r_lo + (R * (gw + 1)) / W : r_lo;
    const int nch = (int)((wr1 - wr0 + CR - 1) / CR);
    // warps covering relative row q: the warp whose range holds q
    auto warp_of = [&](int64_t q) -> int64_t { return ((q + 1) * W - 1) / R; };

    if (lane == 0) {
        for (int s = 0; s < stages; ++s)
            ptx::mbar_init(&bars[s], 1);
        ptx::fence_mbar_init();
    }
    __syncwarp();
    const uint64_t policy = ptx::policy_evict_first();
    const uint8_t *Xb = static_cast<const uint8_t *>(p.X);
    auto issue = [&](int i) {
        const int64_t row0 = wr0 + (int64_t)i * CR;
        const int rows = (int)((wr1 - row0) < CR ? (wr1 - row0) : CR);
        uint64_t *bar = &bars[i % stages];
        ptx::mbar_arrive_expect_tx(bar, (unsigned)(rows * row_bytes));
        ptx::bulk_g2s(ring + (i % stages) * slot_bytes, Xb + row0 * (int64_t)row_bytes,
                      (unsigned)(rows * row_bytes), bar, policy);
    };
    if (lane == 0) {
        const int pre = nch < stages ? nch : stages;
        for (int i = 0; i < pre; ++i)
            issue(i);
    }
    // a slot's labels are loaded one slot ahead and kept as raw bytes until
    // their use, so that no conversion waits for the load where it is issued
    auto load_y = [&](int i) -> unsigned {
        if (i >= nch)
            return 0u;
        const int64_t row = wr0 + (int64_t)i * CR + lane;
        return row < wr1 ? (unsigned)__ldg(p.y + row) : 0u;
    };

    // the non-empty group holding row wr0
    int cur = 0;
    if (nch > 0) {
        int lo = 0, hi = G;          // largest g in [0, G) with off[g] <= wr0
        while (hi - lo > 1) {
            const int mid = (lo + hi) >> 1;
            if (off[mid] <= wr0)
                lo = mid;
            else
                hi = mid;
        }
        cur = lo;
        while (off[cur + 1] <= wr0)
            ++cur;
    }
    int64_t cur_end = nch > 0 ? off[cur + 1] : 0;   // end row of the current group

    // phase-2 lane mapping
    int W2 = 1;
    while (W2 < PCU)
        W2 <<= 1;
    const int RS = 32 / W2;
    const int rs = lane / W2;
    const int ch = lane & (W2 - 1);
    const int rot = ((PC & 1) == 0) ? (lane & 7) % PCU : 0;

    float gacc[EPC];
#pragma unroll
    for (int e = 0; e < EPC; ++e)
        gacc[e] = 0.0f;
    float fseg = 0.0f;
    bool bad = false;
    int fail_at = -1;

    // Coefficients of the current group, times the FP8 column scales, staged
    // in this warp's slice of shared memory for the common case where a whole
    // slot of rows belongs to that group.
    float *bcur = reinterpret_cast<float *>(smem + NW * ring_bytes + NW * stages * 8) +
                  warp * PCU * EPC;
    auto stage_beta = [&](int g) {
        __syncwarp();
        for (int j = lane; j < PCU * EPC; j += 32) {
            float v = 0.0f;
            if (j < P) {
                v = __ldg(p.beta + (size_t)g * P + j);
                if (p.x_scale)
                    v *= __ldg(p.x_scale + j);
            }
            bcur[j] = v;
        }
        __syncwarp();
    };

    // Close the warp's run of rows of group g. A group whose rows all lie in
    // this warp's range is finished here from registers; a group shared with
    // neighbouring warps goes through the fixed-point accumulators and the
    // last contributor finishes it.
    auto flush = [&](int g) {
        double fs = warp_sum_f64((double)fseg);
        for (int m = W2; m < 32; m <<= 1)
#pragma unroll
            for (int e = 0; e < EPC; ++e)
                gacc[e] += __shfl_xor_sync(FULL, gacc[e], m);
        const double nanv = __longlong_as_double(0x7FF8000000000000LL);
        const bool priv = off[g] >= wr0 && off[g + 1] <= wr1;
        if (priv) {
            double dd = 0.0;
            for (int j = lane; j < P; j += 32) {
                const double d = (double)p.beta[(size_t)g * P + j] - (double)p.mu[j];
                dd += d * d;
            }
            dd = warp_sum_f64(dd);
            if (lane == 0)
                p.f_out[g] = (bad ? nanv : fs) - 0.5 * p.inv_t2 * dd - p.prior_const;
            if (rs == 0 && ch < PCU) {
#pragma unroll
                for (int e = 0; e < EPC; ++e) {
                    const int col = ch * EPC + e;
                    if (col < P) {
                        const double sc = p.x_scale ? (double)p.x_scale[col] : 1.0;
                        const double d = (double)p.beta[(size_t)g * P + col] - (double)p.mu[col];
                        const double t = bad ? nanv : (double)gacc[e];
                        p.g_out[(size_t)g * P + col] = (float)(sc * t - d * p.inv_t2);
                    }
                }
            }
        } else {
            unsigned long long *ga = p.acc + (size_t)g * (P + 1) * fx::kLimbs;
            if (rs == 0 && ch < PCU) {
#pragma unroll
                for (int e = 0; e < EPC; ++e) {
                    const int col = ch * EPC + e;
                    if (col < P)
                        fx::add(ga + (size_t)(1 + col) * fx::kLimbs, bad ? nanv : (double)gacc[e],
                                p.gflag + g);
                }
            }
            if (lane == 0)
                fx::add(ga, bad ? nanv : fs, p.gflag + g);
            __threadfence();
            __syncwarp();
            unsigned last = 0;
            if (lane == 0) {
                const int64_t q0 = off[g] - r_lo;
                const int64_t q1 = off[g + 1] - 1 - r_lo;
                const unsigned expect = (unsigned)(warp_of(q1) - warp_of(q0) + 1);
                last = (atomicAdd(p.gticket + g, 1u) + 1u == expect) ? 1u : 0u;
            }
            last = __shfl_sync(FULL, last, 0);
            if (last) {
                __threadfence();
                group_finalize(p, g, true, lane);
            }
        }
#pragma unroll
        for (int e = 0; e < EPC; ++e)
            gacc[e] = 0.0f;
        fseg = 0.0f;
    };

    if (nch > 0)
        stage_beta(cur);
    unsigned ycur = load_y(0);
    for (int i = 0; i < nch; ++i) {
        const int s = i % stages;
        const unsigned parity = (unsigned)(i / stages) & 1u;
        const int64_t row0 = wr0 + (int64_t)i * CR;
        const int nrows = (int)((wr1 - row0) < CR ? (wr1 - row0) : CR);
        const unsigned ynext = load_y(i + 1);
        if (!bad) {
            const bool okw = ptx::mbar_wait_bounded(&bars[s], parity, kSpinLimit);
            if (__any_sync(FULL, !okw)) {
                bad = true;
                fail_at = i;
                if (lane == 0)
                    atomicOr(p.status, kDevTimeout);
            }
        }
        const uint8_t *slot = ring + s * slot_bytes;

        // ---- groups of this slot's rows -------------------------------------------
        const bool valid = lane < nrows;
        const int64_t myrow = row0 + lane;
        int gl = cur;
        if (valid && myrow >= cur_end) {     // rare: this row starts a later group
            gl = cur + 1;
            while (myrow >= off[gl + 1])
                ++gl;
        }
        const int g0 = __shfl_sync(FULL, gl, 0);
        if (g0 != cur) {              // the current group ended with the previous slot
            flush(cur);
            cur = g0;
            cur_end = off[cur + 1];
            stage_beta(cur);
        }
        const bool uniform = __all_sync(FULL, !valid || gl == cur);

        // ---- phase 1: this lane's row ------------------------------------------
        float ell = 0.0f, r = 0.0f;
        if (valid) {
            const uint8_t *xr = slot + lane * row_bytes;
            float eta = 0.0f;
            int cs = rot;
            if (uniform) {
#pragma unroll kU1
                for (int it = 0; it < PCU; ++it) {
                    const int c = PCX ? ((rot + it) & (PCX - 1)) : cs;
                    cs = (cs + 1 == PCU) ? 0 : cs + 1;
                    float xv[EPC];
                    TR::load(xr + c * 16, xv);
                    const float *bk = bcur + c * EPC;
                    float pa = 0.0f;
#pragma unroll
                    for (int e = 0; e < EPC; e += 4) {
                        const float4 bb = *reinterpret_cast<const float4 *>(bk + e);
                        pa = fmaf(xv[e], bb.x, pa);
                        pa = fmaf(xv[e + 1], bb.y, pa);
                        pa = fmaf(xv[e + 2], bb.z, pa);
                        pa = fmaf(xv[e + 3], bb.w, pa);
                    }
                    eta += pa;
                }
            } else {
                const float *bg = p.beta + (size_t)gl * P;
                for (int it = 0; it < PCU; ++it) {
                    const int c = cs;
                    cs = (cs + 1 == PCU) ? 0 : cs + 1;
                    float xv[EPC];
                    TR::load(xr + c * 16, xv);
                    float pa = 0.0f;
#pragma unroll
                    for (int e = 0; e < EPC; ++e) {
                        const int col = c * EPC + e;
                        float bv = col < P ? __ldg(bg + col) : 0.0f;
                        if (p.x_scale && col < P)
                            bv *= __ldg(p.x_scale + col);
                        pa = fmaf(xv[e], bv, pa);
                    }
                    eta += pa;
                }
            }
            tr_map(eta, (float)ycur, ell, r);
        }

        // ---- phase 2: per-group segments of this slot ----------------------------
        int sidx = 0;
        while (sidx < nrows) {
            const int sg = __shfl_sync(FULL, gl, sidx);
            if (sg != cur) {
                flush(cur);
                cur = sg;
                cur_end = off[cur + 1];
                stage_beta(cur);
            }
            const int64_t gend = cur_end;
            const int e_end = (int)((gend - row0) < nrows ? (gend - row0) : nrows);
            if (PCX && sidx == 0 && e_end == CR) {
                // a whole slot of one group: the same steps, fully unrolled,
                // with the row offsets as constants
                const uint8_t *xb = slot + rs * row_bytes + ch * 16;
#pragma unroll
                for (int i0 = 0; i0 < CR; i0 += RS) {
                    const float ri = __shfl_sync(FULL, r, i0 + rs);
                    float xv[EPC];
                    TR::load(xb + i0 * row_bytes, xv);
#pragma unroll
                    for (int e = 0; e < EPC; ++e)
                        gacc[e] = fmaf(ri, xv[e], gacc[e]);
                }
            } else {
#pragma unroll 2
                for (int i0 = sidx; i0 < e_end; i0 += RS) {
                    const int ii = i0 + rs;
                    const bool v2 = ii < e_end;
                    const float ri = __shfl_sync(FULL, r, v2 ? ii : 0);
                    if (v2 && ch < PCU) {
                        float xv[EPC];
                        TR::load(slot + ii * row_bytes + ch * 16, xv);
#pragma unroll
                        for (int e = 0; e < EPC; ++e)
                            gacc[e] = fmaf(ri, xv[e], gacc[e]);
                    }
                }
            }
            if (lane >= sidx && lane < e_end)
                fseg += ell;
            sidx = e_end;
        }
        __syncwarp();
        if (lane == 0 && !bad && i + stages < nch)
            issue(i + stages);
        ycur = ynext;
    }
    if (nch > 0)
        flush(cur);
    if (bad && lane == 0) {
        // let this warp's copies still in flight land (bounded) before exit
        const int last = (fail_at + stages < nch) ? fail_at + stages : nch;
        for (int i = fail_at; i < last; ++i)
            ptx::mbar_wait_bounded(&bars[i % stages], (unsigned)(i / stages) & 1u, kSpinLimit);
    }
}

// ---------------------------------------------------------------------------
// Narrow rows (at most 32 used columns, NCH 16-byte chunks): each lane keeps
// its row, the current group's coefficients and its gradient accumulators in
// registers, so phase 2 is NCH*EPC fused multiply-adds per row with no
// shuffles or shared-memory re-reads. Lane l reads chunk (c + rot_l) mod NCH
// in step c so that 8 consecutive rows hit 8 distinct bank groups; the
// accumulators are therefore in lane-rotated column order and are put back in
// order (through a per-warp shared-memory transpose) only when a group ends.
constexpr int kNarrowMaxThreads = 384;      // registers: row, coefficients, accumulators

template <typename Tag, int NCH>
__global__ void __launch_bounds__(kNarrowMaxThreads, 1)
    grouped_narrow_kernel(GroupedParams p)
{
    using TR = XTraits<Tag>;
    constexpr int EPC = TR::EPC;
    constexpr int ES = TR::ES;
    constexpr unsigned FULL = 0xFFFFFFFFu;
    constexpr int CR = kGroupedRows;
    constexpr int NCOL = NCH * EPC;            // <= 32 columns held per lane
    static_assert(NCOL <= 32, "narrow path holds at most 32 columns per lane");

    extern __shared__ __align__(128) uint8_t smem[];
    const int tid = threadIdx.x;
    const int lane = tid & 31;
    const int warp = tid >> 5;
    const int NW = blockDim.x >> 5;
    const int b = blockIdx.x;
    const int grid = gridDim.x;
    const int P = p.P;
    const int row_bytes = p.ld * ES;
    const int PCS = row_bytes / 16;            // 16-byte chunks per stored row
    const int G = p.G;
    const int stages = p.stages;
    const int U = p.units;                     // 32-row units per TMA slot
    const int SR = CR * U;                     // rows per slot
    const int slot_bytes = SR * row_bytes;
    const int ring_bytes = (stages * slot_bytes + 127) / 128 * 128;
    uint8_t *ring = smem + warp * ring_bytes;
    uint64_t *bars = reinterpret_cast<uint64_t *>(smem + NW * ring_bytes) + warp * stages;
    float *tsp = reinterpret_cast<float *>(smem + NW * ring_bytes + NW * stages * 8 + 64) +
                 warp * 32 * 17;              // per-warp 32 x 17 transpose buffer
    const int64_t *off = p.off;

    ptx::grid_dep_wait();
    bool ok = true;
    for (int g = tid; g < G; g += blockDim.x)
        if (off[g] > off[g + 1])
            ok = false;
    if (tid == 0 && (off[0] < 0 || off[G] > p.N))
        ok = false;
    if (__syncthreads_or(!ok)) {
        for (int i = b * blockDim.x + tid; i < G * (P + 1); i += grid * blockDim.x) {
            const int g = i / (P + 1);
            const int j = i - g * (P + 1);
            const double nanv = __longlong_as_double(0x7FF8000000000000LL);
            if (j == 0)
                p.f_out[g] = nanv;
            else
                p.g_out[(size_t)g * P + j - 1] = (float)nanv;
        }
        return;
    }
    ptx::grid_dep_launch_dependents();

    const int Wall = grid * NW;
    const int gw = b * NW + warp;
    for (int g = gw; g < G; g += Wall)
        if (off[g] == off[g + 1])
            group_finalize(p, g, false, lane);

    const int64_t r_lo = off[0];
    const int64_t R = off[G] - r_lo;
    const int W = (int)(R < (int64_t)Wall ? R : (int64_t)Wall);
    const int64_t wr0 = gw < W ? r_lo + (R * gw) / W : r_lo;
    const int64_t wr1 = gw < W ? r_lo + (R * (gw + 1)) / W : r_lo;
    const int nch = (int)((wr1 - wr0 + SR - 1) / SR);
    auto warp_of = [&](int64_t q) -> int64_t { return ((q + 1) * W - 1) / R; };

    if (lane == 0) {
        for (int s = 0; s < stages; ++s)
            ptx::mbar_init(&bars[s], 1);
        ptx::fence_mbar_init();
    }
    __syncwarp();
    const uint64_t policy = ptx::policy_evict_first();
    const uint8_t *Xb = static_cast<const uint8_t *>(p.X);
    auto issue = [&](int i) {
        const int64_t row0 = wr0 + (int64_t)i * SR;
        const int rows = (int)((wr1 - row0) < SR ? (wr1 - row0) : SR);
        uint64_t *bar = &bars[i % stages];
        ptx::mbar_arrive_expect_tx(bar, (unsigned)(rows * row_bytes));
        ptx::bulk_g2s(ring + (i % stages) * slot_bytes, Xb + row0 * (int64_t)row_bytes,
                      (unsigned)(rows * row_bytes), bar, policy);
    };
    if (lane == 0) {
        const int pre = nch < stages ? nch : stages;
        for (int i = 0; i < pre; ++i)
            issue(i);
    }
    // labels of slot i, one register per 32-row unit (at most 4 units), kept
    // as raw bytes until their use one slot later
    auto load_y = [&](int i, unsigned &a0, unsigned &a1, unsigned &a2, unsigned &a3) {
        unsigned v[4] = {0u, 0u, 0u, 0u};
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const int64_t row = wr0 + (int64_t)i * SR + u * CR + lane;
            if (i < nch && u < U && row < wr1)
                v[u] = (unsigned)__ldg(p.y + row);
        }
        a0 = v[0]; a1 = v[1]; a2 = v[2]; a3 = v[3];
    };

    int cur = 0;
    if (nch > 0) {
        int lo = 0, hi = G;
        while (hi - lo > 1) {
            const int mid = (lo + hi) >> 1;
            if (off[mid] <= wr0)
                lo = mid;
            else
                hi = mid;
        }
        cur = lo;
        while (off[cur + 1] <= wr0)
            ++cur;
    }
    int64_t cur_end = nch > 0 ? off[cur + 1] : 0;   // end row of the current group

    const int rot = (lane * NCH / 8) & (NCH - 1);
    float br[NCH][EPC];                         // current group's coefficients, rotated
    float gr[NCH][EPC];                         // gradient accumulators, rotated
#pragma unroll
    for (int c = 0; c < NCH; ++c)
#pragma unroll
        for (int e = 0; e < EPC; ++e)
            gr[c][e] = 0.0f;
    float fseg = 0.0f;
    bool bad = false;
    int fail_at = -1;

    auto load_beta = [&](int g) {
#pragma unroll
        for (int c = 0; c < NCH; ++c) {
            const int cc = (c + rot) & (NCH - 1);
#pragma unroll
            for (int e = 0; e < EPC; ++e) {
                const int col = cc * EPC + e;
                float v = 0.0f;
                if (col < P) {
                    v = __ldg(p.beta + (size_t)g * P + col);
                    if (p.x_scale)
                        v *= __ldg(p.x_scale + col);
                }
                br[c][e] = v;
            }
        }
    };

    auto flush = [&](int g) {
        const double nanv = __longlong_as_double(0x7FF8000000000000LL);
        const double fs = warp_sum_f64((double)fseg);
        // lane-rotated accumulators back to column order, 16 columns per
        // pass through the warp's transpose buffer; lane j ends with column j
        double half[2] = {0.0, 0.0};
#pragma unroll
        for (int hp = 0; hp < (NCOL + 15) / 16; ++hp) {
            __syncwarp();
#pragma unroll
            for (int c = 0; c < NCH; ++c) {
                const int cc = (c + rot) & (NCH - 1);
#pragma unroll
                for (int e = 0; e < EPC; ++e) {
                    const int col = cc * EPC + e - 16 * hp;
                    if (col >= 0 && col < 16)
                        tsp[lane * 17 + col] = gr[c][e];
                }
            }
            __syncwarp();
            double t = 0.0;
            if (lane < 16 && 16 * hp + lane < NCOL)
                for (int l = 0; l < 32; ++l)
                    t += (double)tsp[l * 17 + lane];
            half[hp] = t;
        }
        __syncwarp();
        const double ga0 = __shfl_sync(FULL, half[0], lane & 15);
        const double ga1 = __shfl_sync(FULL, half[1], lane & 15);
        const double gcol = lane < 16 ? ga0 : ga1;
        const bool priv = off[g] >= wr0 && off[g + 1] <= wr1;
        if (priv) {
            double dd = 0.0;
            if (lane < P) {
                const double d = (double)p.beta[(size_t)g * P + lane] - (double)p.mu[lane];
                dd = d * d;
            }
            dd = warp_sum_f64(dd);
            if (lane == 0)
                p.f_out[g] = (bad ? nanv : fs) - 0.5 * p.inv_t2 * dd - p.prior_const;
            if (lane < P) {
                const double sc = p.x_scale ? (double)p.x_scale[lane] : 1.0;
                const double d = (double)p.beta[(size_t)g * P + lane] - (double)p.mu[lane];
                p.g_out[(size_t)g * P + lane] = (float)(sc * (bad ? nanv : gcol) - d * p.inv_t2);
            }
        } else {
            unsigned long long *ga = p.acc + (size_t)g * (P + 1) * fx::kLimbs;
            if (lane < P)
                fx::add(ga + (size_t)(1 + lane) * fx::kLimbs, bad ? nanv : gcol, p.gflag + g);
            if (lane == 0)
                fx::add(ga, bad ? nanv : fs, p.gflag + g);
            __threadfence();
            __syncwarp();
            unsigned last = 0;
            if (lane == 0) {
                const int64_t q0 = off[g] - r_lo;
                const int64_t q1 = off[g + 1] - 1 - r_lo;
                const unsigned expect = (unsigned)(warp_of(q1) - warp_of(q0) + 1);
                last = (atomicAdd(p.gticket + g, 1u) + 1u == expect) ? 1u : 0u;
            }
            last = __shfl_sync(FULL, last, 0);
            if (last) {
                __threadfence();
                group_finalize(p, g, true, lane);
            }
        }
#pragma unroll
        for (int c = 0; c < NCH; ++c)
#pragma unroll
            for (int e = 0; e < EPC; ++e)
                gr[c][e] = 0.0f;
        fseg = 0.0f;
    };

    if (nch > 0)
        load_beta(cur);
    unsigned yc0, yc1, yc2, yc3;
    load_y(0, yc0, yc1, yc2, yc3);
    for (int i = 0; i < nch; ++i) {
        const int s = i % stages;
        const unsigned parity = (unsigned)(i / stages) & 1u;
        unsigned yn0, yn1, yn2, yn3;
        load_y(i + 1, yn0, yn1, yn2, yn3);
        if (!bad) {
            const bool okw = ptx::mbar_wait_bounded(&bars[s], parity, kSpinLimit);
            if (__any_sync(FULL, !okw)) {
                bad = true;
                fail_at = i;
                if (lane == 0)
                    atomicOr(p.status, kDevTimeout);
            }
        }
        for (int u = 0; u < U; ++u) {
            const float ycur = (float)yc0;        // labels shift down one unit per step
            yc0 = yc1;
            yc1 = yc2;
            yc2 = yc3;
            const int64_t row0 = wr0 + (int64_t)i * SR + u * CR;
            if (row0 >= wr1)
                break;
            const int nrows = (int)((wr1 - row0) < CR ? (wr1 - row0) : CR);
            const uint8_t *xrow = ring + s * slot_bytes + (u * CR + lane) * row_bytes;
            const bool valid = lane < nrows;
            const int64_t myrow = row0 + lane;
            int gl = cur;
            if (valid && myrow >= cur_end) {     // rare: this row starts a later group
                gl = cur + 1;
                while (myrow >= off[gl + 1])
                    ++gl;
            }
            const int g0 = __shfl_sync(FULL, gl, 0);
            if (g0 != cur) {
                flush(cur);
                cur = g0;
                cur_end = off[cur + 1];
                load_beta(cur);
            }
            const bool uniform = __all_sync(FULL, !valid || gl == cur);

            // ---- phase 1 ------------------------------------------------------------
            float xv[NCH][EPC];
            float ell = 0.0f, r = 0.0f;
    #pragma unroll
            for (int c = 0; c < NCH; ++c) {
                // chunks past the stored row (NCH rounds its chunk count up
                // to a power of two) hold no column of this row: zero
                if (valid && ((c + rot) & (NCH - 1)) < PCS) {
                    TR::load(xrow + ((c + rot) & (NCH - 1)) * 16, xv[c]);
                } else {
    #pragma unroll
                    for (int e = 0; e < EPC; ++e)
                        xv[c][e] = 0.0f;
                }
            }
            if (valid) {
                float eta = 0.0f;
                if (uniform) {
    #pragma unroll
                    for (int c = 0; c < NCH; ++c) {
                        float pa = 0.0f;
    #pragma unroll
                        for (int e = 0; e < EPC; ++e)
                            pa = fmaf(xv[c][e], br[c][e], pa);
                        eta += pa;
                    }
                } else {
                    const float *bg = p.beta + (size_t)gl * P;
    #pragma unroll
                    for (int c = 0; c < NCH; ++c) {
                        const int cc = (c + rot) & (NCH - 1);
                        float pa = 0.0f;
    #pragma unroll
                        for (int e = 0; e < EPC; ++e) {
                            const int col = cc * EPC + e;
                            float bv = col < P ? __ldg(bg + col) : 0.0f;
                            if (p.x_scale && col < P)
                                bv *= __ldg(p.x_scale + col);
                            pa = fmaf(xv[c][e], bv, pa);
                        }
                        eta += pa;
                    }
                }
                tr_map(eta, ycur, ell, r);
            }

            // ---- phase 2: one segment per group present in this slot --------------------
            int sidx = 0;
            while (sidx < nrows) {
                const int sg = __shfl_sync(FULL, gl, sidx);
                if (sg != cur) {
                    flush(cur);
                    cur = sg;
                    cur_end = off[cur + 1];
                    load_beta(cur);
                }
                const int64_t gend = cur_end;
                const int e_end = (int)((gend - row0) < nrows ? (gend - row0) : nrows);
                if (lane >= sidx && lane < e_end) {
    #pragma unroll
                    for (int c = 0; c < NCH; ++c)
    #pragma unroll
                        for (int e = 0; e < EPC; ++e)
                            gr[c][e] = fmaf(r, xv[c][e], gr[c][e]);
                    fseg += ell;
                }
                sidx = e_end;
            }
        }
        __syncwarp();
        if (lane == 0 && !bad && i + stages < nch)
            issue(i + stages);
        yc0 = yn0;
        yc1 = yn1;
        yc2 = yn2;
        yc3 = yn3;
    }
    if (nch > 0)
        flush(cur);
    if (bad && lane == 0) {
        const int last = (fail_at + stages < nch) ? fail_at + stages : nch;
        for (int i = fail_at; i < last; ++i)
            ptx::mbar_wait_bounded(&bars[i % stages], (unsigned)(i / stages) & 1u, kSpinLimit);
    }
}

// ---------------------------------------------------------------------------

// Narrow-row path: chunks per row when at most 32 columns are used, else 0.
static int grouped_nch(int p, int epc)
{
    const int pcu = (p + epc - 1) / epc;
    if (pcu * epc > 32)
        return 0;
    int n = 1;
    while (n < pcu)
        n <<= 1;
    return n * epc <= 32 ? n : 0;
}

static int grouped_smem(int row_bytes, int warps, int stages, int pcue, int narrow, int units)
{
    const int ring = (stages * units * kGroupedRows * row_bytes + 127) / 128 * 128;
    const int extra = narrow ? 64 + warps * 32 * 17 * 4 : warps * pcue * 4;
    return warps * ring + warps * stages * 8 + extra + 64;
}

// Launch shape of the grouped pass: warps per CTA and slots per warp ring
// (defaults; glm_autotune can replace them with measured choices).
glm_status_t grouped_configure(glm_ctx *h)
{
    const int es = h->elem_bytes;
    const int epc = 16 / es;
    const int pcu = (h->d.p + epc - 1) / epc;
    if (pcu > 32)
        return GLM_ERR_UNSUPPORTED;
    const int row_bytes = h->d.ld * es;
    const int pcue = pcu * epc;
    // the default is the warp-stream kernel; the autotuner also tries the
    // narrow-row kernel where it applies
    const bool narrow = false;
    int warps = 16;
    const int budget = kSmemOptinBytes;
    const int units = 1;
    int stages = 8;
    while (stages >= 2 && grouped_smem(row_bytes, warps, stages, pcue, narrow, units) > budget)
        --stages;
    while (stages < 2 && warps > 1) {
        warps = warps > 4 ? warps - 4 : warps - 1;
        stages = 8;
        while (stages >= 2 && grouped_smem(row_bytes, warps, stages, pcue, narrow, units) > budget)
            --stages;
    }
    if (stages < 2)
        return GLM_ERR_UNSUPPORTED;
    h->gr_warps = warps;
    h->gr_stages = stages;
    h->gr_units = units;
    h->gr_narrow = narrow ? 1 : 0;
    h->gr_grid = h->sm_count;
    return GLM_OK;
}

glm_status_t launch_grouped(glm_ctx *h, const void *X, const float *x_scale, const uint8_t *y,
                            const int64_t *group_off, int G, const float *beta, const float *mu,
                            double tau, double *f_out, float *g_out, cudaStream_t s)
{
    if (!h->gr_acc || h->gr_warps == 0)
        return GLM_ERR_UNSUPPORTED;
    GroupedParams prm;
    std::memset(&prm, 0, sizeof(prm));
    prm.X = X;
    prm.x_scale = x_scale;
    prm.y = y;
    prm.off = group_off;
    prm.N = h->d.n_rows;
    prm.G = G;
    prm.P = h->d.p;
    prm.ld = h->d.ld;
    prm.stages = h->gr_stages;
    prm.units = h->gr_units;
    prm.beta = beta;
    prm.mu = mu;
    const double t2 = tau * tau;
    prm.inv_t2 = 1.0 / t2;
    prm.prior_const = 0.5 * (double)h->d.p * std::log(2.0 * M_PI * t2);
    prm.acc = h->gr_acc;
    prm.gticket = h->gr_ticket;
    prm.gflag = h->gr_flag;
    prm.status = h->status;
    prm.f_out = f_out;
    prm.g_out = g_out;

    const int epc = 16 / h->elem_bytes;
    const int nchunks = grouped_nch(h->d.p, epc);
    const int smem = grouped_smem(h->d.ld * h->elem_bytes, h->gr_warps, h->gr_stages,
                                  ((h->d.p + epc - 1) / epc) * epc, nchunks > 0, h->gr_units);
    void (*fn)(GroupedParams) = nullptr;
    const bool narrow = nchunks > 0 && h->gr_narrow;
    // rows of exactly eight 16-byte chunks, all holding used columns
    const bool rows8 = h->d.ld * h->elem_bytes == 128 && (h->d.p + epc - 1) / epc == 8;
    switch (h->d.xtype) {
    case GLM_X_F32:
        if (!narrow)
            fn = rows8 ? grouped_logpost_grad_kernel<F32Tag, 8> : grouped_logpost_grad_kernel<F32Tag, 0>;
        else if (nchunks == 1)
            fn = grouped_narrow_kernel<F32Tag, 1>;
        else if (nchunks == 2)
            fn = grouped_narrow_kernel<F32Tag, 2>;
        else if (nchunks == 4)
            fn = grouped_narrow_kernel<F32Tag, 4>;
        else
            fn = grouped_narrow_kernel<F32Tag, 8>;
        break;
    case GLM_X_BF16:
        if (!narrow)
            fn = rows8 ? grouped_logpost_grad_kernel<BF16Tag, 8> : grouped_logpost_grad_kernel<BF16Tag, 0>;
        else if (nchunks == 1)
            fn = grouped_narrow_kernel<BF16Tag, 1>;
        else if (nchunks == 2)
            fn = grouped_narrow_kernel<BF16Tag, 2>;
        else
            fn = grouped_narrow_kernel<BF16Tag, 4>;
        break;
    case GLM_X_FP8E4M3:
        if (!narrow)
            fn = rows8 ? grouped_logpost_grad_kernel<FP8Tag, 8> : grouped_logpost_grad_kernel<FP8Tag, 0>;
        else if (nchunks == 1)
            fn = grouped_narrow_kernel<FP8Tag, 1>;
        else
            fn = grouped_narrow_kernel<FP8Tag, 2>;
        break;
    default: return GLM_ERR_UNSUPPORTED;
    }
    if (allow_max_dynamic_smem(reinterpret_cast<const void *>(fn)) != cudaSuccess)
        return GLM_ERR_CUDA;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)h->gr_grid);
    cfg.blockDim = dim3((unsigned)(h->gr_warps * 32));
    cfg.dynamicSmemBytes = (size_t)smem;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    if (cudaLaunchKernelEx(&cfg, fn, prm) != cudaSuccess)
        return GLM_ERR_CUDA;
    return GLM_OK;
}


// Launch-shape autotuner for the grouped pass: times every feasible
// (kernel variant, warps per CTA, 32-row units per slot, slots per ring, CTAs
// per SM) on the caller's own inputs and keeps the fastest in the handle.
glm_status_t autotune_grouped(glm_ctx *h, const void *X, const float *x_scale, const uint8_t *y,
                              const int64_t *group_off, int G, const float *beta, const float *mu,
                              double tau, double *f_out, float *g_out, cudaStream_t s, int reps)
{
    if (!h->gr_acc || h->gr_warps == 0)
        return GLM_ERR_UNSUPPORTED;
    const int es = h->elem_bytes;
    const int epc = 16 / es;
    const int pcue = ((h->d.p + epc - 1) / epc) * epc;
    const int row_bytes = h->d.ld * es;
    const bool narrow_ok = grouped_nch(h->d.p, epc) > 0;
    cudaEvent_t e0, e1;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess)
        return GLM_ERR_CUDA;
    const int save[5] = {h->gr_narrow, h->gr_warps, h->gr_units, h->gr_stages, h->gr_grid};
    int best[5] = {save[0], save[1], save[2], save[3], save[4]};
    float best_ms = 1e30f;
    glm_status_t st = GLM_OK;
    for (int nar = 0; nar <= (narrow_ok ? 1 : 0) && st == GLM_OK; ++nar) {
        const int wmax = (nar ? kNarrowMaxThreads : kGroupedMaxThreads) / 32;
        const int wc[4] = {4, 8, 12, 16};
        for (int wi = 0; wi < 4 && st == GLM_OK; ++wi) {
            const int warps = wc[wi];
            if (warps > wmax)
                continue;
            for (int units = 1; units <= (nar ? 4 : 1) && st == GLM_OK; units <<= 1) {
                for (int per_sm = 1; per_sm <= 2 && st == GLM_OK; ++per_sm) {
                    const int budget = kSmemOptinBytes / per_sm - (per_sm > 1 ? 1024 : 0);
                    for (int stages = 2; stages <= 4 && st == GLM_OK; ++stages) {
                        if (grouped_smem(row_bytes, warps, stages, pcue, nar, units) > budget)
                            continue;
                        h->gr_narrow = nar;
                        h->gr_warps = warps;
                        h->gr_units = units;
                        h->gr_stages = stages;
                        h->gr_grid = h->sm_count * per_sm;
                        st = launch_grouped(h, X, x_scale, y, group_off, G, beta, mu, tau, f_out,
                                            g_out, s);
                        if (st != GLM_OK)
                            break;
                        cudaEventRecord(e0, s);
                        for (int r = 0; r < reps && st == GLM_OK; ++r)
                            st = launch_grouped(h, X, x_scale, y, group_off, G, beta, mu, tau,
                                                f_out, g_out, s);
                        cudaEventRecord(e1, s);
                        if (cudaEventSynchronize(e1) != cudaSuccess) {
                            st = GLM_ERR_CUDA;
                            break;
                        }
                        float ms = 0.0f;
                        cudaEventElapsedTime(&ms, e0, e1);
                        if (st == GLM_OK && ms < best_ms) {
                            best_ms = ms;
                            best[0] = nar;
                            best[1] = warps;
                            best[2] = units;
                            best[3] = stages;
                            best[4] = h->gr_grid;
                        }
                    }
                }
            }
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    const int *use = (st == GLM_OK) ? best : save;
    h->gr_narrow = use[0];
    h->gr_warps = use[1];
    h->gr_units = use[2];
    h->gr_stages = use[3];
    h->gr_grid = use[4];
    return st;
}

}  // namespace glm

// Explicit launch shapes: the autotuner's candidate space, validated the same
// way (variant, warps per CTA, units per slot, ring slots, CTAs per SM).
extern "C" glm_status_t glm_grouped_set_shape(glm_handle_t h, int32_t variant, int32_t warps,
                                              int32_t units, int32_t stages, int32_t ctas_per_sm)
{
    using namespace glm;
    if (!h)
        return GLM_ERR_INVALID_ARG;
    if (!h->gr_acc || h->gr_warps == 0)
        return GLM_ERR_UNSUPPORTED;
    const int es = h->elem_bytes;
    const int epc = 16 / es;
    const int pcue = ((h->d.p + epc - 1) / epc) * epc;
    const bool narrow_ok = grouped_nch(h->d.p, epc) > 0;
    if (variant < 0 || variant > 1 || (variant == 1 && !narrow_ok))
        return GLM_ERR_INVALID_ARG;
    const int wmax = (variant ? kNarrowMaxThreads : kGroupedMaxThreads) / 32;
    if ((warps != 4 && warps != 8 && warps != 12 && warps != 16) || warps > wmax)
        return GLM_ERR_INVALID_ARG;
    if (units != 1 && !(variant == 1 && (units == 2 || units == 4)))
        return GLM_ERR_INVALID_ARG;
    if (stages < 2 || stages > 4 || ctas_per_sm < 1 || ctas_per_sm > 2)
        return GLM_ERR_INVALID_ARG;
    const int budget = kSmemOptinBytes / ctas_per_sm - (ctas_per_sm > 1 ? 1024 : 0);
    if (grouped_smem(h->d.ld * es, warps, stages, pcue, variant, units) > budget)
        return GLM_ERR_UNSUPPORTED;
    h->gr_narrow = variant;
    h->gr_warps = warps;
    h->gr_units = units;
    h->gr_stages = stages;
    h->gr_grid = h->sm_count * ctas_per_sm;
    return GLM_OK;
}

extern "C" glm_status_t glm_grouped_get_shape(glm_handle_t h, int32_t *variant, int32_t *warps,
                                              int32_t *units, int32_t *stages,
                                              int32_t *ctas_per_sm)
{
    if (!h)
        return GLM_ERR_INVALID_ARG;
    if (!h->gr_acc || h->gr_warps == 0)
        return GLM_ERR_UNSUPPORTED;
    if (variant)
        *variant = h->gr_narrow;
    if (warps)
        *warps = h->gr_warps;
    if (units)
        *units = h->gr_units;
    if (stages)
        *stages = h->gr_stages;
    if (ctas_per_sm)
        *ctas_per_sm = h->sm_count > 0 ? h->gr_grid / h->sm_count : 0;
    return GLM_OK;
}
