// Gibbs sweeps of univariate slice sampling with the differential update of
// X beta, §3.4.4: changing one coefficient beta_k by d changes X beta by
// d X_k, so with eta = X beta kept on the device an evaluation of the
// log-posterior along coordinate k reads only column k of X (X stored
// column-major) instead of all of X. Each coordinate is updated by Neal's
// slice sampler (stepping out with width w and at most m steps, then
// shrinkage), which needs several evaluations of that conditional.
//
// glm_slice_run is one cooperative launch (one CTA per SM, all resident) for
// all sweeps. Each CTA owns a block of rows and keeps their eta and y in
// shared memory for the whole run; column k of its rows arrives by a TMA
// bulk copy (double-buffered: column k+1 loads while k is sampled). An
// evaluation pass computes, for up to 16 candidate values of beta_k at once
// (all the stepping-out points of an update go in one pass), the CTA's sum
// of log-likelihood terms ell(eta_n + (x - beta_k) x_nk); the CTAs meet at a
// grid barrier (a counter with a bounded wait), after which every CTA adds
// the per-CTA sums in the same fixed order and so takes the same stepping-out
// and shrinkage decisions without a second barrier. An accepted move updates
// eta in shared memory (each CTA its own rows) and is written back at the end.
#include <cmath>
#include <cstring>
#include <new>

#include "glm_internal.cuh"

struct glm_slice {
    glm_slice_desc_t d;
    int device;
    int sm_count;
    int grid;                  // CTAs of the cooperative launch
    int rows_max;              // rows per CTA (multiple of 4)
    int smem_bytes;
    void *ws;
    double *part;              // 2 x grid x kSliceMaxCand pass partials
    double *part1;             // standalone evaluation: blocks x kSliceMaxCand
    unsigned *counter;         // grid-barrier arrivals
    unsigned *abort_flag;
    unsigned *status;
};

namespace glm {

constexpr int kSliceThreads = 512;
constexpr int kSliceMaxCand = 16;          // candidates per evaluation pass
constexpr int kSliceMaxShrink = 64;
constexpr int kSliceEvalBlocks = 1024;     // standalone evaluation grid
constexpr int kSliceSpecDefault = 2;       // shrinkage proposals per pass
constexpr unsigned kGridSpinLimit = 1u << 22;
static_assert(kSliceMaxShrink + 2 <= kSliceThreads, "one random number per thread");

struct SliceParams {
    const float *Xt;           // column-major, column k at Xt + k * ld
    const uint8_t *y;
    float *eta;                // N, in/out
    float *beta;               // P, in/out
    double *f_state;           // in/out
    int init_f;
    int64_t N;
    int P;
    int64_t ld;
    int n_sweeps;
    int m;
    int s_max;
    int spec;
    float w;
    double inv_s2;
    double prior_const;
    const double *log_u0;      // n_sweeps x P
    const float *uni;          // n_sweeps x P x (2 + s_max)
    float *xk_out;             // n_sweeps x P (or null)
    double *gk_out;
    int *nsh_out;
    double *part;
    unsigned *counter;
    unsigned *abort_flag;
    unsigned *status;
    int rows_max;
};

namespace sl {

__device__ __forceinline__ unsigned ld_acquire(const unsigned *p)
{
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ void red_add_release(unsigned *p, unsigned v)
{
    asm volatile("red.release.gpu.global.add.u32 [%0], %1;" : : "l"(p), "r"(v) : "memory");
}

// log-likelihood term y t - softplus(t), overflow-free, fast exp/log
__device__ __forceinline__ float ell(float t, float yv)
{
    const float e = __expf(-fabsf(t));
    return fmaf(yv, t, -fmaxf(t, 0.0f)) - __logf(1.0f + e);
}

}  // namespace sl

// The rows of CTA b: [rb(b), rb(b+1)), block starts multiples of 4 (16-byte
// aligned column segments for the bulk copies).
__host__ __device__ inline int64_t slice_row_begin(int64_t N, int grid, int b)
{
    if (b >= grid)
        return N;
    const int64_t r = (N * b) / grid;
    return (r / 4) * 4;
}

struct SliceLayout {
    int eta_off, y_off, x_off, misc_off, total;
};

__host__ __device__ inline SliceLayout slice_layout(int rows_max, int P, int s_max)
{
    SliceLayout L;
    int o = 0;
    L.x_off = o;
    o += 2 * rows_max * 4;                 // two column buffers
    L.eta_off = o;
    o += rows_max * 4;
    L.y_off = o;
    o += (rows_max + 15) / 16 * 16;
    L.misc_off = o;
    // misc: beta (P floats), warp sums (warps x 16 floats), candidates (16 floats),
    // g values (16 doubles), stream buffers 2 x (2 + s_max) floats + 2 doubles,
    // control words, two mbarriers
    o += ((P * 4 + 15) / 16) * 16 + (kSliceThreads / 32) * kSliceMaxCand * 4 + kSliceMaxCand * 4 +
         kSliceMaxCand * 8 + 2 * (((2 + s_max) * 4 + 15) / 16 * 16 + 16) + 256 + 64;
    L.total = o + 128;
    return L;
}

// Candidates per evaluation pass rounded up to a compiled size.
__device__ __forceinline__ int slice_mc(int M)
{
    return M <= 4 ? M : M <= 8 ? 8 : 16;
}

// This thread's sums of ell(eta_i + d[c] x_i) over rows i = tid, tid + NT, ...
// for the MC candidate shifts d[0..MC) (MC a compile-time size: candidates
// beyond M are padding and their sums are not used). Few candidates leave
// little work per row, so those loops are unrolled over rows to keep several
// rows' loads and exp/log in flight.
template <int MC, int U>
__device__ __forceinline__ void slice_rows(const float *xb, const float *etas, const uint8_t *ys,
                                           int R, const float *d, float *acc)
{
#pragma unroll
    for (int c = 0; c < MC; ++c)
        acc[c] = 0.0f;
#pragma unroll U
    for (int i = threadIdx.x; i < R; i += kSliceThreads) {
        const float x = xb[i], e = etas[i], yv = (float)ys[i];
#pragma unroll
        for (int c = 0; c < MC; ++c)
            acc[c] += sl::ell(fmaf(d[c], x, e), yv);
    }
}

__global__ void __launch_bounds__(kSliceThreads, 1) slice_run_kernel(SliceParams p)
{
    constexpr int NT = kSliceThreads;
    constexpr unsigned FULL = 0xFFFFFFFFu;
    extern __shared__ __align__(128) uint8_t smem_raw[];
    uint8_t *smem = smem_raw + ((128u - (ptx::smem_u32(smem_raw) & 127u)) & 127u);
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int b = blockIdx.x, G = gridDim.x;
    const SliceLayout L = slice_layout(p.rows_max, p.P, p.s_max);
    float *xs = reinterpret_cast<float *>(smem + L.x_off);              // [2][rows_max]
    float *etas = reinterpret_cast<float *>(smem + L.eta_off);
    uint8_t *ys = smem + L.y_off;
    uint8_t *misc = smem + L.misc_off;
    float *bs = reinterpret_cast<float *>(misc);                        // beta
    int o = ((p.P * 4 + 15) / 16) * 16;
    float *wsum = reinterpret_cast<float *>(misc + o);                  // [warps][16]
    o += (NT / 32) * kSliceMaxCand * 4;
    float *cand = reinterpret_cast<float *>(misc + o);                  // [16] candidate values
    o += kSliceMaxCand * 4;
    double *gval = reinterpret_cast<double *>(misc + o);                // [16]
    o += kSliceMaxCand * 8;
    const int sb = ((2 + p.s_max) * 4 + 15) / 16 * 16 + 16;            // 16-byte multiple
    uint8_t *stream_buf = misc + o;                                     // [2][sb]
    o += 2 * sb;
    int *ctl = reinterpret_cast<int *>(misc + o);                       // control words
    double *dctl = reinterpret_cast<double *>(misc + o + 64);
    o += 256;
    uint64_t *xbar = reinterpret_cast<uint64_t *>(misc + o);            // [2]

    const int64_t r0 = slice_row_begin(p.N, G, b);
    const int64_t r1 = slice_row_begin(p.N, G, b + 1);
    const int R = (int)(r1 - r0);
    const unsigned col_bytes = (unsigned)(((R + 3) / 4) * 16);   // rounded up: ld >= N rounded

    // own rows' eta and labels into shared memory; coefficients
    for (int i = tid; i < R; i += NT) {
        etas[i] = p.eta[r0 + i];
        ys[i] = p.y[r0 + i];
    }
    for (int j = tid; j < p.P; j += NT)
        bs[j] = p.beta[j];
    if (tid == 0) {
        ptx::mbar_init(&xbar[0], 1);
        ptx::mbar_init(&xbar[1], 1);
        ptx::fence_mbar_init();
    }
    __syncthreads();

    const int n_up = p.n_sweeps * p.P;            // coordinate updates of this run
    const uint64_t policy = ptx::policy_evict_first();
    auto issue_col = [&](int u) {                 // column of update u into buffer u & 1
        const int k = u % p.P;
        uint64_t *bar = &xbar[u & 1];
        ptx::mbar_arrive_expect_tx(bar, col_bytes);
        ptx::bulk_g2s(xs + (u & 1) * p.rows_max, p.Xt + (int64_t)k * p.ld + r0, col_bytes, bar,
                      policy);
    };
    auto load_stream = [&](int u) {               // random numbers of update u
        uint8_t *dst = stream_buf + (u & 1) * sb;
        double *lu = reinterpret_cast<double *>(dst);
        float *un = reinterpret_cast<float *>(dst + 16);
        if (tid == 0)
            *lu = p.log_u0[u];
        for (int j = tid; j < 2 + p.s_max; j += NT)
            un[j] = p.uni[(int64_t)u * (2 + p.s_max) + j];
    };
    bool inflight[2] = {false, false};            // a column copy not yet waited for
    if ((n_up > 0 || p.init_f) && R > 0) {
        if (tid == 0)
            issue_col(0);
        inflight[0] = true;
    }
    if (n_up > 0)
        load_stream(0);

    unsigned pass = 0;                            // grid barriers so far
    bool alive = true;
    // One evaluation pass: the log-posterior at beta with beta_k replaced by
    // x0 + cand[c] for c < M (S2 = |beta|^2 without coordinate k), into
    // gval[]. Uses column buffer xb. Returns false if the run aborted.
    // Candidates are absolute values of beta_k; eta moves by (x - beta_k) X_k.
    auto eval_pass = [&](int M, const float *xb, double S2_wo_k, float x0) -> bool {
        float acc[kSliceMaxCand], dl[kSliceMaxCand];
#pragma unroll
        for (int c = 0; c < kSliceMaxCand; ++c)
            dl[c] = c < M ? __fsub_rn(cand[c], x0) : 0.0f;
        const int MP = slice_mc(M);
        if (MP == 1)
            slice_rows<1, 4>(xb, etas, ys, R, dl, acc);
        else if (MP == 2)
            slice_rows<2, 4>(xb, etas, ys, R, dl, acc);
        else if (MP == 3)
            slice_rows<3, 2>(xb, etas, ys, R, dl, acc);
        else if (MP == 4)
            slice_rows<4, 2>(xb, etas, ys, R, dl, acc);
        else if (MP == 8)
            slice_rows<8, 1>(xb, etas, ys, R, dl, acc);
        else
            slice_rows<16, 1>(xb, etas, ys, R, dl, acc);
#pragma unroll
        for (int c = 0; c < kSliceMaxCand; ++c) {
            if (c < MP) {
                float v = acc[c];
#pragma unroll
                for (int mm = 16; mm > 0; mm >>= 1)
                    v += __shfl_xor_sync(FULL, v, mm);
                if (lane == 0 && c < M)
                    wsum[warp * kSliceMaxCand + c] = v;
            }
        }
        __syncthreads();
        double *part = p.part + (size_t)(pass & 1u) * G * kSliceMaxCand;
        if (tid < M) {
            double v = 0.0;
            for (int w2 = 0; w2 < NT / 32; ++w2)
                v += (double)wsum[w2 * kSliceMaxCand + tid];
            part[(size_t)b * kSliceMaxCand + tid] = v;
        }
        // grid barrier: arrivals counted, bounded wait, abort flag
        __syncthreads();
        if (tid == 0) {
            // release: the partials written before the block barrier are
            // visible to any CTA whose acquire load sees this arrival
            sl::red_add_release(p.counter, 1u);
            const unsigned target = (pass + 1u) * (unsigned)G;
            unsigned it = 0;
            int ok = 1;
            while (sl::ld_acquire(p.counter) < target) {
                // the abort flag is polled every 64th round: one load per round
                if ((it & 63u) == 63u && sl::ld_acquire(p.abort_flag) != 0u) {
                    ok = 0;
                    break;
                }
                if (++it > kGridSpinLimit) {
                    atomicOr(p.status, kDevTimeout);
                    atomicExch(p.abort_flag, 1u);
                    ok = 0;
                    break;
                }
                __nanosleep(32);
            }
            ctl[0] = ok;                          // the acquire load above orders the reads below
        }
        __syncthreads();
        ++pass;
        if (!ctl[0])
            return false;
        // warp c sums the CTAs' partials of candidate c: lane-strided sums,
        // then a shuffle tree (the same fixed order in every CTA)
        for (int c = warp; c < M; c += NT / 32) {
            double v = 0.0;
            for (int q = lane; q < G; q += 32)
                v += __ldcg(part + (size_t)q * kSliceMaxCand + c);
#pragma unroll
            for (int mm = 16; mm > 0; mm >>= 1)
                v += __shfl_xor_sync(FULL, v, mm);
            if (lane == 0) {
                const double x = (double)cand[c];
                gval[c] = v - 0.5 * p.inv_s2 * (S2_wo_k + x * x) - p.prior_const;
            }
        }
        __syncthreads();
        return true;
    };

    // |beta|^2 and the current log-posterior
    if (tid == 0) {
        double s2 = 0.0;
        for (int j = 0; j < p.P; ++j)
            s2 += (double)bs[j] * (double)bs[j];
        dctl[0] = s2;
        dctl[1] = *p.f_state;
    }
    __syncthreads();
    if (p.init_f) {
        // the current point itself: candidate beta_0 on coordinate 0
        if (tid == 0)
            cand[0] = bs[0];
        __syncthreads();
        const double b0 = (double)bs[0];
        if (R > 0 && !ptx::mbar_wait_bounded(&xbar[0], 0u, kSpinLimit) && tid == 0) {
            atomicOr(p.status, kDevTimeout);
            atomicExch(p.abort_flag, 1u);
        }
        alive = eval_pass(1, xs, dctl[0] - b0 * b0, bs[0]);
        if (tid == 0 && alive)
            dctl[1] = gval[0];
        __syncthreads();
    }

    unsigned col_uses[2] = {0u, 0u};
    for (int u = 0; u < n_up && alive; ++u) {
        const int s = u / p.P;
        const int k = u - s * p.P;
        const int buf = u & 1;
        // column k has landed; prefetch the next update's column and numbers
        if (R > 0 && !ptx::mbar_wait_bounded(&xbar[buf], col_uses[buf] & 1u, kSpinLimit)) {
            if (tid == 0) {
                atomicOr(p.status, kDevTimeout);
                atomicExch(p.abort_flag, 1u);
            }
        }
        ++col_uses[buf];
        inflight[buf] = false;
        __syncthreads();
        if (u + 1 < n_up && R > 0) {
            if (tid == 0)
                issue_col(u + 1);
            inflight[buf ^ 1] = true;
        }
        // the next update's random numbers: loaded into registers now, stored
        // to shared memory after this update's passes (latency hidden)
        double nxt_lu = 0.0;
        float nxt_un = 0.0f;
        if (u + 1 < n_up) {
            if (tid == 0)
                nxt_lu = __ldg(p.log_u0 + u + 1);
            if (tid < 2 + p.s_max)
                nxt_un = __ldg(p.uni + (int64_t)(u + 1) * (2 + p.s_max) + tid);
        }
        const float *xb = xs + buf * p.rows_max;
        const uint8_t *sbuf = stream_buf + buf * sb;
        const double log_u0 = *reinterpret_cast<const double *>(sbuf);
        const float *un = reinterpret_cast<const float *>(sbuf + 16);

        // slice level, initial interval and stepping-out split (FP32, each
        // operation rounded separately)
        const float x0 = bs[k];
        const double g0 = dctl[1];
        const double log_y = g0 + log_u0;
        const double S2k = dctl[0] - (double)x0 * (double)x0;
        const float w = p.w;
        const float L0 = __fsub_rn(x0, __fmul_rn(w, un[0]));
        const float R0 = __fadd_rn(L0, w);
        const int J = (int)floorf(__fmul_rn((float)p.m, un[1]));
        const int K = (p.m - 1) - J;
        // stepping-out candidates: L_j (j < J) then R_j (j < K), in one pass
        if (tid == 0) {
            int c = 0;
            for (int j = 0; j < J; ++j)
                cand[c++] = __fsub_rn(L0, __fmul_rn((float)j, w));
            for (int j = 0; j < K; ++j)
                cand[c++] = __fadd_rn(R0, __fmul_rn((float)j, w));
        }
        __syncthreads();
        float Lf = L0, Rf = R0;
        if (J + K > 0) {
            alive = eval_pass(J + K, xb, S2k, x0);
            if (!alive)
                break;
            // apply the sequential stepping-out rule to the evaluated values
            int j = 0;
            for (; j < J; ++j)
                if (!(log_y < gval[j]))
                    break;
            Lf = __fsub_rn(L0, __fmul_rn((float)j, w));
            int kk = 0;
            for (; kk < K; ++kk)
                if (!(log_y < gval[J + kk]))
                    break;
            Rf = __fadd_rn(R0, __fmul_rn((float)kk, w));
        }
        // shrinkage, spec proposals per pass: proposal q of a pass assumes
        // proposals 0..q-1 rejected (each rejection only moves the interval
        // end on its own side), so the first accepted one in order is the
        // sequential result
        float x1 = x0;
        double g1 = g0;
        int nsh = p.s_max;
        for (int t = 0; t < p.s_max && alive;) {
            const int D = min(p.spec, p.s_max - t);
            __syncthreads();                  // the previous pass's cand[] is read
            if (tid == 0) {
                float Lc = Lf, Rc = Rf;
                for (int q = 0; q < D; ++q) {
                    const float xc = __fadd_rn(Lc, __fmul_rn(un[2 + t + q], __fsub_rn(Rc, Lc)));
                    cand[q] = xc;
                    if (xc < x0)
                        Lc = xc;
                    else
                        Rc = xc;
                }
            }
            __syncthreads();
            alive = eval_pass(D, xb, S2k, x0);
            if (!alive)
                break;
            bool acc_ok = false;
            for (int q = 0; q < D; ++q) {
                const float xc = cand[q];
                if (log_y < gval[q]) {
                    x1 = xc;
                    g1 = gval[q];
                    nsh = t + q;
                    acc_ok = true;
                    break;
                }
                if (xc < x0)
                    Lf = xc;
                else
                    Rf = xc;
            }
            if (acc_ok)
                break;
            t += D;
        }
        if (!alive)
            break;
        // materialize: eta += (x1 - x0) X_k on this CTA's rows
        const float dlt = __fsub_rn(x1, x0);
        if (dlt != 0.0f)
            for (int i = tid; i < R; i += NT)
                etas[i] = fmaf(dlt, xb[i], etas[i]);
        if (u + 1 < n_up) {
            uint8_t *dst = stream_buf + (buf ^ 1) * sb;
            if (tid == 0)
                *reinterpret_cast<double *>(dst) = nxt_lu;
            if (tid < 2 + p.s_max)
                reinterpret_cast<float *>(dst + 16)[tid] = nxt_un;
        }
        __syncthreads();
        if (tid == 0) {
            bs[k] = x1;
            dctl[0] = S2k + (double)x1 * (double)x1;
            dctl[1] = g1;
            if (b == 0) {
                if (p.xk_out)
                    p.xk_out[u] = x1;
                if (p.gk_out)
                    p.gk_out[u] = g1;
                if (p.nsh_out)
                    p.nsh_out[u] = nsh;
            }
        }
        __syncthreads();
    }
    // a column copy still in flight (after an abort) lands before the CTA exits
    __syncthreads();
    if (tid == 0) {
        for (int q = 0; q < 2; ++q)
            if (inflight[q])
                ptx::mbar_wait_bounded(&xbar[q], col_uses[q] & 1u, kSpinLimit);
    }
    for (int i = tid; i < R; i += NT)
        p.eta[r0 + i] = etas[i];
    if (b == 0) {
        for (int j = tid; j < p.P; j += NT)
            p.beta[j] = bs[j];
        if (tid == 0)
            *p.f_state = dctl[1];
    }
}

// eta = X beta from the column-major X (k ascending, FP32 accumulation).
__global__ void slice_eta_kernel(const float *__restrict__ Xt, int64_t ld, int64_t N, int P,
                                 const float *__restrict__ beta, float *__restrict__ eta)
{
    for (int64_t n = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; n < N;
         n += (int64_t)gridDim.x * blockDim.x) {
        float s = 0.0f;
        for (int k = 0; k < P; ++k)
            s = fmaf(__ldg(beta + k), __ldg(Xt + (int64_t)k * ld + n), s);
        eta[n] = s;
    }
}

// Standalone evaluation along coordinate k: per-block sums of
// ell(eta_n + (x_c - beta_k) x_nk) for the M candidates.
__global__ void slice_eval_kernel(const float *__restrict__ Xt, int64_t ld, int64_t N,
                                  const uint8_t *__restrict__ y, const float *__restrict__ eta,
                                  const float *__restrict__ beta, int k,
                                  const float *__restrict__ xc, int M, double *__restrict__ part)
{
    __shared__ float wsum[8][kSliceMaxCand];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    float d[kSliceMaxCand], acc[kSliceMaxCand];
    const float bk = beta[k];
#pragma unroll
    for (int c = 0; c < kSliceMaxCand; ++c) {
        d[c] = c < M ? __fsub_rn(xc[c], bk) : 0.0f;
        acc[c] = 0.0f;
    }
    const float *col = Xt + (int64_t)k * ld;
    for (int64_t n = (int64_t)blockIdx.x * blockDim.x + tid; n < N;
         n += (int64_t)gridDim.x * blockDim.x) {
        const float x = __ldg(col + n), e = __ldg(eta + n), yv = (float)__ldg(y + n);
#pragma unroll
        for (int c = 0; c < kSliceMaxCand; ++c)
            if (c < M)
                acc[c] += sl::ell(fmaf(d[c], x, e), yv);
    }
#pragma unroll
    for (int c = 0; c < kSliceMaxCand; ++c) {
        float v = acc[c];
#pragma unroll
        for (int mm = 16; mm > 0; mm >>= 1)
            v += __shfl_xor_sync(0xFFFFFFFFu, v, mm);
        if (lane == 0)
            wsum[warp][c] = v;
    }
    __syncthreads();
    if (tid < M) {
        double v = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w)
            v += (double)wsum[w][tid];
        part[(size_t)blockIdx.x * kSliceMaxCand + tid] = v;
    }
}

__global__ void slice_eval_finish_kernel(const double *__restrict__ part, int blocks, int M,
                                         const float *__restrict__ beta, int P, int k,
                                         const float *__restrict__ xc, double inv_s2,
                                         double prior_const, double *__restrict__ f_out)
{
    const int c = threadIdx.x;
    if (c >= M)
        return;
    double v = 0.0;
    for (int q = 0; q < blocks; ++q)
        v += part[(size_t)q * kSliceMaxCand + c];
    double s2 = 0.0;
    for (int j = 0; j < P; ++j) {
        const double bj = j == k ? (double)xc[c] : (double)beta[j];
        s2 += bj * bj;
    }
    f_out[c] = v - 0.5 * inv_s2 * s2 - prior_const;
}

}  // namespace glm

using namespace glm;

extern "C" {

glm_status_t glm_slice_create(const glm_slice_desc_t *desc, glm_slice_t *out)
{
    if (!out)
        return GLM_ERR_INVALID_ARG;
    *out = nullptr;
    if (!desc)
        return GLM_ERR_INVALID_ARG;
    const glm_slice_desc_t d = *desc;
    if (d.n_rows < 1 || d.p < 1 || d.ld < d.n_rows || d.ld % 4 != 0 || d.m < 1 ||
        d.m > kSliceMaxCand || d.s_max < 1 || d.s_max > kSliceMaxShrink || !(d.w > 0.0f) ||
        !std::isfinite(d.w) || !(d.prior_sigma > 0.0) || !std::isfinite(d.prior_sigma) ||
        d.device < 0 || d.spec < 0 || d.spec > kSliceMaxCand)
        return GLM_ERR_INVALID_ARG;
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev == 0) {
        cudaGetLastError();
        return GLM_ERR_NO_DEVICE;
    }
    if (d.device >= ndev || cudaSetDevice(d.device) != cudaSuccess)
        return GLM_ERR_INVALID_ARG;
    int major = 0, minor = 0, sms = 0, coop = 0;
    cudaDeviceGetAttribute(&major, cudaDevAttrComputeCapabilityMajor, d.device);
    cudaDeviceGetAttribute(&minor, cudaDevAttrComputeCapabilityMinor, d.device);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, d.device);
    cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, d.device);
    if (major != 10 || minor != 3 || !coop)
        return GLM_ERR_NO_DEVICE;
    glm_slice *s = new (std::nothrow) glm_slice;
    if (!s)
        return GLM_ERR_OOM;
    std::memset(s, 0, sizeof(*s));
    s->d = d;
    s->device = d.device;
    s->sm_count = sms;
    s->grid = sms;
    int rmax = 0;
    for (int b = 0; b < s->grid; ++b) {
        const int64_t r = slice_row_begin(d.n_rows, s->grid, b + 1) -
                          slice_row_begin(d.n_rows, s->grid, b);
        if (r > rmax)
            rmax = (int)r;
    }
    s->rows_max = (rmax + 3) / 4 * 4;
    const SliceLayout L = slice_layout(s->rows_max, d.p, d.s_max);
    if (L.total > kSmemDynamicBudget) {
        delete s;
        return GLM_ERR_UNSUPPORTED;        // rows per CTA beyond shared memory
    }
    s->smem_bytes = L.total;
    const size_t part_bytes = (size_t)2 * s->grid * kSliceMaxCand * sizeof(double);
    const size_t part1_bytes = (size_t)kSliceEvalBlocks * kSliceMaxCand * sizeof(double);
    const size_t total = part_bytes + part1_bytes + 256;
    if (cudaMalloc(&s->ws, total) != cudaSuccess) {
        cudaGetLastError();
        delete s;
        return GLM_ERR_OOM;
    }
    uint8_t *base = static_cast<uint8_t *>(s->ws);
    s->part = reinterpret_cast<double *>(base);
    s->part1 = reinterpret_cast<double *>(base + part_bytes);
    s->counter = reinterpret_cast<unsigned *>(base + part_bytes + part1_bytes);
    s->abort_flag = s->counter + 1;
    s->status = s->counter + 2;
    if (cudaMemset(s->ws, 0, total) != cudaSuccess) {
        cudaFree(s->ws);
        delete s;
        return GLM_ERR_CUDA;
    }
    *out = s;
    return GLM_OK;
}

glm_status_t glm_slice_destroy(glm_slice_t s)
{
    if (!s)
        return GLM_OK;
    cudaSetDevice(s->device);
    cudaFree(s->ws);
    delete s;
    return GLM_OK;
}

static bool al(const void *p, unsigned a) { return (reinterpret_cast<uintptr_t>(p) % a) == 0; }

glm_status_t glm_slice_eta(glm_slice_t s, const float *Xt, const float *beta, float *eta,
                           glm_stream_t stream)
{
    if (!s || !Xt || !beta || !eta || !al(Xt, 16))
        return GLM_ERR_INVALID_ARG;
    const int64_t N = s->d.n_rows;
    int blocks = (int)((N + 255) / 256);
    if (blocks > s->sm_count * 8)
        blocks = s->sm_count * 8;
    slice_eta_kernel<<<blocks, 256, 0, reinterpret_cast<cudaStream_t>(stream)>>>(
        Xt, s->d.ld, N, s->d.p, beta, eta);
    return cudaGetLastError() == cudaSuccess ? GLM_OK : GLM_ERR_CUDA;
}

glm_status_t glm_slice_coord_logpost(glm_slice_t s, const float *Xt, const uint8_t *y,
                                     const float *eta, const float *beta, int32_t k,
                                     const float *x, int32_t M, double *f_out,
                                     glm_stream_t stream)
{
    if (!s || !Xt || !y || !eta || !beta || !x || !f_out || k < 0 || k >= s->d.p || M < 1 ||
        M > kSliceMaxCand || !al(Xt, 16) || !al(f_out, 8))
        return GLM_ERR_INVALID_ARG;
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    const int64_t N = s->d.n_rows;
    int blocks = (int)((N + 255) / 256);
    if (blocks > kSliceEvalBlocks)
        blocks = kSliceEvalBlocks;
    const double s2 = s->d.prior_sigma * s->d.prior_sigma;
    slice_eval_kernel<<<blocks, 256, 0, st>>>(Xt, s->d.ld, N, y, eta, beta, k, x, M, s->part1);
    slice_eval_finish_kernel<<<1, 32, 0, st>>>(s->part1, blocks, M, beta, s->d.p, k, x, 1.0 / s2,
                                               0.5 * s->d.p * std::log(2.0 * M_PI * s2), f_out);
    return cudaGetLastError() == cudaSuccess ? GLM_OK : GLM_ERR_CUDA;
}

glm_status_t glm_slice_run(glm_slice_t s, const float *Xt, const uint8_t *y, float *eta,
                           float *beta, double *f_state, int32_t init_f, int32_t n_sweeps,
                           const double *log_u0, const float *uni, float *xk_out,
                           double *gk_out, int32_t *nshrink_out, glm_stream_t stream)
{
    if (!s || !Xt || !y || !eta || !beta || !f_state || n_sweeps < 0 ||
        (n_sweeps > 0 && (!log_u0 || !uni)) || !al(Xt, 16) || !al(f_state, 8) ||
        !al(log_u0 ? (const void *)log_u0 : (const void *)f_state, 8))
        return GLM_ERR_INVALID_ARG;
    // passes: the initial one plus at most 1 + s_max per coordinate update;
    // the arrival counter must not wrap
    const int64_t max_passes = 1 + (int64_t)n_sweeps * s->d.p * (1 + s->d.s_max);
    if (max_passes * s->grid >= 0xFFFFFFFFLL)
        return GLM_ERR_UNSUPPORTED;
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    SliceParams p;
    std::memset(&p, 0, sizeof(p));
    p.Xt = Xt;
    p.y = y;
    p.eta = eta;
    p.beta = beta;
    p.f_state = f_state;
    p.init_f = init_f ? 1 : 0;
    p.N = s->d.n_rows;
    p.P = s->d.p;
    p.ld = s->d.ld;
    p.n_sweeps = n_sweeps;
    p.m = s->d.m;
    p.s_max = s->d.s_max;
    p.spec = s->d.spec > 0 ? s->d.spec : kSliceSpecDefault;
    p.w = s->d.w;
    const double s2 = s->d.prior_sigma * s->d.prior_sigma;
    p.inv_s2 = 1.0 / s2;
    p.prior_const = 0.5 * s->d.p * std::log(2.0 * M_PI * s2);
    p.log_u0 = log_u0;
    p.uni = uni;
    p.xk_out = xk_out;
    p.gk_out = gk_out;
    p.nsh_out = nshrink_out;
    p.part = s->part;
    p.counter = s->counter;
    p.abort_flag = s->abort_flag;
    p.status = s->status;
    p.rows_max = s->rows_max;
    // arrivals and the abort flag start at zero for each run
    if (cudaMemsetAsync(s->counter, 0, 2 * sizeof(unsigned), st) != cudaSuccess)
        return GLM_ERR_CUDA;
    auto fn = &slice_run_kernel;
    if (allow_max_dynamic_smem(reinterpret_cast<const void *>(fn)) != cudaSuccess)
        return GLM_ERR_CUDA;
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, kSliceThreads,
                                                      (size_t)s->smem_bytes) != cudaSuccess ||
        per_sm < 1)
        return GLM_ERR_UNSUPPORTED;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)s->grid);
    cfg.blockDim = dim3(kSliceThreads);
    cfg.dynamicSmemBytes = (size_t)s->smem_bytes;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    if (cudaLaunchKernelEx(&cfg, fn, p) != cudaSuccess)
        return GLM_ERR_CUDA;
    return GLM_OK;
}

glm_status_t glm_slice_sync(glm_slice_t s, glm_stream_t stream)
{
    if (!s)
        return GLM_ERR_INVALID_ARG;
    if (cudaStreamSynchronize(reinterpret_cast<cudaStream_t>(stream)) != cudaSuccess)
        return GLM_ERR_CUDA;
    unsigned word = 0;
    if (cudaMemcpy(&word, s->status, sizeof(word), cudaMemcpyDeviceToHost) != cudaSuccess)
        return GLM_ERR_CUDA;
    if (word) {
        if (cudaMemset(s->status, 0, sizeof(unsigned)) != cudaSuccess)
            return GLM_ERR_CUDA;
        if (word & kDevTimeout)
            return GLM_ERR_TIMEOUT;
    }
    return GLM_OK;
}

}  // extern "C"
