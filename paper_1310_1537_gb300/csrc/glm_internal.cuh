// Internal declarations of the GB300 logistic-GLM library: the handle, the
// kernel parameter blocks and the inline-PTX primitives (mbarrier, bulk TMA
// copies) shared by the kernels. Not part of the public ABI.
#pragma once

#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <cstdint>
#include <cstddef>

#include "../../include/glm.h"

namespace glm {

// Device status word bits (atomicOr'ed by kernels, read by glm_sync).
constexpr unsigned kDevTimeout = 1u;

// Poll limit of every mbarrier wait in the streaming kernels. One failed
// try_wait suspends the thread for a bounded hardware interval, so this cap
// is far above any legitimate wait yet ends in well under a minute.
constexpr unsigned kSpinLimit = 1u << 24;

// Opt-in shared memory per block on sm_103 (227 KB), static and dynamic
// together, and the part of it the configurators leave for the kernels'
// static __shared__ arrays (at most 768 bytes in any kernel here).
constexpr int kSmemOptinBytes = 232448;
constexpr int kSmemStaticReserve = 1024;
constexpr int kSmemDynamicBudget = kSmemOptinBytes - kSmemStaticReserve;

constexpr int kFusedThreads = 256;
constexpr int kMaxStages = 8;

// ---------------------------------------------------------------------------
// Kernel parameter block of the fused CUDA-core pass (glm_fused.cu).
struct FusedParams {
    const void *X;
    const float *x_scale;      // FP8 column scales or nullptr
    const uint8_t *y;
    const float *beta;         // K x P (evaluation mode)
    int64_t N;
    int P;
    int ld;
    int K;                     // vectors in this launch (<= KC)
    int stages;
    int tile_rows;
    double inv_s2;             // 1 / s^2
    double prior_const;        // (P/2) log(2 pi s^2)
    unsigned long long *acc;   // KC x (P+1) fixed-point accumulators (fx::kLimbs each), zero
    unsigned *acc_flag;        // non-finite partial seen, returns to 0
    unsigned *ticket;          // completion counter, returns to 0
    unsigned *status;          // device status word
    double *f_out;             // K (may be null in RWM mode)
    float *g_out;              // K x P (may be null in RWM mode)
    // random-walk Metropolis step (rwm != 0)
    int rwm;
    float step;
    const float *z;            // K x P for this step
    const double *log_u;       // K
    float *state;              // K x P, updated by the last CTA
    double *f_state;           // K
    float *samples;            // K x P or null
    uint8_t *accept;           // K or null
    double *logpost;           // K or null
    int early_prefetch;        // stream X/y before the launch dependency resolves
    int srow;                  // staged row stride in shared memory, bytes
    int box_rows;              // > 0: rows arrive by 3-D tensor copies of this many rows
};

// Kernel parameter block of the grouped (hierarchical-Bayes) pass.
struct GroupedParams {
    const void *X;
    const float *x_scale;      // FP8 column scales or nullptr
    const uint8_t *y;
    const int64_t *off;        // G+1 row offsets
    int64_t N;                 // rows of X (bound on the offsets)
    int G;
    int P;
    int ld;
    int stages;                // slots per warp ring
    int units;                 // 32-row units per slot (narrow-row kernel)
    const float *beta;         // G x P
    const float *mu;           // P
    double inv_t2;             // 1 / tau^2
    double prior_const;        // (P/2) log(2 pi tau^2)
    unsigned long long *acc;   // G x (P+1) fixed-point accumulators, zero
    unsigned *gticket;         // G completion counters, zero
    unsigned *gflag;           // G non-finite flags, zero
    unsigned *status;
    double *f_out;             // G
    float *g_out;              // G x P
};

}  // namespace glm

// ---------------------------------------------------------------------------
// The handle.
struct glm_ctx {
    glm_desc_t d;
    int device;
    int sm_count;
    int elem_bytes;
    // fused CUDA-core kernel configuration
    int grid;
    int tile_rows;
    int split;
    int stages;
    int smem_bytes;
    int kc_max;                 // largest KC instantiation usable for this xtype
    int use_pdl;                // launch with programmatic stream serialization
    // Rows whose 16-byte chunk count is even are staged one zero chunk wider
    // (odd chunk stride: a quarter-warp reading 8 consecutive rows at the
    // same column hits 8 distinct bank groups), through a 3-D tensor map.
    int srow;                   // staged row stride in bytes
    int box_rows;               // rows per tensor copy (0: dense 1-D bulk copies)
    alignas(64) unsigned char fx_map[128];   // CUtensorMap of the last X seen
    const void *fx_map_ptr;
    // workspace
    void *ws;                   // one device allocation
    size_t ws_bytes;
    unsigned long long *acc;    // fixed-point cross-CTA accumulators
    unsigned *acc_flag;
    unsigned *ticket;
    unsigned *status;
    float *scratch;             // quantiser / misc scratch (P floats)
    // host-buffer entry point staging
    float *beta_stage;          // device K_max x P
    double *f_stage;            // device K_max
    float *g_stage;             // device K_max x P
    // tensor-core path
    int tc_enabled;
    int tc_min_k;
    int last_path;              // glm_path_t of the last glm_logpost_grad launched
    alignas(64) unsigned char tc_map[128];   // CUtensorMap of the last X seen
    const void *tc_map_ptr;
    double *tc_part_f;          // per-CTA f partials
    float *tc_part_g;           // per-CTA g partials
    // grouped (hierarchical) path: per-group accumulators, sized by g_max
    unsigned long long *gr_acc;
    unsigned *gr_ticket;
    unsigned *gr_flag;
    int gr_warps;               // warps per CTA
    int gr_stages;              // slots per warp ring
    int gr_units;               // 32-row units per slot
    int gr_narrow;              // 1: register-resident narrow-row kernel
    int gr_grid;
};

namespace glm {

// Launchers implemented in the kernel translation units.
glm_status_t launch_fused(glm_ctx *h, const FusedParams &p, int kc, cudaStream_t s);
glm_status_t fused_configure(glm_ctx *h);
glm_status_t launch_quantize(glm_ctx *h, const float *X32, int ld32, void *Xq, float *x_scale,
                             cudaStream_t s);
glm_status_t launch_wait_timeout(glm_ctx *h, int spin_limit, cudaStream_t s);
// Raise a kernel's dynamic shared-memory cap to the most a block may use on
// the current device (the 227 KB opt-in limit less the kernel's static shared
// memory). The cap is the same on every call, so host threads that launch
// the same kernel concurrently with different sizes cannot lower it between
// another thread's set and launch. Done once per (kernel, device).
cudaError_t allow_max_dynamic_smem(const void *fn);
// cuTensorMapEncodeTiled through the runtime's driver entry point (no link
// against the driver library); nullptr if unavailable.
PFN_cuTensorMapEncodeTiled_v12000 tensor_map_encoder();
// Encode (or reuse) the fused path's padded-row tensor map for X.
glm_status_t fused_tensor_map(glm_ctx *h, const void *X);
glm_status_t grouped_configure(glm_ctx *h);
size_t tc_workspace_bytes(const glm_ctx *h);
glm_status_t launch_grouped(glm_ctx *h, const void *X, const float *x_scale, const uint8_t *y,
                            const int64_t *group_off, int G, const float *beta, const float *mu,
                            double tau, double *f_out, float *g_out, cudaStream_t s);
glm_status_t autotune_grouped(glm_ctx *h, const void *X, const float *x_scale, const uint8_t *y,
                              const int64_t *group_off, int G, const float *beta, const float *mu,
                              double tau, double *f_out, float *g_out, cudaStream_t s, int reps);

}  // namespace glm

// ---------------------------------------------------------------------------
// Inline PTX primitives (device only).
#ifdef __CUDACC__
namespace glm {
namespace ptx {

__device__ __forceinline__ uint32_t smem_u32(const void *p)
{
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t *bar, unsigned count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count)
                 : "memory");
}

// Make mbarrier initialisation visible to the async proxy (TMA).
__device__ __forceinline__ void fence_mbar_init()
{
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void fence_proxy_async_smem()
{
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t *bar, unsigned bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)),
                 "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ void mbar_arrive(uint64_t *bar)
{
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, unsigned parity)
{
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

// Bounded wait: true when the phase completed, false when the limit ran out.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t *bar, unsigned parity, unsigned limit)
{
    for (unsigned i = 0; i < limit; ++i)
        if (mbar_try_wait(bar, parity))
            return true;
    return false;
}

// One-dimensional bulk copy global -> shared through the TMA engine,
// completing `bytes` transactions on `bar`. dst, src 16-byte aligned; bytes a
// multiple of 16.
__device__ __forceinline__ void bulk_g2s(void *dst, const void *src, unsigned bytes, uint64_t *bar,
                                         uint64_t policy)
{
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes.L2::cache_hint "
        "[%0], [%1], %2, [%3], %4;" ::"r"(smem_u32(dst)),
        "l"(src), "r"(bytes), "r"(smem_u32(bar)), "l"(policy)
        : "memory");
}

// Two-dimensional tiled tensor copy global -> shared (coordinates innermost
// first), completing the box's bytes on `bar`. The box lands densely in
// shared memory; elements outside the tensor are written as zeros and are
// not read from memory.
__device__ __forceinline__ void tensor_g2s_2d(void *dst, const CUtensorMap *map, int c0, int c1,
                                              uint64_t *bar, uint64_t policy)
{
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
        ".L2::cache_hint [%0], [%1, {%2, %3}], [%4], %5;" ::"r"(smem_u32(dst)),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(c0), "r"(c1), "r"(smem_u32(bar)), "l"(policy)
        : "memory");
}

__device__ __forceinline__ uint64_t policy_evict_first()
{
    uint64_t pol;
    asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(pol));
    return pol;
}

// Programmatic dependent launch: wait for the previous kernel in the stream
// (and the visibility of its writes) / allow the next one to start launching.
__device__ __forceinline__ void grid_dep_wait()
{
    asm volatile("griddepcontrol.wait;" ::: "memory");
}

__device__ __forceinline__ void grid_dep_launch_dependents()
{
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}

__device__ __forceinline__ double ld_cg_f64(const double *p)
{
    double v;
    asm volatile("ld.global.cg.f64 %0, [%1];" : "=d"(v) : "l"(p));
    return v;
}

}  // namespace ptx

// Deterministic cross-CTA sums in 128-bit two's-complement fixed point with
// 64 fractional bits. A value v is added as the integer floor(v * 2^64),
// split into four 32-bit limbs, each accumulated in its own 64-bit word, so
// no limb sum can overflow for fewer than 2^32 contributions and carries are
// resolved only when the total is read. Integer addition is associative, so
// the total is the same whatever order the CTAs arrive in. |v| must be below
// 2^63; a non-finite or larger value raises the flag word instead.
namespace fx {

constexpr int kLimbs = 4;

__device__ __forceinline__ void add(unsigned long long *acc, double v, unsigned *flag)
{
    if (v == 0.0)
        return;
    if (!isfinite(v) || fabs(v) >= 9.2e18) {
        atomicOr(flag, 1u);
        return;
    }
    int e;
    const double m = frexp(v, &e);                            // v = m 2^e, 0.5 <= |m| < 1
    const long long mi = (long long)ldexp(m, 53);             // exact: |mi| < 2^53
    const int sh = e - 53 + 64;                               // v 2^64 = mi 2^sh
    __int128 t;
    if (sh >= 0)
        t = (__int128)((unsigned __int128)(__int128)mi << sh); // sh <= 74: |t| < 2^127
    else if (sh > -64)
        t = (__int128)(mi >> (-sh));                          // arithmetic shift: floor
    else
        t = mi < 0 ? (__int128)-1 : (__int128)0;
    const unsigned __int128 u = (unsigned __int128)t;
#pragma unroll
    for (int l = 0; l < kLimbs; ++l) {
        const unsigned long long limb = (unsigned long long)((u >> (32 * l)) & 0xFFFFFFFFull);
        if (limb)
            atomicAdd(&acc[l], limb);
    }
}

// Total of an accumulator (then reset to zero for the next launch).
__device__ __forceinline__ double read_and_clear(unsigned long long *acc)
{
    unsigned __int128 T = 0;
#pragma unroll
    for (int l = 0; l < kLimbs; ++l) {
        const unsigned long long w = __ldcg(acc + l);
        T += (unsigned __int128)w << (32 * l);
        acc[l] = 0ull;
    }
    const __int128 sv = (__int128)T;
    const long long hi = (long long)(sv >> 64);               // integer part (floor)
    const unsigned long long lo = (unsigned long long)sv;     // fraction * 2^64
    return (double)hi + ldexp((double)lo, -64);
}

}  // namespace fx
}  // namespace glm
#endif
