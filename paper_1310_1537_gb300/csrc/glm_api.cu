// C ABI of the library: handle lifetime, argument validation, workspace and
// dispatch to the kernels. Every entry point validates on the host and
// launches nothing when it returns an argument error.
#include <cstdlib>
#include <cstring>
#include <cmath>
#include <mutex>
#include <new>
#include <utility>
#include <vector>

#include "glm_internal.cuh"

namespace glm {

glm_status_t launch_fused_f32(glm_ctx *h, const FusedParams &p, int kc, cudaStream_t s);
glm_status_t launch_fused_bf16(glm_ctx *h, const FusedParams &p, int kc, cudaStream_t s);
glm_status_t launch_fused_fp8(glm_ctx *h, const FusedParams &p, int kc, cudaStream_t s);
glm_status_t launch_tc(glm_ctx *h, const void *X, const float *x_scale, const uint8_t *y,
                       const float *beta, int K, double *f_out, float *g_out, cudaStream_t s);
bool tc_supported(const glm_ctx *h);

static int elem_bytes_of(int xtype)
{
    switch (xtype) {
    case GLM_X_F32: return 4;
    case GLM_X_BF16: return 2;
    case GLM_X_FP8E4M3: return 1;
    default: return 0;
    }
}

glm_status_t launch_fused(glm_ctx *h, const FusedParams &p, int kc, cudaStream_t s)
{
    switch (h->d.xtype) {
    case GLM_X_F32: return launch_fused_f32(h, p, kc, s);
    case GLM_X_BF16: return launch_fused_bf16(h, p, kc, s);
    case GLM_X_FP8E4M3: return launch_fused_fp8(h, p, kc, s);
    default: return GLM_ERR_UNSUPPORTED;
    }
}

// Dynamic shared-memory budget per CTA: the 227 KB opt-in limit less room
// for the kernel's static shared arrays.
constexpr int kSmemOptin = kSmemDynamicBudget;

static int fused_smem_total(const glm_ctx *h, int tile_rows, int stages, int kc, int srow)
{
    const int es = h->elem_bytes;
    const int epc = 16 / es;
    const int pce = (h->d.ld / epc) * epc;
    const int stage = tile_rows * srow;
    const int red = kFusedThreads * kc * epc * 4;
    int tiles = stages * stage > red ? stages * stage : red;
    tiles = (tiles + 127) / 128 * 128;
    return tiles + (kc * pce * 4 + 15) / 16 * 16 + (tile_rows * kc * 4 + 15) / 16 * 16 +
           kMaxStages * 8 + 64 + 128;
}

// Choose the phase-1 split (threads per row), the rows per staged tile and the
// ring depth: about 48 KB per stage, at least two stages, at most eight.
glm_status_t fused_configure(glm_ctx *h)
{
    const int es = h->elem_bytes;
    const int epc = 16 / es;
    const int pcu = (h->d.p + epc - 1) / epc;
    if (pcu > kFusedThreads)
        return GLM_ERR_UNSUPPORTED;
    h->kc_max = (epc <= 8) ? 8 : 4;
    const int row_bytes = h->d.ld * es;
    const int pc = row_bytes / 16;
    // Staged row stride for a split: one zero chunk wider when the chunk
    // count is even and rows are read one thread per row (SPLIT <= 4), so
    // that 8 consecutive rows start in distinct bank groups. The extra chunk
    // comes from a 2-D tensor copy of 8-byte words whose box is wider than the
    // row (box dimensions are at most 256 elements, so rows up to 2032 bytes).
    const bool pad_ok = h->d.n_rows > 0 && pc % 2 == 0 && row_bytes + 16 <= 256 * 8 &&
                        tensor_map_encoder() != nullptr;
    auto srow_for = [&](int sp) { return (pad_ok && sp != 32) ? row_bytes + 16 : row_bytes; };
    // Fewest threads per row whose one-batch tile still fits two stages:
    // bigger tiles amortise the per-tile barriers and label loads.
    int split = 32;
    for (int cand = 1; cand <= 4; cand <<= 1) {
        if (fused_smem_total(h, kFusedThreads / cand, 2, h->kc_max, srow_for(cand)) <= kSmemOptin) {
            split = cand;
            break;
        }
    }
    const int budget = kSmemOptin;
    int rb = kFusedThreads / split;
    int srow = srow_for(split);
    const int target = 49152;
    // rows per tile: a multiple of the phase-1 batch, at most four batches
    auto pick_rows = [&](int rbv) {
        int t = (target / srow) / rbv * rbv;
        if (t < rbv)
            t = rbv;
        if (t > 4 * rbv)
            t = 4 * rbv;
        return t;
    };
    int T = pick_rows(rb);
    int stages = kMaxStages;
    while (stages >= 2 && fused_smem_total(h, T, stages, h->kc_max, srow) > budget)
        --stages;
    if (stages < 2 && split != 32) {     // rows too wide: one warp per row, 8-row batches
        split = 32;
        rb = kFusedThreads / split;
        srow = srow_for(split);
        T = pick_rows(rb);
        stages = kMaxStages;
        while (stages >= 2 && fused_smem_total(h, T, stages, h->kc_max, srow) > budget)
            --stages;
    }
    if (stages < 2)
        return GLM_ERR_UNSUPPORTED;
    h->split = split;
    h->stages = stages;
    h->tile_rows = T;
    h->srow = srow;
    h->box_rows = 0;
    if (srow != row_bytes) {
        // rows per tensor copy: the largest power of two up to 256 dividing T
        int br = 256;
        while (br > 8 && T % br != 0)
            br >>= 1;
        h->box_rows = br;
    }
    h->fx_map_ptr = nullptr;
    h->smem_bytes = fused_smem_total(h, T, stages, h->kc_max, srow);
    // one CTA per SM, but no more CTAs than tiles of rows: for small N the
    // extra CTAs would only add to the cross-CTA combine and the ticket
    const int64_t tiles = (h->d.n_rows + T - 1) / T;
    h->grid = tiles < (int64_t)h->sm_count ? (tiles > 0 ? (int)tiles : 1) : h->sm_count;
    h->use_pdl = 1;
    return GLM_OK;
}

__global__ void wait_timeout_kernel(unsigned *status, int spin_limit)
{
    __shared__ __align__(8) uint64_t bar;
    if (threadIdx.x == 0) {
        ptx::mbar_init(&bar, 1);
        ptx::fence_mbar_init();
    }
    __syncthreads();
    // Nothing arrives on this barrier: the bounded wait must give up.
    bool ok = ptx::mbar_wait_bounded(&bar, 0u, (unsigned)spin_limit);
    if (!ok && threadIdx.x == 0)
        atomicOr(status, kDevTimeout);
}

glm_status_t launch_wait_timeout(glm_ctx *h, int spin_limit, cudaStream_t s)
{
    wait_timeout_kernel<<<1, 32, 0, s>>>(h->status, spin_limit);
    return cudaGetLastError() == cudaSuccess ? GLM_OK : GLM_ERR_CUDA;
}

static bool aligned(const void *p, size_t a)
{
    return (reinterpret_cast<uintptr_t>(p) % a) == 0;
}

static glm_status_t check_x_args(const glm_ctx *h, const void *X, const float *x_scale,
                                 const uint8_t *y)
{
    if (h->d.n_rows > 0 && (!X || !y))
        return GLM_ERR_INVALID_ARG;
    if (X && !aligned(X, 16))
        return GLM_ERR_INVALID_ARG;
    const bool fp8 = h->d.xtype == GLM_X_FP8E4M3;
    if (fp8 != (x_scale != nullptr))
        return GLM_ERR_INVALID_ARG;
    if (x_scale && !aligned(x_scale, 4))
        return GLM_ERR_INVALID_ARG;
    return GLM_OK;
}

static FusedParams base_params(const glm_ctx *h, const void *X, const float *x_scale,
                               const uint8_t *y)
{
    FusedParams p;
    std::memset(&p, 0, sizeof(p));
    p.X = X;
    p.x_scale = x_scale;
    p.y = y;
    p.N = h->d.n_rows;
    p.P = h->d.p;
    p.ld = h->d.ld;
    p.stages = h->stages;
    p.tile_rows = h->tile_rows;
    p.srow = h->srow;
    p.box_rows = h->box_rows;
    const double s2 = h->d.prior_sigma * h->d.prior_sigma;
    const bool prior = !(h->d.flags & GLM_FLAG_NO_PRIOR);
    p.inv_s2 = prior ? 1.0 / s2 : 0.0;
    p.prior_const = prior ? 0.5 * (double)h->d.p * std::log(2.0 * M_PI * s2) : 0.0;
    p.acc = h->acc;
    p.acc_flag = h->acc_flag;
    p.ticket = h->ticket;
    p.status = h->status;
    return p;
}

static int kc_for(int remaining, int kc_max)
{
    int kc = 1;
    while (kc < remaining && kc < kc_max)
        kc <<= 1;
    return kc;
}

// Evaluate K vectors on the CUDA cores, KC at a time.
static glm_status_t fused_eval(glm_ctx *h, const void *X, const float *x_scale, const uint8_t *y,
                               const float *beta, int K, double *f_out, float *g_out,
                               cudaStream_t s)
{
    FusedParams p = base_params(h, X, x_scale, y);
    for (int k0 = 0; k0 < K; ) {
        const int kc = kc_for(K - k0, h->kc_max);
        const int kk = (K - k0) < kc ? (K - k0) : kc;
        p.beta = beta + (size_t)k0 * h->d.p;
        p.K = kk;
        p.f_out = f_out + k0;
        p.g_out = g_out + (size_t)k0 * h->d.p;
        glm_status_t st = launch_fused(h, p, kc, s);
        if (st != GLM_OK)
            return st;
        k0 += kk;
    }
    return GLM_OK;
}

PFN_cuTensorMapEncodeTiled_v12000 tensor_map_encoder()
{
    static PFN_cuTensorMapEncodeTiled_v12000 fn = [] {
        cudaDriverEntryPointQueryResult q;
        void *f = nullptr;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &f, 12000, cudaEnableDefault,
                                             &q) != cudaSuccess ||
            q != cudaDriverEntryPointSuccess) {
            cudaGetLastError();
            f = nullptr;
        }
        return reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(f);
    }();
    return fn;
}

// X viewed as rows of 8-byte words: {word within the row, row}. The box is
// two words (one chunk) wider than a row; those words lie outside the
// tensor, so the copy writes them as zeros without reading memory and staged
// rows are srow bytes apart.
glm_status_t fused_tensor_map(glm_ctx *h, const void *X)
{
    if (h->box_rows == 0 || h->fx_map_ptr == X)
        return GLM_OK;
    PFN_cuTensorMapEncodeTiled_v12000 encode = tensor_map_encoder();
    if (!encode)
        return GLM_ERR_CUDA;
    const int row_bytes = h->d.ld * h->elem_bytes;
    const cuuint64_t dims[2] = {(cuuint64_t)(row_bytes / 8), (cuuint64_t)h->d.n_rows};
    const cuuint64_t strides[1] = {(cuuint64_t)row_bytes};
    const cuuint32_t box[2] = {(cuuint32_t)(h->srow / 8), (cuuint32_t)h->box_rows};
    const cuuint32_t estr[2] = {1, 1};
    CUtensorMap *map = reinterpret_cast<CUtensorMap *>(h->fx_map);
    CUresult r = encode(map, CU_TENSOR_MAP_DATA_TYPE_UINT64, 2, const_cast<void *>(X), dims, strides,
                        box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                        CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS)
        return GLM_ERR_CUDA;
    h->fx_map_ptr = X;
    return GLM_OK;
}

cudaError_t allow_max_dynamic_smem(const void *fn)
{
    static std::mutex mu;
    static std::vector<std::pair<const void *, int>> done;   // (kernel, device)
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess)
        return e;
    std::lock_guard<std::mutex> lock(mu);
    for (const auto &d : done)
        if (d.first == fn && d.second == dev)
            return cudaSuccess;
    cudaFuncAttributes a;
    e = cudaFuncGetAttributes(&a, fn);
    if (e != cudaSuccess)
        return e;
    e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             kSmemOptinBytes - (int)a.sharedSizeBytes);
    if (e == cudaSuccess)
        done.push_back({fn, dev});
    return e;
}

}  // namespace glm

using namespace glm;

extern "C" {

const char *glm_status_str(glm_status_t s)
{
    switch (s) {
    case GLM_OK: return "ok";
    case GLM_ERR_INVALID_ARG: return "invalid argument";
    case GLM_ERR_UNSUPPORTED: return "unsupported configuration";
    case GLM_ERR_OOM: return "out of device memory";
    case GLM_ERR_CUDA: return "CUDA error";
    case GLM_ERR_TIMEOUT: return "device wait timed out";
    case GLM_ERR_NO_DEVICE: return "no usable CUDA device";
    case GLM_PENDING: return "pending";
    default: return "unknown status";
    }
}

glm_status_t glm_create(const glm_desc_t *desc, glm_handle_t *out)
{
    if (!out)
        return GLM_ERR_INVALID_ARG;
    *out = nullptr;
    if (!desc)
        return GLM_ERR_INVALID_ARG;
    const glm_desc_t d = *desc;
    const int es = elem_bytes_of(d.xtype);
    if (es == 0 || d.n_rows < 0 || d.p < 1 || d.ld < d.p || d.k_max < 1 || d.k_max > 1024 ||
        !(d.prior_sigma > 0.0) || !std::isfinite(d.prior_sigma) || d.device < 0 ||
        (d.flags & ~(GLM_FLAG_NO_TENSOR_CORES | GLM_FLAG_NO_PRIOR)) != 0)
        return GLM_ERR_INVALID_ARG;
    if (((int64_t)d.ld * es) % 16 != 0 || d.g_max < 0)
        return GLM_ERR_INVALID_ARG;
    if (d.n_rows > ((int64_t)1 << 40) || (int64_t)d.ld * es > (1 << 20))
        return GLM_ERR_UNSUPPORTED;
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev == 0) {
        cudaGetLastError();
        return GLM_ERR_NO_DEVICE;
    }
    if (d.device >= ndev)
        return GLM_ERR_INVALID_ARG;
    if (cudaSetDevice(d.device) != cudaSuccess)
        return GLM_ERR_CUDA;
    cudaDeviceProp prop;
    if (cudaGetDeviceProperties(&prop, d.device) != cudaSuccess)
        return GLM_ERR_CUDA;
    if (prop.major != 10 || prop.minor != 3)
        return GLM_ERR_NO_DEVICE;   // this build carries sm_103a code only

    glm_ctx *h = new (std::nothrow) glm_ctx;
    if (!h)
        return GLM_ERR_OOM;
    std::memset(h, 0, sizeof(*h));
    h->d = d;
    h->device = d.device;
    h->sm_count = prop.multiProcessorCount;
    h->elem_bytes = es;
    glm_status_t st = fused_configure(h);
    if (st != GLM_OK) {
        delete h;
        return st;
    }
    if (d.g_max > 0 && grouped_configure(h) != GLM_OK)
        h->gr_warps = 0;   // rows too wide for the grouped kernel: grouped calls are unsupported
    h->tc_min_k = 16;
    h->tc_enabled = (!(d.flags & GLM_FLAG_NO_TENSOR_CORES)) && tc_supported(h) ? 1 : 0;

    // Workspace: fixed-point accumulators, ticket, flags, status, scratch,
    // host-call staging (all zeroed once here; kernels return them to zero).
    const size_t acc_words = (size_t)8 * (size_t)(d.p + 1) * fx::kLimbs;
    const size_t kp = (size_t)d.k_max * d.p;
    size_t off = 0;
    auto take = [&](size_t bytes) {
        size_t o = off;
        off += (bytes + 255) / 256 * 256;
        return o;
    };
    const size_t o_acc = take(acc_words * 8);
    const size_t o_flag = take(256);
    const size_t o_ticket = take(256);
    const size_t o_status = take(256);
    const size_t o_scratch = take((size_t)d.p * 4 + 256);
    const size_t o_bst = take(kp * 4);
    const size_t o_fst = take((size_t)d.k_max * 8);
    const size_t o_gst = take(kp * 4);
    const size_t gmax = (size_t)(d.g_max > 0 ? d.g_max : 0);
    const size_t o_gacc = take(gmax * (size_t)(d.p + 1) * fx::kLimbs * 8);
    const size_t o_gtk = take(gmax * 4);
    const size_t o_gfl = take(gmax * 4);
    const size_t tcb = h->tc_enabled ? tc_workspace_bytes(h) : 0;
    const size_t o_tc = take(tcb);
    if (cudaMalloc(&h->ws, off) != cudaSuccess) {
        cudaGetLastError();
        delete h;
        return GLM_ERR_OOM;
    }
    h->ws_bytes = off;
    uint8_t *base = static_cast<uint8_t *>(h->ws);
    h->acc = reinterpret_cast<unsigned long long *>(base + o_acc);
    h->acc_flag = reinterpret_cast<unsigned *>(base + o_flag);
    h->ticket = reinterpret_cast<unsigned *>(base + o_ticket);
    h->status = reinterpret_cast<unsigned *>(base + o_status);
    h->scratch = reinterpret_cast<float *>(base + o_scratch);
    h->beta_stage = reinterpret_cast<float *>(base + o_bst);
    h->f_stage = reinterpret_cast<double *>(base + o_fst);
    h->g_stage = reinterpret_cast<float *>(base + o_gst);
    if (tcb) {
        const int MBt = (d.p + 127) / 128;
        h->tc_part_f = reinterpret_cast<double *>(base + o_tc);
        h->tc_part_g = reinterpret_cast<float *>(base + o_tc + (size_t)h->sm_count * 64 * 8);
        (void)MBt;
    }
    if (gmax) {
        h->gr_acc = reinterpret_cast<unsigned long long *>(base + o_gacc);
        h->gr_ticket = reinterpret_cast<unsigned *>(base + o_gtk);
        h->gr_flag = reinterpret_cast<unsigned *>(base + o_gfl);
    }
    if (cudaMemset(h->ws, 0, off) != cudaSuccess || cudaDeviceSynchronize() != cudaSuccess) {
        cudaFree(h->ws);
        delete h;
        return GLM_ERR_CUDA;
    }
    *out = h;
    return GLM_OK;
}

glm_status_t glm_destroy(glm_handle_t h)
{
    if (!h)
        return GLM_OK;
    cudaSetDevice(h->device);
    cudaDeviceSynchronize();
    cudaFree(h->ws);
    delete h;
    return GLM_OK;
}

glm_status_t glm_get_info(glm_handle_t h, glm_info_t *info)
{
    if (!h || !info)
        return GLM_ERR_INVALID_ARG;
    info->sm_count = h->sm_count;
    info->grid = h->grid;
    info->tile_rows = h->tile_rows;
    info->stages = h->stages;
    info->smem_bytes = h->smem_bytes;
    info->tc_enabled = h->tc_enabled;
    info->tc_min_k = h->tc_min_k;
    info->workspace_bytes = (int64_t)h->ws_bytes;
    return GLM_OK;
}

glm_status_t glm_logpost_grad(glm_handle_t h, const void *X, const float *x_scale,
                              const uint8_t *y, const float *beta, int32_t K, double *f_out,
                              float *g_out, glm_stream_t stream)
{
    if (!h)
        return GLM_ERR_INVALID_ARG;
    glm_status_t st = check_x_args(h, X, x_scale, y);
    if (st != GLM_OK)
        return st;
    if (K < 1 || K > h->d.k_max || !beta || !f_out || !g_out || !aligned(beta, 4) ||
        !aligned(f_out, 8) || !aligned(g_out, 4))
        return GLM_ERR_INVALID_ARG;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    h->last_path = GLM_PATH_NONE;
    if (h->tc_enabled && K >= h->tc_min_k && h->d.xtype != GLM_X_F32) {
        st = launch_tc(h, X, x_scale, y, beta, K, f_out, g_out, s);
        if (st != GLM_ERR_UNSUPPORTED) {
            if (st == GLM_OK)
                h->last_path = GLM_PATH_TENSOR_CORES;
            return st;                  // else: the CUDA-core pass below
        }
    }
    st = fused_eval(h, X, x_scale, y, beta, K, f_out, g_out, s);
    if (st == GLM_OK)
        h->last_path = GLM_PATH_CUDA_CORES;
    return st;
}

glm_status_t glm_logpost_grad_host(glm_handle_t h, const void *X, const float *x_scale,
                                   const uint8_t *y, const float *beta_host, int32_t K,
                                   double *f_host, float *g_host, glm_stream_t stream)
{
    if (!h)
        return GLM_ERR_INVALID_ARG;
    if (K < 1 || K > h->d.k_max || !beta_host || !f_host || !g_host)
        return GLM_ERR_INVALID_ARG;
    glm_status_t st = check_x_args(h, X, x_scale, y);
    if (st != GLM_OK)
        return st;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    const size_t kp = (size_t)K * h->d.p;
    if (cudaMemcpyAsync(h->beta_stage, beta_host, kp * 4, cudaMemcpyHostToDevice, s) != cudaSuccess)
        return GLM_ERR_CUDA;
    st = glm_logpost_grad(h, X, x_scale, y, h->beta_stage, K, h->f_stage, h->g_stage, stream);
    if (st != GLM_OK)
        return st;
    if (cudaMemcpyAsync(f_host, h->f_stage, (size_t)K * 8, cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaMemcpyAsync(g_host, h->g_stage, kp * 4, cudaMemcpyDeviceToHost, s) != cudaSuccess)
        return GLM_ERR_CUDA;
    if (cudaStreamSynchronize(s) != cudaSuccess)
        return GLM_ERR_CUDA;
    return GLM_OK;
}

glm_status_t glm_rwm_run(glm_handle_t h, const void *X, const float *x_scale, const uint8_t *y,
                         int32_t K, int32_t n_steps, float step, const float *z,
                         const double *log_u, float *beta_state, double *f_state, int32_t init_f,
                         float *samples, uint8_t *accept, double *logpost, glm_stream_t stream)
{
    if (!h || (h->d.flags & GLM_FLAG_NO_PRIOR))
        return GLM_ERR_INVALID_ARG;     // the accept step needs the whole posterior
    glm_status_t st = check_x_args(h, X, x_scale, y);
    if (st != GLM_OK)
        return st;
    const int kmax = h->d.k_max < h->kc_max ? h->d.k_max : h->kc_max;
    if (K < 1 || K > kmax || n_steps < 0 || !beta_state || !f_state || !std::isfinite(step) ||
        (n_steps > 0 && (!z || !log_u)) || !aligned(beta_state, 4) || !aligned(f_state, 8))
        return GLM_ERR_INVALID_ARG;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    const int kc = kc_for(K, h->kc_max);
    if (init_f) {
        FusedParams p = base_params(h, X, x_scale, y);
        p.beta = beta_state;
        p.K = K;
        p.f_out = f_state;
        p.g_out = h->g_stage;
        st = launch_fused(h, p, kc, s);
        if (st != GLM_OK)
            return st;
    }
    const size_t kp = (size_t)K * h->d.p;
    for (int t = 0; t < n_steps; ++t) {
        FusedParams p = base_params(h, X, x_scale, y);
        // after this call's first launch the previous kernel in the stream is
        // one of ours, which never writes X or y: let it stream them early
        p.early_prefetch = (t > 0 || init_f) ? 1 : 0;
        p.K = K;
        p.rwm = 1;
        p.step = step;
        p.z = z + (size_t)t * kp;
        p.log_u = log_u + (size_t)t * K;
        p.state = beta_state;
        p.f_state = f_state;
        p.samples = samples ? samples + (size_t)t * kp : nullptr;
        p.accept = accept ? accept + (size_t)t * K : nullptr;
        p.logpost = logpost ? logpost + (size_t)t * K : nullptr;
        st = launch_fused(h, p, kc, s);
        if (st != GLM_OK)
            return st;
    }
    return GLM_OK;
}

glm_status_t glm_logpost_grad_grouped(glm_handle_t h, const void *X, const float *x_scale,
                                      const uint8_t *y, const int64_t *group_off, int32_t G,
                                      const float *beta, const float *mu, double tau,
                                      double *f_out, float *g_out, glm_stream_t stream)
{
    if (!h)
        return GLM_ERR_INVALID_ARG;
    glm_status_t st = check_x_args(h, X, x_scale, y);
    if (st != GLM_OK)
        return st;
    if (G < 1 || G > h->d.g_max || !group_off || !beta || !mu || !f_out || !g_out ||
        !(tau > 0.0) || !std::isfinite(tau) || !aligned(group_off, 8) || !aligned(f_out, 8) ||
        !aligned(beta, 4) || !aligned(mu, 4) || !aligned(g_out, 4))
        return GLM_ERR_INVALID_ARG;
    return launch_grouped(h, X, x_scale, y, group_off, G, beta, mu, tau, f_out, g_out,
                          reinterpret_cast<cudaStream_t>(stream));
}

glm_status_t glm_autotune_grouped(glm_handle_t h, const void *X, const float *x_scale,
                                  const uint8_t *y, const int64_t *group_off, int32_t G,
                                  const float *beta, const float *mu, double tau, double *f_out,
                                  float *g_out, int32_t reps, glm_stream_t stream)
{
    if (!h)
        return GLM_ERR_INVALID_ARG;
    glm_status_t st = check_x_args(h, X, x_scale, y);
    if (st != GLM_OK)
        return st;
    if (G < 1 || G > h->d.g_max || !group_off || !beta || !mu || !f_out || !g_out ||
        !(tau > 0.0) || !std::isfinite(tau) || reps < 1 || reps > 1000)
        return GLM_ERR_INVALID_ARG;
    return autotune_grouped(h, X, x_scale, y, group_off, G, beta, mu, tau, f_out, g_out,
                            reinterpret_cast<cudaStream_t>(stream), reps);
}

glm_status_t glm_quantize(glm_handle_t h, const float *X32, int32_t ld32, void *Xq,
                          float *x_scale, glm_stream_t stream)
{
    if (!h)
        return GLM_ERR_INVALID_ARG;
    if (h->d.xtype == GLM_X_F32)
        return GLM_ERR_UNSUPPORTED;
    const bool fp8 = h->d.xtype == GLM_X_FP8E4M3;
    if ((h->d.n_rows > 0 && (!X32 || !Xq)) || ld32 < h->d.p || fp8 != (x_scale != nullptr) ||
        (Xq && !aligned(Xq, 16)))
        return GLM_ERR_INVALID_ARG;
    return launch_quantize(h, X32, ld32, Xq, x_scale, reinterpret_cast<cudaStream_t>(stream));
}

glm_status_t glm_sync(glm_handle_t h, glm_stream_t stream)
{
    if (!h)
        return GLM_ERR_INVALID_ARG;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    if (cudaStreamSynchronize(s) != cudaSuccess)
        return GLM_ERR_CUDA;
    unsigned word = 0;
    if (cudaMemcpy(&word, h->status, sizeof(word), cudaMemcpyDeviceToHost) != cudaSuccess)
        return GLM_ERR_CUDA;
    if (word) {
        if (cudaMemset(h->status, 0, sizeof(unsigned)) != cudaSuccess)
            return GLM_ERR_CUDA;
        if (word & kDevTimeout)
            return GLM_ERR_TIMEOUT;
    }
    return GLM_OK;
}

glm_status_t glm_selftest_wait_timeout(glm_handle_t h, int32_t spin_limit, glm_stream_t stream)
{
    if (!h || spin_limit < 1)
        return GLM_ERR_INVALID_ARG;
    return launch_wait_timeout(h, spin_limit, reinterpret_cast<cudaStream_t>(stream));
}

}  // extern "C"
