// glm_logpost_grad_noalloc: the fused log-posterior + gradient evaluation for
// callers that must not allocate device memory.
//
// Some callers cannot call cudaMalloc at the point where they evaluate: code
// running inside a memory pool or arena that owns all device memory of the
// process, a real-time loop that must not take the allocator's locks or risk
// an out-of-memory failure mid-run, or a plugin whose host application
// forbids allocation. The handle API allocates its workspace in glm_create;
// this entry point instead keeps its scratch (the cross-CTA fixed-point
// accumulators, the completion ticket and the flag/status words) in one
// file-scope device array of a fixed size, so a call allocates nothing.
#include <cuda.h>
#include <cmath>
#include <cstring>
#include <mutex>

#include "glm_internal.cuh"

namespace {

constexpr int kNoAllocMaxP = 1024;          // columns
constexpr int kNoAllocMaxKC = 8;            // vectors per launch (larger K: several launches)
constexpr int kNoAllocMaxDevices = 64;
// accumulators: KC x (P+1) x limbs words, then ticket, flag and status words
constexpr size_t kAccWords = (size_t)kNoAllocMaxKC * (kNoAllocMaxP + 1) * glm::fx::kLimbs;
constexpr size_t kScratchWords = kAccWords + 32;

// The scratch. Every GPU that loads this library holds it (about 263 KB)
// until the process exits. In host code this name is only a host-side
// stand-in for the symbol; its device address comes from
// cudaGetSymbolAddress below.
static __device__ __align__(256) unsigned long long g_glm_noalloc_scratch[kScratchWords];

std::mutex g_setup_mutex;
void *g_scratch_addr[kNoAllocMaxDevices];   // device address per device
void *g_scratch_ctx[kNoAllocMaxDevices];    // the context that address belongs to

typedef CUresult (*CtxGetCurrentFn)(CUcontext *);

CtxGetCurrentFn ctx_get_current()
{
    static CtxGetCurrentFn fn = [] {
        cudaDriverEntryPointQueryResult q;
        void *f = nullptr;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f, 12000, cudaEnableDefault, &q) !=
                cudaSuccess ||
            q != cudaDriverEntryPointSuccess) {
            cudaGetLastError();
            f = nullptr;
        }
        return reinterpret_cast<CtxGetCurrentFn>(f);
    }();
    return fn;
}

// Look up, with the device current, the device address of the scratch array:
// once per device, and again only if the device's context has changed since
// (after cudaDeviceReset the module is loaded anew and the array may move).
glm_status_t scratch_for_device(int dev, void **out)
{
    CtxGetCurrentFn get = ctx_get_current();
    CUcontext ctx = nullptr;
    if (!get || get(&ctx) != CUDA_SUCCESS)
        return GLM_ERR_CUDA;
    std::lock_guard<std::mutex> lock(g_setup_mutex);
    if (!g_scratch_addr[dev] || !ctx || g_scratch_ctx[dev] != (void *)ctx) {
        void *ptr = nullptr;
        if (cudaGetSymbolAddress(&ptr, g_glm_noalloc_scratch) != cudaSuccess || !ptr) {
            cudaGetLastError();
            return GLM_ERR_CUDA;
        }
        // the runtime makes the primary context current on first use: read it again
        if (get(&ctx) != CUDA_SUCCESS)
            return GLM_ERR_CUDA;
        g_scratch_addr[dev] = ptr;
        g_scratch_ctx[dev] = (void *)ctx;
    }
    *out = g_scratch_addr[dev];
    return GLM_OK;
}

int elem_bytes(int xtype)
{
    return xtype == GLM_X_F32 ? 4 : xtype == GLM_X_BF16 ? 2 : xtype == GLM_X_FP8E4M3 ? 1 : 0;
}

}  // namespace

extern "C" glm_status_t glm_logpost_grad_noalloc(const void *X, const float *x_scale,
                                                 const uint8_t *y, int64_t n_rows, int32_t p,
                                                 int32_t ld, int32_t xtype, double prior_sigma,
                                                 const float *beta, int32_t K, double *f_out,
                                                 float *g_out, glm_stream_t stream)
{
    // the same checks as glm_create and glm_logpost_grad
    auto misaligned = [](const void *q, uintptr_t a) { return reinterpret_cast<uintptr_t>(q) % a != 0; };
    const int es = elem_bytes(xtype);
    if (es == 0 || n_rows < 0 || p < 1 || ld < p || K < 1 || K > 1024 ||
        !(prior_sigma > 0.0) || !std::isfinite(prior_sigma) || !beta || !f_out || !g_out)
        return GLM_ERR_INVALID_ARG;
    if (p > kNoAllocMaxP)
        return GLM_ERR_INVALID_ARG;        // the fixed scratch holds P <= 1024 only
    if (((int64_t)ld * es) % 16 != 0 || (n_rows > 0 && (!X || !y)) ||
        (X && misaligned(X, 16)) || (xtype == GLM_X_FP8E4M3) != (x_scale != nullptr) ||
        (x_scale && misaligned(x_scale, 4)) || misaligned(beta, 4) || misaligned(f_out, 8) ||
        misaligned(g_out, 4))
        return GLM_ERR_INVALID_ARG;
    if (n_rows > ((int64_t)1 << 40) || (int64_t)ld * es > (1 << 20))
        return GLM_ERR_UNSUPPORTED;

    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kNoAllocMaxDevices)
        return GLM_ERR_NO_DEVICE;
    int major = 0, minor = 0, sms = 0;
    if (cudaDeviceGetAttribute(&major, cudaDevAttrComputeCapabilityMajor, dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&minor, cudaDevAttrComputeCapabilityMinor, dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        return GLM_ERR_CUDA;
    if (major != 10 || minor != 3)
        return GLM_ERR_NO_DEVICE;
    void *scratch = nullptr;
    glm_status_t st = scratch_for_device(dev, &scratch);
    if (st != GLM_OK)
        return st;

    // A handle on the stack: the same launch configuration the handle API
    // would choose for this shape, pointed at the static scratch.
    glm_ctx c;
    std::memset(&c, 0, sizeof(c));
    c.d.n_rows = n_rows;
    c.d.p = p;
    c.d.ld = ld;
    c.d.k_max = K;
    c.d.xtype = xtype;
    c.d.prior_sigma = prior_sigma;
    c.d.device = dev;
    c.d.flags = GLM_FLAG_NO_TENSOR_CORES;
    c.device = dev;
    c.sm_count = sms;
    c.elem_bytes = es;
    st = glm::fused_configure(&c);
    if (st != GLM_OK)
        return st;
    unsigned long long *words = static_cast<unsigned long long *>(scratch);
    c.acc = words;
    c.ticket = reinterpret_cast<unsigned *>(words + kAccWords);
    c.acc_flag = c.ticket + 1;
    c.status = c.ticket + 2;

    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    // The array keeps whatever the previous call left; the kernel needs its
    // accumulators, ticket and flags at zero, so clear them first.
    const size_t used = (size_t)kNoAllocMaxKC * (p + 1) * glm::fx::kLimbs;
    if (cudaMemsetAsync(words, 0, used * sizeof(unsigned long long), s) != cudaSuccess ||
        cudaMemsetAsync(c.ticket, 0, 4 * sizeof(unsigned), s) != cudaSuccess)
        return GLM_ERR_CUDA;

    const double s2 = prior_sigma * prior_sigma;
    for (int k0 = 0; k0 < K;) {
        int kc = 1;
        while (kc < K - k0 && kc < c.kc_max)
            kc <<= 1;
        const int kk = (K - k0) < kc ? (K - k0) : kc;
        glm::FusedParams prm;
        std::memset(&prm, 0, sizeof(prm));
        prm.X = X;
        prm.x_scale = x_scale;
        prm.y = y;
        prm.beta = beta + (size_t)k0 * p;
        prm.N = n_rows;
        prm.P = p;
        prm.ld = ld;
        prm.K = kk;
        prm.stages = c.stages;
        prm.tile_rows = c.tile_rows;
        prm.srow = c.srow;
        prm.box_rows = c.box_rows;
        prm.inv_s2 = 1.0 / s2;
        prm.prior_const = 0.5 * (double)p * std::log(2.0 * M_PI * s2);
        prm.acc = c.acc;
        prm.acc_flag = c.acc_flag;
        prm.ticket = c.ticket;
        prm.status = c.status;
        prm.f_out = f_out + k0;
        prm.g_out = g_out + (size_t)k0 * p;
        st = glm::launch_fused(&c, prm, kc, s);
        if (st != GLM_OK)
            return st;
        k0 += kk;
    }
    return GLM_OK;
}
