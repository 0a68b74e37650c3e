/*
 * glm.h — C ABI of the GB300 (sm_103a) library for the data-parallel hot path
 * of Mahani & Sharabiani, "SIMD Parallel MCMC Sampling with Applications for
 * Big-Data Bayesian Analytics": the Bayesian logistic-regression log-posterior
 * and its gradient, evaluated for K coefficient vectors in one pass over X.
 *
 * What every evaluation computes (for k = 0..K-1, rows n = 0..N-1):
 *
 *   eta_nk = x_n . beta_k                                   (§3.2, the LA map)
 *   f_k    = sum_n -[(1 - y_n) eta_nk + log(1 + exp(-eta_nk))]
 *            - |beta_k|^2 / (2 s^2) - (P/2) log(2 pi s^2)   (§3.1.1, eq-loglike-binlogit,
 *                                                             plus the N(0, s^2 I) prior)
 *   g_k    = sum_n (y_n - 1/(1 + exp(-eta_nk))) x_n - beta_k / s^2
 *                                                           (§4.2, eq-grad-expanded/-compact)
 *
 * Conventions shared by every entry point below:
 *
 * - Layout. X is row-major N x ld (row n starts at element n*ld); only the
 *   first P columns are used, padding columns must hold finite values
 *   (zeros recommended). ld * element_size must be a multiple of 16 bytes and
 *   X must be 16-byte aligned. y is N bytes, each 0 or 1 (other values give
 *   undefined results). beta is K x P row-major FP32 (beta_k contiguous),
 *   f_out is K FP64, g_out is K x P row-major FP32.
 * - Storage types. GLM_X_F32: X is float. GLM_X_BF16: X is bfloat16.
 *   GLM_X_FP8E4M3: X holds E4M3 codes q and x_scale holds P FP32 column
 *   scales, the stored value being q * x_scale[j]. x_scale must be NULL for
 *   the other types.
 * - Memory. Unless an entry point says "host", every data pointer is device
 *   memory of the handle's device, owned by the caller; the library never
 *   frees or retains it past the call. The handle owns only its workspace.
 * - Streams. glm_stream_t is a cudaStream_t (NULL = legacy default stream).
 *   Device entry points enqueue work and return without synchronising; they
 *   allocate nothing. One handle may be used by one stream at a time.
 * - Errors. Argument errors are detected on the host before anything is
 *   launched and return GLM_ERR_INVALID_ARG / GLM_ERR_UNSUPPORTED. A launch
 *   failure returns GLM_ERR_CUDA. Asynchronous device-side conditions (a
 *   bounded wait that expired) are recorded in the handle's status word and
 *   returned by glm_sync.
 */
#ifndef GLM_H
#define GLM_H

#include <stddef.h>
#include <stdint.h>

#if defined(__GNUC__)
#define GLM_API __attribute__((visibility("default")))
#else
#define GLM_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

typedef struct glm_ctx *glm_handle_t;
typedef struct CUstream_st *glm_stream_t;   /* same type as cudaStream_t */

typedef enum {
    GLM_OK = 0,
    GLM_ERR_INVALID_ARG = 1,   /* bad pointer, size, alignment or value      */
    GLM_ERR_UNSUPPORTED = 2,   /* valid but outside what this build supports */
    GLM_ERR_OOM = 3,           /* workspace allocation failed                 */
    GLM_ERR_CUDA = 4,          /* a CUDA runtime call or launch failed        */
    GLM_ERR_TIMEOUT = 5,       /* a device-side bounded wait expired          */
    GLM_ERR_NO_DEVICE = 6,     /* no usable sm_103 device                     */
    GLM_PENDING = 7            /* glm_server_poll: result not ready yet       */
} glm_status_t;

typedef enum {
    GLM_X_F32 = 0,
    GLM_X_BF16 = 1,
    GLM_X_FP8E4M3 = 2
} glm_xtype_t;

/* Handle descriptor: the shape of the dataset the handle evaluates. */
typedef struct {
    int64_t n_rows;       /* N >= 0                                           */
    int32_t p;            /* P >= 1                                           */
    int32_t ld;           /* row stride in elements, >= P, 16-byte rows       */
    int32_t k_max;        /* largest K any call will pass, 1..1024            */
    int32_t xtype;        /* glm_xtype_t                                      */
    double prior_sigma;   /* s > 0 of the N(0, s^2 I) prior                   */
    int32_t device;       /* CUDA device ordinal                              */
    uint32_t flags;       /* GLM_FLAG_* below                                 */
    int32_t g_max;        /* largest G of any grouped call (0: none)          */
} glm_desc_t;

/* Never route K > 1 evaluations to the tensor-core kernel. */
#define GLM_FLAG_NO_TENSOR_CORES 0x1u

/* f and g without the prior terms: the likelihood sums over this handle's
 * rows only. For row shards of one dataset evaluated separately (on several
 * GPUs, or in pieces) and summed afterwards; one shard keeps the prior so it
 * is counted once (§4.2.2 combine; the prior as in glm_logpost_grad). Applies
 * to glm_logpost_grad and glm_logpost_grad_host; glm_rwm_run refuses such a
 * handle (its accept step needs the whole posterior) and grouped calls always
 * include the group prior. */
#define GLM_FLAG_NO_PRIOR 0x2u

/* Read-only facts about a handle (for reports and tuning). */
typedef struct {
    int32_t sm_count;         /* SMs of the device                            */
    int32_t grid;             /* CTAs of the fused CUDA-core kernel           */
    int32_t tile_rows;        /* rows per staged tile                         */
    int32_t stages;           /* tiles in flight per CTA                      */
    int32_t smem_bytes;       /* dynamic shared memory per CTA                */
    int32_t tc_enabled;       /* 1 if K >= tc_min_k uses tcgen05 tensor cores */
    int32_t tc_min_k;
    int64_t workspace_bytes;  /* device memory owned by the handle            */
} glm_info_t;

/*
 * glm_create — validate *desc, select the device, allocate the handle's
 * workspace (per-CTA partial sums, completion ticket, status word) and choose
 * the kernel configuration. Returns GLM_OK and *out, or an error and
 * *out = NULL. Not stream-ordered: call it before any capture.
 */
GLM_API glm_status_t glm_create(const glm_desc_t *desc, glm_handle_t *out);

/* glm_destroy — synchronise the device, free the workspace and the handle.
 * NULL is accepted and ignored. */
GLM_API glm_status_t glm_destroy(glm_handle_t h);

/* glm_status_str — static English text of a status code. */
GLM_API const char *glm_status_str(glm_status_t s);

/* glm_get_info — fill *info for handle h. */
GLM_API glm_status_t glm_get_info(glm_handle_t h, glm_info_t *info);

/*
 * glm_logpost_grad — log-posterior f_k and gradient g_k (definitions above;
 * §3.1.1, §4.2) for K coefficient vectors in one fused pass over X, for the
 * handle's N rows.
 *   X       device, N x ld of the handle's xtype, 16-byte aligned
 *   x_scale device, P FP32 column scales for GLM_X_FP8E4M3, else NULL
 *   y       device, N bytes in {0, 1}
 *   beta    device, K x P FP32
 *   K       1 <= K <= k_max
 *   f_out   device, K FP64 (8-byte aligned)
 *   g_out   device, K x P FP32
 * f is accumulated per row in FP32 and across CTAs in FP64; g is accumulated
 * in FP32 and combined across CTAs in FP64. Results are deterministic: the
 * same inputs give bitwise the same outputs, whatever else runs. K >= tc_min_k
 * with BF16/FP8 storage and p <= 256 runs on the tcgen05 tensor cores (see
 * glm_get_info): there the coefficients and residuals enter the MMAs as sums
 * of terms of X's type (two BF16 terms; four and five E4M3 terms), the MMAs
 * accumulate in FP32, and the per-CTA partials of g are added in a fixed
 * order in FP32 (f in FP64).
 */
GLM_API glm_status_t glm_logpost_grad(glm_handle_t h, const void *X, const float *x_scale,
                              const uint8_t *y, const float *beta, int32_t K,
                              double *f_out, float *g_out, glm_stream_t stream);

/*
 * glm_logpost_grad_host — the same evaluation with HOST beta and results
 * (the offload pattern of §4.5: copy beta in, evaluate, copy f and g out).
 * X, x_scale and y stay device-resident. beta_host (K x P FP32), f_host (K)
 * and g_host (K x P) are host memory; pinned memory gives the fastest copies.
 * Synchronises `stream` before returning.
 */
GLM_API glm_status_t glm_logpost_grad_host(glm_handle_t h, const void *X, const float *x_scale,
                                   const uint8_t *y, const float *beta_host, int32_t K,
                                   double *f_host, float *g_host, glm_stream_t stream);

/*
 * glm_logpost_grad_grouped — the hierarchical-Bayes batch of §4.1: group m
 * owns rows [group_off[m], group_off[m+1]) of X and coefficient vector
 * beta_m; its conditional log-posterior is L_m(beta_m) + log N(beta_m | mu,
 * tau^2 I) with gradient g_L,m(beta_m) - (beta_m - mu) / tau^2.
 *   group_off device, G+1 int64, non-decreasing, group_off[G] <= N (the
 *             handle's n_rows); rows before group_off[0] are not read
 *   G         1 <= G <= the handle's g_max
 *   beta      device, G x P FP32;  mu device, P FP32;  tau > 0
 *   f_out     device, G FP64;      g_out device, G x P FP32
 * One persistent launch evaluates every group: the rows
 * [group_off[0], group_off[G]) are split evenly over all warps of the grid,
 * each warp streams its rows once through its own TMA ring and keeps one
 * group's sums in registers until the group ends; per-group sums meet in
 * fixed-point accumulators and the last warp to contribute to a group adds
 * the prior and writes its f and g. Empty groups are allowed (their f is the
 * prior alone). Deterministic. Malformed offsets (decreasing, or beyond N)
 * give undefined results; they are not checked on the host because the
 * offsets live in device memory.
 */
GLM_API glm_status_t glm_logpost_grad_grouped(glm_handle_t h, const void *X, const float *x_scale,
                                      const uint8_t *y, const int64_t *group_off, int32_t G,
                                      const float *beta, const float *mu, double tau,
                                      double *f_out, float *g_out, glm_stream_t stream);

/*
 * glm_autotune_grouped — choose the grouped pass's launch shape for this
 * handle by measurement: every feasible combination of kernel variant (row
 * streamed once per lane with shuffles, or register-resident narrow rows for
 * at most 32 used columns), warps per CTA, rows per TMA slot, slots per warp
 * ring and CTAs per SM is run `reps` times (1..1000) on the given inputs and
 * timed with CUDA events; the fastest is kept in the handle and used by later
 * glm_logpost_grad_grouped calls. Arguments as for glm_logpost_grad_grouped;
 * f_out and g_out receive a valid result. Synchronises `stream` and creates
 * CUDA events: call it outside stream capture, not on a latency-critical path.
 */
GLM_API glm_status_t glm_autotune_grouped(glm_handle_t h, const void *X, const float *x_scale,
                                          const uint8_t *y, const int64_t *group_off, int32_t G,
                                          const float *beta, const float *mu, double tau,
                                          double *f_out, float *g_out, int32_t reps,
                                          glm_stream_t stream);

/*
 * glm_grouped_set_shape / glm_grouped_get_shape — the grouped pass's launch
 * shape, set explicitly (for a reproducible configuration without timing) or
 * read back (after glm_autotune_grouped):
 *   variant      0: the warp-stream kernel (lanes split a slot's rows for the
 *                gradient, any P); 1: the narrow-row kernel (each lane keeps
 *                its row, the group's coefficients and the gradient sums in
 *                registers; only when the used columns fit 32 per row)
 *   warps        warps per CTA: 4, 8, 12 or 16 (at most 12 for variant 1)
 *   units        32-row units per copy slot: 1, or 2 or 4 with variant 1
 *   stages       copy slots per warp ring, 2..4
 *   ctas_per_sm  1 or 2 (the grid is that many CTAs per SM)
 * These are the shapes glm_autotune_grouped chooses from. Set returns
 * GLM_ERR_INVALID_ARG for a value outside these ranges or a variant that does
 * not apply to the handle's P, GLM_ERR_UNSUPPORTED if the shape's shared
 * memory does not fit, and GLM_ERR_UNSUPPORTED for a handle created without
 * grouped support (g_max = 0); on an error the shape is unchanged. Get writes
 * each non-null pointer. Neither call touches the device; do not call them
 * while another thread launches on the same handle.
 */
GLM_API glm_status_t glm_grouped_set_shape(glm_handle_t h, int32_t variant, int32_t warps,
                                           int32_t units, int32_t stages, int32_t ctas_per_sm);
GLM_API glm_status_t glm_grouped_get_shape(glm_handle_t h, int32_t *variant, int32_t *warps,
                                           int32_t *units, int32_t *stages,
                                           int32_t *ctas_per_sm);

/*
 * glm_rwm_run — K independent random-walk Metropolis chains (the sampler of
 * §2.2 that consumes the log-posterior), n_steps steps each, entirely on the
 * device: step t proposes beta'_k = fmaf(step, z[t][k], beta_k) in FP32,
 * evaluates f(beta'_k) with the fused kernel (one launch per step), and
 * accepts iff log_u[t][k] < f(beta'_k) - f(beta_k), compared in FP64.
 *   z          device, n_steps x K x P FP32 standard normals
 *   log_u      device, n_steps x K FP64 logs of uniforms
 *   beta_state device, K x P FP32 chain state, updated in place
 *   f_state    device, K FP64 log-posterior at beta_state, updated in place;
 *              computed first when init_f != 0
 *   samples    device, n_steps x K x P FP32 or NULL (state after each step)
 *   accept     device, n_steps x K bytes or NULL (1 = accepted)
 *   logpost    device, n_steps x K FP64 or NULL (f after each step)
 * 1 <= K <= min(k_max, 8). Asynchronous on `stream`.
 */
GLM_API glm_status_t glm_rwm_run(glm_handle_t h, const void *X, const float *x_scale,
                         const uint8_t *y, int32_t K, int32_t n_steps, float step,
                         const float *z, const double *log_u, float *beta_state,
                         double *f_state, int32_t init_f, float *samples,
                         uint8_t *accept, double *logpost, glm_stream_t stream);

/*
 * glm_quantize — convert a device FP32 matrix X32 (N x ld32, first P columns)
 * to the handle's storage type in Xq (N x ld of that type, padding zero):
 * GLM_X_BF16 rounds to nearest even; GLM_X_FP8E4M3 first sets
 * x_scale[j] = the smallest power of two s with 448 s >= max_n |x_nj|
 * (1 for an all-zero column) and stores the E4M3 code nearest to x_nj / s,
 * ties to even, saturating. x_scale must be non-NULL exactly for FP8.
 * Uses the handle's workspace; asynchronous on `stream`.
 */
GLM_API glm_status_t glm_quantize(glm_handle_t h, const float *X32, int32_t ld32, void *Xq,
                          float *x_scale, glm_stream_t stream);

/*
 * glm_sync — synchronise `stream`, then read and clear the handle's
 * device status word. Returns GLM_ERR_TIMEOUT if a bounded device wait
 * expired since the last glm_sync (the outputs of that call are then NaN),
 * GLM_ERR_CUDA on an asynchronous CUDA error, else GLM_OK.
 */
GLM_API glm_status_t glm_sync(glm_handle_t h, glm_stream_t stream);

/*
 * glm_selftest_wait_timeout — launch one CTA that waits on a shared-memory
 * barrier nothing will ever complete, with a limit of `spin_limit` polls;
 * when the limit runs out the kernel records GLM_ERR_TIMEOUT in the status
 * word and returns. Exists so tests can check the bounded-wait path without
 * faulting or hanging the GPU. Read the result with glm_sync.
 */
GLM_API glm_status_t glm_selftest_wait_timeout(glm_handle_t h, int32_t spin_limit,
                                       glm_stream_t stream);

/*
 * glm_logpost_grad_noalloc — the same evaluation as glm_logpost_grad, for
 * callers that cannot allocate device memory when they evaluate: code running
 * under a memory pool or arena that owns all of the process's device memory,
 * a real-time loop that must not take the allocator's locks or risk running
 * out of memory mid-run, or a plugin whose host forbids allocation. The
 * paper has no counterpart; this is a deployment convenience.
 *
 * There is no handle: the dataset shape is passed directly (n_rows, p, ld,
 * xtype, prior_sigma as in glm_desc_t), and the call runs on the calling
 * thread's current CUDA device, where all pointers must live. Arguments and
 * results are as for glm_logpost_grad, with 1 <= K <= 1024.
 *
 * Memory. The call allocates nothing: no cudaMalloc, cudaFree or allocating
 * library routine. Its scratch (cross-CTA accumulators, completion ticket,
 * flag words) is one fixed device array of about 263 KB inside this library,
 * which every GPU that loads the library holds until the process exits. The
 * array sizes the problem: p > 1024 returns GLM_ERR_INVALID_ARG.
 *
 * Sharing. Every call on a device uses the same array, which keeps what the
 * last call left; each call clears it on its stream before launching. Calls
 * whose work overlaps on the GPU (different streams, or different host
 * threads on one device, without ordering between them) race on the array
 * and give wrong results: order them on one stream.
 *
 * Set-up. The first call on each device looks up the array's device address
 * (cudaGetSymbolAddress, with that device current); make that first call
 * before any stream capture. The address is kept per device together with
 * the CUDA context it belongs to: after cudaDeviceReset (a new context) the
 * next call looks it up again, so that call is a set-up call too.
 *
 * Errors: as glm_create and glm_logpost_grad (GLM_ERR_INVALID_ARG for a
 * non-finite prior_sigma or misaligned pointers; GLM_ERR_UNSUPPORTED for
 * rows wider than 1 MiB), nothing launched. A bounded device wait that
 * expires shows up as NaN results.
 */
GLM_API glm_status_t glm_logpost_grad_noalloc(const void *X, const float *x_scale,
                                              const uint8_t *y, int64_t n_rows, int32_t p,
                                              int32_t ld, int32_t xtype, double prior_sigma,
                                              const float *beta, int32_t K, double *f_out,
                                              float *g_out, glm_stream_t stream);

/* ------------------------------------------------------------------------
 * Serving loop with continuous batching.
 *
 * The paper evaluates one posterior at a time; it has no serving layer. This
 * is a deployment layer over glm_logpost_grad for many clients that ask for
 * f and g of their own coefficient vectors against datasets held resident on
 * one GPU.
 *
 * A server owns a scheduler thread, a pool of `streams` CUDA streams and
 * pinned host staging per stream. Requests are queued in arrival order. The
 * scheduler takes the oldest waiting request, merges later waiting requests
 * for the same dataset while the merged batch holds at most max_batch_k
 * vectors, and runs the batch on a free stream once memory admits it.
 * Batches for different datasets run concurrently on different streams.
 *
 * Device memory admission. The server keeps one account of the device memory
 * it stands for, against a budget (hbm_budget_bytes; 0 = the device's free
 * memory when the server is created, less one sixteenth kept back):
 *  - resident: each registered dataset's X, y and x_scale (the caller's
 *    memory, counted at its size) plus the evaluation workspaces the server
 *    creates for it, one per stream slot;
 *  - in flight: each running batch's coefficient, f and g buffers, taken
 *    from a stream-ordered pool the server owns and returned when the batch's
 *    copies are done.
 * A dataset whose footprint does not fit what the budget leaves, or whose
 * workspaces the device cannot allocate, is refused (GLM_ERR_OOM, nothing
 * kept). A request whose batch could not fit even with nothing in flight is
 * refused at submit (GLM_ERR_OOM). Otherwise a batch that does not fit now
 * is first trimmed to the requests that do (the oldest always stays in it)
 * and, when even the oldest does not fit, deferred until a running batch
 * completes; the same holds when the pool cannot get the memory from the
 * device. Deferred requests keep their place in the queue.
 *
 * Each vector's result is the one glm_logpost_grad gives for it in a batch
 * of that batch's size: batches of 16 or more BF16 or FP8 vectors take the
 * tensor-core pass where the shape allows it (p <= 256), the others the
 * CUDA-core pass, so a result alone and inside a mix agree to the evaluation
 * tolerance. Each request reports the pass that served its batch.
 * ---------------------------------------------------------------------- */
typedef struct glm_server *glm_server_t;

typedef struct {
    int32_t device;            /* CUDA device                                  */
    int32_t streams;           /* stream slots, 1..16                          */
    int32_t max_batch_k;       /* largest merged batch in vectors, 1..1024     */
    int32_t max_pending;       /* queue limit; submit past it returns OOM      */
    int64_t hbm_budget_bytes;  /* device memory account (0 = default, above)   */
} glm_server_desc_t;

/* The evaluation pass that served a batch (glm_request_info_t.path). */
typedef enum {
    GLM_PATH_NONE = 0,             /* not run (failed before the evaluation)  */
    GLM_PATH_CUDA_CORES = 1,       /* fused CUDA-core pass                    */
    GLM_PATH_TENSOR_CORES = 2      /* tcgen05 pass (BF16 or FP8 operands)     */
} glm_path_t;

typedef struct {
    int64_t submit_ns;         /* steady-clock times of the request's life     */
    int64_t start_ns;          /* batch launched                               */
    int64_t done_ns;           /* results copied back to the host              */
    int32_t batch_k;           /* vectors in the batch that carried it         */
    int32_t batch_requests;    /* requests merged into that batch              */
    int32_t k;                 /* this request's vectors                       */
    int32_t status;            /* glm_status_t of the request                  */
    int32_t path;              /* glm_path_t of the batch that carried it      */
    int32_t deferrals;         /* times its batch was deferred for memory      */
} glm_request_info_t;

typedef struct {
    int64_t requests_done;
    int64_t requests_failed;
    int64_t requests_waiting;
    int64_t batches;
    int64_t vectors_done;
    int64_t hbm_budget_bytes;
    int64_t hbm_in_flight_bytes;
    int64_t hbm_resident_bytes;   /* registered datasets and their workspaces   */
    int64_t batches_tensor_cores; /* batches served by the tensor-core pass     */
    int64_t deferrals;            /* dispatches deferred for memory             */
    int64_t trimmed_batches;      /* batches cut short to fit the budget        */
    int64_t refused_requests;     /* submits refused: batch can never fit       */
    int32_t max_concurrent_batches;
    int32_t last_cuda_error;   /* cudaError_t of the last failed step (0: none) */
    int32_t last_error_site;   /* glm_server_error_site_t of that step          */
} glm_server_stats_t;

/* Where a failed batch failed (glm_server_stats_t.last_error_site). */
typedef enum {
    GLM_SERVER_SITE_NONE = 0,
    GLM_SERVER_SITE_COPY_IN = 1,      /* coefficients host -> device         */
    GLM_SERVER_SITE_EVALUATE = 2,     /* glm_logpost_grad refused or failed  */
    GLM_SERVER_SITE_COPY_OUT = 3,     /* f, g or status device -> host       */
    GLM_SERVER_SITE_COMPLETION = 4,   /* completion callback not enqueued    */
    GLM_SERVER_SITE_DEVICE_WAIT = 5   /* a bounded device wait expired       */
} glm_server_error_site_t;

/* Create a server on desc->device. Returns GLM_ERR_NO_DEVICE without a GPU,
 * GLM_ERR_INVALID_ARG on a bad descriptor, GLM_ERR_OOM if the budget is
 * below 64 KB or the batch memory pool or staging cannot be created. */
GLM_API glm_status_t glm_server_create(const glm_server_desc_t *desc, glm_server_t *out);

/* Register a device-resident dataset (same layout and storage types as the
 * handle API: X row-major n_rows x ld, y n_rows bytes, x_scale for FP8). The
 * caller keeps X, x_scale and y alive and unchanged until the dataset is
 * removed or the server destroyed. Creates one evaluation handle per stream
 * slot. Returns the dataset's id, or GLM_ERR_OOM (nothing registered) when
 * the dataset's footprint does not fit the budget that is left or the
 * device cannot allocate its workspaces. */
GLM_API glm_status_t glm_server_add_dataset(glm_server_t s, const void *X, const float *x_scale,
                                            const uint8_t *y, int64_t n_rows, int32_t p,
                                            int32_t ld, int32_t xtype, double prior_sigma,
                                            int32_t *dataset_id);

/* Unregister a dataset: GLM_PENDING (nothing changed) while requests for it
 * are waiting or running, else its workspaces are freed, its footprint leaves
 * the account and later submits for it return GLM_ERR_INVALID_ARG. The
 * caller may free X, x_scale and y once this returns GLM_OK. */
GLM_API glm_status_t glm_server_remove_dataset(glm_server_t s, int32_t dataset_id);

/* Queue a request: K (1..max_batch_k) FP32 vectors beta_host[K x P] in HOST
 * memory, copied before the call returns. Returns a request id, or
 * GLM_ERR_OOM when max_pending requests are already waiting or when a batch
 * of K vectors for this dataset could not fit the budget even with nothing
 * in flight. Thread-safe. */
GLM_API glm_status_t glm_server_submit(glm_server_t s, int32_t dataset_id, const float *beta_host,
                                       int32_t K, uint64_t *request_id);

/* Non-blocking: GLM_PENDING while the request runs; when it has finished,
 * copies f (K FP64) and g (K x P FP32) into the HOST buffers given (either
 * may be NULL), fills *info if not NULL, forgets the request and returns its
 * status: GLM_OK, the error glm_logpost_grad returned for its batch,
 * GLM_ERR_CUDA when a copy or launch of the batch failed, or GLM_ERR_TIMEOUT
 * when a bounded device wait of the batch expired (results not valid). An
 * unknown id returns GLM_ERR_INVALID_ARG. */
GLM_API glm_status_t glm_server_poll(glm_server_t s, uint64_t request_id, double *f_host,
                                     float *g_host, glm_request_info_t *info);

/* Blocking form of glm_server_poll, waiting up to timeout_ms milliseconds
 * (GLM_ERR_TIMEOUT if the request has not finished by then; it stays queued). */
GLM_API glm_status_t glm_server_wait(glm_server_t s, uint64_t request_id, double *f_host,
                                     float *g_host, glm_request_info_t *info, int32_t timeout_ms);

/* Counters since creation. */
GLM_API glm_status_t glm_server_stats(glm_server_t s, glm_server_stats_t *stats);

/* Stop the scheduler, drain the streams and free everything the server owns
 * (not the datasets' memory). Requests still waiting are dropped. */
GLM_API glm_status_t glm_server_destroy(glm_server_t s);

/* ------------------------------------------------------------------------
 * Gibbs sweeps of univariate slice sampling with the differential update of
 * X beta (§3.4.4). The sampler updates one coefficient at a time; changing
 * beta_k by d changes eta = X beta by d X_k, so with eta kept on the device a
 * log-posterior evaluation along coordinate k reads column k of X only.
 * X is stored column-major here ("Xt": column k at Xt + k * ld, FP32).
 *
 * Each coordinate update is Neal's slice sampler: slice level
 * log y = f(beta) + log u0; initial interval L0 = x0 - w U, R0 = L0 + w;
 * stepping out at most J = floor(m V) steps left and K = m - 1 - J right
 * (L_j = L0 - j w, R_j = R0 + j w); then shrinkage proposals
 * x1 = L + S_t (R - L) until log y < f(x1), moving the interval end on the
 * side of x1 toward x1 otherwise. Interval arithmetic is FP32 with each
 * operation rounded separately. After s_max rejected proposals the
 * coordinate keeps x0. The device evaluates the next `spec` proposals of
 * the shrinkage sequence in one pass (each assuming the earlier ones are
 * rejected, as the sequence is fixed by the random numbers until the first
 * acceptance) and applies them in order: the result equals one proposal at a
 * time. f is the full log-posterior (likelihood plus the
 * N(0, s^2 I) prior, as for glm_logpost_grad). Random numbers are inputs:
 * log_u0 (n_sweeps x P FP64) and uni (n_sweeps x P x (2 + s_max) FP32: U, V,
 * then the shrinkage uniforms S_t), all uniforms in (0, 1).
 * ---------------------------------------------------------------------- */
typedef struct glm_slice *glm_slice_t;

typedef struct {
    int64_t n_rows;       /* N >= 1                                            */
    int64_t ld;           /* column stride of Xt in elements: >= N, multiple of 4 */
    int32_t p;            /* P >= 1                                            */
    int32_t m;            /* stepping-out limit, 1..16                         */
    int32_t s_max;        /* shrinkage proposals per update, 1..64             */
    int32_t device;
    float w;              /* initial interval width > 0                        */
    int32_t spec;         /* shrinkage proposals per evaluation pass, 1..16;
                             0 selects the default (2)                        */
    double prior_sigma;   /* s > 0                                             */
} glm_slice_desc_t;

/* Create a sampler for one dataset shape. GLM_ERR_UNSUPPORTED when a CTA's
 * rows (about N / 152) do not fit in shared memory (N above about 2.5 M). */
GLM_API glm_status_t glm_slice_create(const glm_slice_desc_t *desc, glm_slice_t *out);
GLM_API glm_status_t glm_slice_destroy(glm_slice_t s);

/* eta = X beta (device N FP32) from Xt and beta (device P FP32). Needed
 * before the first glm_slice_run of a chain and whenever beta is set by the
 * caller. */
GLM_API glm_status_t glm_slice_eta(glm_slice_t s, const float *Xt, const float *beta, float *eta,
                                   glm_stream_t stream);

/* The log-posterior at beta with beta_k replaced by x[c], c < M <= 16
 * (device FP32 candidates), into f_out[c] (device FP64): one pass over column
 * k and eta, which must equal X beta. */
GLM_API glm_status_t glm_slice_coord_logpost(glm_slice_t s, const float *Xt, const uint8_t *y,
                                             const float *eta, const float *beta, int32_t k,
                                             const float *x, int32_t M, double *f_out,
                                             glm_stream_t stream);

/* n_sweeps Gibbs sweeps (coordinates 0..P-1 in order) from the state
 * (beta, eta = X beta, f_state = f(beta); init_f = 1 computes f_state first),
 * one cooperative launch. Updates beta, eta and f_state in place (device).
 * Optional per-update outputs (device, n_sweeps x P, or NULL): xk_out the
 * coordinate's new value, gk_out f after the update, nshrink_out rejected
 * shrinkage proposals (s_max: kept x0). Asynchronous; a bounded device wait
 * that expires is reported by glm_slice_sync as GLM_ERR_TIMEOUT (the state
 * is then not valid). */
GLM_API glm_status_t glm_slice_run(glm_slice_t s, const float *Xt, const uint8_t *y, float *eta,
                                   float *beta, double *f_state, int32_t init_f, int32_t n_sweeps,
                                   const double *log_u0, const float *uni, float *xk_out,
                                   double *gk_out, int32_t *nshrink_out, glm_stream_t stream);

/* Synchronise the stream and return the sampler's device status. */
GLM_API glm_status_t glm_slice_sync(glm_slice_t s, glm_stream_t stream);

/* ------------------------------------------------------------------------
 * Square-lattice Ising model, checkerboard Gibbs sampling (§4.3.1).
 * Spins s_i in {0, 1} on a rows x cols lattice (cols even), each node
 * coupled to its 4 lattice neighbours with weight w, free boundary (a
 * missing neighbour contributes nothing). Gibbs conditional:
 * P(s_i = 1 | rest) = 1 / (1 + exp(-z_i)), z_i = b_i + w * sum_j s_j over
 * the neighbours j of i (the energy is E(s) = -sum b_i s_i - w sum_<ij>
 * s_i s_j). Colour c holds the sites with (row + col) % 2 == c; a sweep
 * updates colour 0, then colour 1, setting s_i = 1 iff u_i < P(s_i = 1).
 *
 * Layout: each colour in its own dense plane of rows x (cols / 2) elements,
 * plane entry (r, j) = site (r, 2j + (r + c) % 2) (the unit-stride colour
 * layout of §4.3.1). All buffers are device memory owned by the caller.
 * Spins must be 0 or 1.
 * ---------------------------------------------------------------------- */

/* Natural row-major rows x cols array (elem_bytes 1 or 4) into its two
 * colour planes, and back. */
GLM_API glm_status_t glm_ising_split(const void *nat, int32_t elem_bytes, int32_t rows, int32_t cols,
                                     void *plane0, void *plane1, glm_stream_t stream);
GLM_API glm_status_t glm_ising_merge(const void *plane0, const void *plane1, int32_t elem_bytes,
                                     int32_t rows, int32_t cols, void *nat, glm_stream_t stream);

/* n_sweeps checkerboard sweeps in place on the spin planes s0, s1 (uint8)
 * with bias planes b0, b1 (FP32) and coupling w. u: the batch of uniforms in
 * [0, 1), n_sweeps x 2 x rows x (cols / 2) FP32 (sweep, colour, then plane
 * order). ones_out (optional, 8-byte aligned, n_sweeps x 2 int64): the number
 * of 1s in plane c after half-sweep (t, c). Asynchronous: one launch per
 * half-sweep. Unit-stride vector path when cols / 2 is a multiple of 8 and
 * all planes and u are 16-byte aligned, else per-site. */
GLM_API glm_status_t glm_ising_sweeps(uint8_t *s0, uint8_t *s1, const float *b0, const float *b1,
                                      int32_t rows, int32_t cols, float w, int32_t n_sweeps,
                                      const float *u, int64_t *ones_out, glm_stream_t stream);

/* ------------------------------------------------------------------------
 * Log-posterior, gradient and Hessian in one pass (§4.2's derivatives one
 * order further, which §5.2 proposes for Newton-type and Riemannian
 * samplers), one coefficient vector, FP32 X with P <= 64:
 *   f, g as glm_logpost_grad (prior N(0, s^2 I));
 *   H = -X^T diag(mu (1 - mu)) X - I / s^2, mu_n = 1 / (1 + exp(-x_n . beta)).
 * ---------------------------------------------------------------------- */
typedef struct glm_hess *glm_hess_t;

/* A Hessian evaluator for N x P row-major FP32 X with row stride ld
 * (P <= ld <= 64, ld a multiple of 4): per-CTA partials are allocated here. */
GLM_API glm_status_t glm_hess_create(int64_t n_rows, int32_t p, int32_t ld, double prior_sigma,
                                     int32_t device, glm_hess_t *out);
GLM_API glm_status_t glm_hess_destroy(glm_hess_t h);

/* f_out (1 FP64), g_out (P FP32), H_out (P x P FP32 row-major, symmetric) at
 * beta (P FP32), all device memory; X 16-byte aligned, y N bytes in {0, 1}.
 * Asynchronous: one pass over X plus a fixed-order combine (deterministic). */
GLM_API glm_status_t glm_hess_eval(glm_hess_t h, const float *X, const uint8_t *y,
                                   const float *beta, double *f_out, float *g_out, float *H_out,
                                   glm_stream_t stream);

/* Synchronise the stream and return the evaluator's device status
 * (GLM_ERR_TIMEOUT if a bounded wait expired; the results are then NaN). */
GLM_API glm_status_t glm_hess_sync(glm_hess_t h, glm_stream_t stream);

#ifdef __cplusplus
}
#endif

#endif /* GLM_H */
