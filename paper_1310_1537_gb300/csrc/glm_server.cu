// Serving loop with continuous batching over device-resident datasets.
//
// Requests (a dataset id and K coefficient vectors on the host) are queued by
// glm_server_submit and returned through glm_server_poll / glm_server_wait. A
// scheduler thread forms batches: it takes the oldest waiting request, merges
// later requests for the same dataset while the batch stays within
// max_batch_k vectors, and launches the batch on a free stream slot once the
// device memory account admits it. Batches for different datasets run
// concurrently on different streams; requests that arrive while others are
// on the GPU join the next batch formed. Each slot copies its batch's
// coefficients in (pinned staging), evaluates it with the dataset's handle
// for that slot, copies f and g out and completes through a host callback
// that scatters results to the requests.
//
// Device memory account. One budget covers what the server stands for on the
// device: every registered dataset (X, y, x_scale at their size, plus the
// workspaces of its per-slot handles: "resident") and every running batch's
// coefficient, f and g buffers ("in flight"). Batch buffers come from a
// stream-ordered memory pool owned by the server (cudaMallocFromPoolAsync on
// the slot's stream, freed on the same stream after the copies out), with
// reuse across streams limited to frees that have completed, so the pool
// never makes one slot's stream wait for another's. Admission: a dataset
// that does not fit the budget is refused at registration; a request whose
// batch could never fit is refused at submit; a batch that does not fit now
// is trimmed to the requests that do, or deferred until a completion when
// even the oldest request does not fit; a pool allocation the device cannot
// serve defers the same way (or fails the request with GLM_ERR_OOM when
// nothing is in flight that could give memory back).
//
// The evaluation of a vector does not depend on which other vectors share its
// batch beyond the kernel path chosen for the batch size (CUDA cores below 16
// vectors, tensor cores from 16 where the shape allows), so a result alone
// and in a mix agree to the evaluation tolerance; each request reports the
// path that served it.
#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <thread>
#include <vector>

#include "glm_internal.cuh"

namespace {

int64_t now_ns()
{
    return std::chrono::duration_cast<std::chrono::nanoseconds>(
               std::chrono::steady_clock::now().time_since_epoch())
        .count();
}

struct Dataset {
    const void *X;
    const float *x_scale;
    const uint8_t *y;
    int64_t n;
    int p;
    int ld;
    int xtype;
    double sigma;
    std::vector<glm_handle_t> handles;      // one per slot
    size_t footprint = 0;                   // bytes counted as resident
    int outstanding = 0;                    // requests waiting or running
    bool live = true;                       // false once removed
};

struct Request {
    int ds;
    int K;
    std::vector<float> beta;
    std::vector<double> f;
    std::vector<float> g;
    int64_t submit_ns = 0;
    int64_t start_ns = 0;
    int64_t done_ns = 0;
    int batch_k = 0;
    int batch_requests = 0;
    int path = GLM_PATH_NONE;
    int deferrals = 0;
    bool deferred_now = false;              // counted in the current deferral
    int state = 0;                          // 0 waiting, 1 running, 2 done, 3 failed
    glm_status_t status = GLM_OK;
};

struct Slot {
    cudaStream_t stream = nullptr;
    bool busy = false;
    float *beta_pin = nullptr;              // pinned host staging
    double *f_pin = nullptr;
    float *g_pin = nullptr;
    unsigned *status_pin = nullptr;         // the batch handle's device status word
    size_t cap_kp = 0;                      // floats of beta/g staging
    // current batch (staging pointers fixed at dispatch: add_dataset may
    // replace the slot's buffers while the batch runs)
    float *b_beta = nullptr;
    double *b_f = nullptr;
    float *b_g = nullptr;
    std::vector<uint64_t> ids;
    int ds = -1;
    int K = 0;
    void *dev = nullptr;                    // batch buffers from the pool
    size_t dev_bytes = 0;                   // bytes counted as in flight
    int path = GLM_PATH_NONE;
    glm_status_t launch_status = GLM_OK;
    int index = 0;                          // position in the slot pool
    struct glm_server *srv = nullptr;
};

}  // namespace

struct glm_server {
    glm_server_desc_t d;
    int device = 0;
    std::mutex mu;
    std::condition_variable cv;             // scheduler wake-ups
    std::condition_variable done_cv;        // request completions
    std::vector<Dataset> datasets;
    std::map<uint64_t, Request> requests;
    std::deque<uint64_t> waiting;           // request ids, ascending = arrival order
    std::vector<std::unique_ptr<Slot>> slots;
    uint64_t next_id = 1;
    bool stop = false;
    std::thread sched;
    cudaMemPool_t pool = nullptr;           // batch buffers
    std::vector<void *> retired;            // outgrown pinned staging buffers
    // device memory account
    size_t budget = 0;
    size_t resident = 0;
    size_t in_flight = 0;
    // statistics
    uint64_t n_done = 0, n_failed = 0, n_batches = 0, vectors_done = 0;
    uint64_t n_batches_tc = 0, n_deferrals = 0, n_trimmed = 0, n_refused = 0;
    int max_concurrent = 0;
    int last_cuda_error = 0;                // cudaError_t of the last failed step
    int last_error_site = 0;                // glm_server_error_site_t of that step
};

namespace {

size_t round256(size_t b) { return (b + 255) / 256 * 256; }

// Device bytes of a batch of K vectors of P coefficients: beta, f and g.
size_t batch_bytes(int K, int p)
{
    return round256((size_t)K * p * 4) + round256((size_t)K * 8) + round256((size_t)K * p * 4);
}

// What the budget leaves for batches (called with the lock held).
size_t batch_room(const glm_server *s)
{
    const size_t used = s->resident + s->in_flight;
    return used >= s->budget ? 0 : s->budget - used;
}

// Fail one waiting request (lock held); it is no longer in `waiting`.
void fail_request(glm_server *s, Request &r, glm_status_t st)
{
    r.state = 3;
    r.status = st;
    r.done_ns = now_ns();
    s->n_failed++;
    s->datasets[(size_t)r.ds].outstanding--;
}

// Host callback at the end of a batch: scatter results, free the slot. The
// batch buffers went back to the pool on the stream before this runs.
void CUDART_CB batch_done(void *arg)
{
    Slot *sl = static_cast<Slot *>(arg);
    glm_server *s = sl->srv;
    const int64_t t = now_ns();
    {
        std::lock_guard<std::mutex> lock(s->mu);
        Dataset &D = s->datasets[(size_t)sl->ds];
        const int p = D.p;
        if (sl->launch_status == GLM_OK && (*sl->status_pin & glm::kDevTimeout)) {
            sl->launch_status = GLM_ERR_TIMEOUT;
            s->last_error_site = GLM_SERVER_SITE_DEVICE_WAIT;
        }
        if (sl->launch_status == GLM_OK && sl->path == GLM_PATH_TENSOR_CORES)
            s->n_batches_tc++;
        int k0 = 0;
        for (uint64_t id : sl->ids) {
            auto it = s->requests.find(id);
            if (it == s->requests.end())
                continue;
            Request &r = it->second;
            r.path = sl->launch_status == GLM_OK ? sl->path : GLM_PATH_NONE;
            if (sl->launch_status == GLM_OK) {
                std::memcpy(r.f.data(), sl->b_f + k0, sizeof(double) * (size_t)r.K);
                std::memcpy(r.g.data(), sl->b_g + (size_t)k0 * p, sizeof(float) * (size_t)r.K * p);
                r.state = 2;
                s->n_done++;
                s->vectors_done += (uint64_t)r.K;
            } else {
                r.state = 3;
                r.status = sl->launch_status;
                s->n_failed++;
            }
            r.done_ns = t;
            D.outstanding--;
            k0 += r.K;
        }
        s->in_flight -= sl->dev_bytes;
        sl->dev = nullptr;
        sl->dev_bytes = 0;
        sl->busy = false;
        sl->ids.clear();
    }
    s->cv.notify_all();
    s->done_cv.notify_all();
}

// Put requests taken for a batch back into the queue in arrival order.
void requeue_locked(glm_server *s, const std::vector<uint64_t> &ids)
{
    for (uint64_t id : ids)
        s->waiting.push_back(id);
    std::sort(s->waiting.begin(), s->waiting.end());
}

// Count one deferral episode for the request at the head of the queue.
void note_deferral_locked(glm_server *s, Request &r)
{
    if (!r.deferred_now) {
        r.deferred_now = true;
        r.deferrals++;
        s->n_deferrals++;
    }
}

// Called with the lock held: form and launch batches while slots and memory allow.
void dispatch_locked(glm_server *s, std::unique_lock<std::mutex> &lock)
{
    for (;;) {
        if (s->waiting.empty())
            return;
        Slot *sl = nullptr;
        for (auto &u : s->slots)
            if (!u->busy) {
                sl = u.get();
                break;
            }
        if (!sl)
            return;
        // the oldest waiting request decides the dataset
        const uint64_t first = s->waiting.front();
        Request &r0 = s->requests[first];
        const int ds = r0.ds;
        const int p = s->datasets[(size_t)ds].p;
        const size_t room = batch_room(s);
        if (batch_bytes(r0.K, p) > room) {
            if (s->in_flight == 0) {
                // nothing running could give memory back: the budget shrank
                // under it (datasets registered after it was queued)
                s->waiting.pop_front();
                s->n_refused++;
                fail_request(s, r0, GLM_ERR_OOM);
                s->done_cv.notify_all();
                continue;
            }
            note_deferral_locked(s, r0);
            return;                         // a completion wakes the scheduler
        }
        // merge later same-dataset requests that keep the batch within
        // max_batch_k vectors and within the room the budget leaves
        std::vector<uint64_t> ids;
        int K = 0;
        bool trimmed = false;
        for (auto it = s->waiting.begin(); it != s->waiting.end();) {
            Request &r = s->requests[*it];
            if (r.ds == ds && K + r.K <= s->d.max_batch_k) {
                if (batch_bytes(K + r.K, p) <= room) {
                    ids.push_back(*it);
                    K += r.K;
                    it = s->waiting.erase(it);
                    continue;
                }
                trimmed = true;
            }
            ++it;
        }
        const size_t bytes = batch_bytes(K, p);
        s->in_flight += bytes;              // reserved before the lock is dropped
        sl->busy = true;
        sl->ids = ids;
        sl->ds = ds;
        sl->K = K;
        sl->dev = nullptr;
        sl->dev_bytes = bytes;
        sl->path = GLM_PATH_NONE;
        sl->launch_status = GLM_OK;
        sl->b_beta = sl->beta_pin;
        sl->b_f = sl->f_pin;
        sl->b_g = sl->g_pin;
        int k0 = 0;
        for (uint64_t id : ids) {
            Request &r = s->requests[id];
            std::memcpy(sl->b_beta + (size_t)k0 * p, r.beta.data(), sizeof(float) * (size_t)r.K * p);
            k0 += r.K;
        }
        // copy what the launch needs: add_dataset may grow the vector meanwhile
        const Dataset &D = s->datasets[(size_t)ds];
        glm_handle_t h = D.handles[(size_t)sl->index];
        const void *X = D.X;
        const float *x_scale = D.x_scale;
        const uint8_t *y = D.y;
        // allocate and launch without the lock: the callback takes it
        lock.unlock();
        void *dev = nullptr;
        cudaError_t ce = cudaMallocFromPoolAsync(&dev, bytes, s->pool, sl->stream);
        if (ce != cudaSuccess) {
            cudaGetLastError();
            lock.lock();
            s->in_flight -= bytes;
            sl->busy = false;
            sl->ids.clear();
            requeue_locked(s, ids);
            Request &h0 = s->requests[s->waiting.front()];
            if (s->in_flight == 0) {
                // the device cannot give even this with nothing else running
                for (uint64_t id : ids) {
                    auto w = std::find(s->waiting.begin(), s->waiting.end(), id);
                    if (w != s->waiting.end())
                        s->waiting.erase(w);
                    s->n_refused++;
                    fail_request(s, s->requests[id], GLM_ERR_OOM);
                }
                s->last_cuda_error = (int)ce;
                s->last_error_site = GLM_SERVER_SITE_COPY_IN;
                s->done_cv.notify_all();
                continue;
            }
            note_deferral_locked(s, h0);
            return;
        }
        sl->dev = dev;
        uint8_t *base = static_cast<uint8_t *>(dev);
        float *dbeta = reinterpret_cast<float *>(base);
        double *df = reinterpret_cast<double *>(base + round256((size_t)K * p * 4));
        float *dg = reinterpret_cast<float *>(reinterpret_cast<uint8_t *>(df) +
                                              round256((size_t)K * 8));
        glm_status_t st = GLM_OK;
        int site = 0;
        *sl->status_pin = 0;
        if ((ce = cudaMemcpyAsync(dbeta, sl->b_beta, sizeof(float) * (size_t)K * p,
                                  cudaMemcpyHostToDevice, sl->stream)) != cudaSuccess) {
            st = GLM_ERR_CUDA;
            site = GLM_SERVER_SITE_COPY_IN;
        }
        if (st == GLM_OK) {
            st = glm_logpost_grad(h, X, x_scale, y, dbeta, K, df, dg,
                                  reinterpret_cast<glm_stream_t>(sl->stream));
            if (st != GLM_OK) {
                site = GLM_SERVER_SITE_EVALUATE;
                ce = cudaGetLastError();
            } else {
                sl->path = h->last_path;    // this slot's handle: only this thread uses it
            }
        }
        if (st == GLM_OK &&
            ((ce = cudaMemcpyAsync(sl->b_f, df, sizeof(double) * (size_t)K,
                                   cudaMemcpyDeviceToHost, sl->stream)) != cudaSuccess ||
             (ce = cudaMemcpyAsync(sl->b_g, dg, sizeof(float) * (size_t)K * p,
                                   cudaMemcpyDeviceToHost, sl->stream)) != cudaSuccess ||
             (ce = cudaMemcpyAsync(sl->status_pin, h->status, sizeof(unsigned),
                                   cudaMemcpyDeviceToHost, sl->stream)) != cudaSuccess ||
             (ce = cudaMemsetAsync(h->status, 0, sizeof(unsigned), sl->stream)) != cudaSuccess)) {
            st = GLM_ERR_CUDA;
            site = GLM_SERVER_SITE_COPY_OUT;
        }
        // back to the pool once the stream has passed the copies
        if (cudaFreeAsync(dev, sl->stream) != cudaSuccess)
            cudaGetLastError();
        sl->launch_status = st;
        {
            std::lock_guard<std::mutex> g(s->mu);
            if (st != GLM_OK) {
                s->last_cuda_error = (int)ce;
                s->last_error_site = site;
            }
            int busy_now = 0;
            for (auto &u : s->slots)
                busy_now += u->busy ? 1 : 0;
            s->max_concurrent = std::max(s->max_concurrent, busy_now);
            s->n_batches++;
            s->n_trimmed += trimmed ? 1 : 0;
            const int64_t t = now_ns();
            for (uint64_t id : ids) {
                Request &r = s->requests[id];
                r.state = 1;
                r.start_ns = t;
                r.batch_k = K;
                r.batch_requests = (int)ids.size();
                r.deferred_now = false;
            }
        }
        if ((ce = cudaLaunchHostFunc(sl->stream, batch_done, sl)) != cudaSuccess) {
            cudaGetLastError();
            {
                std::lock_guard<std::mutex> g(s->mu);
                s->last_cuda_error = (int)ce;
                s->last_error_site = GLM_SERVER_SITE_COMPLETION;
            }
            sl->launch_status = GLM_ERR_CUDA;
            batch_done(sl);
        }
        lock.lock();
    }
}

void scheduler_main(glm_server *s)
{
    cudaSetDevice(s->device);
    std::unique_lock<std::mutex> lock(s->mu);
    while (!s->stop) {
        dispatch_locked(s, lock);
        s->cv.wait_for(lock, std::chrono::milliseconds(50));
    }
}

glm_status_t ensure_slot_capacity(glm_server *s, int p)
{
    // Called with the lock held. A slot may be running a batch from its
    // current buffers, so buffers that are too small are retired (freed at
    // destroy), never freed here.
    const size_t need = (size_t)s->d.max_batch_k * (size_t)p;
    for (auto &sl : s->slots) {
        if (!sl->status_pin) {
            if (cudaHostAlloc((void **)&sl->status_pin, 64, cudaHostAllocDefault) != cudaSuccess) {
                cudaGetLastError();
                sl->status_pin = nullptr;
                return GLM_ERR_OOM;
            }
        }
        if (sl->cap_kp >= need)
            continue;
        float *b = nullptr, *g = nullptr;
        double *f = nullptr;
        if (cudaHostAlloc((void **)&b, need * 4, cudaHostAllocDefault) != cudaSuccess ||
            cudaHostAlloc((void **)&g, need * 4, cudaHostAllocDefault) != cudaSuccess ||
            cudaHostAlloc((void **)&f, (size_t)s->d.max_batch_k * 8, cudaHostAllocDefault) !=
                cudaSuccess) {
            cudaGetLastError();
            if (b)
                cudaFreeHost(b);
            if (g)
                cudaFreeHost(g);
            return GLM_ERR_OOM;
        }
        for (void *old : {(void *)sl->beta_pin, (void *)sl->g_pin, (void *)sl->f_pin})
            if (old)
                s->retired.push_back(old);
        sl->beta_pin = b;
        sl->g_pin = g;
        sl->f_pin = f;
        sl->cap_kp = need;
    }
    return GLM_OK;
}

}  // namespace

extern "C" {

glm_status_t glm_server_create(const glm_server_desc_t *desc, glm_server_t *out)
{
    if (!out)
        return GLM_ERR_INVALID_ARG;
    *out = nullptr;
    if (!desc || desc->streams < 1 || desc->streams > 16 || desc->max_batch_k < 1 ||
        desc->max_batch_k > 1024 || desc->hbm_budget_bytes < 0 || desc->max_pending < 1 ||
        desc->device < 0)
        return GLM_ERR_INVALID_ARG;
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev == 0) {
        cudaGetLastError();
        return GLM_ERR_NO_DEVICE;
    }
    if (desc->device >= ndev || cudaSetDevice(desc->device) != cudaSuccess)
        return GLM_ERR_INVALID_ARG;
    size_t free_b = 0, total_b = 0;
    if (cudaMemGetInfo(&free_b, &total_b) != cudaSuccess) {
        cudaGetLastError();
        return GLM_ERR_CUDA;
    }
    const size_t budget = desc->hbm_budget_bytes > 0 ? (size_t)desc->hbm_budget_bytes
                                                     : free_b - free_b / 16;
    if (budget < 65536)
        return GLM_ERR_OOM;
    glm_server *s = new (std::nothrow) glm_server;
    if (!s)
        return GLM_ERR_OOM;
    s->d = *desc;
    s->device = desc->device;
    s->budget = budget;
    // batch buffers: a pool that keeps what it got from the device (no
    // release threshold) and reuses a block across streams only once its free
    // has completed, never by making one stream wait for another
    cudaMemPoolProps props;
    std::memset(&props, 0, sizeof(props));
    props.allocType = cudaMemAllocationTypePinned;
    props.handleTypes = cudaMemHandleTypeNone;
    props.location.type = cudaMemLocationTypeDevice;
    props.location.id = desc->device;
    uint64_t keep = ~0ull;
    int no = 0;
    if (cudaMemPoolCreate(&s->pool, &props) != cudaSuccess ||
        cudaMemPoolSetAttribute(s->pool, cudaMemPoolAttrReleaseThreshold, &keep) != cudaSuccess ||
        cudaMemPoolSetAttribute(s->pool, cudaMemPoolReuseAllowInternalDependencies, &no) !=
            cudaSuccess) {
        cudaGetLastError();
        if (s->pool)
            cudaMemPoolDestroy(s->pool);
        delete s;
        return GLM_ERR_OOM;
    }
    for (int i = 0; i < desc->streams; ++i) {
        auto sl = std::make_unique<Slot>();
        sl->srv = s;
        sl->index = i;
        if (cudaStreamCreateWithFlags(&sl->stream, cudaStreamNonBlocking) != cudaSuccess) {
            cudaGetLastError();
            for (auto &u : s->slots)
                cudaStreamDestroy(u->stream);
            cudaMemPoolDestroy(s->pool);
            delete s;
            return GLM_ERR_CUDA;
        }
        s->slots.push_back(std::move(sl));
    }
    s->sched = std::thread(scheduler_main, s);
    *out = s;
    return GLM_OK;
}

glm_status_t glm_server_add_dataset(glm_server_t s, const void *X, const float *x_scale,
                                    const uint8_t *y, int64_t n_rows, int32_t p, int32_t ld,
                                    int32_t xtype, double prior_sigma, int32_t *dataset_id)
{
    if (!s || !dataset_id)
        return GLM_ERR_INVALID_ARG;
    Dataset D;
    D.X = X;
    D.x_scale = x_scale;
    D.y = y;
    D.n = n_rows;
    D.p = p;
    D.ld = ld;
    D.xtype = xtype;
    D.sigma = prior_sigma;
    glm_desc_t hd;
    std::memset(&hd, 0, sizeof(hd));
    hd.n_rows = n_rows;
    hd.p = p;
    hd.ld = ld;
    hd.k_max = s->d.max_batch_k;
    hd.xtype = xtype;
    hd.prior_sigma = prior_sigma;
    hd.device = s->device;
    // the first handle validates the shape and gives the workspace size
    glm_handle_t h0 = nullptr;
    glm_status_t st = glm_create(&hd, &h0);
    if (st != GLM_OK)
        return st;
    glm_info_t info;
    glm_get_info(h0, &info);
    const size_t nslots = s->slots.size();
    const size_t es = xtype == GLM_X_F32 ? 4 : xtype == GLM_X_BF16 ? 2 : 1;
    const size_t data = round256((size_t)n_rows * (size_t)ld * es) + round256((size_t)n_rows) +
                        (x_scale ? round256((size_t)p * 4) : 0);
    D.footprint = data + (size_t)info.workspace_bytes * nslots;
    {
        // reserve the footprint before the other handles allocate
        std::lock_guard<std::mutex> lock(s->mu);
        if (s->resident + s->in_flight + D.footprint + batch_bytes(1, p) > s->budget) {
            glm_destroy(h0);
            return GLM_ERR_OOM;
        }
        s->resident += D.footprint;
    }
    auto undo = [&](glm_status_t e) {
        for (auto hh : D.handles)
            glm_destroy(hh);
        std::lock_guard<std::mutex> lock(s->mu);
        s->resident -= D.footprint;
        return e;
    };
    D.handles.push_back(h0);
    size_t free_b = 0, total_b = 0;
    if (cudaMemGetInfo(&free_b, &total_b) != cudaSuccess) {
        cudaGetLastError();
        return undo(GLM_ERR_CUDA);
    }
    if ((size_t)info.workspace_bytes * (nslots - 1) + ((size_t)16 << 20) > free_b)
        return undo(GLM_ERR_OOM);           // the device has not got the workspaces
    for (size_t i = 1; i < nslots; ++i) {
        glm_handle_t h = nullptr;
        st = glm_create(&hd, &h);
        if (st != GLM_OK)
            return undo(st);
        D.handles.push_back(h);
    }
    {
        std::lock_guard<std::mutex> lock(s->mu);
        st = ensure_slot_capacity(s, p);
        if (st == GLM_OK) {
            *dataset_id = (int32_t)s->datasets.size();
            s->datasets.push_back(std::move(D));
            return GLM_OK;
        }
    }
    // glm_destroy synchronises the device, which waits for completion
    // callbacks that take the lock: never destroy with the lock held
    return undo(st);
}

glm_status_t glm_server_remove_dataset(glm_server_t s, int32_t dataset_id)
{
    if (!s)
        return GLM_ERR_INVALID_ARG;
    std::vector<glm_handle_t> handles;
    {
        std::lock_guard<std::mutex> lock(s->mu);
        if (dataset_id < 0 || dataset_id >= (int32_t)s->datasets.size() ||
            !s->datasets[(size_t)dataset_id].live)
            return GLM_ERR_INVALID_ARG;
        Dataset &D = s->datasets[(size_t)dataset_id];
        if (D.outstanding > 0)
            return GLM_PENDING;
        D.live = false;
        handles.swap(D.handles);
        s->resident -= D.footprint;
        D.footprint = 0;
    }
    for (auto h : handles)
        glm_destroy(h);
    s->cv.notify_all();                     // memory came back: deferred work may fit
    return GLM_OK;
}

glm_status_t glm_server_submit(glm_server_t s, int32_t dataset_id, const float *beta_host,
                               int32_t K, uint64_t *request_id)
{
    if (!s || !beta_host || !request_id)
        return GLM_ERR_INVALID_ARG;
    const int64_t t = now_ns();
    uint64_t id;
    {
        std::lock_guard<std::mutex> lock(s->mu);
        if (dataset_id < 0 || dataset_id >= (int32_t)s->datasets.size() ||
            !s->datasets[(size_t)dataset_id].live || K < 1 || K > s->d.max_batch_k)
            return GLM_ERR_INVALID_ARG;
        if ((int)s->waiting.size() >= s->d.max_pending)
            return GLM_ERR_OOM;   // queue full: refuse rather than grow without bound
        Dataset &D = s->datasets[(size_t)dataset_id];
        const int p = D.p;
        if (s->resident >= s->budget || batch_bytes(K, p) > s->budget - s->resident) {
            s->n_refused++;
            return GLM_ERR_OOM;   // could not fit even with nothing in flight
        }
        id = s->next_id++;
        Request &r = s->requests[id];
        r.ds = dataset_id;
        r.K = K;
        r.beta.assign(beta_host, beta_host + (size_t)K * p);
        r.f.assign((size_t)K, 0.0);
        r.g.assign((size_t)K * p, 0.0f);
        r.submit_ns = t;
        D.outstanding++;
        s->waiting.push_back(id);
    }
    s->cv.notify_all();
    *request_id = id;
    return GLM_OK;
}

static glm_status_t take_result(glm_server_t s, Request &r, double *f_host, float *g_host,
                                glm_request_info_t *info)
{
    const int p = s->datasets[r.ds].p;
    if (info) {
        info->submit_ns = r.submit_ns;
        info->start_ns = r.start_ns;
        info->done_ns = r.done_ns;
        info->batch_k = r.batch_k;
        info->batch_requests = r.batch_requests;
        info->k = r.K;
        info->status = r.state == 2 ? GLM_OK : r.status;
        info->path = r.path;
        info->deferrals = r.deferrals;
    }
    if (r.state == 2) {
        if (f_host)
            std::memcpy(f_host, r.f.data(), sizeof(double) * (size_t)r.K);
        if (g_host)
            std::memcpy(g_host, r.g.data(), sizeof(float) * (size_t)r.K * p);
        return GLM_OK;
    }
    return r.status == GLM_OK ? GLM_ERR_CUDA : r.status;
}

glm_status_t glm_server_poll(glm_server_t s, uint64_t request_id, double *f_host, float *g_host,
                             glm_request_info_t *info)
{
    if (!s)
        return GLM_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> lock(s->mu);
    auto it = s->requests.find(request_id);
    if (it == s->requests.end())
        return GLM_ERR_INVALID_ARG;
    if (it->second.state < 2)
        return GLM_PENDING;
    glm_status_t st = take_result(s, it->second, f_host, g_host, info);
    s->requests.erase(it);
    return st;
}

glm_status_t glm_server_wait(glm_server_t s, uint64_t request_id, double *f_host, float *g_host,
                             glm_request_info_t *info, int32_t timeout_ms)
{
    if (!s || timeout_ms < 0)
        return GLM_ERR_INVALID_ARG;
    std::unique_lock<std::mutex> lock(s->mu);
    auto deadline = std::chrono::steady_clock::now() + std::chrono::milliseconds(timeout_ms);
    for (;;) {
        auto it = s->requests.find(request_id);
        if (it == s->requests.end())
            return GLM_ERR_INVALID_ARG;
        if (it->second.state >= 2) {
            glm_status_t st = take_result(s, it->second, f_host, g_host, info);
            s->requests.erase(it);
            return st;
        }
        if (s->done_cv.wait_until(lock, deadline) == std::cv_status::timeout) {
            auto it2 = s->requests.find(request_id);
            if (it2 != s->requests.end() && it2->second.state >= 2)
                continue;
            return GLM_ERR_TIMEOUT;
        }
    }
}

glm_status_t glm_server_stats(glm_server_t s, glm_server_stats_t *st)
{
    if (!s || !st)
        return GLM_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> lock(s->mu);
    st->requests_done = (int64_t)s->n_done;
    st->requests_failed = (int64_t)s->n_failed;
    st->requests_waiting = (int64_t)s->waiting.size();
    st->batches = (int64_t)s->n_batches;
    st->vectors_done = (int64_t)s->vectors_done;
    st->hbm_budget_bytes = (int64_t)s->budget;
    st->hbm_in_flight_bytes = (int64_t)s->in_flight;
    st->hbm_resident_bytes = (int64_t)s->resident;
    st->batches_tensor_cores = (int64_t)s->n_batches_tc;
    st->deferrals = (int64_t)s->n_deferrals;
    st->trimmed_batches = (int64_t)s->n_trimmed;
    st->refused_requests = (int64_t)s->n_refused;
    st->max_concurrent_batches = s->max_concurrent;
    st->last_cuda_error = s->last_cuda_error;
    st->last_error_site = s->last_error_site;
    return GLM_OK;
}

glm_status_t glm_server_destroy(glm_server_t s)
{
    if (!s)
        return GLM_OK;
    {
        std::lock_guard<std::mutex> lock(s->mu);
        s->stop = true;
    }
    s->cv.notify_all();
    if (s->sched.joinable())
        s->sched.join();
    cudaSetDevice(s->device);
    for (auto &sl : s->slots)
        cudaStreamSynchronize(sl->stream);
    for (auto &D : s->datasets)
        for (auto h : D.handles)
            glm_destroy(h);
    for (auto &sl : s->slots) {
        cudaStreamDestroy(sl->stream);
        cudaFreeHost(sl->beta_pin);
        cudaFreeHost(sl->g_pin);
        cudaFreeHost(sl->f_pin);
        if (sl->status_pin)
            cudaFreeHost(sl->status_pin);
    }
    for (void *p : s->retired)
        cudaFreeHost(p);
    cudaMemPoolDestroy(s->pool);
    delete s;
    return GLM_OK;
}

}  // extern "C"
