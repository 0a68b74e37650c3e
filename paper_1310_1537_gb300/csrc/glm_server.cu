// Serving loop with continuous batching over device-resident datasets.
//
// Requests (a dataset id and K coefficient vectors on the host) are queued by
// glm_server_submit and returned through glm_server_poll / glm_server_wait. A
// scheduler thread forms batches: it takes the oldest waiting request, merges
// later requests for the same dataset while the batch stays within
// max_batch_k vectors, and launches the batch on a free stream slot as soon as
// one is free and the batch's device buffers fit the HBM budget (admission by
// free memory). Batches for different datasets run concurrently on different
// streams; requests that arrive while others are on the GPU join the next
// batch formed. Each slot copies its batch's coefficients in (pinned staging),
// evaluates it with the dataset's handle for that slot, copies f and g out and
// completes through a host callback that scatters results to the requests.
// The evaluation of a vector does not depend on which other vectors share its
// batch beyond the kernel path chosen for the batch size (CUDA cores below 16
// vectors, tensor cores from 16), so a result alone and in a mix agree to the
// evaluation tolerance.
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
    size_t dev_off = 0;                     // arena offset of the batch buffers
    size_t dev_bytes = 0;
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
    std::deque<uint64_t> waiting;
    std::vector<std::unique_ptr<Slot>> slots;
    uint64_t next_id = 1;
    bool stop = false;
    std::thread sched;
    // device arena for batch buffers (first fit over a free list)
    uint8_t *arena = nullptr;
    size_t arena_bytes = 0;
    std::vector<std::pair<size_t, size_t>> free_list;   // (offset, size)
    std::vector<void *> retired;            // outgrown pinned staging buffers
    size_t in_flight_bytes = 0;
    // statistics
    uint64_t n_done = 0, n_failed = 0, n_batches = 0, vectors_done = 0;
    int max_concurrent = 0;
    int last_cuda_error = 0;                // cudaError_t of the last failed step
    int last_error_site = 0;                // glm_server_error_site_t of that step
};

namespace {

bool arena_alloc(glm_server *s, size_t bytes, size_t *off)
{
    bytes = (bytes + 255) / 256 * 256;
    for (size_t i = 0; i < s->free_list.size(); ++i) {
        if (s->free_list[i].second >= bytes) {
            *off = s->free_list[i].first;
            s->free_list[i].first += bytes;
            s->free_list[i].second -= bytes;
            if (s->free_list[i].second == 0)
                s->free_list.erase(s->free_list.begin() + (long)i);
            s->in_flight_bytes += bytes;
            return true;
        }
    }
    return false;
}

void arena_free(glm_server *s, size_t off, size_t bytes)
{
    bytes = (bytes + 255) / 256 * 256;
    s->in_flight_bytes -= bytes;
    s->free_list.push_back({off, bytes});
    std::sort(s->free_list.begin(), s->free_list.end());
    std::vector<std::pair<size_t, size_t>> merged;
    for (auto &r : s->free_list) {
        if (!merged.empty() && merged.back().first + merged.back().second == r.first)
            merged.back().second += r.second;
        else
            merged.push_back(r);
    }
    s->free_list.swap(merged);
}

size_t batch_bytes(int K, int p)
{
    return ((size_t)K * p * 4 + 255) / 256 * 256 + ((size_t)K * 8 + 255) / 256 * 256 +
           ((size_t)K * p * 4 + 255) / 256 * 256;
}

// Host callback at the end of a batch: scatter results, free the slot.
void CUDART_CB batch_done(void *arg)
{
    Slot *sl = static_cast<Slot *>(arg);
    glm_server *s = sl->srv;
    const int64_t t = now_ns();
    {
        std::lock_guard<std::mutex> lock(s->mu);
        const int p = s->datasets[sl->ds].p;
        if (sl->launch_status == GLM_OK && (*sl->status_pin & glm::kDevTimeout)) {
            sl->launch_status = GLM_ERR_TIMEOUT;
            s->last_error_site = GLM_SERVER_SITE_DEVICE_WAIT;
        }
        int k0 = 0;
        for (uint64_t id : sl->ids) {
            auto it = s->requests.find(id);
            if (it == s->requests.end())
                continue;
            Request &r = it->second;
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
            k0 += r.K;
        }
        arena_free(s, sl->dev_off, sl->dev_bytes);
        sl->busy = false;
        sl->ids.clear();
    }
    s->cv.notify_all();
    s->done_cv.notify_all();
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
        // oldest waiting request decides the dataset; merge same-dataset requests
        const uint64_t first = s->waiting.front();
        Request &r0 = s->requests[first];
        const int ds = r0.ds;
        const int p = s->datasets[ds].p;
        std::vector<uint64_t> ids;
        int K = 0;
        for (auto it = s->waiting.begin(); it != s->waiting.end();) {
            Request &r = s->requests[*it];
            if (r.ds == ds && K + r.K <= s->d.max_batch_k) {
                ids.push_back(*it);
                K += r.K;
                it = s->waiting.erase(it);
            } else {
                ++it;
            }
        }
        const size_t bytes = batch_bytes(K, p);
        size_t off = 0;
        if (!arena_alloc(s, bytes, &off)) {
            // not enough free device memory right now: put the batch back in
            // arrival order and wait for a completion
            for (auto it = ids.rbegin(); it != ids.rend(); ++it)
                s->waiting.push_front(*it);
            std::sort(s->waiting.begin(), s->waiting.end());
            return;
        }
        sl->busy = true;
        sl->ids = ids;
        sl->ds = ds;
        sl->K = K;
        sl->dev_off = off;
        sl->dev_bytes = bytes;
        sl->launch_status = GLM_OK;
        sl->b_beta = sl->beta_pin;
        sl->b_f = sl->f_pin;
        sl->b_g = sl->g_pin;
        int busy_now = 0;
        for (auto &u : s->slots)
            busy_now += u->busy ? 1 : 0;
        s->max_concurrent = std::max(s->max_concurrent, busy_now);
        s->n_batches++;
        const int64_t t = now_ns();
        int k0 = 0;
        for (uint64_t id : ids) {
            Request &r = s->requests[id];
            r.state = 1;
            r.start_ns = t;
            r.batch_k = K;
            r.batch_requests = (int)ids.size();
            std::memcpy(sl->b_beta + (size_t)k0 * p, r.beta.data(), sizeof(float) * (size_t)r.K * p);
            k0 += r.K;
        }
        // copy what the launch needs: add_dataset may grow the vector meanwhile
        const Dataset &D = s->datasets[ds];
        glm_handle_t h = D.handles[(size_t)sl->index];
        const void *X = D.X;
        const float *x_scale = D.x_scale;
        const uint8_t *y = D.y;
        uint8_t *base = s->arena + off;
        float *dbeta = reinterpret_cast<float *>(base);
        double *df = reinterpret_cast<double *>(base + ((size_t)K * p * 4 + 255) / 256 * 256);
        float *dg = reinterpret_cast<float *>(reinterpret_cast<uint8_t *>(df) +
                                              ((size_t)K * 8 + 255) / 256 * 256);
        // launch without the lock: the callback takes it
        lock.unlock();
        glm_status_t st = GLM_OK;
        int site = 0;
        cudaError_t ce = cudaSuccess;
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
        sl->launch_status = st;
        if (st != GLM_OK) {
            std::lock_guard<std::mutex> g(s->mu);
            s->last_cuda_error = (int)ce;
            s->last_error_site = site;
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
    glm_server *s = new (std::nothrow) glm_server;
    if (!s)
        return GLM_ERR_OOM;
    s->d = *desc;
    s->device = desc->device;
    size_t free_b = 0, total_b = 0;
    cudaMemGetInfo(&free_b, &total_b);
    size_t budget = desc->hbm_budget_bytes > 0 ? (size_t)desc->hbm_budget_bytes : free_b / 8;
    if (budget > free_b / 2)
        budget = free_b / 2;
    budget = budget / 256 * 256;
    if (budget < 4096 || cudaMalloc((void **)&s->arena, budget) != cudaSuccess) {
        cudaGetLastError();
        delete s;
        return GLM_ERR_OOM;
    }
    s->arena_bytes = budget;
    s->free_list.push_back({0, budget});
    for (int i = 0; i < desc->streams; ++i) {
        auto sl = std::make_unique<Slot>();
        sl->srv = s;
        sl->index = i;
        if (cudaStreamCreateWithFlags(&sl->stream, cudaStreamNonBlocking) != cudaSuccess) {
            cudaGetLastError();
            for (auto &u : s->slots)
                cudaStreamDestroy(u->stream);
            cudaFree(s->arena);
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
    for (size_t i = 0; i < s->slots.size(); ++i) {
        glm_handle_t h = nullptr;
        glm_status_t st = glm_create(&hd, &h);
        if (st != GLM_OK) {
            for (auto hh : D.handles)
                glm_destroy(hh);
            return st;
        }
        D.handles.push_back(h);
    }
    std::lock_guard<std::mutex> lock(s->mu);
    glm_status_t st = ensure_slot_capacity(s, p);
    if (st != GLM_OK) {
        for (auto hh : D.handles)
            glm_destroy(hh);
        return st;
    }
    if (batch_bytes(s->d.max_batch_k, p) > s->arena_bytes) {
        for (auto hh : D.handles)
            glm_destroy(hh);
        return GLM_ERR_OOM;
    }
    *dataset_id = (int32_t)s->datasets.size();
    s->datasets.push_back(std::move(D));
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
        if (dataset_id < 0 || dataset_id >= (int32_t)s->datasets.size() || K < 1 ||
            K > s->d.max_batch_k)
            return GLM_ERR_INVALID_ARG;
        if ((int)s->waiting.size() >= s->d.max_pending)
            return GLM_ERR_OOM;   // queue full: refuse rather than grow without bound
        const int p = s->datasets[dataset_id].p;
        id = s->next_id++;
        Request &r = s->requests[id];
        r.ds = dataset_id;
        r.K = K;
        r.beta.assign(beta_host, beta_host + (size_t)K * p);
        r.f.assign((size_t)K, 0.0);
        r.g.assign((size_t)K * p, 0.0f);
        r.submit_ns = t;
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
    st->max_concurrent_batches = s->max_concurrent;
    st->last_cuda_error = s->last_cuda_error;
    st->last_error_site = s->last_error_site;
    st->hbm_budget_bytes = (int64_t)s->arena_bytes;
    st->hbm_in_flight_bytes = (int64_t)s->in_flight_bytes;
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
    cudaFree(s->arena);
    delete s;
    return GLM_OK;
}

}  // extern "C"
