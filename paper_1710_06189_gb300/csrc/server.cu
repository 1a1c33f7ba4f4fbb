// Serving loop: continuous batching of host requests (glcm_server_*).
//
// The paper hides host-to-device transfers behind computation by splitting an
// image into stripes on several CUDA streams (Sec. III, Eqs. 7-9).  A server
// applies the same overlap across requests: one scheduler thread admits
// requests by device footprint into an arena, copies their images on a copy
// stream, and launches whatever has been admitted as one batch on the next
// idle lane (a context with its own stream), so copies of new requests run
// under the kernels of earlier batches and several batches can be on the GPU
// at once.  The compute itself goes through the public context API
// (glcm_enqueue_batch, glcm_synchronize, glcm_get_timing); each lane context
// also leaves a few SMs to the image copy kernel.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <deque>
#include <mutex>
#include <string>
#include <thread>
#include <unordered_map>
#include <vector>

#include "arena.h"
#include "glcm.h"
#include "glcm_internal.cuh"

namespace {

using Clock = std::chrono::steady_clock;

struct Req {
    long long id = 0;
    glcm_desc d{};  // the caller's host pointers
    std::vector<glcm_offset> offs;
    size_t dpitch = 0, img_bytes = 0, counts_bytes = 0, norm_bytes = 0, feat_bytes = 0;
    size_t off = 0, foot = 0;  // arena block
    cudaEvent_t copied = nullptr;
    Clock::time_point t_submit, t_done;
    int status = GLCM_OK;
    bool finished = false;
};

struct Lane {
    glcm_ctx* ctx = nullptr;
    cudaStream_t stream = nullptr;
    bool busy = false;
};

struct Batch {
    int lane = 0;
    std::vector<Req*> reqs;
    cudaEvent_t done = nullptr;
};

size_t r256(size_t b) { return glcm_arena::Arena::round_up(b); }

// Image bytes in one batch, at most (a batch always takes at least one
// request): a batch waits for all its copies before it votes, so a burst cut
// into batches of about 1 ms of copying at 210 GB/s votes batch by batch
// while the next batches still copy, instead of copying everything first.
constexpr size_t kBatchImageBytes = 256ull << 20;

// SMs every lane's vote launches leave to the image copy kernel, and the
// copy kernel's CTAs (two per SM).  A burst of served requests is bound by
// the copies: measured on the all-at-once burst of the served stream, 8 SMs
// and 24 CTAs gave 780 Gpairs/s, 16 SMs 864, 24 SMs and 48 CTAs 1042, 32 SMs
// and 64 CTAs 1024, 48 SMs and 96 CTAs 997.
constexpr int kServerCopySMs = 24;
constexpr int kServerCopyCTAs = 2 * kServerCopySMs;

std::string g_server_create_error;

}  // namespace

struct glcm_server {
    int device = 0;
    int max_batch = 256, max_queue = 4096;
    uint8_t* base = nullptr;
    glcm_arena::Arena arena;  // guarded by mu
    std::vector<Lane> lanes;
    cudaStream_t copy = nullptr;
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    std::deque<Req*> queue;                    // submitted, not admitted (mu)
    std::unordered_map<long long, Req*> reqs;  // live tickets (mu)
    long long next_id = 1;
    bool stop = false;
    glcm_server_counters st{};  // mu
    std::string err;            // mu
    std::thread worker;
    // Scheduler-thread state.
    std::vector<Req*> staged;  // admitted, copy enqueued, not launched
    std::deque<Batch> running;
    std::vector<cudaEvent_t> events;
};

namespace {

cudaEvent_t take_event(glcm_server* s)
{
    if (!s->events.empty()) {
        cudaEvent_t e = s->events.back();
        s->events.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    if (cudaEventCreateWithFlags(&e, cudaEventDisableTiming) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    return e;
}

// Mark requests done (scheduler thread); frees their arena blocks.
void finish(glcm_server* s, const std::vector<Req*>& rs, int status, const char* why)
{
    const auto now = Clock::now();
    std::lock_guard<std::mutex> lk(s->mu);
    for (Req* r : rs) {
        if (r->copied) {
            s->events.push_back(r->copied);
            r->copied = nullptr;
        }
        s->arena.release(r->off, r->foot);
        r->status = status;
        r->t_done = now;
        r->finished = true;
        if (status == GLCM_OK)
            s->st.completed++;
        else
            s->st.failed++;
    }
    if (status != GLCM_OK && why)
        s->err = why;
    s->cv_done.notify_all();
}

bool retire(glcm_server* s)
{
    bool progress = false;
    for (auto it = s->running.begin(); it != s->running.end();) {
        const cudaError_t q = cudaEventQuery(it->done);
        if (q == cudaErrorNotReady) {
            ++it;
            continue;
        }
        Lane& ln = s->lanes[it->lane];
        int rc = GLCM_OK;
        std::string why;
        if (q != cudaSuccess) {
            rc = GLCM_ERR_CUDA;
            why = std::string("batch failed: ") + cudaGetErrorString(q);
            cudaGetLastError();
        } else {
            rc = glcm_synchronize(ln.ctx);
            if (rc != GLCM_OK)
                why = glcm_last_error(ln.ctx);
        }
        long long nk = 0;
        glcm_get_timing(ln.ctx, nullptr, nullptr, &nk, 1);
        {
            std::lock_guard<std::mutex> lk(s->mu);
            s->st.kernel_launches += nk;
        }
        finish(s, it->reqs, rc, why.empty() ? nullptr : why.c_str());
        s->events.push_back(it->done);
        ln.busy = false;
        it = s->running.erase(it);
        progress = true;
    }
    return progress;
}

bool admit(glcm_server* s)
{
    std::vector<Req*> take;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        while (!s->queue.empty()) {
            Req* r = s->queue.front();
            size_t off = 0;
            if (!s->arena.alloc(r->foot, &off))
                break;  // arrival order: later requests wait behind this one
            r->off = off;
            s->queue.pop_front();
            take.push_back(r);
        }
        s->st.arena_peak = std::max(s->st.arena_peak, s->arena.peak());
    }
    for (Req* r : take) {
        const int bpp = r->d.dtype == GLCM_U8 ? 1 : 2;
        cudaError_t e = glcm::copy_rows_to_device(s->base + r->off, r->dpitch, r->d.image, r->d.pitch_bytes,
                                                  (size_t)r->d.width * bpp, r->d.height, s->copy, true,
                                                  kServerCopyCTAs);
        r->copied = take_event(s);
        if (e == cudaSuccess && r->copied)
            e = cudaEventRecord(r->copied, s->copy);
        if (e != cudaSuccess || !r->copied) {
            cudaGetLastError();
            cudaStreamSynchronize(s->copy);
            char why[256];
            snprintf(why, sizeof why, "image copy of request %lld failed: %s", r->id,
                     e != cudaSuccess ? cudaGetErrorString(e) : "no event");
            finish(s, {r}, GLCM_ERR_CUDA, why);
            continue;
        }
        s->staged.push_back(r);
    }
    return !take.empty();
}

bool launch(glcm_server* s)
{
    bool progress = false;
    while (!s->staged.empty()) {
        int li = -1;
        for (int k = 0; k < (int)s->lanes.size(); ++k)
            if (!s->lanes[k].busy) {
                li = k;
                break;
            }
        if (li < 0)
            break;
        Lane& ln = s->lanes[li];
        // The batch: staged requests in admission order; a levels-mode
        // request runs alone so that a range error is its own.
        std::vector<Req*> b;
        size_t k = 0, bytes = 0;
        for (; k < s->staged.size() && (int)b.size() < s->max_batch; ++k) {
            Req* r = s->staged[k];
            const bool alone = (r->d.flags & GLCM_INPUT_LEVELS) != 0;
            if (alone && !b.empty())
                break;
            if (!b.empty() && bytes + r->img_bytes > kBatchImageBytes)
                break;
            bytes += r->img_bytes;
            b.push_back(r);
            if (alone) {
                ++k;
                break;
            }
        }
        s->staged.erase(s->staged.begin(), s->staged.begin() + k);
        std::vector<glcm_desc> descs(b.size());
        int rc = GLCM_OK;
        std::string why;
        for (size_t i = 0; i < b.size(); ++i) {
            Req* r = b[i];
            uint8_t* p = s->base + r->off;
            glcm_desc& d = descs[i];
            d = r->d;
            d.image = p;
            d.pitch_bytes = r->dpitch;
            d.offsets = r->offs.data();
            d.counts = reinterpret_cast<uint32_t*>(p + r256(r->img_bytes));
            uint8_t* q = reinterpret_cast<uint8_t*>(d.counts) + r256(r->counts_bytes);
            d.normalized = r->d.normalized ? reinterpret_cast<float*>(q) : nullptr;
            q += r->d.normalized ? r256(r->norm_bytes) : 0;
            d.features = r->d.features ? reinterpret_cast<float*>(q) : nullptr;
            if (cudaStreamWaitEvent(ln.stream, r->copied, 0) != cudaSuccess) {
                cudaGetLastError();
                rc = GLCM_ERR_CUDA;
                why = "cudaStreamWaitEvent failed";
            }
        }
        if (rc == GLCM_OK) {
            rc = glcm_enqueue_batch(ln.ctx, descs.data(), (int)descs.size());
            if (rc != GLCM_OK)
                why = glcm_last_error(ln.ctx);
        }
        for (size_t i = 0; rc == GLCM_OK && i < b.size(); ++i) {
            Req* r = b[i];
            const glcm_desc& d = descs[i];
            cudaError_t e = cudaMemcpyAsync(r->d.counts, d.counts, r->counts_bytes, cudaMemcpyDeviceToHost, ln.stream);
            if (e == cudaSuccess && r->d.normalized)
                e = cudaMemcpyAsync(r->d.normalized, d.normalized, r->norm_bytes, cudaMemcpyDeviceToHost, ln.stream);
            if (e == cudaSuccess && r->d.features)
                e = cudaMemcpyAsync(r->d.features, d.features, r->feat_bytes, cudaMemcpyDeviceToHost, ln.stream);
            if (e != cudaSuccess) {
                cudaGetLastError();
                rc = GLCM_ERR_CUDA;
                why = std::string("result copy failed: ") + cudaGetErrorString(e);
            }
        }
        Batch bt;
        bt.lane = li;
        bt.reqs = b;
        bt.done = rc == GLCM_OK ? take_event(s) : nullptr;
        if (rc == GLCM_OK && (!bt.done || cudaEventRecord(bt.done, ln.stream) != cudaSuccess)) {
            cudaGetLastError();
            rc = GLCM_ERR_CUDA;
            why = "cudaEventRecord failed";
        }
        if (rc != GLCM_OK) {
            // Nothing of this batch may still use its arena blocks.
            cudaStreamSynchronize(ln.stream);
            cudaStreamSynchronize(s->copy);
            glcm_synchronize(ln.ctx);
            if (bt.done)
                s->events.push_back(bt.done);
            finish(s, b, rc, why.c_str());
            progress = true;
            continue;
        }
        ln.busy = true;
        {
            std::lock_guard<std::mutex> lk(s->mu);
            s->st.batches++;
            s->st.max_batch = std::max<long long>(s->st.max_batch, (long long)b.size());
        }
        s->running.push_back(std::move(bt));
        progress = true;
    }
    return progress;
}

void scheduler(glcm_server* s)
{
    cudaSetDevice(s->device);
    for (;;) {
        bool progress = retire(s);
        progress |= admit(s);
        progress |= launch(s);
        std::unique_lock<std::mutex> lk(s->mu);
        if (s->stop && s->queue.empty() && s->staged.empty() && s->running.empty())
            break;
        if (!progress) {
            // Short naps while batches are on the GPU (their completion is
            // polled), longer ones when idle (submissions notify).
            const auto nap = s->running.empty() && s->staged.empty() ? std::chrono::microseconds(2000)
                                                                      : std::chrono::microseconds(20);
            s->cv_work.wait_for(lk, nap);
        }
    }
}

bool host_pointer(const void* p)
{
    if (!p)
        return false;
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return true;
    }
    return a.type != cudaMemoryTypeDevice && a.type != cudaMemoryTypeManaged;
}

}  // namespace

extern "C" const char* glcm_server_last_error(const glcm_server* s)
{
    return s ? s->err.c_str() : g_server_create_error.c_str();
}

extern "C" int glcm_server_create(glcm_server** out, int device, size_t hbm_budget_bytes, int lanes, int max_batch,
                                  int max_queue)
{
    if (!out) {
        g_server_create_error = "out is NULL";
        return GLCM_ERR_ARG;
    }
    *out = nullptr;
    if (lanes < 0 || lanes > 8 || max_batch < 0 || max_queue < 0) {
        g_server_create_error = "lanes must be 0..8, max_batch and max_queue >= 0";
        return GLCM_ERR_ARG;
    }
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev) {
        cudaGetLastError();
        g_server_create_error = "no such CUDA device";
        return GLCM_ERR_ARG;
    }
    cudaSetDevice(device);
    glcm_server* s = new glcm_server();
    s->device = device;
    s->max_batch = max_batch ? max_batch : 256;
    s->max_queue = max_queue ? max_queue : 4096;
    const size_t budget = hbm_budget_bytes ? hbm_budget_bytes : ((size_t)4 << 30);
    int rc = GLCM_OK;
    if (cudaMalloc(&s->base, budget) != cudaSuccess) {
        cudaGetLastError();
        s->base = nullptr;
        g_server_create_error = "could not allocate the server arena";
        rc = GLCM_ERR_NOMEM;
    }
    s->arena.reset(budget);
    s->st.arena_bytes = s->arena.capacity();
    if (rc == GLCM_OK && cudaStreamCreateWithFlags(&s->copy, cudaStreamNonBlocking) != cudaSuccess) {
        cudaGetLastError();
        g_server_create_error = "copy stream creation failed";
        rc = GLCM_ERR_CUDA;
    }
    const int nl = lanes ? lanes : 2;
    for (int k = 0; rc == GLCM_OK && k < nl; ++k) {
        Lane ln;
        if (cudaStreamCreateWithFlags(&ln.stream, cudaStreamNonBlocking) != cudaSuccess) {
            cudaGetLastError();
            g_server_create_error = "lane stream creation failed";
            rc = GLCM_ERR_CUDA;
            break;
        }
        rc = glcm_create(&ln.ctx, device, (size_t)256 << 20, ln.stream);
        if (rc != GLCM_OK) {
            g_server_create_error = glcm_last_error(nullptr);
            cudaStreamDestroy(ln.stream);
            break;
        }
        // Image copies go through the copy kernel (copy-engine transfers from
        // host memory held back the lanes' kernels until every queued transfer
        // was done); the lanes' votes leave it kServerCopySMs SMs.
        glcm::set_vote_sm_reserve(ln.ctx, kServerCopySMs);
        s->lanes.push_back(ln);
    }
    if (rc != GLCM_OK) {
        glcm_server_destroy(s);
        return rc;
    }
    s->worker = std::thread(scheduler, s);
    *out = s;
    return GLCM_OK;
}

extern "C" int glcm_server_submit(glcm_server* s, const glcm_desc* r, long long* ticket)
{
    if (!s || !r || !ticket)
        return GLCM_ERR_ARG;
    auto bad = [&](int code, const char* msg) {
        std::lock_guard<std::mutex> lk(s->mu);
        s->err = msg;
        return code;
    };
    if (!r->image || !r->counts || r->width < 1 || r->height < 1 || (r->dtype != GLCM_U8 && r->dtype != GLCM_U16) ||
        r->levels < 2 || r->levels > GLCM_MAX_COUNT_LEVELS || !r->offsets || r->n_offsets < 1 ||
        r->n_offsets > GLCM_MAX_OFFSETS ||
        (r->flags & ~(GLCM_SYMMETRIC | GLCM_NORMALIZE | GLCM_INPUT_LEVELS | GLCM_FLAT_WRAP)))
        return bad(GLCM_ERR_ARG, "invalid request");
    if ((r->normalized || r->features) && r->levels > GLCM_MAX_LEVELS)
        return bad(GLCM_ERR_UNSUPPORTED, "normalized GLCMs and features need levels <= 256");
    const int bpp = r->dtype == GLCM_U8 ? 1 : 2;
    if (r->pitch_bytes < (size_t)r->width * bpp)
        return bad(GLCM_ERR_ARG, "pitch_bytes < width * bytes per pixel");
    for (int o = 0; o < r->n_offsets; ++o)
        if (r->offsets[o].dx <= -65536 || r->offsets[o].dx >= 65536 || r->offsets[o].dy <= -65536 ||
            r->offsets[o].dy >= 65536)
            return bad(GLCM_ERR_ARG, "offset out of range");
    cudaSetDevice(s->device);
    if (!host_pointer(r->image) || !host_pointer(r->counts) || (r->normalized && !host_pointer(r->normalized)) ||
        (r->features && !host_pointer(r->features)))
        return bad(GLCM_ERR_ARG, "server requests take host pointers");
    Req* q = new Req();
    q->d = *r;
    q->offs.assign(r->offsets, r->offsets + r->n_offsets);
    q->d.offsets = q->offs.data();
    const size_t nn = (size_t)r->levels * r->levels;
    q->dpitch = ((size_t)r->width * bpp + 15) & ~(size_t)15;
    q->img_bytes = q->dpitch * r->height;
    q->counts_bytes = r->n_offsets * nn * 4;
    q->norm_bytes = r->normalized ? r->n_offsets * nn * 4 : 0;
    q->feat_bytes = r->features ? (size_t)r->n_offsets * GLCM_N_FEATURES * 4 : 0;
    q->foot = r256(q->img_bytes) + r256(q->counts_bytes) + r256(q->norm_bytes) + r256(q->feat_bytes);
    std::lock_guard<std::mutex> lk(s->mu);
    if (s->stop) {
        delete q;
        s->err = "server is shutting down";
        return GLCM_ERR_BUSY;
    }
    if (q->foot > s->arena.capacity()) {
        char buf[160];
        snprintf(buf, sizeof buf, "request footprint %zu bytes exceeds the %zu-byte arena", q->foot,
                 s->arena.capacity());
        s->err = buf;
        delete q;
        return GLCM_ERR_NOMEM;
    }
    if ((int)s->queue.size() >= s->max_queue) {
        delete q;
        s->err = "admission queue full";
        return GLCM_ERR_BUSY;
    }
    q->id = s->next_id++;
    q->t_submit = Clock::now();
    s->queue.push_back(q);
    s->reqs[q->id] = q;
    s->st.submitted++;
    s->st.queue_peak = std::max<long long>(s->st.queue_peak, (long long)s->queue.size());
    *ticket = q->id;
    s->cv_work.notify_one();
    return GLCM_OK;
}

extern "C" int glcm_server_wait(glcm_server* s, long long ticket, int timeout_ms, double* latency_ms)
{
    if (!s)
        return GLCM_ERR_ARG;
    std::unique_lock<std::mutex> lk(s->mu);
    auto ready = [&] {
        auto f = s->reqs.find(ticket);
        return f == s->reqs.end() || f->second->finished;
    };
    if (timeout_ms < 0)
        s->cv_done.wait(lk, ready);
    else if (!s->cv_done.wait_for(lk, std::chrono::milliseconds(timeout_ms), ready))
        return GLCM_ERR_BUSY;
    auto f = s->reqs.find(ticket);
    if (f == s->reqs.end()) {
        s->err = "unknown ticket";
        return GLCM_ERR_ARG;
    }
    Req* r = f->second;
    const int status = r->status;
    if (latency_ms)
        *latency_ms = std::chrono::duration<double, std::milli>(r->t_done - r->t_submit).count();
    s->reqs.erase(f);
    delete r;
    return status;
}

extern "C" int glcm_server_stats(glcm_server* s, glcm_server_counters* out)
{
    if (!s || !out)
        return GLCM_ERR_ARG;
    std::lock_guard<std::mutex> lk(s->mu);
    *out = s->st;
    return GLCM_OK;
}

extern "C" int glcm_server_destroy(glcm_server* s)
{
    if (!s)
        return GLCM_OK;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        s->stop = true;
        for (Req* r : s->queue) {
            r->status = GLCM_ERR_BUSY;
            r->t_done = Clock::now();
            r->finished = true;
            s->st.failed++;
        }
        s->queue.clear();
        s->cv_work.notify_all();
        s->cv_done.notify_all();
    }
    if (s->worker.joinable())
        s->worker.join();
    cudaSetDevice(s->device);
    for (Lane& ln : s->lanes) {
        glcm_destroy(ln.ctx);
        cudaStreamDestroy(ln.stream);
    }
    if (s->copy) {
        cudaStreamSynchronize(s->copy);
        cudaStreamDestroy(s->copy);
    }
    for (cudaEvent_t e : s->events)
        cudaEventDestroy(e);
    for (auto& kv : s->reqs) {
        if (kv.second->copied)
            cudaEventDestroy(kv.second->copied);
        delete kv.second;
    }
    if (s->base)
        cudaFree(s->base);
    delete s;
    return GLCM_OK;
}
