// Serving engine: continuous batching of edge-map requests on one GPU.
//
// submit() copies the request into pinned staging (or, when the staging
// pool is full, into heap memory until staging frees up) and queues it.  An
// engine thread admits queued requests in arrival order while the device
// pool (the HBM budget) has room for the request's packed image and edge
// map and fewer than max_inflight batches are on the GPU; each admitted
// group becomes one batch:
//     H2D copies (stream h2d) -> persistent batch kernel under a CUDA graph
//     (stream compute) -> D2H copies (stream d2h) -> completion event.
// The three streams let the uploads of the next batch and the downloads of
// the previous one overlap the running kernel.  The engine retires batches
// in order as their events complete, frees their device memory and wakes
// pollers; poll() copies a finished edge map out of staging and forgets the
// ticket.  All waits are bounded by the caller's timeouts or by the engine
// tick; nothing here spins on the GPU.
#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstdlib>
#include <cstring>
#include <deque>
#include <memory>
#include <mutex>
#include <thread>
#include <unordered_map>
#include <vector>

#include "me_alloc.h"
#include "me_internal.h"

using namespace me;

namespace {

using Clock = std::chrono::steady_clock;

double us_since(Clock::time_point a, Clock::time_point b) {
    return std::chrono::duration<double, std::micro>(b - a).count();
}

constexpr size_t kAlign = 256;

enum State { QUEUED, ADMITTED, DONE, FAILED };

struct Req {
    uint64_t ticket = 0;
    int32_t w = 0, h = 0, stride = 0, boundary = 0;
    size_t bytes = 0, span = 0;        // packed size; rounded to kAlign
    bool pinned = false;               // input is in staging (else in heap)
    size_t pin_off = 0;                // staging: input at +0, output at +span
    std::unique_ptr<uint32_t[]> heap;  // input while staging was full
    size_t dev_off = 0;                // device pool: input at +0, output at +span
    State state = QUEUED;
    bool cancelled = false;
    Clock::time_point t_submit, t_admit, t_done;
};

struct Batch {
    std::vector<Req *> reqs;
    cudaEvent_t up = nullptr, kern = nullptr, done = nullptr;
};

}  // namespace

struct me_server {
    me_serve_cfg cfg{};
    char *dev_base = nullptr;
    char *pin_base = nullptr;
    RangeAlloc dev_alloc, pin_alloc;
    cudaStream_t s_h2d = nullptr, s_comp = nullptr, s_d2h = nullptr;
    std::unique_ptr<BatchRing> ring;

    std::mutex mu;
    std::condition_variable cv_engine, cv_done;
    std::deque<Req *> queue;
    std::unordered_map<uint64_t, Req *> reqs;
    std::deque<Batch> inflight;
    std::vector<Batch> spare;          // batches whose events can be reused
    std::thread engine;
    bool closing = false, stop = false;
    uint64_t next_ticket = 1;
    int64_t submitted = 0, completed = 0, batches = 0;

    // ------------------------------------------------------------------
    void free_req(Req *r) {          // caller holds mu
        if (r->pinned) pin_alloc.release(r->pin_off, 2 * r->span);
        delete r;
    }

    bool new_batch(Batch *b) {
        if (!spare.empty()) {
            *b = spare.back();
            spare.pop_back();
            b->reqs.clear();
            return true;
        }
        const unsigned f = cudaEventDisableTiming;
        if (cudaEventCreateWithFlags(&b->up, f) != cudaSuccess ||
            cudaEventCreateWithFlags(&b->kern, f) != cudaSuccess ||
            cudaEventCreateWithFlags(&b->done, f) != cudaSuccess) {
            cudaGetLastError();
            return false;
        }
        return true;
    }

    // Retire finished batches (in order); caller holds mu.
    void retire() {
        bool any = false;
        while (!inflight.empty()) {
            Batch &b = inflight.front();
            const cudaError_t q = cudaEventQuery(b.done);
            if (q == cudaErrorNotReady) break;
            const State st = q == cudaSuccess ? DONE : FAILED;
            if (q != cudaSuccess) cudaGetLastError();
            const auto now = Clock::now();
            for (Req *r : b.reqs) {
                dev_alloc.release(r->dev_off, 2 * r->span);
                r->t_done = now;
                r->state = st;
                ++completed;
                if (r->cancelled) free_req(r);
            }
            b.reqs.clear();
            spare.push_back(std::move(b));
            inflight.pop_front();
            any = true;
        }
        if (any) cv_done.notify_all();
    }

    // Give staging to queued requests still held in heap memory, in order.
    void stage_heap_requests() {
        for (Req *r : queue) {
            if (r->pinned) continue;
            size_t off;
            if (!pin_alloc.alloc(2 * r->span, &off)) break;
            std::memcpy(pin_base + off, r->heap.get(), r->bytes);
            r->heap.reset();
            r->pin_off = off;
            r->pinned = true;
        }
    }

    // Issue one admitted batch; called without mu.
    void launch(Batch &b) {
        cudaError_t e = cudaSuccess;
        std::vector<me_desc> descs;
        descs.reserve(b.reqs.size());
        for (Req *r : b.reqs) {
            char *din = dev_base + r->dev_off;
            if (e == cudaSuccess)
                e = cudaMemcpyAsync(din, pin_base + r->pin_off, r->bytes,
                                    cudaMemcpyHostToDevice, s_h2d);
            descs.push_back({reinterpret_cast<const uint32_t *>(din),
                             reinterpret_cast<uint32_t *>(din + r->span), r->w, r->h, r->stride,
                             r->boundary});
        }
        if (e == cudaSuccess) e = cudaEventRecord(b.up, s_h2d);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(s_comp, b.up, 0);
        if (e == cudaSuccess) {
            const int rc = ring->launch(descs.data(), (int)descs.size(), s_comp);
            if (rc != ME_OK) e = cudaErrorLaunchFailure;
        }
        if (e == cudaSuccess) e = cudaEventRecord(b.kern, s_comp);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(s_d2h, b.kern, 0);
        for (Req *r : b.reqs)
            if (e == cudaSuccess)
                e = cudaMemcpyAsync(pin_base + r->pin_off + r->span,
                                    dev_base + r->dev_off + r->span, r->bytes,
                                    cudaMemcpyDeviceToHost, s_d2h);
        // the done event is recorded even after a failure so that the batch
        // retires once whatever was enqueued has finished
        cudaError_t f = cudaEventRecord(b.done, s_d2h);
        if (e != cudaSuccess || f != cudaSuccess) {
            cudaGetLastError();
            std::lock_guard<std::mutex> lk(mu);
            failed_launch = true;              // run() fails the batch's requests
        }
    }
    bool failed_launch = false;

    void run() {
        cudaSetDevice(cfg.device);
        std::unique_lock<std::mutex> lk(mu);
        for (;;) {
            retire();
            stage_heap_requests();
            Batch b;
            bool have = false;
            if (!stop && (int)inflight.size() < cfg.max_inflight && !queue.empty() &&
                queue.front()->pinned) {
                if (!new_batch(&b)) break;
                have = true;
                const auto now = Clock::now();
                while (!queue.empty() && (int)b.reqs.size() < cfg.max_batch) {
                    Req *r = queue.front();
                    if (!r->pinned) break;
                    size_t off;
                    if (!dev_alloc.alloc(2 * r->span, &off)) break;   // wait for memory
                    r->dev_off = off;
                    r->state = ADMITTED;
                    r->t_admit = now;
                    queue.pop_front();
                    b.reqs.push_back(r);
                }
                if (b.reqs.empty()) {
                    spare.push_back(std::move(b));
                    have = false;
                }
            }
            if (have) {
                lk.unlock();
                launch(b);
                lk.lock();
                if (failed_launch) {
                    // keep the requests failed: their copies or kernel never ran
                    failed_launch = false;
                    cudaEventSynchronize(b.done);
                    cudaGetLastError();
                    const auto now = Clock::now();
                    for (Req *r : b.reqs) {
                        dev_alloc.release(r->dev_off, 2 * r->span);
                        r->t_done = now;
                        r->state = FAILED;
                        ++completed;
                        if (r->cancelled) free_req(r);
                    }
                    b.reqs.clear();
                    spare.push_back(std::move(b));
                    cv_done.notify_all();
                } else {
                    inflight.push_back(std::move(b));
                    ++batches;
                }
                continue;
            }
            if (stop && inflight.empty()) break;
            if (!inflight.empty())
                cv_engine.wait_for(lk, std::chrono::microseconds(std::max(1, cfg.tick_us)));
            else
                cv_engine.wait_for(lk, std::chrono::milliseconds(50));
        }
    }
};

namespace {

void destroy(me_server *s) {
    int cur = 0;
    cudaGetDevice(&cur);
    cudaSetDevice(s->cfg.device);
    for (cudaStream_t st : {s->s_h2d, s->s_comp, s->s_d2h})
        if (st) cudaStreamSynchronize(st);
    for (auto &b : s->inflight) s->spare.push_back(b);
    for (auto &b : s->spare) {
        if (b.up) cudaEventDestroy(b.up);
        if (b.kern) cudaEventDestroy(b.kern);
        if (b.done) cudaEventDestroy(b.done);
    }
    s->ring.reset();
    for (cudaStream_t st : {s->s_h2d, s->s_comp, s->s_d2h})
        if (st) cudaStreamDestroy(st);
    for (auto &kv : s->reqs) delete kv.second;
    if (s->dev_base) cudaFree(s->dev_base);
    if (s->pin_base) cudaFreeHost(s->pin_base);
    cudaGetLastError();
    cudaSetDevice(cur);
    delete s;
}

int fail_open(me_server *s, cudaError_t e, int cur) {
    cudaGetLastError();
    destroy(s);
    cudaSetDevice(cur);
    return record_cuda(e);
}

}  // namespace

extern "C" {

int me_serve_open(const me_serve_cfg *cfg, me_server **out) {
    if (cfg == nullptr || out == nullptr) return ME_ERR_ARG;
    *out = nullptr;
    if (cfg->hbm_budget_bytes <= 0 || cfg->staging_bytes < 0 || cfg->max_inflight < 1 ||
        cfg->max_batch < 1 || cfg->tick_us < 0 || cfg->device < 0)
        return ME_ERR_ARG;
    int ndev = 0;
    cudaError_t e = cudaGetDeviceCount(&ndev);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return record_cuda(e);
    }
    if (cfg->device >= ndev) return ME_ERR_ARG;
    int cur = 0;
    cudaGetDevice(&cur);
    if ((e = cudaSetDevice(cfg->device)) != cudaSuccess) return record_cuda(e);

    me_server *s = new (std::nothrow) me_server();
    if (!s) return ME_ERR_NOMEM;
    s->cfg = *cfg;
    const size_t budget = (size_t)cfg->hbm_budget_bytes;
    const size_t staging = cfg->staging_bytes > 0 ? (size_t)cfg->staging_bytes : budget;
    if ((e = cudaMalloc(&s->dev_base, budget)) != cudaSuccess) {
        s->dev_base = nullptr;
        return fail_open(s, e, cur);
    }
    if ((e = cudaHostAlloc(&s->pin_base, staging, cudaHostAllocDefault)) != cudaSuccess) {
        s->pin_base = nullptr;
        return fail_open(s, e, cur);
    }
    s->dev_alloc.reset(budget, kAlign);
    s->pin_alloc.reset(staging, kAlign);
    for (cudaStream_t *st : {&s->s_h2d, &s->s_comp, &s->s_d2h})
        if ((e = cudaStreamCreateWithFlags(st, cudaStreamNonBlocking)) != cudaSuccess)
            return fail_open(s, e, cur);
    s->ring.reset(new BatchRing(cfg->max_inflight + 1));
    try {
        s->engine = std::thread([s] { s->run(); });
    } catch (...) {
        destroy(s);
        cudaSetDevice(cur);
        return ME_ERR_NOMEM;
    }
    cudaSetDevice(cur);
    *out = s;
    return ME_OK;
}

int me_serve_submit(me_server *s, const uint32_t *host_img, int32_t w, int32_t h,
                    int32_t stride_words, int32_t boundary, uint64_t *ticket) {
    if (s == nullptr || host_img == nullptr || ticket == nullptr) return ME_ERR_ARG;
    if (w <= 0 || h <= 0 || stride_words < (int32_t)(((int64_t)w + 31) / 32) ||
        (boundary != ME_BOUNDARY_WHITE && boundary != ME_BOUNDARY_BLACK))
        return ME_ERR_ARG;
    std::unique_ptr<Req> r(new (std::nothrow) Req());
    if (!r) return ME_ERR_NOMEM;
    r->w = w;
    r->h = h;
    r->stride = stride_words;
    r->boundary = boundary;
    r->bytes = (size_t)h * (size_t)stride_words * 4;
    r->span = (r->bytes + kAlign - 1) / kAlign * kAlign;
    r->t_submit = Clock::now();
    {
        std::lock_guard<std::mutex> lk(s->mu);
        if (s->closing) return ME_ERR_CLOSED;
        if (2 * r->span > s->dev_alloc.capacity() || 2 * r->span > s->pin_alloc.capacity())
            return ME_ERR_BUDGET;
        r->pinned = s->pin_alloc.alloc(2 * r->span, &r->pin_off);
    }
    // copy the image while the request is not yet visible to the engine
    if (r->pinned) {
        std::memcpy(s->pin_base + r->pin_off, host_img, r->bytes);
    } else {
        r->heap.reset(new (std::nothrow) uint32_t[r->bytes / 4]);
        if (!r->heap) return ME_ERR_NOMEM;
        std::memcpy(r->heap.get(), host_img, r->bytes);
    }
    std::lock_guard<std::mutex> lk(s->mu);
    if (s->closing) {
        s->free_req(r.release());
        return ME_ERR_CLOSED;
    }
    Req *p = r.release();
    p->ticket = s->next_ticket++;
    s->reqs[p->ticket] = p;
    s->queue.push_back(p);
    ++s->submitted;
    *ticket = p->ticket;
    s->cv_engine.notify_one();
    return ME_OK;
}

int me_serve_poll(me_server *s, uint64_t ticket, uint32_t *host_edge, int64_t timeout_us,
                  me_timing *t) {
    if (s == nullptr || host_edge == nullptr) return ME_ERR_ARG;
    std::unique_lock<std::mutex> lk(s->mu);
    auto it = s->reqs.find(ticket);
    if (it == s->reqs.end()) return ME_ERR_TICKET;
    Req *r = it->second;
    auto ready = [r] { return r->state == DONE || r->state == FAILED; };
    if (!ready()) {
        if (timeout_us == 0) return ME_PENDING;
        if (timeout_us < 0) {
            s->cv_done.wait(lk, ready);
        } else if (!s->cv_done.wait_for(lk, std::chrono::microseconds(timeout_us), ready)) {
            return ME_TIMEOUT;
        }
        // the request may have been collected or cancelled by another thread
        it = s->reqs.find(ticket);
        if (it == s->reqs.end() || it->second != r) return ME_ERR_TICKET;
    }
    s->reqs.erase(it);
    if (r->state == FAILED) {
        s->free_req(r);
        return ME_ERR_CUDA;
    }
    lk.unlock();
    std::memcpy(host_edge, s->pin_base + r->pin_off + r->span, r->bytes);
    if (t) {
        t->queue_us = us_since(r->t_submit, r->t_admit);
        t->device_us = us_since(r->t_admit, r->t_done);
        t->total_us = us_since(r->t_submit, r->t_done);
    }
    lk.lock();
    s->free_req(r);
    s->cv_engine.notify_one();           // staging freed: queued requests may move in
    return ME_OK;
}

int me_serve_cancel(me_server *s, uint64_t ticket) {
    if (s == nullptr) return ME_ERR_ARG;
    std::lock_guard<std::mutex> lk(s->mu);
    auto it = s->reqs.find(ticket);
    if (it == s->reqs.end()) return ME_ERR_TICKET;
    Req *r = it->second;
    s->reqs.erase(it);
    if (r->state == QUEUED) {
        s->queue.erase(std::find(s->queue.begin(), s->queue.end(), r));
        s->free_req(r);
    } else if (r->state == ADMITTED) {
        r->cancelled = true;                // freed when its batch retires
    } else {
        s->free_req(r);
    }
    s->cv_engine.notify_one();
    return ME_OK;
}

int me_serve_stats(me_server *s, int64_t *submitted, int64_t *completed, int64_t *batches,
                   int64_t *peak_bytes) {
    if (s == nullptr) return ME_ERR_ARG;
    std::lock_guard<std::mutex> lk(s->mu);
    if (submitted) *submitted = s->submitted;
    if (completed) *completed = s->completed;
    if (batches) *batches = s->batches;
    if (peak_bytes) *peak_bytes = (int64_t)s->dev_alloc.peak();
    return ME_OK;
}

int me_serve_close(me_server *s, int64_t drain_timeout_us) {
    if (s == nullptr) return ME_ERR_ARG;
    int rc = ME_OK;
    {
        std::unique_lock<std::mutex> lk(s->mu);
        s->closing = true;
        // uncollected results are dropped now, so their staging can take
        // requests still waiting in heap memory
        for (auto it = s->reqs.begin(); it != s->reqs.end();) {
            if (it->second->state == DONE || it->second->state == FAILED) {
                s->free_req(it->second);
                it = s->reqs.erase(it);
            } else {
                ++it;
            }
        }
        auto drained = [s] { return s->queue.empty() && s->inflight.empty(); };
        s->cv_engine.notify_one();
        if (drain_timeout_us < 0) {
            while (!drained()) s->cv_done.wait_for(lk, std::chrono::milliseconds(10));
        } else {
            const auto until = Clock::now() + std::chrono::microseconds(drain_timeout_us);
            while (!drained() && Clock::now() < until)
                s->cv_done.wait_for(lk, std::chrono::milliseconds(1));
            if (!drained()) rc = ME_TIMEOUT;
        }
        // requests never admitted are dropped
        for (Req *r : s->queue) {
            s->reqs.erase(r->ticket);
            s->free_req(r);
        }
        s->queue.clear();
        s->stop = true;
        s->cv_engine.notify_one();
    }
    if (s->engine.joinable()) s->engine.join();
    destroy(s);
    return rc;
}

}  // extern "C"
