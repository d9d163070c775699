// Serving engine: continuous batching of edge-map requests on one GPU.
//
// submit() takes a range of pinned staging (or, when staging is full, heap
// memory until staging frees up), queues the request and copies the image
// in.  An engine thread admits queued requests in arrival order while the
// device pool (the HBM budget) has room for the request's packed image and
// edge map and fewer than max_inflight batches are on the GPU; each
// admitted group becomes one batch:
//     H2D copies (stream h2d) -> persistent batch kernel under a CUDA graph
//     (stream compute) -> D2H copies (stream d2h) -> completion event.
// The three streams let the uploads of the next batch and the downloads of
// the previous one overlap the running kernel.  A completion thread watches
// the oldest batch's event, retires batches in order as they finish, frees
// their device memory and wakes the pollers of their requests and the
// engine; poll() copies a finished edge map out of staging and forgets the
// ticket.
//
// Both pools are split in two halves, inputs in the lower and edge maps in
// the upper, and a request takes the same offset in both halves of a pool.
// Staging is handed out by next fit at submit and device memory by next fit
// at admission, both in arrival order, so the requests of a batch usually
// sit back to back in staging and on the device alike: the engine merges
// such neighbours into one copy each way (a batch of hundreds of requests
// moves in a handful of copies instead of two per request).
//
// Locks, taken only in this order when nested: qmu (the queue, staging,
// admission order, the engine's sleep), dev_mu (the device pool, batches in
// flight, the completion thread's sleep), then one of kShards ticket shards
// (ticket -> request, a request's completion state, its poller's wake-up).
// A submit takes qmu and a shard once each; a poll takes a shard and hands
// the request's staging back through a lock-free list that the next submit
// (or the engine) empties under qmu.  The engine sleeps only after stating
// what it waits for (engine_waiting, waits_for) and re-checking it, and
// every thread that may unblock it bumps wake_seq and then looks at
// engine_waiting, so no wake-up is lost and none is sent for nothing.
//
// All waits are bounded by the caller's timeouts, by `stop`, or by the
// GPU's own progress; nothing here spins on a flag the GPU sets.
#include <algorithm>
#include <atomic>
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
constexpr int kShards = 16;
// A poller watches its request this long before it sleeps: most requests
// finish meanwhile, and the completion thread then makes no wake-up call.
// At saturation a request takes about 110-150 us in the server; 100 us
// measured 4-6% more requests per second than 30 us, and 300 or 1000 us no
// more than 100.
constexpr int kSpinUs = 100;

enum State { QUEUED, ADMITTED, DONE, FAILED };

struct Req {
    uint64_t ticket = 0;
    int32_t w = 0, h = 0, stride = 0, boundary = 0;
    size_t bytes = 0, span = 0;        // packed size; rounded to kAlign
    bool pinned = false;               // input is in staging (else in heap), or
                                       // a direct request; qmu
    std::atomic<bool> copied{false};   // the input copy into staging is done
    Req *next_free = nullptr;          // link in the server's list of freed requests
    size_t pin_off = 0;                // staging: input at in + off, output at out + off
    std::unique_ptr<uint32_t[]> heap;  // input while staging was full
    size_t dev_off = 0;                // device: input at in + off, output at out + off
    // QUEUED -> ADMITTED under dev_mu (the engine has taken the request off
    // the queue then), then DONE or FAILED under the shard;
    // atomic so that a poller may watch it without the lock
    std::atomic<State> state{QUEUED};
    bool cancelled = false;            // under qmu and the shard
    bool open = false;                 // reserved, not yet committed (qmu and the shard)
    // direct request: the kernel reads host_in and writes host_out, the
    // caller's own host buffers, over the CPU-GPU link (no staging, no
    // device memory, no copies)
    const uint32_t *host_in = nullptr;
    uint32_t *host_out = nullptr;
    bool direct() const { return host_out != nullptr; }
    // the condition the poller waiting for this request sleeps on (only that
    // poller is woken when the request's batch retires); under the shard
    std::condition_variable *waiter = nullptr;
    Clock::time_point t_submit, t_admit, t_done;
};

struct Batch {
    std::vector<Req *> reqs;
    cudaEvent_t up = nullptr, kern = nullptr, done = nullptr;
    bool failed = false;               // a CUDA call of its launch failed
};

struct Shard {
    std::mutex mu;
    std::unordered_map<uint64_t, Req *> map;
};

// Maximal runs of a batch's requests that lie back to back both in staging
// and on the device; f(first, last).
template <class F>
void for_each_run(const std::vector<Req *> &reqs, F &&f) {
    size_t i = 0;
    while (i < reqs.size()) {
        if (reqs[i]->direct()) {       // nothing to copy
            ++i;
            continue;
        }
        size_t j = i;
        while (j + 1 < reqs.size() && !reqs[j + 1]->direct() &&
               reqs[j + 1]->pin_off == reqs[j]->pin_off + reqs[j]->span &&
               reqs[j + 1]->dev_off == reqs[j]->dev_off + reqs[j]->span)
            ++j;
        f(reqs[i], reqs[j]);
        i = j + 1;
    }
}

bool finished(const Req *r) {
    const State st = r->state.load();
    return st == DONE || st == FAILED;
}

// Wait until r has finished, at most timeout_us (negative: no limit).  sl
// holds r's shard lock on entry and on return.  ME_OK, ME_PENDING (timeout
// 0), ME_TIMEOUT, or ME_ERR_ARG when another thread already waits for r.
int wait_finished(std::unique_lock<std::mutex> &sl, Req *r, int64_t timeout_us) {
    if (finished(r)) return ME_OK;
    if (timeout_us == 0) return ME_PENDING;
    if (r->waiter != nullptr) return ME_ERR_ARG;
    std::condition_variable cv;
    r->waiter = &cv;                   // from here on cancel refuses the ticket
    const auto t0 = Clock::now();
    const int64_t spin = timeout_us < 0 ? kSpinUs : std::min<int64_t>(kSpinUs, timeout_us);
    sl.unlock();
    const auto spin_end = t0 + std::chrono::microseconds(spin);
    while (!finished(r) && Clock::now() < spin_end) std::this_thread::yield();
    sl.lock();
    bool ok = true;
    if (timeout_us < 0)
        cv.wait(sl, [r] { return finished(r); });
    else
        ok = cv.wait_until(sl, t0 + std::chrono::microseconds(timeout_us),
                           [r] { return finished(r); });
    r->waiter = nullptr;
    return ok ? ME_OK : ME_TIMEOUT;
}

}  // namespace

struct me_server {
    me_serve_cfg cfg{};
    char *dev_base = nullptr;          // [inputs | edge maps], dev_half bytes each
    char *pin_base = nullptr;          // [inputs | edge maps], pin_half bytes each
    size_t dev_half = 0, pin_half = 0;
    cudaStream_t s_h2d = nullptr, s_comp = nullptr, s_d2h = nullptr;
    std::unique_ptr<BatchRing> ring;
    std::thread engine, retirer;

    // qmu: the queue, staging, closing/stop, the engine's sleep
    std::mutex qmu;
    std::condition_variable cv_engine;
    std::deque<Req *> queue;
    RangeAlloc pin_alloc;              // offsets within one staging half
    bool closing = false, stop = false;
    std::atomic<int> heap_waiting{0};  // queued requests still in heap memory
    uint64_t next_ticket = 1;

    // the engine's sleep: what it waits for, and a counter every waker bumps
    std::atomic<bool> engine_waiting{false};
    std::atomic<Req *> waits_for{nullptr};  // the request whose copy it needs
    std::atomic<uint64_t> wake_seq{0};
    // collected requests whose staging is still to be released (under qmu)
    std::atomic<Req *> freed{nullptr};

    // dev_mu: the device pool, batches in flight, the completion thread's sleep
    std::mutex dev_mu;
    std::condition_variable cv_retire;
    RangeAlloc dev_alloc;              // offsets within one device half
    std::deque<Batch> inflight;
    std::vector<Batch> spare;          // batches whose events can be reused
    bool stop_retirer = false;

    Shard shards[kShards];

    std::atomic<int64_t> submitted{0}, completed{0}, batches{0}, copies{0};

    Shard &shard(uint64_t ticket) { return shards[ticket % kShards]; }
    char *dev_in(const Req *r) const { return dev_base + r->dev_off; }
    char *dev_out(const Req *r) const { return dev_base + dev_half + r->dev_off; }
    char *pin_in(const Req *r) const { return pin_base + r->pin_off; }
    char *pin_out(const Req *r) const { return pin_base + pin_half + r->pin_off; }

    // ------------------------------------------------------------------
    void free_req(Req *r) {            // caller holds qmu
        if (r->pinned && !r->direct()) pin_alloc.release(r->pin_off, r->span);
        delete r;
    }

    // Hand a finished request to the next holder of qmu (no lock taken).
    void push_freed(Req *r) {
        Req *h = freed.load(std::memory_order_relaxed);
        do {
            r->next_free = h;
        } while (!freed.compare_exchange_weak(h, r, std::memory_order_release,
                                              std::memory_order_relaxed));
    }
    // Give the staging of the requests on the freed list back (caller holds
    // qmu) and return the list, whose requests the caller deletes once it
    // has let go of qmu (they were allocated by other threads, whose heap
    // arenas a delete may have to lock).
    Req *drain_freed() {
        Req *head = freed.exchange(nullptr, std::memory_order_acquire);
        for (Req *r = head; r != nullptr; r = r->next_free)
            if (r->pinned && !r->direct()) pin_alloc.release(r->pin_off, r->span);
        return head;
    }
    static void delete_list(Req *r) {
        while (r) {
            Req *n = r->next_free;
            delete r;
            r = n;
        }
    }

    // Something the engine may wait for has changed.
    void wake_engine_locked() {        // caller holds qmu
        wake_seq.fetch_add(1);
        if (engine_waiting.load()) cv_engine.notify_one();
    }
    void wake_engine() {               // caller holds no server lock
        wake_seq.fetch_add(1);
        if (engine_waiting.load()) {
            std::lock_guard<std::mutex> lk(qmu);
            cv_engine.notify_one();
        }
    }

    bool new_batch(Batch *b) {         // caller holds dev_mu
        if (!spare.empty()) {
            *b = std::move(spare.back());
            spare.pop_back();
            b->reqs.clear();
            b->failed = false;
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

    // Give staging to queued requests still held in heap memory, in order.
    // Called with qmu held through lk; the copies run with it released (the
    // requests are not admitted meanwhile: copied is false).
    void stage_heap_requests(std::unique_lock<std::mutex> &lk) {
        if (heap_waiting.load() == 0) return;
        std::vector<Req *> moved;
        for (Req *r : queue) {
            if (r->pinned) continue;
            size_t off;
            if (!pin_alloc.alloc_next(r->span, &off)) break;
            r->pin_off = off;
            r->pinned = true;
            r->copied = false;
            --heap_waiting;
            moved.push_back(r);
        }
        if (moved.empty()) return;
        lk.unlock();
        for (Req *r : moved) {
            std::memcpy(pin_in(r), r->heap.get(), r->bytes);
            r->heap.reset();
        }
        lk.lock();
        // requests cancelled (or dropped by close) during the copy are
        // freed here, by the thread that held them
        for (Req *r : moved) {
            if (r->cancelled) free_req(r);
            else r->copied.store(true);
        }
    }

    // Issue one admitted batch; called without locks.  Returns false if any
    // CUDA call failed (the done event is still recorded behind whatever
    // was enqueued).
    bool launch(Batch &b, int64_t *ncopies) {
        cudaError_t e = cudaSuccess;
        int64_t nc = 0;
        std::vector<me_desc> descs;
        descs.reserve(b.reqs.size());
        for_each_run(b.reqs, [&](const Req *a, const Req *z) {
            const size_t n = z->pin_off + z->bytes - a->pin_off;
            if (e == cudaSuccess)
                e = cudaMemcpyAsync(dev_in(a), pin_in(a), n, cudaMemcpyHostToDevice, s_h2d);
            ++nc;
        });
        // a batch of direct requests only has no copies: the kernel and the
        // done event are all it enqueues
        const bool copying = nc > 0;
        for (Req *r : b.reqs) {
            if (r->direct())
                descs.push_back({r->host_in, r->host_out, r->w, r->h, r->stride, r->boundary});
            else
                descs.push_back({reinterpret_cast<const uint32_t *>(dev_in(r)),
                                 reinterpret_cast<uint32_t *>(dev_out(r)), r->w, r->h, r->stride,
                                 r->boundary});
        }
        if (copying && e == cudaSuccess) e = cudaEventRecord(b.up, s_h2d);
        if (copying && e == cudaSuccess) e = cudaStreamWaitEvent(s_comp, b.up, 0);
        if (e == cudaSuccess) {
            const int rc = ring->launch(descs.data(), (int)descs.size(), s_comp);
            if (rc != ME_OK) e = cudaErrorLaunchFailure;
        }
        if (copying) {
            if (e == cudaSuccess) e = cudaEventRecord(b.kern, s_comp);
            if (e == cudaSuccess) e = cudaStreamWaitEvent(s_d2h, b.kern, 0);
            for_each_run(b.reqs, [&](const Req *a, const Req *z) {
                const size_t n = z->pin_off + z->bytes - a->pin_off;
                if (e == cudaSuccess)
                    e = cudaMemcpyAsync(pin_out(a), dev_out(a), n, cudaMemcpyDeviceToHost,
                                        s_d2h);
                ++nc;
            });
        }
        // recorded even after a failure, so that the batch retires once
        // whatever was enqueued has finished
        const cudaError_t f = cudaEventRecord(b.done, copying ? s_d2h : s_comp);
        *ncopies = nc;
        if (e != cudaSuccess || f != cudaSuccess) {
            cudaGetLastError();
            return false;
        }
        return true;
    }

    // Engine thread: admission and launches.
    enum Blocked { NOTHING, EMPTY, NOT_COPIED, HEAP, NO_SLOT, NO_MEMORY };

    // Admit a batch from the head of the queue into b.  lk holds qmu on
    // entry and on return; the ready requests at the head are taken off the
    // queue under it, and their device memory is given with it released
    // (submitters are not held up meanwhile).  Those that do not fit go back
    // to the head of the queue, in order.
    Blocked admit(Batch *b, std::unique_lock<std::mutex> &lk) {
        if (queue.empty()) return EMPTY;
        Req *f = queue.front();
        if (!f->pinned) return HEAP;
        if (!f->copied.load()) return NOT_COPIED;
        {
            std::lock_guard<std::mutex> dl(dev_mu);
            if ((int)inflight.size() >= cfg.max_inflight) return NO_SLOT;
            if (!new_batch(b)) return NO_SLOT;
        }
        std::vector<Req *> &take = b->reqs;
        while (!queue.empty() && (int)take.size() < cfg.max_batch) {
            Req *r = queue.front();
            if (!r->pinned || !r->copied.load()) break;
            queue.pop_front();
            take.push_back(r);
        }
        lk.unlock();
        size_t k = 0;
        {
            std::lock_guard<std::mutex> dl(dev_mu);
            const auto now = Clock::now();
            for (; k < take.size(); ++k) {
                Req *r = take[k];
                if (!r->direct()) {
                    size_t off;
                    if (!dev_alloc.alloc_next(r->span, &off)) break;   // wait for memory
                    r->dev_off = off;
                }
                r->t_admit = now;
                r->state = ADMITTED;
            }
        }
        lk.lock();
        for (size_t j = take.size(); j-- > k;) queue.push_front(take[j]);
        take.resize(k);
        if (take.empty()) {
            std::lock_guard<std::mutex> dl(dev_mu);
            spare.push_back(std::move(*b));
            return NO_MEMORY;
        }
        return NOTHING;
    }

    void run_engine() {
        cudaSetDevice(cfg.device);
        std::unique_lock<std::mutex> lk(qmu);
        for (;;) {
            const uint64_t seq = wake_seq.load();
            if (Req *dead = drain_freed()) {
                lk.unlock();
                delete_list(dead);
                lk.lock();
            }
            stage_heap_requests(lk);
            if (stop) break;
            Batch b;
            const Blocked why = admit(&b, lk);
            if (why == NOTHING) {
                lk.unlock();
                int64_t nc = 0;
                const bool ok = launch(b, &nc);
                if (!ok) cudaEventSynchronize(b.done);   // let enqueued work end
                copies += nc;
                ++batches;
                {
                    // a batch whose copies or kernel never ran: its requests
                    // fail, in order, once the batches before it have retired
                    std::lock_guard<std::mutex> dl(dev_mu);
                    b.failed = !ok;
                    inflight.push_back(std::move(b));
                    cv_retire.notify_one();
                }
                lk.lock();
                continue;
            }
            // state what is awaited, then look again: a waker changes its
            // state first and reads engine_waiting / waits_for after
            Req *f = why == NOT_COPIED && !queue.empty() ? queue.front() : nullptr;
            waits_for.store(f);
            engine_waiting.store(true);
            const bool changed = wake_seq.load() != seq || (f && f->copied.load());
            if (!changed) cv_engine.wait_for(lk, std::chrono::milliseconds(20));
            engine_waiting.store(false);
            waits_for.store(nullptr);
        }
    }

    // Completion thread: retires batches in order as their events complete.
    // While batches are in flight it queries the oldest one's event every
    // tick_us microseconds (0: continuously, yielding between queries).
    void run_retirer() {
        cudaSetDevice(cfg.device);
        std::vector<Req *> reqs, gone;
        for (;;) {
            cudaEvent_t ev;
            {
                std::unique_lock<std::mutex> dl(dev_mu);
                while (inflight.empty()) {
                    if (stop_retirer) return;
                    cv_retire.wait_for(dl, std::chrono::milliseconds(20));
                }
                ev = inflight.front().done;
            }
            cudaError_t q = cudaEventQuery(ev);
            while (q == cudaErrorNotReady) {
                if (cfg.tick_us > 0)
                    std::this_thread::sleep_for(std::chrono::microseconds(cfg.tick_us));
                else
                    std::this_thread::yield();
                q = cudaEventQuery(ev);
            }
            if (q != cudaSuccess) cudaGetLastError();
            {
                std::lock_guard<std::mutex> dl(dev_mu);
                Batch &b = inflight.front();
                if (b.failed) q = cudaErrorLaunchFailure;
                for (Req *r : b.reqs)
                    if (!r->direct()) dev_alloc.release(r->dev_off, r->span);
                reqs.swap(b.reqs);
                spare.push_back(std::move(b));
                inflight.pop_front();
            }
            const State st = q == cudaSuccess ? DONE : FAILED;
            const auto now = Clock::now();
            gone.clear();
            for (Req *r : reqs) {
                Shard &sh = shard(r->ticket);
                std::lock_guard<std::mutex> sl(sh.mu);
                r->t_done = now;
                r->state = st;
                if (r->waiter) r->waiter->notify_one();
                if (r->cancelled) gone.push_back(r);
            }
            completed += (int64_t)reqs.size();
            reqs.clear();
            for (Req *r : gone) push_freed(r);
            wake_engine();                  // a slot and device memory are free
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
    for (auto &b : s->inflight) {
        // admitted requests that were cancelled live only in their batch
        for (Req *r : b.reqs)
            if (r->cancelled) delete r;
        b.reqs.clear();
        s->spare.push_back(std::move(b));
    }
    s->inflight.clear();
    for (auto &b : s->spare) {
        if (b.up) cudaEventDestroy(b.up);
        if (b.kern) cudaEventDestroy(b.kern);
        if (b.done) cudaEventDestroy(b.done);
    }
    s->ring.reset();
    for (cudaStream_t st : {s->s_h2d, s->s_comp, s->s_d2h})
        if (st) cudaStreamDestroy(st);
    for (auto &sh : s->shards)
        for (auto &kv : sh.map) delete kv.second;
    // cancelled requests the engine put back on the queue after close
    // emptied it are in no map
    for (Req *r : s->queue)
        if (r->cancelled) delete r;
    for (Req *r = s->freed.exchange(nullptr); r != nullptr;) {
        Req *n = r->next_free;
        delete r;
        r = n;
    }
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
    // each pool in two halves of whole kAlign units
    const size_t budget = (size_t)cfg->hbm_budget_bytes / (2 * kAlign) * (2 * kAlign);
    const size_t staging0 = cfg->staging_bytes > 0 ? (size_t)cfg->staging_bytes : budget;
    const size_t staging = staging0 / (2 * kAlign) * (2 * kAlign);
    if (budget == 0 || staging == 0) return ME_ERR_ARG;
    int cur = 0;
    cudaGetDevice(&cur);
    if ((e = cudaSetDevice(cfg->device)) != cudaSuccess) return record_cuda(e);

    me_server *s = new (std::nothrow) me_server();
    if (!s) {
        cudaSetDevice(cur);
        return ME_ERR_NOMEM;
    }
    s->cfg = *cfg;
    s->dev_half = budget / 2;
    s->pin_half = staging / 2;
    if ((e = cudaMalloc(&s->dev_base, budget)) != cudaSuccess) {
        s->dev_base = nullptr;
        return fail_open(s, e, cur);
    }
    if ((e = cudaHostAlloc(&s->pin_base, staging, cudaHostAllocDefault)) != cudaSuccess) {
        s->pin_base = nullptr;
        return fail_open(s, e, cur);
    }
    s->dev_alloc.reset(s->dev_half, kAlign);
    s->pin_alloc.reset(s->pin_half, kAlign);
    for (cudaStream_t *st : {&s->s_h2d, &s->s_comp, &s->s_d2h})
        if ((e = cudaStreamCreateWithFlags(st, cudaStreamNonBlocking)) != cudaSuccess)
            return fail_open(s, e, cur);
    s->ring.reset(new BatchRing(cfg->max_inflight + 1));
    try {
        s->engine = std::thread([s] { s->run_engine(); });
        s->retirer = std::thread([s] { s->run_retirer(); });
    } catch (...) {
        {
            std::lock_guard<std::mutex> lk(s->qmu);
            s->stop = true;
        }
        {
            std::lock_guard<std::mutex> dl(s->dev_mu);
            s->stop_retirer = true;
        }
        s->cv_engine.notify_all();
        s->cv_retire.notify_all();
        if (s->engine.joinable()) s->engine.join();
        if (s->retirer.joinable()) s->retirer.join();
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
    Req *p = r.get();
    Req *dead = nullptr;
    {
        std::lock_guard<std::mutex> lk(s->qmu);
        if (s->closing) return ME_ERR_CLOSED;
        if (p->span > s->dev_half || p->span > s->pin_half) return ME_ERR_BUDGET;
        dead = s->drain_freed();
        p->pinned = s->pin_alloc.alloc_next(p->span, &p->pin_off);
        p->ticket = s->next_ticket++;
        if (p->pinned) {
            // queued at once, in staging order, but not admitted before the
            // copy below has finished (copied == false); an engine asleep on
            // an empty queue now waits for this request's copy
            s->queue.push_back(p);
            if (s->queue.size() == 1 && s->engine_waiting.load()) s->waits_for.store(p);
        }
    }
    me_server::delete_list(dead);
    if (!p->pinned) {
        p->heap.reset(new (std::nothrow) uint32_t[p->bytes / 4]);
        if (!p->heap) return ME_ERR_NOMEM;      // p was never queued
        std::memcpy(p->heap.get(), host_img, p->bytes);
    }
    {
        Shard &sh = s->shard(p->ticket);
        std::lock_guard<std::mutex> sl(sh.mu);
        sh.map[p->ticket] = p;
    }
    r.release();
    *ticket = p->ticket;
    ++s->submitted;
    if (p->pinned) {
        std::memcpy(s->pin_in(p), host_img, p->bytes);
        p->copied.store(true);
        if (s->waits_for.load() == p) s->wake_engine();
        return ME_OK;
    }
    std::lock_guard<std::mutex> lk(s->qmu);
    p->copied.store(true);
    s->queue.push_back(p);
    ++s->heap_waiting;
    s->wake_engine_locked();
    return ME_OK;
}

int me_serve_poll(me_server *s, uint64_t ticket, uint32_t *host_edge, int64_t timeout_us,
                  me_timing *t) {
    if (s == nullptr) return ME_ERR_ARG;
    Shard &sh = s->shard(ticket);
    std::unique_lock<std::mutex> sl(sh.mu);
    auto it = sh.map.find(ticket);
    if (it == sh.map.end()) return ME_ERR_TICKET;
    Req *r = it->second;
    if (host_edge == nullptr && !r->direct()) return ME_ERR_ARG;
    if (!finished(r)) {
        const int rc = wait_finished(sl, r, timeout_us);
        if (rc != ME_OK) return rc;
        it = sh.map.find(ticket);           // the map may have rehashed meanwhile
    }
    sh.map.erase(it);
    sl.unlock();
    const bool ok = r->state == DONE;
    if (ok) {
        if (!r->direct())
            std::memcpy(host_edge, s->pin_out(r), r->bytes);
        else if (host_edge != nullptr && host_edge != r->host_out)
            std::memcpy(host_edge, r->host_out, r->bytes);
        if (t) {
            t->queue_us = us_since(r->t_submit, r->t_admit);
            t->device_us = us_since(r->t_admit, r->t_done);
            t->total_us = us_since(r->t_submit, r->t_done);
        }
    }
    // its staging goes back at the next submit or engine round; requests
    // waiting in heap memory need the engine to take it
    s->push_freed(r);
    if (s->heap_waiting.load() > 0) s->wake_engine();
    return ok ? ME_OK : ME_ERR_CUDA;
}

int me_serve_cancel(me_server *s, uint64_t ticket) {
    if (s == nullptr) return ME_ERR_ARG;
    std::lock_guard<std::mutex> lk(s->qmu);
    Shard &sh = s->shard(ticket);
    std::lock_guard<std::mutex> sl(sh.mu);
    auto it = sh.map.find(ticket);
    if (it == sh.map.end()) return ME_ERR_TICKET;
    Req *r = it->second;
    if (r->waiter != nullptr) return ME_ERR_ARG;   // a poll is waiting for it
    sh.map.erase(it);
    const auto qit = std::find(s->queue.begin(), s->queue.end(), r);
    if (r->state == QUEUED && qit == s->queue.end()) {
        r->cancelled = true;                // being admitted: freed when its batch retires
    } else if (r->state == QUEUED) {
        s->queue.erase(qit);
        if (r->open) {
            s->free_req(r);                 // reserved, never committed
        } else if (!r->copied.load()) {
            r->cancelled = true;            // the engine is copying it in; it frees it
        } else {
            if (!r->pinned) --s->heap_waiting;
            s->free_req(r);
        }
    } else if (r->state == ADMITTED) {
        r->cancelled = true;                // freed when its batch retires
    } else {
        s->free_req(r);
    }
    s->wake_engine_locked();
    return ME_OK;
}

int me_serve_reserve(me_server *s, int32_t w, int32_t h, int32_t stride_words,
                     int32_t boundary, uint64_t *ticket, uint32_t **host_img) {
    if (s == nullptr || ticket == nullptr || host_img == nullptr) return ME_ERR_ARG;
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
    r->open = true;
    Req *p = r.get();
    Req *dead = nullptr;
    bool room = false;
    {
        std::lock_guard<std::mutex> lk(s->qmu);
        if (s->closing) return ME_ERR_CLOSED;
        if (p->span > s->dev_half || p->span > s->pin_half) return ME_ERR_BUDGET;
        dead = s->drain_freed();
        room = s->pin_alloc.alloc_next(p->span, &p->pin_off);
        if (room) {
            p->pinned = true;
            p->ticket = s->next_ticket++;
            s->queue.push_back(p);
            if (s->queue.size() == 1 && s->engine_waiting.load()) s->waits_for.store(p);
        }
    }
    me_server::delete_list(dead);
    if (!room) return ME_PENDING;
    {
        Shard &sh = s->shard(p->ticket);
        std::lock_guard<std::mutex> sl(sh.mu);
        sh.map[p->ticket] = p;
    }
    r.release();
    ++s->submitted;
    *ticket = p->ticket;
    *host_img = reinterpret_cast<uint32_t *>(s->pin_in(p));
    return ME_OK;
}

int me_serve_submit_direct(me_server *s, const uint32_t *host_img, uint32_t *host_edge,
                           int32_t w, int32_t h, int32_t stride_words, int32_t boundary,
                           uint64_t *ticket) {
    if (s == nullptr || host_img == nullptr || host_edge == nullptr || ticket == nullptr)
        return ME_ERR_ARG;
    if (w <= 0 || h <= 0 || stride_words < (int32_t)(((int64_t)w + 31) / 32) ||
        (boundary != ME_BOUNDARY_WHITE && boundary != ME_BOUNDARY_BLACK) ||
        ((uintptr_t)host_img & 3) || ((uintptr_t)host_edge & 3))
        return ME_ERR_ARG;
    const size_t bytes = (size_t)h * (size_t)stride_words * 4;
    if (ranges_overlap(host_img, bytes, host_edge, bytes)) return ME_ERR_ALIAS;
    // both buffers must be host memory the device can reach (pinned or
    // registered with CUDA)
    for (const void *q : {static_cast<const void *>(host_img), static_cast<const void *>(host_edge)}) {
        cudaPointerAttributes a;
        const cudaError_t e = cudaPointerGetAttributes(&a, q);
        if (e != cudaSuccess) {
            cudaGetLastError();
            return ME_ERR_ARG;
        }
        if (a.type != cudaMemoryTypeHost) return ME_ERR_ARG;
    }
    std::unique_ptr<Req> r(new (std::nothrow) Req());
    if (!r) return ME_ERR_NOMEM;
    r->w = w;
    r->h = h;
    r->stride = stride_words;
    r->boundary = boundary;
    r->bytes = bytes;
    r->span = (bytes + kAlign - 1) / kAlign * kAlign;
    r->host_in = host_img;
    r->host_out = host_edge;
    r->pinned = true;                       // ready for admission as it stands
    r->copied.store(true);
    r->t_submit = Clock::now();
    Req *p = r.get();
    {
        std::lock_guard<std::mutex> lk(s->qmu);
        if (s->closing) return ME_ERR_CLOSED;
        p->ticket = s->next_ticket++;
        Shard &sh = s->shard(p->ticket);
        {
            std::lock_guard<std::mutex> sl(sh.mu);
            sh.map[p->ticket] = p;
        }
        s->queue.push_back(p);
        r.release();
        ++s->submitted;
        *ticket = p->ticket;
        if (s->queue.front() == p) s->wake_engine_locked();
    }
    return ME_OK;
}

int me_serve_commit(me_server *s, uint64_t ticket) {
    if (s == nullptr) return ME_ERR_ARG;
    Req *p = nullptr;
    {
        Shard &sh = s->shard(ticket);
        std::lock_guard<std::mutex> sl(sh.mu);
        auto it = sh.map.find(ticket);
        if (it == sh.map.end()) return ME_ERR_TICKET;
        p = it->second;
        if (!p->open) return ME_ERR_ARG;      // not reserved, or committed already
        p->open = false;
    }
    p->copied.store(true);
    if (s->waits_for.load() == p) s->wake_engine();
    return ME_OK;
}

int me_serve_poll_view(me_server *s, uint64_t ticket, int64_t timeout_us,
                       const uint32_t **host_edge, me_timing *t) {
    if (s == nullptr || host_edge == nullptr) return ME_ERR_ARG;
    Shard &sh = s->shard(ticket);
    std::unique_lock<std::mutex> sl(sh.mu);
    auto it = sh.map.find(ticket);
    if (it == sh.map.end()) return ME_ERR_TICKET;
    Req *r = it->second;
    const int rc = wait_finished(sl, r, timeout_us);
    if (rc != ME_OK) return rc;
    if (r->state == FAILED) return ME_ERR_CUDA;
    *host_edge = r->direct() ? r->host_out : reinterpret_cast<const uint32_t *>(s->pin_out(r));
    if (t) {
        t->queue_us = us_since(r->t_submit, r->t_admit);
        t->device_us = us_since(r->t_admit, r->t_done);
        t->total_us = us_since(r->t_submit, r->t_done);
    }
    return ME_OK;
}

int me_serve_release(me_server *s, uint64_t ticket) {
    if (s == nullptr) return ME_ERR_ARG;
    Req *r = nullptr;
    {
        Shard &sh = s->shard(ticket);
        std::lock_guard<std::mutex> sl(sh.mu);
        auto it = sh.map.find(ticket);
        if (it == sh.map.end()) return ME_ERR_TICKET;
        r = it->second;
        if (r->state != DONE && r->state != FAILED) return ME_ERR_ARG;
        sh.map.erase(it);
    }
    s->push_freed(r);
    if (s->heap_waiting.load() > 0) s->wake_engine();
    return ME_OK;
}

int me_serve_stats(me_server *s, int64_t *submitted, int64_t *completed, int64_t *batches,
                   int64_t *peak_bytes) {
    if (s == nullptr) return ME_ERR_ARG;
    if (submitted) *submitted = s->submitted.load();
    if (completed) *completed = s->completed.load();
    if (batches) *batches = s->batches.load();
    if (peak_bytes) {
        std::lock_guard<std::mutex> dl(s->dev_mu);
        *peak_bytes = 2 * (int64_t)s->dev_alloc.peak();
    }
    return ME_OK;
}

int me_serve_copies(me_server *s, int64_t *copies) {
    if (s == nullptr || copies == nullptr) return ME_ERR_ARG;
    *copies = s->copies.load();
    return ME_OK;
}

int me_serve_close(me_server *s, int64_t drain_timeout_us) {
    if (s == nullptr) return ME_ERR_ARG;
    int rc = ME_OK;
    {
        std::lock_guard<std::mutex> lk(s->qmu);
        s->closing = true;
        s->wake_engine_locked();
    }
    // uncollected results are dropped now, so their staging can take
    // requests still waiting in heap memory
    std::vector<Req *> dropped;
    for (auto &sh : s->shards) {
        std::lock_guard<std::mutex> sl(sh.mu);
        for (auto it = sh.map.begin(); it != sh.map.end();) {
            if (it->second->state == DONE || it->second->state == FAILED) {
                dropped.push_back(it->second);
                it = sh.map.erase(it);
            } else {
                ++it;
            }
        }
    }
    {
        std::lock_guard<std::mutex> lk(s->qmu);
        for (Req *r : dropped) s->free_req(r);
        s->wake_engine_locked();
    }
    auto drained = [s] {
        std::lock_guard<std::mutex> lk(s->qmu);
        std::lock_guard<std::mutex> dl(s->dev_mu);
        return s->queue.empty() && s->inflight.empty();
    };
    const auto until = Clock::now() + std::chrono::microseconds(drain_timeout_us);
    while (!drained()) {
        if (drain_timeout_us >= 0 && Clock::now() >= until) {
            rc = ME_TIMEOUT;
            break;
        }
        std::this_thread::sleep_for(std::chrono::microseconds(200));
    }
    {
        // requests never admitted are dropped (one the engine is copying
        // into staging is freed by the engine when the copy is done)
        std::lock_guard<std::mutex> lk(s->qmu);
        for (Req *r : s->queue) {
            Shard &sh = s->shard(r->ticket);
            {
                std::lock_guard<std::mutex> sl(sh.mu);
                sh.map.erase(r->ticket);
            }
            if (!r->copied.load() && !r->open) r->cancelled = true;
            else s->free_req(r);
        }
        s->queue.clear();
        s->heap_waiting.store(0);
        s->stop = true;
        s->wake_seq.fetch_add(1);
        s->cv_engine.notify_all();
    }
    if (s->engine.joinable()) s->engine.join();
    {
        // the engine has launched its last batch; the completion thread
        // retires what is in flight and then stops
        std::lock_guard<std::mutex> dl(s->dev_mu);
        s->stop_retirer = true;
        s->cv_retire.notify_all();
    }
    if (s->retirer.joinable()) s->retirer.join();
    destroy(s);
    return rc;
}

}  // extern "C"
