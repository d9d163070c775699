// Load generator for the serving engine (libme_loadgen.so).
//
// Drives a server through the public C ABI of include/me.h only, from host
// threads, so that the offered load is bounded by the server and the host
// link rather than by the client.  Each client is one thread that submits
// its share of the requests and collects their results oldest first: in a
// closed loop it keeps up to `window` requests outstanding; in an open loop
// it submits every request at its scheduled arrival time and, between
// arrivals, waits for the oldest result no longer than until the next
// arrival.  Latency is measured from the scheduled arrival (open loop) or
// from the submit call (closed loop) to the return of the poll that
// delivered the result, so a client or server that falls behind its
// schedule shows in it.  Every result can be compared with the edge map it
// must equal.  Three ways to hand requests over (mode): 0, me_serve_submit
// and me_serve_poll (one copy in, one copy out); 1, the zero-copy calls
// (each client writes its image straight into the staging it reserved and
// reads the edge map where the server left it); 2, me_serve_submit_direct
// (the images already sit in host memory the GPU reaches, and each client
// has a ring of such output slots the kernel writes into).  In modes 1 and 2
// an XOR over the edge map's words stands for the client consuming it.
//
// Not part of libme's C ABI; bench.py and the serving tests load it.
#include <algorithm>
#include <atomic>
#include <chrono>
#include <cstdint>
#include <cstring>
#include <deque>
#include <thread>
#include <vector>

#include <sys/prctl.h>

#include "me.h"

namespace {

using Clock = std::chrono::steady_clock;

double us_between(Clock::time_point a, Clock::time_point b) {
    return std::chrono::duration<double, std::micro>(b - a).count();
}

// Sleep until t: coarse sleep to 100 us before it, then yield.
void wait_until(Clock::time_point t) {
    for (;;) {
        const auto now = Clock::now();
        if (now >= t) return;
        const double left = us_between(now, t);
        if (left > 150.0)
            std::this_thread::sleep_for(std::chrono::microseconds((int64_t)(left - 100.0)));
        else
            std::this_thread::yield();
    }
}

}  // namespace

extern "C" {

typedef struct me_load_item {
    const uint32_t *img;       // host image: h rows of stride_words words
    const uint32_t *expect;    // NULL, or the edge map the result must equal
    int32_t w, h, stride_words, boundary;
} me_load_item;

typedef struct me_load_result {
    double wall_s;             // first submit to last result
    int64_t mismatches;        // results that differed from expect
    int64_t errors;            // failed submits or polls
    int32_t first_error;       // status of the first failure (0: none)
    int32_t pad;               // zero-copy clients: bits of the XOR of what they read
} me_load_result;

// XOR of every word of a result: the client reads it once, the way an
// application consuming the edge map would (rows are whole words, so the
// byte count is a multiple of 4; the buffers are 4-byte aligned).
static uint64_t fold(const uint32_t *p, size_t bytes) {
    const size_t n = bytes / 4;
    size_t k = 0;
    uint64_t x = 0;
    if (n && ((uintptr_t)p & 7)) x ^= p[k++];
    const unsigned char *q = reinterpret_cast<const unsigned char *>(p + k);
    auto at = [q](size_t j) {
        uint64_t v;
        std::memcpy(&v, q + 8 * j, 8);
        return v;
    };
    const size_t m = (n - k) / 2;
    uint64_t a = 0, b = 0, c = 0, d = 0;
    size_t j = 0;
    for (; j + 4 <= m; j += 4) {
        a ^= at(j);
        b ^= at(j + 1);
        c ^= at(j + 2);
        d ^= at(j + 3);
    }
    for (; j < m; ++j) a ^= at(j);
    x ^= a ^ b ^ c ^ d;
    for (k += 2 * m; k < n; ++k) x ^= p[k];
    return x;
}

/*
 * Run n requests through srv.  Request i goes to client i % clients.
 * mode: 0 me_serve_submit / me_serve_poll; 1 me_serve_reserve /
 * me_serve_commit and me_serve_poll_view / me_serve_release; 2
 * me_serve_submit_direct into out_ring (slots of slot_words words, `slots`
 * per client, client c taking slots c * slots .. c * slots + slots - 1;
 * the images and the ring must be memory the GPU reaches) and me_serve_poll
 * with no buffer.  A client holds at most `slots` direct requests.
 * arrival_us: NULL for a closed loop (each client keeps up to `window`
 * requests outstanding), else the arrival time of each request in
 * microseconds from the start (open loop; window is ignored).
 * latency_us[i] (may be NULL): arrival (open) or submit (closed) to result
 * delivered; server_us[i] (may be NULL): the server's submit-to-ready time
 * (me_timing.total_us).  Returns ME_OK or ME_ERR_ARG; failures of single
 * requests are counted in *res.
 */
int me_load_run(me_server *srv, const me_load_item *items, int64_t n,
                const double *arrival_us, int32_t clients, int32_t window, int32_t mode,
                uint32_t *out_ring, int64_t slot_words, int32_t slots,
                double *latency_us, double *server_us, me_load_result *res) {
    if (srv == nullptr || items == nullptr || n <= 0 || clients < 1 || res == nullptr ||
        (arrival_us == nullptr && window < 1) || mode < 0 || mode > 2 ||
        (mode == 2 && (out_ring == nullptr || slots < 1 || slot_words < 1)))
        return ME_ERR_ARG;
    const bool zero_copy = mode == 1, direct = mode == 2;
    std::atomic<int64_t> mismatches{0}, errors{0};
    std::atomic<uint64_t> checksum{0};
    std::atomic<int32_t> first_error{0};
    auto fail = [&](int rc) {
        errors.fetch_add(1);
        int32_t z = 0;
        first_error.compare_exchange_strong(z, rc);
    };
    size_t max_bytes = 0;
    for (int64_t i = 0; i < n; ++i)
        max_bytes = std::max(max_bytes, (size_t)items[i].h * (size_t)items[i].stride_words * 4);
    if (direct && max_bytes > (size_t)slot_words * 4) return ME_ERR_ARG;   // a slot too small
    std::memset(res, 0, sizeof(*res));

    std::atomic<int> ready{0};
    std::atomic<bool> go{false};
    Clock::time_point t0;
    std::vector<Clock::time_point> t_last((size_t)clients);
    const bool open = arrival_us != nullptr;
    auto arrival = [&](int64_t i) {
        return t0 + std::chrono::nanoseconds((int64_t)(arrival_us[i] * 1e3));
    };

    std::vector<std::thread> th;
    for (int c = 0; c < clients; ++c) {
        th.emplace_back([&, c] {
            std::vector<uint32_t> scratch(max_bytes / 4 + 1);
            struct Out {
                int64_t i;
                uint64_t ticket;
                Clock::time_point from;
                uint32_t *slot;        // direct: the output slot
            };
            int64_t next_slot = 0;
            std::deque<Out> out;
            prctl(PR_SET_TIMERSLACK, 1000UL, 0, 0, 0);   // 1 us sleep precision
            ready.fetch_add(1);
            while (!go.load(std::memory_order_acquire)) std::this_thread::yield();
            Clock::time_point last = t0;
            int64_t next = c;
            // Take the oldest result; false when it is not ready within
            // timeout_us (0: not at all).
            auto collect_oldest = [&](int64_t timeout_us) {
                me_timing tm{};
                const Out o = out.front();
                const uint32_t *view = nullptr;
                const int rc = zero_copy ? me_serve_poll_view(srv, o.ticket, timeout_us, &view, &tm)
                               : direct  ? me_serve_poll(srv, o.ticket, nullptr, timeout_us, &tm)
                                         : me_serve_poll(srv, o.ticket, scratch.data(), timeout_us,
                                                         &tm);
                if (rc == ME_PENDING || rc == ME_TIMEOUT) return false;
                out.pop_front();
                if (rc != ME_OK) {
                    fail(rc);
                    if (zero_copy) me_serve_release(srv, o.ticket);
                    last = Clock::now();
                    return true;
                }
                const me_load_item &it = items[o.i];
                const size_t bytes = (size_t)it.h * (size_t)it.stride_words * 4;
                const uint32_t *got = zero_copy ? view : direct ? o.slot : scratch.data();
                if (it.expect) {
                    if (std::memcmp(got, it.expect, bytes) != 0) mismatches.fetch_add(1);
                } else if (zero_copy || direct) {
                    checksum.fetch_xor(fold(got, bytes), std::memory_order_relaxed);
                }
                if (zero_copy) me_serve_release(srv, o.ticket);
                last = Clock::now();
                if (latency_us) latency_us[o.i] = us_between(o.from, last);
                if (server_us) server_us[o.i] = tm.total_us;
                return true;
            };
            // the longest the oldest result may be waited for: until the
            // next arrival (open loop) or without limit
            auto patience = [&] {
                if (!open || next >= n) return (int64_t)-1;
                return (int64_t)std::max(0.0, us_between(Clock::now(), arrival(next)));
            };
            while (next < n || !out.empty()) {
                // whatever has finished is collected first: a client that
                // falls behind its schedule must not leave results holding
                // staging while it submits
                if (!out.empty() && collect_oldest(0)) continue;
                const auto now = Clock::now();
                // a direct client also needs a free output slot
                const bool due = next < n && (open ? arrival(next) <= now
                                                   : (int)out.size() < window) &&
                                 (!direct || (int)out.size() < slots);
                if (due) {
                    const me_load_item &it = items[next];
                    const auto from = open ? arrival(next) : Clock::now();
                    uint64_t tk = 0;
                    int rc;
                    uint32_t *slot = nullptr;
                    if (direct) {
                        slot = out_ring + ((int64_t)c * slots + next_slot % slots) * slot_words;
                        ++next_slot;
                        rc = me_serve_submit_direct(srv, it.img, slot, it.w, it.h,
                                                    it.stride_words, it.boundary, &tk);
                    } else if (zero_copy) {
                        uint32_t *dst = nullptr;
                        rc = me_serve_reserve(srv, it.w, it.h, it.stride_words, it.boundary,
                                              &tk, &dst);
                        if (rc == ME_PENDING) {
                            // no staging now: wait for the oldest result
                            if (!out.empty()) collect_oldest(-1);
                            else std::this_thread::yield();
                            continue;
                        }
                        if (rc == ME_OK) {
                            std::memcpy(dst, it.img, (size_t)it.h * (size_t)it.stride_words * 4);
                            rc = me_serve_commit(srv, tk);
                        }
                    } else {
                        rc = me_serve_submit(srv, it.img, it.w, it.h, it.stride_words,
                                             it.boundary, &tk);
                    }
                    if (rc == ME_OK) out.push_back({next, tk, from, slot}); else fail(rc);
                    next += clients;
                    continue;
                }
                if (out.empty()) {                       // open loop, idle
                    wait_until(arrival(next));
                    continue;
                }
                // every output slot taken: the oldest result frees one
                collect_oldest(direct && (int)out.size() >= slots ? -1 : patience());
            }
            t_last[c] = last;
        });
    }
    while (ready.load() < (int)th.size()) std::this_thread::yield();
    t0 = Clock::now();
    go.store(true, std::memory_order_release);
    for (auto &t : th) t.join();
    Clock::time_point end = t0;
    for (auto &t : t_last) end = std::max(end, t);
    res->wall_s = us_between(t0, end) * 1e-6;
    res->mismatches = mismatches.load();
    res->errors = errors.load();
    res->first_error = first_error.load();
    res->pad = (int32_t)(checksum.load() & 0x7fffffff);
    return ME_OK;
}

}  // extern "C"
