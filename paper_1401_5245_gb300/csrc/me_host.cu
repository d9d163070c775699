// me_edges_batch_host: a ragged batch in host memory, end to end.
//
// Images are grouped into chunks in order and every chunk's batch plan is
// uploaded up front in one small copy.  Chunk k then goes to device slot
// k % kSlots: one host-to-device copy of the chunk's input span (stream `up`),
// one persistent batch launch over it (stream `comp`), and one device-to-
// host copy per run of adjacent images (stream `down`).  Events chain the
// three streams, so the upload of chunk k+1 and the download of chunk k-1
// overlap the kernel of chunk k; a slot is refilled only after its previous
// download finished.  Copies start at host page boundaries wherever the
// caller's buffers allow, and the slots mirror the host addresses modulo the
// page size.
#include <algorithm>
#include <memory>
#include <mutex>
#include <vector>

#include "me_internal.h"

namespace me {

namespace {

// Three slots: while chunk k computes, chunk k-1 can still be downloading
// and chunk k+1 already uploading, each in its own slot.
constexpr int kSlots = 3;
// 16 MiB chunks measured fastest on the 4096-image batch (2.042 ms against
// 2.055-2.080 ms for 12, 20, 24 and 32 MiB, 2.12-2.20 ms for 6-8 MiB).
constexpr int64_t kDefaultChunk = 16ll << 20;
// Host-to-device and device-to-host copies ran about 20% slower on GB300
// from host addresses off a page boundary: a 298 MB upload/compute/download
// pipeline in 32 MiB chunks took 1.97 ms from page-aligned host addresses
// and 2.44 ms from addresses 16 bytes past them.
constexpr uintptr_t kHostPage = 4096;

struct HostPipe {
    std::mutex mu;
    cudaStream_t up = nullptr, comp = nullptr, down = nullptr;
    cudaEvent_t start = nullptr, plans_done = nullptr;
    cudaEvent_t up_done[kSlots] = {}, comp_done[kSlots] = {}, down_done[kSlots] = {};
    char *slot[kSlots] = {};           // input half [0, cap), output half [cap, 2 cap)
    size_t cap = 0;
    char *plan_host = nullptr;         // pinned: every chunk's batch plan
    char *plan_dev = nullptr;
    size_t plan_cap = 0;
    bool ready = false;

    int reserve_plans(size_t bytes) {
        if (plan_cap >= bytes) return ME_OK;
        if (plan_host) cudaFreeHost(plan_host);
        if (plan_dev) cudaFree(plan_dev);
        plan_host = plan_dev = nullptr;
        plan_cap = 0;
        size_t c = 64 * 1024;
        while (c < bytes) c <<= 1;
        cudaError_t e = cudaHostAlloc((void **)&plan_host, c, cudaHostAllocDefault);
        if (e == cudaSuccess) e = cudaMalloc((void **)&plan_dev, c);
        if (e != cudaSuccess) {
            cudaGetLastError();
            if (plan_host) cudaFreeHost(plan_host);
            plan_host = nullptr;
            plan_dev = nullptr;
            return record_cuda(e);
        }
        plan_cap = c;
        return ME_OK;
    }

    int init() {
        if (ready) return ME_OK;
        cudaError_t e = cudaSuccess;
        for (cudaStream_t *s : {&up, &comp, &down})
            if (e == cudaSuccess) e = cudaStreamCreateWithFlags(s, cudaStreamNonBlocking);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&start, cudaEventDisableTiming);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&plans_done, cudaEventDisableTiming);
        for (int s = 0; s < kSlots && e == cudaSuccess; ++s) {
            e = cudaEventCreateWithFlags(&up_done[s], cudaEventDisableTiming);
            if (e == cudaSuccess) e = cudaEventCreateWithFlags(&comp_done[s], cudaEventDisableTiming);
            if (e == cudaSuccess) e = cudaEventCreateWithFlags(&down_done[s], cudaEventDisableTiming);
        }
        if (e != cudaSuccess) {
            cudaGetLastError();
            return record_cuda(e);
        }
        ready = true;
        return ME_OK;
    }
    int reserve(size_t span) {
        if (cap >= span) return ME_OK;
        if (down) cudaStreamSynchronize(down);
        for (int s = 0; s < kSlots; ++s) {
            if (slot[s]) cudaFree(slot[s]);
            slot[s] = nullptr;
        }
        cap = 0;
        const size_t c = (span + 255) / 256 * 256;
        for (int s = 0; s < kSlots; ++s) {
            cudaError_t e = cudaMalloc(&slot[s], 2 * c);
            if (e != cudaSuccess) {
                cudaGetLastError();
                return record_cuda(e);
            }
        }
        cap = c;
        return ME_OK;
    }
    void release() {
        if (down) cudaStreamSynchronize(down);
        if (plan_host) cudaFreeHost(plan_host);
        if (plan_dev) cudaFree(plan_dev);
        for (int s = 0; s < kSlots; ++s) {
            if (slot[s]) cudaFree(slot[s]);
            for (cudaEvent_t ev : {up_done[s], comp_done[s], down_done[s]})
                if (ev) cudaEventDestroy(ev);
        }
        if (start) cudaEventDestroy(start);
        if (plans_done) cudaEventDestroy(plans_done);
        for (cudaStream_t s : {up, comp, down})
            if (s) cudaStreamDestroy(s);
    }
};

std::mutex g_pipes_mu;
HostPipe *g_pipes[64] = {};

HostPipe *pipe_for(int dev) {
    std::lock_guard<std::mutex> lk(g_pipes_mu);
    if (!g_pipes[dev]) g_pipes[dev] = new HostPipe();
    return g_pipes[dev];
}

struct Chunk {
    int first, count;       // images [first, first + count)
    int64_t lo, hi;         // input span in words, lo a multiple of 4
    // host page at or below the span's first input / output byte; a host
    // address a of the chunk lives at slot offset a - base
    uintptr_t in_base, out_base;
};

// A host<->device copy issued as the bytes before the first host page
// boundary, then the rest from that boundary.
cudaError_t copy_paged(void *dst, const void *src, size_t bytes, cudaMemcpyKind kind,
                       cudaStream_t s) {
    const uintptr_t h = kind == cudaMemcpyHostToDevice ? (uintptr_t)src : (uintptr_t)dst;
    const size_t head = std::min(bytes, (size_t)((kHostPage - h % kHostPage) % kHostPage));
    cudaError_t e = cudaSuccess;
    if (head > 0) e = cudaMemcpyAsync(dst, src, head, kind, s);
    if (e == cudaSuccess && bytes > head)
        e = cudaMemcpyAsync(static_cast<char *>(dst) + head,
                            static_cast<const char *>(src) + head, bytes - head, kind, s);
    return e;
}

int fail(cudaError_t e) {
    cudaGetLastError();
    return record_cuda(e);
}

// After a failure part way through: let what was enqueued finish, so the
// call never returns with its copies still reading or writing host memory.
int fail_drain(HostPipe *p, int rc) {
    for (cudaStream_t s : {p->up, p->comp, p->down})
        if (s) cudaStreamSynchronize(s);
    cudaGetLastError();
    return rc;
}

}  // namespace

int host_pipes_shutdown() {
    int cur = 0;
    cudaGetDevice(&cur);
    std::lock_guard<std::mutex> lk(g_pipes_mu);
    for (int d = 0; d < 64; ++d) {
        if (!g_pipes[d]) continue;
        cudaSetDevice(d);
        g_pipes[d]->release();
        delete g_pipes[d];
        g_pipes[d] = nullptr;
    }
    cudaSetDevice(cur);
    return ME_OK;
}

}  // namespace me

using namespace me;

extern "C" int me_edges_batch_host(const uint32_t *host_in, uint32_t *host_out,
                                   const me_host_image *imgs, int32_t n, int64_t chunk_bytes,
                                   me_stream_t stream) {
    if (n < 0 || (n > 0 && (imgs == nullptr || host_in == nullptr || host_out == nullptr)) ||
        chunk_bytes < 0)
        return ME_ERR_ARG;
    if (n == 0) return ME_OK;
    if (chunk_bytes == 0) chunk_bytes = kDefaultChunk;
    // arguments, and the extent of the batch in both buffers
    int64_t extent = 0;
    for (int i = 0; i < n; ++i) {
        const me_host_image &m = imgs[i];
        if (m.offset_words < 0 || m.w <= 0 || m.h <= 0 ||
            m.stride_words < (int32_t)(((int64_t)m.w + 31) / 32) ||
            (m.boundary != ME_BOUNDARY_WHITE && m.boundary != ME_BOUNDARY_BLACK))
            return ME_ERR_ARG;
        extent = std::max<int64_t>(extent, m.offset_words + (int64_t)m.h * m.stride_words);
    }
    if (ranges_overlap(host_in, (size_t)extent * 4, host_out, (size_t)extent * 4))
        return ME_ERR_ALIAS;

    // chunks of consecutive images whose input span stays within chunk_bytes
    std::vector<Chunk> chunks;
    int64_t max_span = 0;
    for (int i = 0; i < n;) {
        Chunk c{i, 0, 0, 0, 0, 0};
        c.lo = imgs[i].offset_words & ~int64_t(3);
        c.hi = imgs[i].offset_words + (int64_t)imgs[i].h * imgs[i].stride_words;
        c.count = 1;
        int j = i + 1;
        for (; j < n; ++j) {
            const int64_t lo = std::min(c.lo, imgs[j].offset_words & ~int64_t(3));
            const int64_t hi =
                std::max(c.hi, imgs[j].offset_words + (int64_t)imgs[j].h * imgs[j].stride_words);
            if ((hi - lo) * 4 > chunk_bytes) break;
            c.lo = lo;
            c.hi = hi;
            ++c.count;
        }
        max_span = std::max(max_span, c.hi - c.lo);
        c.in_base = (uintptr_t)(host_in + c.lo) & ~(kHostPage - 1);
        c.out_base = (uintptr_t)(host_out + c.lo) & ~(kHostPage - 1);
        chunks.push_back(c);
        i = j;
    }

    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return fail(e);
    if (dev < 0 || dev >= 64) return ME_ERR_UNSUPPORTED;
    HostPipe *p = pipe_for(dev);
    std::lock_guard<std::mutex> lk(p->mu);
    int rc = p->init();
    if (rc != ME_OK) return rc;
    if ((rc = p->reserve((size_t)max_span * 4 + kHostPage)) != ME_OK) return rc;

    // Start chunk 0's upload, then plan every chunk's batch while it runs and
    // upload all the plans in one small copy: a plan copied per chunk would
    // queue on the copy engine behind the next chunk's upload and hold its
    // kernel back.
    auto upload = [&](size_t k) -> cudaError_t {
        const Chunk &c = chunks[k];
        const int s = (int)(k % kSlots);
        cudaError_t r = cudaSuccess;
        if (k >= (size_t)kSlots) r = cudaStreamWaitEvent(p->up, p->down_done[s], 0);
        // from the page boundary below the span, where that is still inside
        // the caller's input buffer (the extra bytes are only read)
        const uintptr_t from = std::max(c.in_base, (uintptr_t)host_in);
        const uintptr_t to = (uintptr_t)(host_in + c.hi);
        if (r == cudaSuccess)
            r = copy_paged(p->slot[s] + (from - c.in_base), reinterpret_cast<const void *>(from),
                           to - from, cudaMemcpyHostToDevice, p->up);
        if (r == cudaSuccess) r = cudaEventRecord(p->up_done[s], p->up);
        return r;
    };
    if ((e = cudaEventRecord(p->start, (cudaStream_t)stream)) != cudaSuccess) return fail(e);
    if ((e = cudaStreamWaitEvent(p->up, p->start, 0)) != cudaSuccess) return fail_drain(p, fail(e));
    if ((e = upload(0)) != cudaSuccess) return fail_drain(p, fail(e));

    std::vector<BatchSetup> setups(chunks.size());
    std::vector<size_t> arena_at(chunks.size());
    std::vector<me_desc> descs((size_t)n);     // device-side view of every image
    size_t plans = 0;
    for (size_t k = 0; k < chunks.size(); ++k) {
        const Chunk &c = chunks[k];
        char *din = p->slot[k % kSlots], *dout = p->slot[k % kSlots] + p->cap;
        for (int i = c.first; i < c.first + c.count; ++i) {
            const me_host_image &m = imgs[i];
            const size_t at_in = (uintptr_t)(host_in + m.offset_words) - c.in_base;
            const size_t at_out = (uintptr_t)(host_out + m.offset_words) - c.out_base;
            descs[i] = {reinterpret_cast<const uint32_t *>(din + at_in),
                        reinterpret_cast<uint32_t *>(dout + at_out), m.w, m.h, m.stride_words,
                        m.boundary};
        }
        if ((rc = setup_batch(&descs[c.first], c.count, batch_cfg(&descs[c.first], c.count),
                              &setups[k])) != ME_OK)
            return fail_drain(p, rc);
        arena_at[k] = plans;
        plans += (setups[k].arena + 255) / 256 * 256;
    }
    if ((rc = p->reserve_plans(plans)) != ME_OK) return fail_drain(p, rc);
    for (size_t k = 0; k < chunks.size(); ++k)
        if ((rc = fill_arena(&descs[chunks[k].first], chunks[k].count, setups[k],
                             p->plan_host + arena_at[k])) != ME_OK)
            return fail_drain(p, rc);
    if ((e = cudaMemcpyAsync(p->plan_dev, p->plan_host, plans, cudaMemcpyHostToDevice, p->up)) !=
        cudaSuccess)
        return fail_drain(p, fail(e));
    if ((e = cudaEventRecord(p->plans_done, p->up)) != cudaSuccess) return fail_drain(p, fail(e));
    if ((e = cudaStreamWaitEvent(p->comp, p->plans_done, 0)) != cudaSuccess)
        return fail_drain(p, fail(e));

    for (size_t k = 0; k < chunks.size(); ++k) {
        const Chunk &c = chunks[k];
        const int s = (int)(k % kSlots);
        char *dout = p->slot[s] + p->cap;
        if (k > 0 && (e = upload(k)) != cudaSuccess) return fail_drain(p, fail(e));
        if ((e = cudaStreamWaitEvent(p->comp, p->up_done[s], 0)) != cudaSuccess) return fail_drain(p, fail(e));
        // a plain launch: an event wait stands before every chunk's kernel
        if ((e = launch_planned(setups[k], p->plan_dev + arena_at[k], p->comp, false)) !=
            cudaSuccess)
            return fail_drain(p, fail(e));
        if ((e = cudaEventRecord(p->comp_done[s], p->comp)) != cudaSuccess) return fail_drain(p, fail(e));
        if ((e = cudaStreamWaitEvent(p->down, p->comp_done[s], 0)) != cudaSuccess) return fail_drain(p, fail(e));
        // one download per run of images that follow each other without gaps
        int i = c.first;
        while (i < c.first + c.count) {
            const int64_t r0 = imgs[i].offset_words;
            int64_t r1 = r0 + (int64_t)imgs[i].h * imgs[i].stride_words;
            int j = i + 1;
            while (j < c.first + c.count && imgs[j].offset_words == r1) {
                r1 += (int64_t)imgs[j].h * imgs[j].stride_words;
                ++j;
            }
            if ((e = copy_paged(host_out + r0, dout + ((uintptr_t)(host_out + r0) - c.out_base),
                                (size_t)(r1 - r0) * 4, cudaMemcpyDeviceToHost, p->down)) !=
                cudaSuccess)
                return fail_drain(p, fail(e));
            i = j;
        }
        if ((e = cudaEventRecord(p->down_done[s], p->down)) != cudaSuccess) return fail_drain(p, fail(e));
    }
    if ((e = cudaStreamSynchronize(p->down)) != cudaSuccess) return fail_drain(p, fail(e));
    return ME_OK;
}
