// me_edges_batch and batch plans: many images in one persistent launch,
// replayed from CUDA graphs.
//
// A call plans the batch on the host (descriptors, tile ranges per warp),
// writes the plan into a pinned staging slot and launches that slot's
// graph: one memcpy node (staging -> device arena) and one kernel node (the
// persistent batch kernel reading the arena).  Slots form a ring of
// kRing per device; a slot is reused only after the event recorded behind
// its last launch has completed, so in-flight graphs never see their
// staging or arena overwritten.  Graphs are cached per slot and keyed by the
// tile configuration and grid; the memcpy node's size is set per launch.
#include <algorithm>
#include <cstring>
#include <memory>
#include <mutex>
#include <unordered_map>
#include <vector>

#include "me_internal.h"

namespace me {

namespace {

constexpr int kRing = 4;
constexpr size_t kMinSlot = 64 * 1024;

struct GraphEntry {
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    cudaGraphNode_t copy = nullptr;
};

struct Slot {
    size_t cap = 0;
    void *host = nullptr;
    void *dev = nullptr;
    cudaEvent_t done = nullptr;
    bool pending = false;
    std::unordered_map<uint64_t, GraphEntry> graphs;

    void drop_graphs() {
        for (auto &kv : graphs) {
            if (kv.second.exec) cudaGraphExecDestroy(kv.second.exec);
            if (kv.second.graph) cudaGraphDestroy(kv.second.graph);
        }
        graphs.clear();
    }
    void release() {
        if (pending && done) cudaEventSynchronize(done);
        pending = false;
        drop_graphs();
        if (host) cudaFreeHost(host);
        if (dev) cudaFree(dev);
        if (done) cudaEventDestroy(done);
        host = dev = nullptr;
        done = nullptr;
        cap = 0;
    }
};

struct DevBatch {
    std::mutex mu;
    Slot slots[kRing];
    int next = 0;
};

std::mutex g_devs_mu;
DevBatch *g_devs[64] = {};

DevBatch *dev_state(int dev) {
    std::lock_guard<std::mutex> lk(g_devs_mu);
    if (!g_devs[dev]) g_devs[dev] = new DevBatch();
    return g_devs[dev];
}

size_t round_pow2(size_t v) {
    size_t c = kMinSlot;
    while (c < v) c <<= 1;
    return c;
}

// Graph: copy `cap` bytes host -> arena, then the persistent kernel.
cudaError_t build_graph(const void *host, void *dev, size_t bytes, int grid,
                        int threads, int rpt, GraphEntry *out) {
    cudaGraph_t g = nullptr;
    cudaError_t e = cudaGraphCreate(&g, 0);
    if (e != cudaSuccess) return e;
    cudaGraphNode_t copy = nullptr, kern = nullptr;
    e = cudaGraphAddMemcpyNode1D(&copy, g, nullptr, 0, dev, host, bytes,
                                 cudaMemcpyHostToDevice);
    if (e == cudaSuccess) {
        cudaKernelNodeParams kp = {};
        void *arena = dev;
        void *args[] = {&arena};
        kp.func = const_cast<void *>(batch_kernel(rpt));
        kp.gridDim = dim3(grid);
        kp.blockDim = dim3(threads);
        kp.sharedMemBytes = 0;
        kp.kernelParams = args;
        e = cudaGraphAddKernelNode(&kern, g, &copy, 1, &kp);
    }
    cudaGraphExec_t exec = nullptr;
    if (e == cudaSuccess) e = cudaGraphInstantiate(&exec, g, 0);
    if (e != cudaSuccess) {
        cudaGraphDestroy(g);
        return e;
    }
    out->graph = g;
    out->exec = exec;
    out->copy = copy;
    return cudaSuccess;
}

int fail(cudaError_t e) {
    cudaGetLastError();
    return record_cuda(e);
}

}  // namespace

int batch_shutdown_all() {
    int cur = 0;
    cudaGetDevice(&cur);
    std::lock_guard<std::mutex> lk(g_devs_mu);
    for (int d = 0; d < 64; ++d) {
        if (!g_devs[d]) continue;
        cudaSetDevice(d);
        {
            std::lock_guard<std::mutex> lk2(g_devs[d]->mu);
            for (auto &s : g_devs[d]->slots) s.release();
        }
        delete g_devs[d];
        g_devs[d] = nullptr;
    }
    cudaSetDevice(cur);
    return ME_OK;
}

}  // namespace me

using namespace me;

struct me_batch_plan {
    int device = 0;
    void *dev = nullptr;
    size_t bytes = 0;
    int64_t algo_bytes = 0;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
};

extern "C" {

int me_edges_batch(const me_desc *descs, int32_t n, me_stream_t stream) {
    if (n < 0 || (n > 0 && descs == nullptr)) return ME_ERR_ARG;
    if (n == 0) return ME_OK;
    me_tile_cfg cfg = tile_cfg(ME_KIND_BATCH);
    if (cfg.ctas_per_sm <= 0) cfg.ctas_per_sm = 4;
    int64_t tasks = 0;
    int rc = batch_tasks(descs, n, cfg, &tasks);
    if (rc != ME_OK) return rc;
    DevInfo di;
    if ((rc = device_info(&di)) != ME_OK) return rc;
    int grid = 0, threads = 0;
    batch_grid(cfg, di, (int)tasks, &grid, &threads);
    const int total_warps = grid * (threads / 32);
    const size_t need = arena_bytes(n, total_warps);

    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return fail(e);
    DevBatch *st = dev_state(dev);
    std::lock_guard<std::mutex> lk(st->mu);
    Slot &slot = st->slots[st->next];
    st->next = (st->next + 1) % kRing;
    if (slot.pending) {
        e = cudaEventSynchronize(slot.done);
        if (e != cudaSuccess) return fail(e);
        slot.pending = false;
    }
    if (slot.cap < need) {
        slot.release();
        const size_t cap = round_pow2(need);
        if ((e = cudaHostAlloc(&slot.host, cap, cudaHostAllocDefault)) != cudaSuccess) {
            slot.host = nullptr;
            return fail(e);
        }
        if ((e = cudaMalloc(&slot.dev, cap)) != cudaSuccess) {
            slot.dev = nullptr;
            slot.release();
            return fail(e);
        }
        if ((e = cudaEventCreateWithFlags(&slot.done, cudaEventDisableTiming)) != cudaSuccess) {
            slot.done = nullptr;
            slot.release();
            return fail(e);
        }
        slot.cap = cap;
    }
    int bad = -1;
    if ((rc = plan_batch(descs, n, cfg, total_warps, slot.host, &bad)) != ME_OK) return rc;

    const uint64_t key = cfg_key(cfg) ^ ((uint64_t)grid << 44);
    auto it = slot.graphs.find(key);
    if (it == slot.graphs.end()) {
        GraphEntry ge;
        if ((e = build_graph(slot.host, slot.dev, slot.cap, grid, threads,
                             cfg.rows_per_lane, &ge)) != cudaSuccess)
            return fail(e);
        it = slot.graphs.emplace(key, ge).first;
    }
    // copy only what this batch filled
    e = cudaGraphExecMemcpyNodeSetParams1D(it->second.exec, it->second.copy, slot.dev,
                                           slot.host, need, cudaMemcpyHostToDevice);
    if (e != cudaSuccess) return fail(e);
    if ((e = cudaGraphLaunch(it->second.exec, (cudaStream_t)stream)) != cudaSuccess)
        return fail(e);
    if ((e = cudaEventRecord(slot.done, (cudaStream_t)stream)) != cudaSuccess) return fail(e);
    slot.pending = true;
    return ME_OK;
}

int me_batch_plan_create(const me_desc *descs, int32_t n, me_stream_t stream,
                         me_batch_plan **out) {
    if (out == nullptr || n <= 0 || descs == nullptr) return ME_ERR_ARG;
    *out = nullptr;
    me_tile_cfg cfg = tile_cfg(ME_KIND_BATCH);
    if (cfg.ctas_per_sm <= 0) cfg.ctas_per_sm = 4;
    int64_t tasks = 0;
    int rc = batch_tasks(descs, n, cfg, &tasks);
    if (rc != ME_OK) return rc;
    DevInfo di;
    if ((rc = device_info(&di)) != ME_OK) return rc;
    int grid = 0, threads = 0;
    batch_grid(cfg, di, (int)tasks, &grid, &threads);
    const int total_warps = grid * (threads / 32);
    const size_t need = arena_bytes(n, total_warps);
    std::vector<unsigned char> host;
    try {
        host.resize(need);
    } catch (...) {
        return ME_ERR_NOMEM;
    }
    if ((rc = plan_batch(descs, n, cfg, total_warps, host.data(), nullptr)) != ME_OK) return rc;

    std::unique_ptr<me_batch_plan> p(new (std::nothrow) me_batch_plan());
    if (!p) return ME_ERR_NOMEM;
    cudaError_t e = cudaGetDevice(&p->device);
    if (e != cudaSuccess) return fail(e);
    if ((e = cudaMalloc(&p->dev, need)) != cudaSuccess) return fail(e);
    p->bytes = need;
    p->algo_bytes = reinterpret_cast<BatchHeader *>(host.data())->bytes;
    e = cudaMemcpyAsync(p->dev, host.data(), need, cudaMemcpyHostToDevice,
                        (cudaStream_t)stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize((cudaStream_t)stream);
    if (e == cudaSuccess) e = cudaGraphCreate(&p->graph, 0);
    if (e == cudaSuccess) {
        cudaKernelNodeParams kp = {};
        void *arena = p->dev;
        void *args[] = {&arena};
        kp.func = const_cast<void *>(batch_kernel(cfg.rows_per_lane));
        kp.gridDim = dim3(grid);
        kp.blockDim = dim3(threads);
        kp.kernelParams = args;
        cudaGraphNode_t node;
        e = cudaGraphAddKernelNode(&node, p->graph, nullptr, 0, &kp);
    }
    if (e == cudaSuccess) e = cudaGraphInstantiate(&p->exec, p->graph, 0);
    if (e != cudaSuccess) {
        me_batch_plan_destroy(p.release());
        return fail(e);
    }
    *out = p.release();
    return ME_OK;
}

int me_batch_run(me_batch_plan *plan, me_stream_t stream) {
    if (plan == nullptr || plan->exec == nullptr) return ME_ERR_ARG;
    cudaError_t e = cudaGraphLaunch(plan->exec, (cudaStream_t)stream);
    return e == cudaSuccess ? ME_OK : fail(e);
}

int64_t me_batch_plan_bytes(const me_batch_plan *plan) {
    return plan ? plan->algo_bytes : 0;
}

int me_batch_plan_destroy(me_batch_plan *plan) {
    if (plan == nullptr) return ME_OK;
    cudaDeviceSynchronize();
    if (plan->exec) cudaGraphExecDestroy(plan->exec);
    if (plan->graph) cudaGraphDestroy(plan->graph);
    if (plan->dev) cudaFree(plan->dev);
    delete plan;
    return ME_OK;
}

}  // extern "C"

extern "C" int me_shutdown(void) { return me::batch_shutdown_all(); }
