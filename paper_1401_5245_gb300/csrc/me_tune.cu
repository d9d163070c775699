// Autotuner: times candidate tile configurations on the caller's images
// with CUDA events and keeps the fastest.  Optional cache file named by
// ME_TUNE_CACHE, one line per (device name, kind):
//     <device name>|<kind>|<engine> <rows> <vec> <threads> <ctas_per_sm> <stage_kb> <stages> <chunk>
#include <algorithm>
#include <atomic>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <fstream>
#include <mutex>
#include <sstream>
#include <string>
#include <vector>

#include "me_internal.h"

namespace me {

namespace {

std::vector<me_tile_cfg> candidates(int kind) {
    std::vector<me_tile_cfg> out;
    const int threads[] = {128, 256, 512};
    if (kind == ME_KIND_SINGLE) {
        for (int r : {4, 8, 16, 32})
            for (int t : threads)
                for (int c : {0, 2, 4, 8}) out.push_back({ME_ENGINE_REGS, r, 4, t, c, 32, 4, 0});
    } else {
        // rows per lane x CTA size x persistence x tiles per chunk
        for (int r : {4, 8, 16})
            for (int t : threads)
                for (int c : {0, 1, 2, 4, 8})
                    for (int ch : {2, 4, 8})
                        out.push_back({ME_ENGINE_REGS, r, 4, t, c, 32, 4, ch});
    }
    // bulk engine: stage size x ring depth x CTA size, as many CTAs as fit
    for (int kb : {8, 16, 32, 48, 64})
        for (int st : {2, 3, 4, 6})
            for (int t : {256, 512})
                if (kb * st <= 216) out.push_back({ME_ENGINE_BULK, 8, 4, t, 0, kb, st, 0});
    return out;
}

std::string key_of(const DevInfo &di, int kind) {
    return std::string(di.name) + "|" + std::to_string(kind);
}

bool read_cache(const char *path, const std::string &key, me_tile_cfg *out) {
    std::ifstream f(path);
    std::string line;
    bool found = false;
    while (std::getline(f, line)) {
        const size_t bar = line.rfind('|');
        if (bar == std::string::npos || line.substr(0, bar) != key) continue;
        std::istringstream is(line.substr(bar + 1));
        me_tile_cfg c;
        if (is >> c.engine >> c.rows_per_lane >> c.vec_words >> c.cta_threads >> c.ctas_per_sm >>
                c.stage_kb >> c.stages >> c.chunk_tiles &&
            valid_cfg(c)) {
            *out = c;
            found = true;
        }
    }
    return found;
}

void write_cache(const char *path, const std::string &key, const me_tile_cfg &c) {
    std::vector<std::string> keep;
    {
        std::ifstream f(path);
        std::string line;
        while (std::getline(f, line)) {
            const size_t bar = line.rfind('|');
            if (bar != std::string::npos && line.substr(0, bar) == key) continue;
            if (!line.empty()) keep.push_back(line);
        }
    }
    std::ofstream f(path, std::ios::trunc);
    for (auto &l : keep) f << l << "\n";
    f << key << "|" << c.engine << " " << c.rows_per_lane << " " << c.vec_words << " "
      << c.cta_threads << " " << c.ctas_per_sm << " " << c.stage_kb << " " << c.stages << " "
      << c.chunk_tiles << "\n";
}

int run_once(int kind, const me_desc *s, int n, cudaStream_t st) {
    if (kind != ME_KIND_SINGLE) return me_edges_batch(s, n, (me_stream_t)st);
    for (int i = 0; i < n; ++i) {
        int rc = me_edges(s[i].img, s[i].w, s[i].h, s[i].stride_words, s[i].edge,
                          s[i].boundary, (me_stream_t)st);
        if (rc != ME_OK) return rc;
    }
    return ME_OK;
}

}  // namespace

// Apply a cached choice for this device once per process and kind.
void apply_tune_cache(int kind) {
    static std::mutex mu;
    static std::atomic<bool> done[3] = {false, false, false};
    const int k = kind == ME_KIND_BATCH || kind == ME_KIND_BATCH_ANY ? kind : ME_KIND_SINGLE;
    if (done[k].load(std::memory_order_acquire)) return;
    std::lock_guard<std::mutex> lk(mu);
    if (done[k].load(std::memory_order_relaxed)) return;
    done[k].store(true, std::memory_order_release);
    const char *path = std::getenv("ME_TUNE_CACHE");
    if (!path || !*path) return;
    DevInfo di;
    if (device_info(&di) != ME_OK) return;
    me_tile_cfg c;
    if (read_cache(path, key_of(di, kind), &c)) me_set_tile_cfg(kind, &c);
}

}  // namespace me

using namespace me;

extern "C" int me_autotune(int32_t kind, const me_desc *sample, int32_t n, int32_t reps,
                           me_stream_t stream, me_tile_cfg *best) {
    if ((kind != ME_KIND_SINGLE && kind != ME_KIND_BATCH && kind != ME_KIND_BATCH_ANY) ||
        sample == nullptr || n <= 0 || reps <= 0 || best == nullptr)
        return ME_ERR_ARG;
    // the sample's launches take the configuration of its own batch kind
    if (kind != ME_KIND_SINGLE && batch_any(sample, n) != (kind == ME_KIND_BATCH_ANY))
        return ME_ERR_ARG;
    DevInfo di;
    int rc = device_info(&di);
    if (rc != ME_OK) return rc;
    const cudaStream_t st = (cudaStream_t)stream;
    const me_tile_cfg saved = tile_cfg(kind);
    cudaEvent_t a = nullptr, b = nullptr;
    cudaError_t e = cudaEventCreate(&a);
    if (e == cudaSuccess) e = cudaEventCreate(&b);
    if (e != cudaSuccess) {
        if (a) cudaEventDestroy(a);
        return record_cuda(e);
    }
    float best_ms = 1e30f;
    me_tile_cfg best_cfg = saved;
    for (const me_tile_cfg &c : candidates(kind)) {
        if (me_set_tile_cfg(kind, &c) != ME_OK) continue;   // engine not available
        // warm-up (also builds the graphs of this configuration)
        if (run_once(kind, sample, n, st) != ME_OK || run_once(kind, sample, n, st) != ME_OK) {
            cudaGetLastError();
            continue;
        }
        // steady-state throughput: `reps` calls back to back between two
        // events (host planning overlaps the GPU as it does in a stream of
        // batches), best of three such runs
        float best_run = 1e30f;
        bool ok = true;
        for (int run = 0; run < 3 && ok; ++run) {
            cudaEventRecord(a, st);
            for (int r = 0; r < reps && ok; ++r) ok = run_once(kind, sample, n, st) == ME_OK;
            cudaEventRecord(b, st);
            cudaEventSynchronize(b);
            float ms = 0;
            cudaEventElapsedTime(&ms, a, b);
            best_run = std::min(best_run, ms / reps);
        }
        if (!ok) {
            cudaGetLastError();
            continue;
        }
        if (best_run < best_ms) {
            best_ms = best_run;
            best_cfg = c;
        }
    }
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    me_set_tile_cfg(kind, &best_cfg);
    *best = best_cfg;
    const char *path = std::getenv("ME_TUNE_CACHE");
    if (path && *path) write_cache(path, key_of(di, kind), best_cfg);
    return best_ms < 1e30f ? ME_OK : ME_ERR_CUDA;
}
