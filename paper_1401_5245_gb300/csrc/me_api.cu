// C ABI of libme: argument checks, device facts, tile configurations and
// the single-image entry points.  Every compute step runs in the kernels of
// me_window.cu, me_bulk.cu and me_staged.cu.
#include <algorithm>
#include <cstdio>
#include <cstring>
#include <mutex>

#include "me_internal.h"

namespace me {

static thread_local int t_last_cuda = 0;

int record_cuda(cudaError_t e) {
    t_last_cuda = (int)e;
    return ME_ERR_CUDA;
}

int check_device_ptr(const void *p) {
    cudaPointerAttributes a;
    cudaError_t e = cudaPointerGetAttributes(&a, p);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return record_cuda(e);
    }
    if (a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged) return ME_OK;
    return ME_ERR_ARG;
}

int device_info(DevInfo *out) {
    static std::mutex mu;
    static DevInfo cache[64];
    static bool have[64] = {};
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return record_cuda(e);
    if (dev < 0 || dev >= 64) return ME_ERR_UNSUPPORTED;
    std::lock_guard<std::mutex> lk(mu);
    if (!have[dev]) {
        cudaDeviceProp p;
        e = cudaGetDeviceProperties(&p, dev);
        if (e != cudaSuccess) return record_cuda(e);
        DevInfo &d = cache[dev];
        d.sm_count = p.multiProcessorCount;
        d.max_threads_per_sm = p.maxThreadsPerMultiProcessor;
        d.cc_major = p.major;
        d.cc_minor = p.minor;
        std::snprintf(d.name, sizeof(d.name), "%s", p.name);
        have[dev] = true;
    }
    *out = cache[dev];
    return ME_OK;
}

int ceil_log2(int v) {
    int l = 0;
    while ((1 << l) < v) ++l;
    return l;
}

// ------------------------------------------------------------ tile configs
static std::mutex g_cfg_mu;
static me_tile_cfg g_cfg[3] = {
    {ME_ENGINE_REGS, 4, 4, 128, 0, 32, 4, 0},     // single image
    {ME_ENGINE_REGS, 4, 4, 512, 8, 32, 4, 4},     // batch, 128-bit accesses throughout
    {ME_ENGINE_REGS, 4, 4, 128, 0, 32, 4, 4},     // batch with narrower accesses
};

static bool valid_kind(int kind) {
    return kind == ME_KIND_SINGLE || kind == ME_KIND_BATCH || kind == ME_KIND_BATCH_ANY;
}

void apply_tune_cache(int kind);

me_tile_cfg tile_cfg(int kind) {
    apply_tune_cache(kind);
    std::lock_guard<std::mutex> lk(g_cfg_mu);
    return g_cfg[valid_kind(kind) ? kind : ME_KIND_SINGLE];
}

bool batch_any(const me_desc *descs, int n) {
    for (int i = 0; i < n; ++i)
        if (!vec16_ok(descs[i].img, descs[i].edge, descs[i].stride_words)) return true;
    return false;
}

me_tile_cfg batch_cfg(const me_desc *descs, int n) {
    return tile_cfg(batch_any(descs, n) ? ME_KIND_BATCH_ANY : ME_KIND_BATCH);
}

bool valid_cfg(const me_tile_cfg &c) {
    const bool rows = c.rows_per_lane == 4 || c.rows_per_lane == 8 ||
                      c.rows_per_lane == 16 || c.rows_per_lane == 32;
    const bool vec = c.vec_words == 1 || c.vec_words == 4;
    const bool thr = c.cta_threads == 128 || c.cta_threads == 256 || c.cta_threads == 512;
    const bool eng = c.engine == ME_ENGINE_REGS || c.engine == ME_ENGINE_BULK;
    const bool stage = c.stage_kb >= 4 && c.stage_kb <= 64 && c.stages >= 2 && c.stages <= 8 &&
                       c.stage_kb * c.stages <= 216;
    const bool chunk = c.chunk_tiles >= 0 && c.chunk_tiles <= 64;
    return rows && vec && thr && eng && stage && chunk && c.ctas_per_sm >= 0 &&
           c.ctas_per_sm <= 32;
}

uint64_t cfg_key(const me_tile_cfg &c) {
    uint64_t k = (uint64_t)c.engine;
    for (int32_t v : {c.rows_per_lane, c.vec_words, c.cta_threads, c.ctas_per_sm, c.stage_kb,
                      c.stages, c.chunk_tiles})
        k = k * 1000003ull + (uint64_t)v;
    return k;
}

}  // namespace me

using namespace me;

extern "C" {

const char *me_status_string(int s) {
    switch (s) {
        case ME_OK: return "ME_OK";
        case ME_PENDING: return "ME_PENDING";
        case ME_TIMEOUT: return "ME_TIMEOUT";
        case ME_ERR_ARG: return "ME_ERR_ARG";
        case ME_ERR_ALIAS: return "ME_ERR_ALIAS";
        case ME_ERR_ALIGN: return "ME_ERR_ALIGN";
        case ME_ERR_BUDGET: return "ME_ERR_BUDGET";
        case ME_ERR_CUDA: return "ME_ERR_CUDA";
        case ME_ERR_CLOSED: return "ME_ERR_CLOSED";
        case ME_ERR_TICKET: return "ME_ERR_TICKET";
        case ME_ERR_NOMEM: return "ME_ERR_NOMEM";
        case ME_ERR_UNSUPPORTED: return "ME_ERR_UNSUPPORTED";
        case ME_ERR_TOO_BIG: return "ME_ERR_TOO_BIG";
        default: return "ME_UNKNOWN_STATUS";
    }
}

int me_last_cuda_error(void) {
    const int e = t_last_cuda;
    t_last_cuda = 0;
    return e;
}

int me_version(void) { return 10000; }

int me_device_faults(int32_t clear, uint32_t *flags) {
    if (flags == nullptr) return ME_ERR_ARG;
    cudaError_t e = cudaDeviceSynchronize();
    if (e != cudaSuccess) return record_cuda(e);
    *flags = device_fault_flags(clear != 0) | window_fault_flags(clear != 0);
    return ME_OK;
}

int me_get_tile_cfg(int32_t kind, me_tile_cfg *out) {
    if (out == nullptr || !valid_kind(kind)) return ME_ERR_ARG;
    *out = tile_cfg(kind);
    return ME_OK;
}

int me_set_tile_cfg(int32_t kind, const me_tile_cfg *cfg) {
    if (cfg == nullptr || !valid_kind(kind)) return ME_ERR_ARG;
    if (!valid_cfg(*cfg)) return ME_ERR_ARG;
    if (cfg->engine == ME_ENGINE_BULK && !bulk_available()) return ME_ERR_UNSUPPORTED;
    std::lock_guard<std::mutex> lk(g_cfg_mu);
    g_cfg[kind] = *cfg;
    return ME_OK;
}

// Shared front end of the one-output single-image calls.
static int single_call(int mode, const uint32_t *img, int32_t w, int32_t h,
                       int32_t stride_words, uint32_t *out, int32_t boundary,
                       me_stream_t stream) {
    int rc = check_image_args(img, out, w, h, stride_words, boundary);
    if (rc != ME_OK) return rc;
    if ((rc = check_device_ptr(img)) != ME_OK) return rc;
    if ((rc = check_device_ptr(out)) != ME_OK) return rc;
    const me_tile_cfg cfg = tile_cfg(ME_KIND_SINGLE);
    const Geo g = make_geo(img, w, h, stride_words, boundary, pick_vw(cfg.vec_words),
                           vec16_ok(img, out, stride_words), vec8_ok(img, out, stride_words));
    cudaError_t e;
    if (mode == MODE_EDGE && cfg.engine == ME_ENGINE_BULK) {
        e = launch_bulk(g, out, cfg, (cudaStream_t)stream);
    } else {
        Outs o = {{out, nullptr, nullptr, nullptr}};
        e = launch_window(mode, g, o, cfg, (cudaStream_t)stream);
    }
    return e == cudaSuccess ? ME_OK : record_cuda(e);
}

int me_edges(const uint32_t *img, int32_t w, int32_t h, int32_t stride_words,
             uint32_t *edge, int32_t boundary, me_stream_t stream) {
    return single_call(MODE_EDGE, img, w, h, stride_words, edge, boundary, stream);
}

int me_edges_display(const uint32_t *img, int32_t w, int32_t h,
                     int32_t stride_words, uint32_t *out, int32_t boundary,
                     me_stream_t stream) {
    return single_call(MODE_DISPLAY, img, w, h, stride_words, out, boundary, stream);
}

int me_end_points(const uint32_t *img, int32_t w, int32_t h,
                  int32_t stride_words, uint32_t *out, int32_t boundary,
                  me_stream_t stream) {
    return single_call(MODE_END, img, w, h, stride_words, out, boundary, stream);
}

int me_fundamental_edges(const uint32_t *img, int32_t w, int32_t h,
                         int32_t stride_words, uint32_t *left, uint32_t *right,
                         uint32_t *up, uint32_t *down, int32_t boundary,
                         me_stream_t stream) {
    uint32_t *outs[4] = {left, right, up, down};
    int rc;
    for (int k = 0; k < 4; ++k)
        if ((rc = check_image_args(img, outs[k], w, h, stride_words, boundary)) != ME_OK)
            return rc;
    const size_t bytes = (size_t)h * (size_t)stride_words * 4;
    for (int a = 0; a < 4; ++a)
        for (int b = a + 1; b < 4; ++b)
            if (ranges_overlap(outs[a], bytes, outs[b], bytes)) return ME_ERR_ALIAS;
    if ((rc = check_device_ptr(img)) != ME_OK) return rc;
    for (int k = 0; k < 4; ++k)
        if ((rc = check_device_ptr(outs[k])) != ME_OK) return rc;
    const me_tile_cfg cfg = tile_cfg(ME_KIND_SINGLE);
    bool vec16 = true;
    bool vec8 = true;
    for (int k = 0; k < 4; ++k) {
        vec16 = vec16 && vec16_ok(img, outs[k], stride_words);
        vec8 = vec8 && vec8_ok(img, outs[k], stride_words);
    }
    const Geo g = make_geo(img, w, h, stride_words, boundary, pick_vw(cfg.vec_words), vec16,
                           vec8);
    Outs o = {{left, right, up, down}};
    cudaError_t e = launch_window(MODE_FUND, g, o, cfg, (cudaStream_t)stream);
    return e == cudaSuccess ? ME_OK : record_cuda(e);
}

int me_edges_staged(const uint32_t *img, int32_t w, int32_t h,
                    int32_t stride_words, uint32_t *edge, int32_t boundary,
                    me_stream_t stream) {
    int rc = check_image_args(img, edge, w, h, stride_words, boundary);
    if (rc != ME_OK) return rc;
    if ((rc = check_device_ptr(img)) != ME_OK) return rc;
    if ((rc = check_device_ptr(edge)) != ME_OK) return rc;
    if ((uint64_t)h * (uint64_t)stride_words >= (1ull << 32)) return ME_ERR_ARG;
    const cudaStream_t s = (cudaStream_t)stream;
    const Geo g = make_geo(img, w, h, stride_words, boundary, 1);
    uint32_t *mask = nullptr;
    cudaError_t e = scratch_alloc((void **)&mask, (size_t)h * stride_words * 4, s);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return record_cuda(e);
    }
    e = launch_staged(g, mask, edge, s);
    cudaError_t f = scratch_free(mask, s);
    if (e == cudaSuccess) e = f;
    return e == cudaSuccess ? ME_OK : record_cuda(e);
}

}  // extern "C"
