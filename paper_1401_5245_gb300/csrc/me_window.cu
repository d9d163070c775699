// Fused method-of-masks kernels on the register-window engine: one image
// per launch (all output modes) and the persistent batch kernel.
#include <algorithm>
#include <cstring>
#include <mutex>
#include <utility>
#include <vector>

#include "me_internal.h"
#include "me_window.cuh"

namespace me {

// ------------------------------------------------------------ single image
// Warp tiles are numbered with the column block fastest, so warps that run
// together cover whole row bands and share the halo rows in L2.
template <int VW, int RPT, int MODE>
__global__ void __launch_bounds__(512)
k_window(Geo g, Outs o, int ntasks) {
    const int lane = threadIdx.x & 31;
    const int warp = (int)((blockIdx.x * (unsigned)blockDim.x + threadIdx.x) >> 5);
    const int nwarps = (int)((gridDim.x * (unsigned)blockDim.x) >> 5);
    for (int t = warp; t < ntasks; t += nwarps) {
        const int cb = t % g.ncb;
        const int rb = t / g.ncb;
        window_tile<VW, RPT, MODE>(g, o, cb, rb, lane);
    }
}

using WindowFn = void (*)(Geo, Outs, int);

template <int VW, int MODE>
static WindowFn pick_rpt(int rpt) {
    switch (rpt) {
        case 4: return k_window<VW, 4, MODE>;
        case 8: return k_window<VW, 8, MODE>;
        case 16: return k_window<VW, 16, MODE>;
        case 32: return k_window<VW, 32, MODE>;
        default: return nullptr;
    }
}

template <int VW>
static WindowFn pick_mode(int mode, int rpt) {
    switch (mode) {
        case MODE_EDGE: return pick_rpt<VW, MODE_EDGE>(rpt);
        case MODE_DISPLAY: return pick_rpt<VW, MODE_DISPLAY>(rpt);
        case MODE_FUND: return pick_rpt<VW, MODE_FUND>(rpt);
        case MODE_END: return pick_rpt<VW, MODE_END>(rpt);
        default: return nullptr;
    }
}

static int64_t tasks_of(int h, int segs, int ncb, int rpt) {
    const int64_t rows_per_task = (int64_t)rpt * segs;
    const int64_t nrb = (h + rows_per_task - 1) / rows_per_task;
    return (int64_t)ncb * nrb;
}

cudaError_t launch_window(int mode, const Geo &g, const Outs &o,
                          const me_tile_cfg &cfg, cudaStream_t s) {
    WindowFn fn = (g.vw == 4) ? pick_mode<4>(mode, cfg.rows_per_lane)
                              : pick_mode<1>(mode, cfg.rows_per_lane);
    if (fn == nullptr) return cudaErrorInvalidValue;
    const int64_t ntasks = tasks_of(g.h, g.segs, g.ncb, cfg.rows_per_lane);
    if (ntasks > INT32_MAX) return cudaErrorInvalidValue;
    const int threads = cfg.cta_threads;
    const int warps_per_cta = threads / 32;
    int64_t grid = (ntasks + warps_per_cta - 1) / warps_per_cta;
    if (cfg.ctas_per_sm > 0) {
        DevInfo di;
        if (device_info(&di) != ME_OK) return cudaErrorInvalidDevice;
        int occ = 0;
        if (regs_ctas_per_sm(reinterpret_cast<const void *>(fn), threads, &occ) != ME_OK)
            return cudaErrorInvalidValue;
        const int per_sm = std::max(1, std::min(cfg.ctas_per_sm, occ));
        grid = std::min<int64_t>(grid, (int64_t)di.sm_count * per_sm);
    }
    grid = std::max<int64_t>(1, std::min<int64_t>(grid, INT32_MAX));
    fn<<<(unsigned)grid, threads, 0, s>>>(g, o, (int)ntasks);
    return cudaGetLastError();
}

// ------------------------------------------------------------- batch
// Every warp owns a contiguous range of the batch's tiles, so consecutive
// tiles of one warp are usually vertically adjacent in the same image and
// the halo rows it re-reads are still in L1/L2.  The host gives every warp
// the same number of tiles and writes each warp's first tile and its image;
// the warp then walks forward.
template <int RPT>
__global__ void __launch_bounds__(512)
k_batch(const BatchHeader *__restrict__ hdr) {
    const BDesc *descs = reinterpret_cast<const BDesc *>(hdr + 1);
    const int W = hdr->total_warps;
    const int32_t *warp_first_image = reinterpret_cast<const int32_t *>(descs + hdr->n);
    const int32_t *warp_first_task = reinterpret_cast<const int32_t *>(
        reinterpret_cast<const char *>(warp_first_image) + owner_table_bytes(W));
    const int lane = threadIdx.x & 31;
    const int warp = (int)((blockIdx.x * (unsigned)blockDim.x + threadIdx.x) >> 5);
    if (warp >= W) return;
    const int t0 = warp_first_task[warp];
    const int t1 = warp_first_task[warp + 1];
    int i = warp_first_image[warp];
    for (int t = t0; t < t1; ++t) {
        while (t >= descs[i].task_base + descs[i].ntasks) ++i;
        const BDesc &d = descs[i];
        Geo g;
        g.img = d.img;
        g.w = 0;
        g.h = d.h;
        g.stride = d.stride;
        g.nw = d.nw;
        g.lastmask = d.lastmask;
        g.fill = d.fill;
        g.vw = d.vw;
        g.nv = d.nv;
        g.seg_w = d.seg_w;
        g.segs = d.segs;
        g.ncb = d.ncb;
        Outs o;
        o.p[0] = d.edge;
        o.p[1] = o.p[2] = o.p[3] = nullptr;
        const int local = t - d.task_base;
        const int cb = local % d.ncb;
        const int rb = local / d.ncb;
        if (d.vw == 4)
            window_tile<4, RPT, MODE_EDGE>(g, o, cb, rb, lane);
        else
            window_tile<1, RPT, MODE_EDGE>(g, o, cb, rb, lane);
    }
}

using BatchFn = void (*)(const BatchHeader *);

static BatchFn pick_batch(int rpt) {
    switch (rpt) {
        case 4: return k_batch<4>;
        case 8: return k_batch<8>;
        case 16: return k_batch<16>;
        case 32: return k_batch<32>;
        default: return nullptr;
    }
}

int regs_ctas_per_sm(const void *fn, int threads, int *out) {
    return cached_occupancy(fn, threads, 0, out);
}

int cached_occupancy(const void *fn, int threads, size_t smem, int *out) {
    // cudaOccupancyMaxActiveBlocksPerMultiprocessor costs microseconds per
    // call; launches ask it every time, so remember answers per device
    struct Key {
        const void *fn;
        int threads, dev;
        size_t smem;
        bool operator==(const Key &o) const {
            return fn == o.fn && threads == o.threads && dev == o.dev && smem == o.smem;
        }
    };
    static std::mutex mu;
    static std::vector<std::pair<Key, int>> seen;
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return record_cuda(e);
    const Key k{fn, threads, dev, smem};
    {
        std::lock_guard<std::mutex> lk(mu);
        for (auto &kv : seen)
            if (kv.first == k) {
                *out = kv.second;
                return ME_OK;
            }
    }
    int n = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, fn, threads, smem);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return record_cuda(e);
    }
    std::lock_guard<std::mutex> lk(mu);
    seen.push_back({k, n});
    *out = n;
    return ME_OK;
}

int batch_grid(const me_tile_cfg &cfg, const DevInfo &di, int *grid, int *threads) {
    int occ = 0;
    int rc = regs_ctas_per_sm(reinterpret_cast<const void *>(pick_batch(cfg.rows_per_lane)),
                              cfg.cta_threads, &occ);
    if (rc != ME_OK) return rc;
    const int per_sm = std::max(1, std::min(cfg.ctas_per_sm > 0 ? cfg.ctas_per_sm : occ, occ));
    *grid = di.sm_count * per_sm;
    *threads = cfg.cta_threads;
    return ME_OK;
}

cudaError_t launch_batch(const void *arena_dev, int grid, int threads,
                         int rows_per_lane, cudaStream_t s) {
    BatchFn fn = pick_batch(rows_per_lane);
    if (fn == nullptr) return cudaErrorInvalidValue;
    fn<<<grid, threads, 0, s>>>(static_cast<const BatchHeader *>(arena_dev));
    return cudaGetLastError();
}

static void fill_bdesc(const me_desc &d, const me_tile_cfg &cfg, BDesc *out) {
    const int vw = pick_vw(d.img, d.edge, d.stride_words, cfg.vec_words);
    Geo g = make_geo(d.img, d.w, d.h, d.stride_words, d.boundary, vw);
    out->img = d.img;
    out->edge = d.edge;
    out->segs = g.segs;
    out->h = g.h;
    out->stride = g.stride;
    out->nw = g.nw;
    out->lastmask = g.lastmask;
    out->fill = g.fill;
    out->vw = g.vw;
    out->seg_w = g.seg_w;
    out->ncb = g.ncb;
    out->nv = g.nv;
}

int batch_tasks(const me_desc *descs, int n, const me_tile_cfg &cfg,
                int64_t *total_tasks) {
    int64_t total = 0;
    for (int i = 0; i < n; ++i) {
        const me_desc &d = descs[i];
        int rc = check_image_args(d.img, d.edge, d.w, d.h, d.stride_words, d.boundary);
        if (rc != ME_OK) return rc;
        BDesc b;
        fill_bdesc(d, cfg, &b);
        total += tasks_of(b.h, b.segs, b.ncb, cfg.rows_per_lane);
    }
    *total_tasks = total;
    return total > INT32_MAX ? ME_ERR_ARG : ME_OK;
}

int plan_batch(const me_desc *descs, int n, const me_tile_cfg &cfg,
               int total_warps, void *host_arena, int *bad) {
    BatchHeader *hdr = static_cast<BatchHeader *>(host_arena);
    BDesc *bd = reinterpret_cast<BDesc *>(hdr + 1);
    int32_t *first_image = reinterpret_cast<int32_t *>(bd + n);
    int32_t *first_task = reinterpret_cast<int32_t *>(reinterpret_cast<char *>(first_image) +
                                                      owner_table_bytes(total_warps));
    std::memset(hdr, 0, sizeof(*hdr));
    int64_t total = 0, bytes = 0;
    for (int i = 0; i < n; ++i) {
        const me_desc &d = descs[i];
        int rc = check_image_args(d.img, d.edge, d.w, d.h, d.stride_words, d.boundary);
        if (rc != ME_OK) {
            if (bad) *bad = i;
            return rc;
        }
        fill_bdesc(d, cfg, &bd[i]);
        const int64_t nt = tasks_of(bd[i].h, bd[i].segs, bd[i].ncb, cfg.rows_per_lane);
        if (total + nt > INT32_MAX) {
            if (bad) *bad = i;
            return ME_ERR_ARG;
        }
        bd[i].task_base = (int32_t)total;
        bd[i].ntasks = (int32_t)nt;
        total += nt;
        bytes += 2 * (int64_t)d.h * d.stride_words * 4;
    }
    hdr->n = n;
    hdr->total_tasks = (int32_t)total;
    hdr->total_warps = total_warps;
    hdr->rows_per_lane = cfg.rows_per_lane;
    hdr->bytes = bytes;
    // Equal numbers of tiles per warp.  A tile costs about one memory round
    // trip whatever its width, so equal counts finish together better than
    // equal bytes (measured on the uneven 4096-image batch).
    for (int w = 0; w <= total_warps; ++w)
        first_task[w] = (int32_t)((total * w) / total_warps);
    // the image holding each warp's first tile (both sequences increase)
    int k = 0;
    for (int w = 0; w <= total_warps; ++w) {
        while (k < n - 1 && first_task[w] >= bd[k].task_base + bd[k].ntasks) ++k;
        first_image[w] = k;
    }
    return ME_OK;
}

}  // namespace me

namespace me {
const void *batch_kernel(int rows_per_lane) {
    return reinterpret_cast<const void *>(pick_batch(rows_per_lane));
}
}  // namespace me
