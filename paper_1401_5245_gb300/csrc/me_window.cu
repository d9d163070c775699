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
template <int VW, int RPT, int MODE, int VEC>
__global__ void __launch_bounds__(512)
k_window(Geo g, Outs o, int ntasks) {
    pdl_enter();
    const int lane = threadIdx.x & 31;
    const int warp = (int)((blockIdx.x * (unsigned)blockDim.x + threadIdx.x) >> 5);
    const int nwarps = (int)((gridDim.x * (unsigned)blockDim.x) >> 5);
    for (int t = warp; t < ntasks; t += nwarps) {
        const int rb = (int)(((uint64_t)t * g.ncb_m) >> g.ncb_s);    // t / ncb
        const int cb = t - rb * g.ncb;
        window_tile<VW, RPT, MODE, VEC>(g, o, cb, rb, lane);
    }
}

using WindowFn = void (*)(Geo, Outs, int);

template <int VW, int MODE, int VEC>
static WindowFn pick_rpt(int rpt) {
    switch (rpt) {
        case 4: return k_window<VW, 4, MODE, VEC>;
        case 8: return k_window<VW, 8, MODE, VEC>;
        case 16: return k_window<VW, 16, MODE, VEC>;
        case 32: return k_window<VW, 32, MODE, VEC>;
        default: return nullptr;
    }
}

template <int VW, int VEC>
static WindowFn pick_mode(int mode, int rpt) {
    switch (mode) {
        case MODE_EDGE: return pick_rpt<VW, MODE_EDGE, VEC>(rpt);
        case MODE_DISPLAY: return pick_rpt<VW, MODE_DISPLAY, VEC>(rpt);
        case MODE_FUND: return pick_rpt<VW, MODE_FUND, VEC>(rpt);
        case MODE_END: return pick_rpt<VW, MODE_END, VEC>(rpt);
        default: return nullptr;
    }
}

// Row blocks of RPT * segs rows times column blocks.  ceil(h / (rpt segs))
// = ceil(ceil(h / rpt) / segs); rpt is a power of two.
static int64_t tasks_of(int h, int segs, int ncb, int rpt) {
    const unsigned rows = ((unsigned)h + (unsigned)rpt - 1) >> __builtin_ctz((unsigned)rpt);
    const unsigned nrb = (rows + (unsigned)segs - 1) / (unsigned)segs;
    return (int64_t)ncb * nrb;
}

cudaError_t launch_window(int mode, const Geo &g, const Outs &o,
                          const me_tile_cfg &cfg, cudaStream_t s) {
    WindowFn fn = g.vw != 4 ? pick_mode<1, 4>(mode, cfg.rows_per_lane)
                  : g.vec16 ? pick_mode<4, 16>(mode, cfg.rows_per_lane)
                  : g.vec8  ? pick_mode<4, 8>(mode, cfg.rows_per_lane)
                            : pick_mode<4, 4>(mode, cfg.rows_per_lane);
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
    const cudaError_t e = launch_pdl(fn, dim3((unsigned)grid), dim3(threads), 0, s, g, o,
                                     (int)ntasks);
    if (e != cudaSuccess) cudaGetLastError();
    return e;
}

// ------------------------------------------------------------- batch
// The batch's tiles, image by image and top to bottom within an image, are
// cut into chunks of C consecutive tiles; warp w of W takes chunks w,
// w + W, w + 2W, ...  The warps running at any moment thus work on one
// window of neighbouring memory that sweeps through the batch, as a copy
// does (on the uneven 4096-image batch this measured 6.6% faster than
// giving each warp one contiguous range), and within a chunk a warp's
// tiles are vertically adjacent, so the halo rows it re-reads are still in
// L1.  A table gives the image of every (1 << block_shift)-th tile; a warp
// bisects between two entries for the image of its chunk's first tile and
// walks forward from there.
// Set by the 128-bit-only batch kernel if it meets an image it cannot take
// (the host picks the kernel from the same flags, so this stays 0); read and
// cleared by me_device_faults.
__device__ unsigned int g_me_window_faults = 0;
constexpr unsigned int kFaultUnalignedTile = 2u;

// Tiles c0 .. t1 - 1 of the batch, which are consecutive.
template <int RPT, bool ANY>
__device__ __forceinline__ void batch_tiles(const BDesc *__restrict__ descs,
                                            const int32_t *__restrict__ block_image, int shift,
                                            int c0, int t1, int lane) {
    // the image of tile c0: bisect the images the table brackets it with
    int i = block_image[c0 >> shift];
    int hi = block_image[(c0 >> shift) + 1];
    while (i < hi) {
        const int mid = (i + hi + 1) >> 1;
        if (descs[mid].task_base <= c0) i = mid; else hi = mid - 1;
    }
    for (int t = c0; t < t1; ++t) {
        while (t >= descs[i].task_base + descs[i].ntasks) ++i;
        // the 64-byte descriptor as four 128-bit loads
        const uint4 *dv = reinterpret_cast<const uint4 *>(descs + i);
        const uint4 d0 = dv[0], d1 = dv[1], d2 = dv[2], d3 = dv[3];
        Geo g;
        g.img = reinterpret_cast<const uint32_t *>(((uint64_t)d0.y << 32) | d0.x);
        g.w = 0;
        g.segs = (int)d1.x;
        g.h = (int)d1.y;
        g.stride = (int)d1.z;
        g.nw = (int)d1.w;
        g.lastmask = d2.x;
        g.fill = d2.y;
        g.vw = (int)(d2.z & 0xff);
        g.vec16 = (int)((d2.z >> 8) & 1);
        g.vec8 = (int)((d2.z >> 9) & 1);
        g.seg_w = (int)d2.w;
        g.ncb = (int)d3.x;
        g.nv = (int)d3.y;
        Outs o;
        o.p[0] = reinterpret_cast<uint32_t *>(((uint64_t)d0.w << 32) | d0.z);
        o.p[1] = o.p[2] = o.p[3] = nullptr;
        const int local = t - (int)d3.z;             // task_base
        // rows of at most 32 vector columns have one column block: no
        // division
        const int cb = g.ncb == 1 ? 0 : local % g.ncb;
        const int rb = g.ncb == 1 ? local : local / g.ncb;
        if (g.vec16) {
            window_tile<4, RPT, MODE_EDGE, 16>(g, o, cb, rb, lane);
        } else if constexpr (ANY) {
            if (g.vec8)
                window_tile<4, RPT, MODE_EDGE, 8>(g, o, cb, rb, lane);
            else
                window_tile<4, RPT, MODE_EDGE, 4>(g, o, cb, rb, lane);
        } else if (lane == 0)
            atomicOr(&g_me_window_faults, kFaultUnalignedTile);
    }
}

// Two 512-thread CTAs per SM for 4 rows per lane (64 registers).  ANY:
// images whose rows are not whole 16-byte groups (or whose buffers are not
// 16-byte aligned) may occur, so the kernel also carries the tile that
// moves four words per lane as 32-bit accesses; batches without such images
// take the kernel without it, whose registers it would otherwise raise.
// The loop's constants come by value (BatchArgs), from the constant bank:
// loaded from the arena they would hold registers the tile needs.
template <int RPT, bool ANY>
__global__ void __launch_bounds__(512, RPT == 4 ? 2 : 1)
k_batch(const BatchHeader *__restrict__ hdr, const BatchArgs a) {
    // launched while the kernel before it on the stream may still run
    // (programmatic dependent launch): wait for it before any global access
    pdl_enter();
    const BDesc *descs = reinterpret_cast<const BDesc *>(hdr + 1);
    const int32_t *block_image = reinterpret_cast<const int32_t *>(descs + hdr->n);
    const int lane = threadIdx.x & 31;
    const unsigned warp = (blockIdx.x * (unsigned)blockDim.x + threadIdx.x) >> 5;
    const unsigned W = (gridDim.x * (unsigned)blockDim.x) >> 5;
    // Tile indices are below 2^31 and item indices below the tiles plus a
    // grid's warps, so no unsigned sum below wraps.
    for (unsigned k = warp;; k += W) {
        const bool chunk = k < (unsigned)a.nchunks;
        const unsigned c0 = chunk ? k * (unsigned)a.chunk
                                  : k + (unsigned)(a.chunked - a.nchunks);
        if (c0 >= (unsigned)a.total) break;
        batch_tiles<RPT, ANY>(descs, block_image, a.shift, (int)c0,
                              (int)(c0 + (chunk ? (unsigned)a.chunk : 1u)), lane);
    }
}

using BatchFn = void (*)(const BatchHeader *, BatchArgs);

static BatchFn pick_batch(int rpt, bool any) {
    switch (rpt) {
        case 4: return any ? k_batch<4, true> : k_batch<4, false>;
        case 8: return any ? k_batch<8, true> : k_batch<8, false>;
        case 16: return any ? k_batch<16, true> : k_batch<16, false>;
        case 32: return any ? k_batch<32, true> : k_batch<32, false>;
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

int batch_grid(const me_tile_cfg &cfg, const DevInfo &di, int64_t total_tasks, bool any,
               int *grid, int *threads) {
    *threads = cfg.cta_threads;
    if (cfg.ctas_per_sm == 0) {
        const int64_t chunks = (total_tasks + chunk_of(cfg) - 1) / chunk_of(cfg);
        const int64_t warps = cfg.cta_threads / 32;
        *grid = (int)std::max<int64_t>(1, std::min<int64_t>((chunks + warps - 1) / warps,
                                                            INT32_MAX));
        return ME_OK;
    }
    int occ = 0;
    int rc = regs_ctas_per_sm(reinterpret_cast<const void *>(pick_batch(cfg.rows_per_lane, any)),
                              cfg.cta_threads, &occ);
    if (rc != ME_OK) return rc;
    const int per_sm = std::max(1, std::min(cfg.ctas_per_sm, occ));
    *grid = di.sm_count * per_sm;
    return ME_OK;
}

static void fill_bdesc(const me_desc &d, const me_tile_cfg &cfg, BDesc *out) {
    // batches always take 4 words per lane; vec_words = 1 asks for 32-bit
    // accesses
    Geo g = make_geo(d.img, d.w, d.h, d.stride_words, d.boundary, 4,
                     cfg.vec_words == 4 && vec16_ok(d.img, d.edge, d.stride_words),
                     cfg.vec_words == 4 && vec8_ok(d.img, d.edge, d.stride_words));
    out->img = d.img;
    out->edge = d.edge;
    out->segs = g.segs;
    out->h = g.h;
    out->stride = g.stride;
    out->nw = g.nw;
    out->lastmask = g.lastmask;
    out->fill = g.fill;
    // words per lane; 128-bit (bit 8) or 64-bit (bit 9) accesses
    out->vw = g.vw | (g.vec16 << 8) | (g.vec8 << 9);
    out->seg_w = g.seg_w;
    out->ncb = g.ncb;
    out->nv = g.nv;
}

int plan_batch(const me_desc *descs, int n, const me_tile_cfg &cfg, void *host_arena,
               int64_t *total_tasks, bool *any, int *bad) {
    BatchHeader *hdr = static_cast<BatchHeader *>(host_arena);
    BDesc *bd = reinterpret_cast<BDesc *>(hdr + 1);
    int32_t *block_image = reinterpret_cast<int32_t *>(bd + n);
    std::memset(hdr, 0, sizeof(*hdr));
    int64_t total = 0, bytes = 0;
    bool narrow = false;        // some image takes 64- or 32-bit accesses
    for (int i = 0; i < n; ++i) {
        const me_desc &d = descs[i];
        int rc = check_image_args(d.img, d.edge, d.w, d.h, d.stride_words, d.boundary);
        if (rc != ME_OK) {
            if (bad) *bad = i;
            return rc;
        }
        fill_bdesc(d, cfg, &bd[i]);
        narrow |= ((bd[i].vw >> 8) & 1) == 0;   // not the 128-bit path
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
    hdr->rows_per_lane = cfg.rows_per_lane;
    hdr->chunk_tiles = chunk_of(cfg);
    hdr->bytes = bytes;
    // entries 0 .. ceil(total / 2^shift) inclusive, the last one n - 1
    int shift = 0;
    while (((total - 1) >> shift) + 2 > task_table_entries(n)) ++shift;
    hdr->block_shift = shift;
    // the image holding tile b << shift: image k covers the entries whose
    // first tile lies in [task_base, task_base + ntasks)
    const int64_t unit = (int64_t)1 << shift;
    int64_t b = 0;
    for (int k = 0; k < n; ++k) {
        const int64_t end = (int64_t)bd[k].task_base + bd[k].ntasks;
        for (; b * unit < end; ++b) block_image[b] = k;
    }
    block_image[b] = n - 1;
    if (total_tasks) *total_tasks = total;
    if (any) *any = narrow;
    return ME_OK;
}

BatchArgs batch_args(const void *host_arena, int grid, int threads) {
    const BatchHeader *hdr = static_cast<const BatchHeader *>(host_arena);
    BatchArgs a;
    a.total = hdr->total_tasks;
    a.chunk = hdr->chunk_tiles;
    a.shift = hdr->block_shift;
    const int64_t step = (int64_t)grid * (threads / 32) * a.chunk;
    int64_t chunked = step > 0 ? (int64_t)a.total / step * step : 0;
    if (chunked == 0) chunked = (int64_t)a.total / a.chunk * a.chunk;
    a.chunked = (int32_t)chunked;
    a.nchunks = (int32_t)(chunked / a.chunk);
    return a;
}

unsigned int window_fault_flags(bool clear) {
    unsigned int v = 0;
    if (cudaMemcpyFromSymbol(&v, g_me_window_faults, sizeof(v)) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    if (clear) {
        const unsigned int z = 0;
        cudaMemcpyToSymbol(g_me_window_faults, &z, sizeof(z));
    }
    return v;
}

}  // namespace me

namespace me {
const void *batch_kernel(int rows_per_lane, bool any) {
    return reinterpret_cast<const void *>(pick_batch(rows_per_lane, any));
}
}  // namespace me
