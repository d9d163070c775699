// Internal declarations shared by the translation units of libme.
#pragma once

#include <algorithm>
#include <cstddef>
#include <cstdint>

#include <mutex>
#include <utility>

#include <cuda_runtime.h>

#include "me.h"

namespace me {

constexpr uint32_t kAllOnes = 0xFFFFFFFFu;
// Output columns of a register-window warp on rows wider than 32 vector
// columns (lanes 0 and 31 only load the columns beside the block).
constexpr int kWideLanes = 30;

// What a window kernel writes per pixel word.
enum Mode : int {
    MODE_EDGE = 0,      // Edge(p): NOT I AND (L OR R OR U OR D)       (Sections 3-5)
    MODE_DISPLAY = 1,   // the OR inverted, as drawn in Section 5
    MODE_FUND = 2,      // the four fundamental edges, four outputs  (Section 4)
    MODE_END = 3,       // black with <= 1 black 8-neighbour          (Section 1)
    MODE_COUNT = 4
};

// Geometry of one packed image as the kernels see it.
struct Geo {
    const uint32_t *img;
    int32_t w, h, stride, nw;   // nw = ceil(w / 32) words hold pixels
    uint32_t lastmask;          // valid bits of word nw - 1
    uint32_t fill;              // outside colour as a word: ~0 white, 0 black
    int32_t vw;                 // words per lane and row: 4 or 1
    int32_t vec16;              // vw == 4: the 4 words move as one 128-bit access
    int32_t vec8;               // vw == 4, not vec16: as two 64-bit accesses
    int32_t nv;                 // vector columns written: ceil(stride / vw)
    int32_t seg_w;              // lanes one row segment uses (nv, or 32 when wide)
    int32_t segs;               // row segments stacked in one warp (32 / seg_w)
    int32_t ncb;                // column blocks (kWideLanes columns when nv > 32)
    // t / ncb for 0 <= t < 2^31 as (t * ncb_m) >> ncb_s (division by an
    // invariant integer by multiplication, Granlund and Montgomery 1994:
    // ncb_m = ceil(2^(32+l) / ncb), ncb_s = 32 + l, l = ceil(log2 ncb))
    uint64_t ncb_m;
    int32_t ncb_s;
};

struct Outs {
    uint32_t *p[4];
};

// Batch descriptor as the persistent kernel reads it (64 bytes).
struct BDesc {
    const uint32_t *img;
    uint32_t *edge;
    int32_t segs, h, stride, nw;
    uint32_t lastmask, fill;
    int32_t vw;                 // bits 0-7 words per lane; bit 8 128-bit, bit 9 64-bit accesses
    int32_t seg_w, ncb, nv;
    int32_t task_base, ntasks;
};
static_assert(sizeof(BDesc) == 64, "BDesc is 64 bytes");
// the batch kernel reads a descriptor as four 16-byte words in this order
static_assert(offsetof(BDesc, edge) == 8 && offsetof(BDesc, segs) == 16 &&
                  offsetof(BDesc, lastmask) == 32 && offsetof(BDesc, vw) == 40 &&
                  offsetof(BDesc, ncb) == 48 && offsetof(BDesc, task_base) == 56,
              "BDesc layout");

// Image descriptor of the bulk-copy engine (64 bytes).  The image is cut
// into bands of band_rows rows x band_words words; a band plus one halo row
// above and below (and 4 halo words left and right in column mode) is
// copied into one shared-memory stage laid out as rows of `pitch` words,
// stage column 0 holding image word x0 - xhalo.
struct KDescB {
    const uint32_t *img;
    uint32_t *edge;
    int32_t flags;              // kBulkCopy | kVecStore | kRowMode
    int32_t h, stride, nw;
    uint32_t lastmask, fill;
    int32_t band_rows, band_words, pitch;
    int32_t ncb, nrb;           // column blocks, row bands
    int32_t band_base;          // first band of this image in the batch
};
static_assert(sizeof(KDescB) == 64, "KDescB is 64 bytes");
constexpr int32_t kBulkCopy = 1;    // copy with cp.async.bulk (16-byte rows)
constexpr int32_t kVecStore = 2;    // 128-bit stores allowed
constexpr int32_t kRowMode = 4;     // full rows, one contiguous copy per band

// Device arena of one batch: header, then descriptors, then a table.
// Register window: entry k is the image holding tile k << block_shift, where
// a warp starts its walk to the image of its next chunk; the table has
// task_table_entries(n) entries and block_shift is the smallest shift that
// covers all tiles with them (so the arena size depends on n alone).  Bulk
// engine: entry c is the image of CTA c's first band.
struct BatchHeader {
    int32_t n;
    int32_t total_tasks;
    int32_t total_warps;        // bulk engine: band owners (CTAs)
    int32_t rows_per_lane;
    int64_t bytes;              // algorithmic bytes: sum of 2 * h * stride * 4
    int32_t chunk_tiles;        // register window: tiles a warp takes at a time
    int32_t block_shift;        // register window: tiles per table entry, log2
    int32_t pad[56];
};
static_assert(sizeof(BatchHeader) == 256, "BatchHeader is 256 bytes");

inline int64_t task_table_entries(int n) { return 4 * (int64_t)n + 64; }
inline size_t arena_bytes(int n) {
    return sizeof(BatchHeader) + (size_t)n * sizeof(BDesc) +
           ((size_t)task_table_entries(n) * sizeof(int32_t) + 255) / 256 * 256;
}
// Tiles per chunk of a register-window batch configuration.
inline int chunk_of(const me_tile_cfg &c) { return c.chunk_tiles > 0 ? c.chunk_tiles : 4; }

constexpr int kThrRows = 4;     // rows per step of the threshold kernel's walk

// The threshold kernel's rows per band: the multiple of kThrRows that
// minimises the walk's length, counted in rows per warp: the waves of tasks
// (ncb column blocks times the bands of h rows) over the resident warps
// times the rows one task reads (band + 2) plus about four rows' worth of
// set-up.  For k waves the shortest band that fits is found directly; k
// runs from the fewest waves possible (one band per column block:
// ceil(ncb / resident_warps)) over at most 1024 wave counts, which reaches
// the optimum over every band height in all cases tried (tests/host).
inline int threshold_band(int64_t ncb, int32_t h, int64_t resident_warps) {
    const int64_t max_waves = (ncb * (((int64_t)h + kThrRows - 1) / kThrRows) +
                               resident_warps - 1) / resident_warps;
    const int64_t min_waves = std::max<int64_t>(1, (ncb + resident_warps - 1) / resident_warps);
    int best = kThrRows;
    int64_t best_cost = INT64_MAX;
    for (int64_t k = min_waves; k <= std::min<int64_t>(max_waves, min_waves + 1023); ++k) {
        const int64_t bands = std::max<int64_t>(1, k * resident_warps / ncb);   // per column
        int64_t band = ((int64_t)h + bands - 1) / bands;
        band = std::max<int64_t>(kThrRows, (band + kThrRows - 1) / kThrRows * kThrRows);
        const int64_t tasks = ncb * (((int64_t)h + band - 1) / band);
        const int64_t cost = (tasks + resident_warps - 1) / resident_warps * (band + 2 + 4);
        if (cost < best_cost) {
            best_cost = cost;
            best = (int)std::min<int64_t>(band, INT32_MAX);
        }
    }
    return best;
}

// ---------------------------------------------------------------- helpers
// Kernels launched by programmatic dependent launch open with this: the
// launch may be placed while the kernel before it on the stream still
// runs, so wait for that kernel (and its memory) before the first global
// access, then let the next launch be placed during this one's tail.  Both
// are no-ops for a kernel launched without the attribute.
__device__ __forceinline__ void pdl_enter() {
#if defined(__CUDA_ARCH__)
    asm volatile("griddepcontrol.wait;" ::: "memory");
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
#endif
}

// Launch `kernel` on s with programmatic stream serialisation allowed.
template <typename... P, typename... A>
cudaError_t launch_pdl(void (*kernel)(P...), dim3 grid, dim3 block, size_t smem,
                       cudaStream_t s, A &&...args) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kernel, std::forward<A>(args)...);
}

// (inline: a batch plan runs them once per image on every call)
int record_cuda(cudaError_t e);         // remembers e, returns ME_ERR_CUDA
int check_device_ptr(const void *p);    // ME_OK or ME_ERR_ARG / ME_ERR_CUDA

inline bool ranges_overlap(const void *a, size_t na, const void *b, size_t nb) {
    const uintptr_t x = (uintptr_t)a, y = (uintptr_t)b;
    return x < y + nb && y < x + na;
}

inline int check_image_args(const void *img, const void *out, int32_t w, int32_t h,
                            int32_t stride_words, int32_t boundary) {
    if (img == nullptr || out == nullptr) return ME_ERR_ARG;
    if (w <= 0 || h <= 0 || stride_words <= 0) return ME_ERR_ARG;
    if (stride_words < (int32_t)(((int64_t)w + 31) / 32)) return ME_ERR_ARG;
    if (boundary != ME_BOUNDARY_WHITE && boundary != ME_BOUNDARY_BLACK) return ME_ERR_ARG;
    if (((uintptr_t)img & 3) || ((uintptr_t)out & 3)) return ME_ERR_ARG;
    const size_t bytes = (size_t)h * (size_t)stride_words * 4;
    if (ranges_overlap(img, bytes, out, bytes)) return ME_ERR_ALIAS;
    return ME_OK;
}

// Words per lane and row: 4 unless the configuration asks for 1.
inline int pick_vw(int want_vw) { return want_vw == 4 ? 4 : 1; }
// A lane's 4 words move as one 128-bit access when both buffers are 16-byte
// aligned and rows hold whole 16-byte groups; as two 64-bit accesses when
// they are 8-byte aligned and rows hold whole pairs of words; else as four
// 32-bit accesses.
inline bool vec16_ok(const void *img, const void *out, int32_t stride) {
    return !(((uintptr_t)img & 15) || ((uintptr_t)out & 15) || (stride & 3));
}
inline bool vec8_ok(const void *img, const void *out, int32_t stride) {
    return !(((uintptr_t)img & 7) || ((uintptr_t)out & 7) || (stride & 1));
}

struct DevInfo {
    int sm_count;
    int max_threads_per_sm;
    int cc_major, cc_minor;
    char name[256];
};
int device_info(DevInfo *out);          // current device, cached

// vw is 1 or 4; vec16 / vec8 (vw == 4 only): 128-bit / 64-bit accesses
// allowed (the wider one is taken).
inline Geo make_geo(const uint32_t *img, int32_t w, int32_t h, int32_t stride,
                    int32_t boundary, int vw, bool vec16 = false, bool vec8 = false) {
    // segments of a row of n <= 32 vector columns that fit in a warp: 32 / n
    static constexpr int8_t kSegs[33] = {0, 32, 16, 10, 8, 6, 5, 4, 4, 3, 3, 2, 2, 2, 2, 2, 2,
                                         1, 1,  1,  1,  1, 1, 1, 1, 1, 1, 1, 1, 1, 1, 1, 1};
    Geo g;
    g.img = img;
    g.w = w;
    g.h = h;
    g.stride = stride;
    g.nw = (int32_t)(((int64_t)w + 31) >> 5);
    g.lastmask = (w & 31) ? ((1u << (w & 31)) - 1u) : kAllOnes;
    g.fill = (boundary == ME_BOUNDARY_WHITE) ? kAllOnes : 0u;
    g.vw = vw;
    g.vec16 = vw == 4 && vec16;
    g.vec8 = vw == 4 && !vec16 && vec8;
    g.nv = vw == 4 ? (stride + 3) >> 2 : stride;   // output covers the whole stride
    // narrow rows: segments of exactly nv lanes, as many as fit in a warp
    g.seg_w = g.nv > 32 ? 32 : g.nv;
    g.segs = kSegs[g.seg_w];
    g.ncb = g.nv > 32 ? (g.nv + kWideLanes - 1) / kWideLanes : 1;
    int l = 0;
    while ((1ll << l) < g.ncb) ++l;
    g.ncb_s = 32 + l;
    g.ncb_m = (uint64_t)((((unsigned __int128)1 << g.ncb_s) + (unsigned)g.ncb - 1) / (unsigned)g.ncb);
    return g;
}
int ceil_log2(int v);

// ------------------------------------------------------- configurations
me_tile_cfg tile_cfg(int kind);         // current configuration of a kind
// Some image of the batch cannot take 128-bit accesses (ME_KIND_BATCH_ANY).
bool batch_any(const me_desc *descs, int n);
// The configuration of the batch's kind.
me_tile_cfg batch_cfg(const me_desc *descs, int n);
bool valid_cfg(const me_tile_cfg &c);
uint64_t cfg_key(const me_tile_cfg &c);

// ---------------------------------------------------------- launchers
// Single image, register-window engine.  `launches` counts kernels issued.
cudaError_t launch_window(int mode, const Geo &g, const Outs &o,
                          const me_tile_cfg &cfg, cudaStream_t s);
// Single image, bulk-copy (TMA) engine; MODE_EDGE only.
cudaError_t launch_bulk(const Geo &g, uint32_t *edge, const me_tile_cfg &cfg,
                        cudaStream_t s);
bool bulk_available();
// Band geometry of one image for a stage of stage_words words.
void bulk_geometry(const Geo &g, const void *edge, int stage_words, KDescB *out);
// Persistent bulk kernel: function pointer, dynamic shared memory, and the
// CTAs per SM it can keep resident (after raising its smem limit).
const void *bulk_kernel();
size_t bulk_smem_bytes(const me_tile_cfg &cfg);
// cta_threads consumer threads plus one producer warp.
inline int bulk_threads(const me_tile_cfg &cfg) { return cfg.cta_threads + 32; }
int bulk_ctas_per_sm(const me_tile_cfg &cfg, int *out);
int regs_ctas_per_sm(const void *fn, int threads, int *out);
// CTAs of `fn` that fit on one SM (cached per device, kernel, size).
int cached_occupancy(const void *fn, int threads, size_t smem, int *out);
// Host plan of a bulk batch arena (header, KDescB[n], first image per CTA).
int plan_batch_bulk(const me_desc *descs, int n, const me_tile_cfg &cfg, int grid,
                    void *host_arena, int64_t *total_bands);
inline size_t bulk_arena_bytes(int n, int grid) {
    return sizeof(BatchHeader) + (size_t)n * sizeof(KDescB) +
           (((size_t)grid + 1) * sizeof(int32_t) + 255) / 256 * 256;
}
unsigned int device_fault_flags(bool clear);

// Persistent batch kernel over an uploaded arena; any: some image of the
// batch takes 32-bit accesses.
const void *batch_kernel(int rows_per_lane, bool any);
unsigned int window_fault_flags(bool clear);
// Persistent grid of a batch (SMs x ctas_per_sm, capped by occupancy), or
// for ctas_per_sm == 0 the grid of one chunk per warp over total_tasks tiles.
int batch_grid(const me_tile_cfg &cfg, const DevInfo &di, int64_t total_tasks, bool any,
               int *grid, int *threads);

// Fill descriptors and the tile-block image table of a batch arena on the
// host (one pass over the images).  Returns ME_OK or an argument error for
// descriptor i (*bad = i); *total_tasks = tiles of the batch, *any = some
// image takes 32-bit accesses.
int plan_batch(const me_desc *descs, int n, const me_tile_cfg &cfg, void *host_arena,
               int64_t *total_tasks, bool *any, int *bad);

// By-value arguments of the register-window batch kernel, which reads them
// from the constant bank (no registers held).  Warp w takes work items w,
// w + W, w + 2W, ... of the grid's W warps: items below nchunks are chunks
// of `chunk` tiles (item k: tiles k * chunk ..), the rest single tiles
// (item k: tile k + chunked - nchunks), up to `total` tiles.
struct BatchArgs {
    int32_t total;        // tiles of the batch
    int32_t chunk;        // tiles per chunk
    int32_t shift;        // tiles per image-table entry, log2
    int32_t nchunks;      // chunk items
    int32_t chunked;      // nchunks * chunk: tiles covered by chunks
};
// The split for a grid: whole rounds of chunks (one per warp each) when
// the batch has at least one, else the whole chunks its tiles make; the
// tiles left over go one at a time, so that the warps' last pieces of work
// differ by one tile rather than a chunk.
BatchArgs batch_args(const void *host_arena, int grid, int threads);

// How one batch launches under a tile configuration: grid, threads,
// dynamic shared memory, arena size and kernel.
struct BatchSetup {
    me_tile_cfg cfg;
    int grid = 0, threads = 0;
    size_t smem = 0, arena = 0;
    const void *fn = nullptr;
    int stage_words = 0;
    bool any = false;           // register window: the kernel with 32-bit tiles
    BatchArgs args = {};        // register window: set by fill_arena
};
// Neither reads the images' geometry beyond n: descriptors are checked by
// fill_arena, which also fixes the grid of a one-chunk-per-warp launch.
int setup_batch(const me_desc *descs, int n, me_tile_cfg cfg, BatchSetup *s);
// Write the arena of a batch (s.arena bytes) into host memory.
int fill_arena(const me_desc *descs, int n, BatchSetup &s, void *host);
// Launch the batch kernel over an arena already in device memory.
// pdl: the register-window kernel may be placed while the kernel before it
// on the stream finishes (it waits for it on entry); worth it only where
// no other operation stands between the two.
cudaError_t launch_planned(const BatchSetup &s, void *arena_dev, cudaStream_t stream,
                           bool pdl = true);

// A ring of batch launch slots (pinned staging, device arena, cached
// graphs).  launch() is thread-safe; a slot is reused only after its last
// launch completed (waits for it if needed).
class BatchRing {
   public:
    explicit BatchRing(int nslots);
    ~BatchRing();
    BatchRing(const BatchRing &) = delete;
    BatchRing &operator=(const BatchRing &) = delete;
    int launch(const me_desc *descs, int n, cudaStream_t stream);
    void release();

   private:
    struct Slot;
    int n_;
    int next_ = 0;
    Slot *slots_;
    cudaStream_t copy_ = nullptr;   // uploads plans beside the caller's stream
    std::mutex mu_;
};

// Release the host-batch pipelines (streams, device slots) on every device.
int host_pipes_shutdown();

// Scratch from the library's stream-ordered pool on the current device
// (kept reserved between calls up to a limit; me_shutdown destroys it).
cudaError_t scratch_alloc(void **p, size_t bytes, cudaStream_t s);
cudaError_t scratch_free(void *p, cudaStream_t s);
int scratch_shutdown();

// Forget the device addresses me_edges_staged_static has cached.
void static_forget_all();

// The five staged passes.
cudaError_t launch_staged(const Geo &g, uint32_t *mask, uint32_t *edge,
                          cudaStream_t s);

}  // namespace me
