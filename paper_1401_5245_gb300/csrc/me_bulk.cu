// Bulk-copy (TMA) engine of the fused method of masks.
//
// Persistent CTAs; CTA g owns a contiguous run of bands (row bands of one
// image, top to bottom, column strip after column strip), so the halo rows
// a band re-reads were copied moments before for the previous band and come
// from L2.  One producer warp walks the run ahead of the consumers: as soon
// as a stage is released it arms the stage's mbarrier with the byte count
// and issues cp.async.bulk copies (one per band when the band is whole rows
// -- contiguous in memory -- else one per row).  The consumer warps wait on
// a stage, compute every output word of its band from shared memory, store
// them with 128-bit streaming stores and release the stage.  Images whose
// rows are not 16-byte aligned take the same path with plain cooperative
// loads into the stage.
//
// Per output word (least significant bit = leftmost pixel):
//   E = ~I & ((I << 1 | prev >> 31) | (I >> 1 | next << 31) | up | down)
// i.e. the mask (Section 3) ANDed with the image moved one pixel right,
// left, down and up (Section 4), the four results ORed (Section 5).
#include <algorithm>
#include <cstring>
#include <mutex>

#include "me_internal.h"
#include "me_ptx.cuh"

namespace me {

// Set when a bounded wait ran out; read and cleared by me_device_faults.
__device__ unsigned int g_me_fault_flags = 0;
constexpr unsigned int kFaultBulkWait = 1u;

constexpr int kMaxStages = 8;
constexpr int kMaxBulkThreads = 512 + 32;  // consumers + one producer warp
constexpr int kHalo = 4;                 // halo words each side in column mode

namespace {

// Where band `local` of image d sits, and what to copy for it.
struct Band {
    int y0, rows;           // output rows [y0, y0 + rows)
    int x0, words;          // output words [x0, x0 + words)
    int ya, yb;             // copied rows [ya, yb)
    int xb;                 // image word held by stage column 0
    int xs, xe;             // copied words [xs, xe)
};

__device__ __forceinline__ Band band_of(const KDescB &d, int local) {
    Band b;
    const int cb = local / d.nrb;
    const int rb = local - cb * d.nrb;
    b.y0 = rb * d.band_rows;
    b.rows = min(d.band_rows, d.h - b.y0);
    b.x0 = cb * d.band_words;
    b.words = min(d.band_words, d.stride - b.x0);     // padding words are written 0
    b.ya = max(0, b.y0 - 1);
    b.yb = min(d.h, b.y0 + d.band_rows + 1);
    if (d.flags & kRowMode) {
        b.xb = 0;
        b.xs = 0;
        b.xe = d.stride;
    } else {
        b.xb = b.x0 - kHalo;
        b.xs = max(0, b.xb);
        b.xe = min(d.stride, b.x0 + d.band_words + kHalo);
    }
    return b;
}

// Bits of image word x that hold pixels (0 for words outside the row).
__device__ __forceinline__ uint32_t col_keep(const KDescB &d, int x) {
    return x < d.nw - 1 ? kAllOnes : (x == d.nw - 1 ? d.lastmask : 0u);
}

// Warp 0: start the copies of band `local` of image d into `stage`.
__device__ __forceinline__ void produce(const KDescB &d, int local, uint32_t *stage,
                                        uint64_t *bar, int lane) {
    const Band b = band_of(d, local);
    if (!(d.flags & kBulkCopy)) {
        // the consumers load this band themselves; just complete the phase
        if (lane == 0) mbar_arrive(bar);
        return;
    }
    const int nrows = b.yb - b.ya;
    const int nwords = b.xe - b.xs;
    if (lane == 0) {
        fence_proxy_async_smem();
        mbar_arrive_expect_tx(bar, (uint32_t)(nrows * nwords * 4));
    }
    __syncwarp();
    if (d.flags & kRowMode) {
        if (lane == 0)
            bulk_g2s(stage, d.img + (size_t)b.ya * d.stride, (uint32_t)(nrows * nwords * 4), bar);
    } else {
        for (int r = lane; r < nrows; r += 32)
            bulk_g2s(stage + (size_t)r * d.pitch + (b.xs - b.xb),
                     d.img + (size_t)(b.ya + r) * d.stride + b.xs, (uint32_t)(nwords * 4), bar);
    }
}

// Barrier among the consumer warps only (the producer warp keeps running).
__device__ __forceinline__ void consumers_sync(int nthreads) {
    asm volatile("bar.sync 1, %0;" ::"r"(nthreads) : "memory");
}

// Consumer threads tid = 0 .. nthreads-1: the band's output words from the
// stage.
__device__ __forceinline__ void consume(const KDescB &d, int local, uint32_t *stage, int tid,
                                        int nthreads) {
    const Band b = band_of(d, local);
    if (!(d.flags & kBulkCopy)) {
        const int nrows = b.yb - b.ya, nwords = b.xe - b.xs;
        for (int i = tid; i < nrows * nwords; i += nthreads) {
            const int r = i / nwords, c = i - r * nwords;
            stage[r * d.pitch + (b.xs - b.xb) + c] =
                __ldg(d.img + (size_t)(b.ya + r) * d.stride + b.xs + c);
        }
        consumers_sync(nthreads);
    }
    // Lanes form row segments of nvp lanes, one 4-word group each (narrow
    // bands fold the warp).  A segment walks a run of rows of one column
    // block, keeping the rows above, at and below the output row in
    // registers; the words left and right of its group come from shared
    // memory, so segments never exchange data and may diverge freely.
    const int ncol4 = (b.words + 3) >> 2;
    const int seg_log2 = ncol4 >= 32 ? 5 : 32 - __clz(ncol4 - 1);
    const int nvp = 1 << seg_log2;
    const int ncb = (ncol4 + nvp - 1) >> seg_log2;
    const int nseg = (nthreads >> 5) << (5 - seg_log2);
    const int rr = max(4, (b.rows * ncb + nseg - 1) / nseg);
    const int nruns = (b.rows + rr - 1) / rr;
    const int units = ncb * nruns;
    const int lane = tid & 31;
    const int col = lane & (nvp - 1);
    const int gseg = ((tid >> 5) << (5 - seg_log2)) + (lane >> seg_log2);
    const bool vec_store = (d.flags & kVecStore) != 0;
    for (int u = gseg; u < units; u += nseg) {
        const int cb = u % ncb, run = u / ncb;
        const int x = b.x0 + 4 * (cb * 32 + col);
        if (x >= b.x0 + b.words) continue;
        const int ys = b.y0 + run * rr;
        const int ye = min(ys + rr, b.y0 + b.rows);
        // outside colour per word of the group: fixed = (raw & keep) | fb
        uint32_t keep[4], fb[4];
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            keep[k] = col_keep(d, x + k);
            fb[k] = d.fill & ~keep[k];
        }
        const uint32_t nkeep = col_keep(d, x + 4), nfb = d.fill & ~nkeep;
        const uint32_t pkeep = x > 0 ? kAllOnes : 0u, pfb = d.fill & ~pkeep;
        const int cx = x - b.xb;                         // stage column of word x
        const int cp = max(cx - 1, 0), cn = min(cx + 4, d.pitch - 1);
        const uint32_t *srow = stage + (size_t)(ys - b.ya) * d.pitch;
        uint32_t up[4], cur[4], cur_p, cur_n;
        if (ys > 0) {
            const uint4 v = lds128(srow - d.pitch + cx);
            up[0] = (v.x & keep[0]) | fb[0]; up[1] = (v.y & keep[1]) | fb[1];
            up[2] = (v.z & keep[2]) | fb[2]; up[3] = (v.w & keep[3]) | fb[3];
        } else {
            up[0] = up[1] = up[2] = up[3] = d.fill;
        }
        {
            const uint4 v = lds128(srow + cx);
            cur[0] = (v.x & keep[0]) | fb[0]; cur[1] = (v.y & keep[1]) | fb[1];
            cur[2] = (v.z & keep[2]) | fb[2]; cur[3] = (v.w & keep[3]) | fb[3];
            cur_p = (srow[cp] & pkeep) | pfb;
            cur_n = (srow[cn] & nkeep) | nfb;
        }
        uint32_t *orow = d.edge + (size_t)ys * d.stride + x;
        for (int y = ys; y < ye; ++y) {
            srow += d.pitch;
            uint32_t dn[4], dn_p, dn_n;
            if (y + 1 < d.h) {
                const uint4 v = lds128(srow + cx);
                dn[0] = (v.x & keep[0]) | fb[0]; dn[1] = (v.y & keep[1]) | fb[1];
                dn[2] = (v.z & keep[2]) | fb[2]; dn[3] = (v.w & keep[3]) | fb[3];
                dn_p = (srow[cp] & pkeep) | pfb;
                dn_n = (srow[cn] & nkeep) | nfb;
            } else {
                dn[0] = dn[1] = dn[2] = dn[3] = dn_p = dn_n = d.fill;
            }
            uint32_t e[4];
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                const uint32_t pv = k == 0 ? cur_p : cur[k - 1];
                const uint32_t nx = k == 3 ? cur_n : cur[k + 1];
                const uint32_t L = __funnelshift_l(pv, cur[k], 1);   // I(x-1, y)
                const uint32_t R = __funnelshift_r(cur[k], nx, 1);   // I(x+1, y)
                e[k] = ~cur[k] & (L | R | up[k] | dn[k]) & keep[k];
            }
            if (vec_store) {
                // stride % 4 == 0: the group lies inside the row
                __stcs(reinterpret_cast<uint4 *>(orow), make_uint4(e[0], e[1], e[2], e[3]));
            } else {
#pragma unroll
                for (int k = 0; k < 4; ++k)
                    if (x + k < d.stride) __stcs(orow + k, e[k]);
            }
            orow += d.stride;
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                up[k] = cur[k];
                cur[k] = dn[k];
            }
            cur_p = dn_p;
            cur_n = dn_n;
        }
    }
}

}  // namespace

// SINGLE: one image passed by value (nbands bands); else the batch arena.
// Warp-specialised: the last warp produces, the others consume.  Stage s
// has two barriers: full[s] (armed by the producer with the copy's byte
// count, completed by the copies) and empty[s] (one arrival per consumer
// warp once it has finished reading the stage).  The producer refills a
// stage as soon as it is empty, so all other stages stay in flight while the
// consumers work; no CTA-wide barrier runs inside the loop.
template <bool SINGLE>
__global__ void __launch_bounds__(kMaxBulkThreads)
k_bulk(const BatchHeader *__restrict__ hdr, KDescB one, int nbands, int stage_words,
       int stages) {
    extern __shared__ __align__(128) uint32_t smem[];
    __shared__ uint64_t full[kMaxStages], empty[kMaxStages];
    const KDescB *descs = SINGLE ? nullptr : reinterpret_cast<const KDescB *>(hdr + 1);
    const int G = SINGLE ? (int)gridDim.x : hdr->total_warps;
    const int64_t B = SINGLE ? nbands : hdr->total_tasks;
    if ((int)blockIdx.x >= G) return;
    const int b_begin = (int)((B * blockIdx.x) / G);
    const int b_end = (int)((B * (blockIdx.x + 1)) / G);
    if (b_begin >= b_end) return;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int ncons = (int)(blockDim.x >> 5) - 1;

    if (threadIdx.x == 0) {
        for (int s = 0; s < stages; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], (uint32_t)ncons);
        }
        fence_mbar_init();
    }
    __syncthreads();

    int cur = 0;                 // image cursor of this warp
    if (!SINGLE) {
        const int32_t *first = reinterpret_cast<const int32_t *>(descs + hdr->n);
        cur = first[blockIdx.x];
    }
    auto image_of = [&](int b) -> KDescB {
        if constexpr (SINGLE) {
            return one;
        } else {
            while (b >= descs[cur].band_base + descs[cur].ncb * descs[cur].nrb) ++cur;
            return descs[cur];
        }
    };

    if (warp == ncons) {
        // producer
        for (int b = b_begin, i = 0; b < b_end; ++b, ++i) {
            const int s = i % stages;
            if (i >= stages && !mbar_wait(&empty[s], (uint32_t)(((i / stages) - 1) & 1))) {
                if (lane == 0) atomicOr(&g_me_fault_flags, kFaultBulkWait);
                break;
            }
            const KDescB d = image_of(b);
            produce(d, b - (SINGLE ? 0 : d.band_base), smem + (size_t)s * stage_words, &full[s],
                    lane);
        }
    } else {
        // consumers
        const int nthreads = ncons * 32;
        for (int b = b_begin, i = 0; b < b_end; ++b, ++i) {
            const int s = i % stages;
            if (!mbar_wait(&full[s], (uint32_t)((i / stages) & 1))) {
                if (lane == 0) atomicOr(&g_me_fault_flags, kFaultBulkWait);
                break;
            }
            const KDescB d = image_of(b);
            consume(d, b - (SINGLE ? 0 : d.band_base), smem + (size_t)s * stage_words,
                    (int)threadIdx.x, nthreads);
            __syncwarp();
            if (lane == 0) mbar_arrive(&empty[s]);
        }
    }
}

// ------------------------------------------------------------------ host
bool bulk_available() { return true; }

void bulk_geometry(const Geo &g, const void *edge, int stage_words, KDescB *d) {
    std::memset(d, 0, sizeof(*d));
    d->img = g.img;
    d->edge = static_cast<uint32_t *>(const_cast<void *>(edge));
    d->h = g.h;
    d->stride = g.stride;
    d->nw = g.nw;
    d->lastmask = g.lastmask;
    d->fill = g.fill;
    const bool aligned = ((uintptr_t)g.img % 16 == 0) && (g.stride % 4 == 0);
    d->flags = (aligned ? kBulkCopy : 0) |
               (((uintptr_t)edge % 16 == 0 && g.stride % 4 == 0) ? kVecStore : 0);
    const int row_words = (g.stride + 3) / 4 * 4;     // stage pitch of whole rows
    // option A: whole rows, one contiguous copy per band (needs aligned rows)
    double cost_a = 1e9;
    int rows_a = 0;
    if (stage_words / row_words >= 3) {
        rows_a = stage_words / row_words - 2;
        const int eff = std::min(rows_a, g.h);
        cost_a = (double)(std::min(eff + 2, g.h) - eff) / eff;
    }
    // option B: column strips of band_words words with 4 halo words a side
    double cost_b = 1e9;
    int rows_b = 0, words_b = 0;
    for (int r : {8, 16, 32, 64, 128}) {
        const int pitch = stage_words / (r + 2) / 4 * 4;
        const int bw = pitch - 2 * kHalo;
        if (bw < 32) continue;
        const int eff_r = std::min(r, g.h);
        const double c = (double)(std::min(eff_r + 2, g.h) - eff_r) / eff_r +
                         (double)(2 * kHalo) / std::min(bw, g.stride + 2 * kHalo);
        if (c < cost_b) {
            cost_b = c;
            rows_b = r;
            words_b = bw;
        }
    }
    if (rows_a > 0 && cost_a <= cost_b) {
        d->flags |= kRowMode;
        d->band_rows = rows_a;
        d->band_words = g.stride;
        d->pitch = aligned ? g.stride : row_words;
        d->ncb = 1;
    } else {
        d->band_rows = rows_b;
        d->band_words = words_b;
        d->pitch = words_b + 2 * kHalo;
        d->ncb = (g.stride + words_b - 1) / words_b;
    }
    d->nrb = (g.h + d->band_rows - 1) / d->band_rows;
}

const void *bulk_kernel() { return reinterpret_cast<const void *>(k_bulk<false>); }

size_t bulk_smem_bytes(const me_tile_cfg &cfg) {
    return (size_t)cfg.stages * cfg.stage_kb * 1024;
}

static int ensure_smem_attr(const void *fn, size_t bytes) {
    static std::mutex mu;
    static size_t done[64][2] = {};
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return record_cuda(e);
    const int k = (fn == reinterpret_cast<const void *>(k_bulk<true>)) ? 0 : 1;
    std::lock_guard<std::mutex> lk(mu);
    if (dev < 64 && done[dev][k] >= bytes) return ME_OK;
    e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return record_cuda(e);
    }
    if (dev < 64) done[dev][k] = bytes;
    return ME_OK;
}

int bulk_ctas_per_sm(const me_tile_cfg &cfg, int *out) {
    const void *fn = bulk_kernel();
    const size_t smem = bulk_smem_bytes(cfg);
    int rc = ensure_smem_attr(fn, smem);
    if (rc != ME_OK) return rc;
    return cached_occupancy(fn, bulk_threads(cfg), smem, out);
}

cudaError_t launch_bulk(const Geo &g, uint32_t *edge, const me_tile_cfg &cfg, cudaStream_t s) {
    const void *fn = reinterpret_cast<const void *>(k_bulk<true>);
    const size_t smem = bulk_smem_bytes(cfg);
    if (ensure_smem_attr(fn, smem) != ME_OK) return cudaErrorInvalidValue;
    KDescB d;
    bulk_geometry(g, edge, (int)(smem / cfg.stages / 4), &d);
    const int64_t nbands = (int64_t)d.ncb * d.nrb;
    if (nbands > INT32_MAX) return cudaErrorInvalidValue;
    DevInfo di;
    if (device_info(&di) != ME_OK) return cudaErrorInvalidDevice;
    int occ = 0;
    if (cached_occupancy(fn, bulk_threads(cfg), smem, &occ) != ME_OK)
        return cudaErrorInvalidValue;
    if (occ < 1) return cudaErrorInvalidConfiguration;
    const int per_sm = cfg.ctas_per_sm > 0 ? std::min(cfg.ctas_per_sm, occ) : occ;
    const int grid = (int)std::max<int64_t>(1, std::min<int64_t>(nbands, (int64_t)di.sm_count * per_sm));
    k_bulk<true><<<grid, bulk_threads(cfg), smem, s>>>(nullptr, d, (int)nbands,
                                                     (int)(smem / cfg.stages / 4), cfg.stages);
    return cudaGetLastError();
}

int plan_batch_bulk(const me_desc *descs, int n, const me_tile_cfg &cfg, int grid,
                    void *host_arena, int64_t *total_bands) {
    const int stage_words = (int)(bulk_smem_bytes(cfg) / cfg.stages / 4);
    BatchHeader *hdr = static_cast<BatchHeader *>(host_arena);
    KDescB *kd = reinterpret_cast<KDescB *>(hdr + 1);
    int32_t *first = reinterpret_cast<int32_t *>(kd + n);
    std::memset(hdr, 0, sizeof(*hdr));
    int64_t total = 0, bytes = 0;
    for (int i = 0; i < n; ++i) {
        const me_desc &d = descs[i];
        int rc = check_image_args(d.img, d.edge, d.w, d.h, d.stride_words, d.boundary);
        if (rc != ME_OK) return rc;
        bulk_geometry(make_geo(d.img, d.w, d.h, d.stride_words, d.boundary, 1), d.edge,
                      stage_words, &kd[i]);
        kd[i].band_base = (int32_t)total;
        total += (int64_t)kd[i].ncb * kd[i].nrb;
        if (total > INT32_MAX) return ME_ERR_ARG;
        bytes += 2 * (int64_t)d.h * d.stride_words * 4;
    }
    hdr->n = n;
    hdr->total_tasks = (int32_t)total;
    hdr->total_warps = grid;                  // band owners: CTAs
    hdr->rows_per_lane = 0;
    hdr->bytes = bytes;
    int i = 0;
    for (int g = 0; g < grid; ++g) {
        const int64_t b0 = (total * g) / grid;
        while (i < n - 1 && b0 >= (int64_t)kd[i].band_base + (int64_t)kd[i].ncb * kd[i].nrb) ++i;
        first[g] = i;
    }
    first[grid] = n > 0 ? n - 1 : 0;
    *total_bands = total;
    return ME_OK;
}

unsigned int device_fault_flags(bool clear) {
    unsigned int v = 0;
    if (cudaMemcpyFromSymbol(&v, g_me_fault_flags, sizeof(v)) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    if (clear) {
        const unsigned int z = 0;
        cudaMemcpyToSymbol(g_me_fault_flags, &z, sizeof(z));
    }
    return v;
}

}  // namespace me
