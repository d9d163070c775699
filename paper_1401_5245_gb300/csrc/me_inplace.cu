// me_edges_inplace: the edge map written over the image it is computed from.
//
// Every output row needs the original rows above and below it, so a row may
// be overwritten only once nobody still has to read it.  The image is cut
// into bands of band_rows rows; one CTA owns a band across the whole row
// width and walks it top to bottom, G rows at a time.  Each thread owns up
// to C vector columns of 4 words and copies its columns of the rows ahead
// (cp.async, one commit group per row) into a ring of Q rows in shared
// memory.  Per group: wait for this thread's copies up to the group's last
// row below, one barrier (everyone's copies are then visible, and everyone
// has finished the previous group, whose oldest ring slots are refilled
// next), issue the next G rows, then compute the group's rows from the ring
// -- own columns and the neighbouring columns' end words alike -- and
// overwrite them in global memory.  A thread reads global memory only at
// its own columns, and each row's copy has landed before the row is
// overwritten.
//
// Between CTAs the only shared rows are at the band seams: the last row of
// a band is the row above the next band, and the first row of a band is the
// row below the previous one.  A first small kernel saves those two rows
// of every seam into scratch before any band starts, and bands read their
// outer halo rows from there.
//
// A band is one row wide in threads and a chain of memory round trips in
// time, so images of a few bands per SM leave the GPU mostly idle.  Images
// up to kCopyMax bytes (or ME_INPLACE_COPY_MAX) are instead copied to
// scratch whole and computed by
// the out-of-place kernel from the copy onto the image: twice the traffic,
// but all of it parallel (measured on GB300: a 4096 x 4096 image in about
// 7 us against 20 us by bands; at 16384 x 16384 the two meet).
#include <algorithm>
#include <cstdlib>
#include <mutex>

#include "me_internal.h"
#include "me_ptx.cuh"

namespace me {

namespace {

constexpr int kIpMaxThreads = 1024;
constexpr size_t kCopyMax = 32ull << 20;   // whole-image copy up to 32 MiB

// The whole-image copy limit: ME_INPLACE_COPY_MAX (bytes) if set, else kCopyMax.
size_t copy_max() {
    const char *v = std::getenv("ME_INPLACE_COPY_MAX");
    if (v == nullptr || *v == 0) return kCopyMax;
    char *end = nullptr;
    const unsigned long long x = std::strtoull(v, &end, 10);
    return (end != nullptr && *end == 0) ? (size_t)x : kCopyMax;
}

struct IpGeo {
    uint32_t *img;
    const uint32_t *seam;               // rows 2k, 2k+1: seam k (bands k, k+1)
    int32_t h, stride, nw, nv;          // nv = vector columns of 4 words
    uint32_t lastmask, fill;
    int32_t band_rows, nbands;
};

__device__ __forceinline__ uint32_t ip_keep(const IpGeo &g, int c) {
    return (c >= 0 && c < g.nw - 1) ? kAllOnes : (c == g.nw - 1 ? g.lastmask : 0u);
}

// Where row y comes from for band b: the image inside the band, the seam
// copies for the rows just outside it, nothing (boundary colour) beyond.
__device__ __forceinline__ const uint32_t *ip_row(const IpGeo &g, int b, int y0, int y1, int y) {
    if (y >= y0 && y < y1) return g.img + (size_t)y * (size_t)g.stride;
    if (y == y0 - 1 && y >= 0) return g.seam + (size_t)(2 * (b - 1)) * (size_t)g.stride;
    if (y == y1 && y < g.h) return g.seam + (size_t)(2 * b + 1) * (size_t)g.stride;
    return nullptr;
}

template <int C, bool V16, int Q, int G>
__global__ void __launch_bounds__(kIpMaxThreads)
k_inplace(IpGeo g) {
    static_assert(Q >= 2 * G + 2, "the ring holds a group, its halo rows and the rows ahead");
    extern __shared__ uint4 s_ring[];              // [Q][C * T]
    const int b = blockIdx.x;
    const int y0 = b * g.band_rows;
    const int y1 = min(y0 + g.band_rows, g.h);
    const int T = blockDim.x;
    const int CT = C * T;

    int vcol[C];
    bool active[C];
#pragma unroll
    for (int k = 0; k < C; ++k) {
        vcol[k] = threadIdx.x + k * T;
        active[k] = vcol[k] < g.nv;
    }
    // ring slot of row r (r >= y0 - 1)
    auto slot = [&](int r) { return (r - y0 + 1) % Q; };
    // this thread's columns of row r into the ring (nothing for rows
    // without a source); one commit group per row in any case
    auto issue = [&](int r) {
        const uint32_t *row = ip_row(g, b, y0, y1, r);
        if (row != nullptr) {
            uint4 *dst = s_ring + slot(r) * CT;
#pragma unroll
            for (int k = 0; k < C; ++k) {
                const int c0 = vcol[k] * 4;
                if (!active[k]) continue;
                if constexpr (V16) {
                    if (c0 < g.nw) cp_async16(dst + vcol[k], row + c0);
                } else {
#pragma unroll
                    for (int i = 0; i < 4; ++i)
                        if (c0 + i < g.nw)
                            cp_async4(reinterpret_cast<uint32_t *>(dst + vcol[k]) + i, row + c0 + i);
                }
            }
        }
        cp_async_commit();
    };
    // this thread's keep masks: its 4 words, and the words just beside them
    uint32_t keep[C][4], keep_l[C], keep_r[C];
#pragma unroll
    for (int k = 0; k < C; ++k) {
#pragma unroll
        for (int i = 0; i < 4; ++i) keep[k][i] = ip_keep(g, vcol[k] * 4 + i);
        keep_l[k] = ip_keep(g, vcol[k] * 4 - 1);
        keep_r[k] = ip_keep(g, vcol[k] * 4 + 4);
    }
    const uint4 fill4 = make_uint4(g.fill, g.fill, g.fill, g.fill);
    auto fix = [&](uint32_t raw, uint32_t keep) { return (raw & keep) | (g.fill & ~keep); };
    auto fix4 = [&](uint4 r, const uint32_t (&kp)[4]) {
        return make_uint4(fix(r.x, kp[0]), fix(r.y, kp[1]), fix(r.z, kp[2]), fix(r.w, kp[3]));
    };

    // launched while the seam kernel may still run (programmatic dependent
    // launch): wait for it to finish before the first read of the image or
    // the seam rows
    asm volatile("griddepcontrol.wait;" ::: "memory");
    for (int r = y0 - 1; r <= y0 + Q - G - 2; ++r) issue(r);

    const int lane = threadIdx.x & 31;
#pragma unroll 1
    for (int y = y0; y < y1; y += G) {
        cp_async_wait<Q - 2 * G - 2>();            // own copies of rows <= y + G
        __syncthreads();
        for (int r = y + Q - G - 1; r <= y + Q - 2; ++r) issue(r);
        int s_up = slot(y - 1);                    // ring slots of rows y - 1, y, y + 1
        int s_cur = s_up + 1 == Q ? 0 : s_up + 1;
#pragma unroll
        for (int j = 0; j < G; ++j) {
            const int yy = y + j;
            if (yy >= y1) break;
            const int s_dn = s_cur + 1 == Q ? 0 : s_cur + 1;
            // rows y0 - 1 .. y1 all have a source when they lie in the image
            const bool have_up = yy >= 1, have_dn = yy + 1 < g.h;
#pragma unroll
            for (int k = 0; k < C; ++k) {
                const int v = vcol[k];
                // the row's own words are fixed (their padding bits reach
                // pixels through the shifts); above and below, padding bits
                // meet only output bits that keep clears
                const uint4 c = fix4(s_ring[s_cur * CT + v], keep[k]);
                const uint4 u = have_up ? s_ring[s_up * CT + v] : fill4;
                const uint4 d = have_dn ? s_ring[s_dn * CT + v] : fill4;
                // the words beside: warp neighbours, the ring at the warp's ends
                uint32_t lw = __shfl_up_sync(0xFFFFFFFFu, c.w, 1);
                uint32_t rw = __shfl_down_sync(0xFFFFFFFFu, c.x, 1);
                if (lane == 0)
                    lw = v > 0 ? fix(reinterpret_cast<const uint32_t *>(
                                         s_ring + s_cur * CT + v - 1)[3], keep_l[k])
                               : g.fill;
                if (lane == 31)
                    rw = v + 1 < CT ? fix(s_ring[s_cur * CT + v + 1].x, keep_r[k]) : g.fill;
                const uint32_t cw[6] = {lw, c.x, c.y, c.z, c.w, rw};
                const uint32_t uw[4] = {u.x, u.y, u.z, u.w}, dw[4] = {d.x, d.y, d.z, d.w};
                uint32_t e[4];
#pragma unroll
                for (int i = 0; i < 4; ++i) {
                    const uint32_t x = cw[1 + i];
                    const uint32_t L = __funnelshift_l(cw[i], x, 1);       // I(x-1, y)
                    const uint32_t R = __funnelshift_r(x, cw[2 + i], 1);   // I(x+1, y)
                    e[i] = ~x & (L | R | uw[i] | dw[i]) & keep[k][i];
                }
                if (active[k]) {
                    uint32_t *out = g.img + (size_t)yy * (size_t)g.stride + v * 4;
                    if constexpr (V16) {
                        *reinterpret_cast<uint4 *>(out) = make_uint4(e[0], e[1], e[2], e[3]);
                    } else {
#pragma unroll
                        for (int i = 0; i < 4; ++i)
                            if (v * 4 + i < g.stride) out[i] = e[i];
                    }
                }
            }
            s_up = s_cur;
            s_cur = s_dn;
        }
    }
    cp_async_wait<0>();
}

// The seam rows into scratch before any band starts: CTA k copies rows
// (k+1) B - 1 and (k+1) B, which lie next to each other, as one run of
// 2 * stride words (16-byte units when the rows allow them).
template <bool V16>
__global__ void __launch_bounds__(256)
k_seams(const uint32_t *img, uint32_t *seam, int32_t stride, int32_t band_rows) {
    // launched while the kernel before it on the stream may still run (an
    // earlier call's bands, possibly on this image): wait for it to end
    // before reading; the band kernel may be scheduled now, and it waits
    // for this grid to end before it reads anything
    asm volatile("griddepcontrol.wait;" ::: "memory");
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
    const size_t words = 2 * (size_t)stride;
    const uint32_t *src = img + ((size_t)(blockIdx.x + 1) * band_rows - 1) * (size_t)stride;
    uint32_t *dst = seam + (size_t)blockIdx.x * words;
    if constexpr (V16) {
        const uint4 *s4 = reinterpret_cast<const uint4 *>(src);
        uint4 *d4 = reinterpret_cast<uint4 *>(dst);
        for (size_t i = threadIdx.x; i < words / 4; i += blockDim.x) d4[i] = s4[i];
    } else {
        for (size_t i = threadIdx.x; i < words; i += blockDim.x) dst[i] = src[i];
    }
}

template <int C, int Q>
constexpr size_t inplace_smem(int threads) {
    return (size_t)Q * C * threads * sizeof(uint4);
}

template <int C, bool V16, int Q, int G>
cudaError_t launch_inplace(const IpGeo &g, int threads, cudaStream_t s) {
    // the ring exceeds the default 48 KiB for wide rows; raise the limit
    // once per device (the attribute belongs to the device's context)
    static std::mutex mu;
    static bool done[64] = {};
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    {
        std::lock_guard<std::mutex> lk(mu);
        if (dev >= 64 || !done[dev]) {
            e = cudaFuncSetAttribute(k_inplace<C, V16, Q, G>,
                                     cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)inplace_smem<C, Q>(kIpMaxThreads));
            if (e != cudaSuccess) return e;
            if (dev < 64) done[dev] = true;
        }
    }
    // programmatic dependent launch: the band kernel's CTAs are placed and
    // set up while the seam kernel before it finishes
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(g.nbands);
    cfg.blockDim = dim3(threads);
    cfg.dynamicSmemBytes = inplace_smem<C, Q>(threads);
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    e = cudaLaunchKernelEx(&cfg, k_inplace<C, V16, Q, G>, g);
    if (e != cudaSuccess) cudaGetLastError();
    return e;
}

}  // namespace

}  // namespace me

using namespace me;

extern "C" int me_edges_inplace(uint32_t *img, int32_t w, int32_t h, int32_t stride_words,
                                int32_t boundary, me_stream_t stream) {
    if (img == nullptr || w <= 0 || h <= 0 || stride_words <= 0 ||
        stride_words < (int32_t)(((int64_t)w + 31) / 32) ||
        (boundary != ME_BOUNDARY_WHITE && boundary != ME_BOUNDARY_BLACK) ||
        ((uintptr_t)img & 3))
        return ME_ERR_ARG;
    int rc = check_device_ptr(img);
    if (rc != ME_OK) return rc;
    const cudaStream_t s = (cudaStream_t)stream;
    const size_t img_bytes = (size_t)h * (size_t)stride_words * 4;
    if (img_bytes <= copy_max()) {
        uint32_t *copy = nullptr;
        cudaError_t e = scratch_alloc(reinterpret_cast<void **>(&copy), img_bytes, s);
        if (e != cudaSuccess) {
            cudaGetLastError();
            return record_cuda(e);
        }
        e = cudaMemcpyAsync(copy, img, img_bytes, cudaMemcpyDeviceToDevice, s);
        if (e == cudaSuccess) {
            rc = me_edges(copy, w, h, stride_words, img, boundary, stream);
            if (rc != ME_OK) e = cudaErrorLaunchFailure;
        }
        const cudaError_t f = scratch_free(copy, s);
        if (e != cudaSuccess || f != cudaSuccess) {
            cudaGetLastError();
            return rc != ME_OK ? rc : record_cuda(e != cudaSuccess ? e : f);
        }
        return ME_OK;
    }
    DevInfo di;
    if ((rc = device_info(&di)) != ME_OK) return rc;
    const Geo geo = make_geo(img, w, h, stride_words, boundary, 4,
                             vec16_ok(img, img, stride_words));
    const int nv = geo.nv;
    const int C = nv <= kIpMaxThreads ? 1 : 2;
    if (nv > 2 * kIpMaxThreads) return ME_ERR_TOO_BIG;
    const int threads = std::max(32, ((nv + C - 1) / C + 31) / 32 * 32);

    IpGeo g;
    g.img = img;
    g.seam = nullptr;
    g.h = h;
    g.stride = stride_words;
    g.nw = geo.nw;
    g.nv = nv;
    g.lastmask = geo.lastmask;
    g.fill = geo.fill;
    // bands: about four CTAs per SM, at least 32 rows (seam copies stay
    // below 2 rows in 32 of extra traffic)
    const int64_t want = (int64_t)di.sm_count * 4;
    g.band_rows = (int32_t)std::max<int64_t>(32, (h + want - 1) / want);
    g.nbands = (int32_t)(((int64_t)h + g.band_rows - 1) / g.band_rows);

    uint32_t *seam = nullptr;
    cudaError_t e = cudaSuccess;
    if (g.nbands > 1) {
        const size_t bytes = (size_t)2 * (g.nbands - 1) * (size_t)stride_words * 4;
        if ((e = scratch_alloc(reinterpret_cast<void **>(&seam), bytes, s)) != cudaSuccess) {
            cudaGetLastError();
            return record_cuda(e);
        }
        g.seam = seam;
        cudaLaunchConfig_t lc = {};
        lc.gridDim = dim3(g.nbands - 1);
        lc.blockDim = dim3(256);
        lc.stream = s;
        cudaLaunchAttribute attr[1];
        attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
        attr[0].val.programmaticStreamSerializationAllowed = 1;
        lc.attrs = attr;
        lc.numAttrs = 1;
        const uint32_t *cimg = img;
        e = geo.vec16 ? cudaLaunchKernelEx(&lc, k_seams<true>, cimg, seam, stride_words,
                                           g.band_rows)
                      : cudaLaunchKernelEx(&lc, k_seams<false>, cimg, seam, stride_words,
                                           g.band_rows);
    }
    if (e == cudaSuccess) {
        // rows of up to 1024 columns: a 12-row ring, 4 rows per barrier;
        // wider ones: 6 rows, 2 per barrier (at most 192 KiB either way)
        if (geo.vec16)
            e = C == 1 ? launch_inplace<1, true, 12, 4>(g, threads, s)
                       : launch_inplace<2, true, 6, 2>(g, threads, s);
        else
            e = C == 1 ? launch_inplace<1, false, 12, 4>(g, threads, s)
                       : launch_inplace<2, false, 6, 2>(g, threads, s);
    }
    if (seam != nullptr) {
        const cudaError_t f = scratch_free(seam, s);
        if (e == cudaSuccess) e = f;
    }
    if (e != cudaSuccess) {
        cudaGetLastError();
        return record_cuda(e);
    }
    return ME_OK;
}
