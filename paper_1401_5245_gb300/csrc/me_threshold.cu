// Thresholding ahead of the method of masks, fused (Section 7: a grey
// photograph is made binary, then its edges are found).  One pass reads the
// 8-bit image, makes each 32-pixel word on the fly (white where grey >= t),
// and writes the edge map (and, if asked, the binary image) packed.
//
// A warp walks a band of rows of one column block of kWideLanes packed
// words, top to bottom: lanes 1..30 produce those words, lanes 0 and 31 make
// the words just left and right of the block, so every neighbour word comes
// from a shuffle.  Each row of the band (and the one row above and below it)
// is loaded and thresholded once, and the words of the rows above and at the
// current row are carried down.  A task starts by requesting its first six
// rows at once; after that, each row's load is issued as the row four above
// it is consumed, so four rows per warp stay in flight.  The band height is
// chosen on the host from the number of resident warps (few waves, little
// idle tail).
//
// With Otsu's rule the threshold comes from the image itself, on the
// device: a histogram pass, one CTA that scores every threshold, and the
// same walk reading the chosen threshold from device memory.
#include <algorithm>

#include "me_internal.h"

namespace me {

namespace {

constexpr int kThrWarps = 8;    // warps per CTA

struct TGeo {
    const uint8_t *grey;
    uint32_t *edge, *binary;            // binary may be null
    int32_t w, h, pitch;                // pitch: bytes per grey row
    int32_t stride, nw, ncb;            // output words per row, words with pixels, blocks
    int32_t band;                       // rows per task (a multiple of kThrRows)
    uint32_t lastmask, fill;
    uint32_t t4;                        // 256 - threshold in every byte
};

struct Raw {
    uint4 a, b;                         // 32 grey bytes
};

// The 32 grey bytes of one packed word from row pointer p (zero where not
// ok): two 128-bit loads when V16 and the 32 bytes lie inside the row's
// pitch (vec), else the nb bytes of the row one by one (fully unrolled, so
// the eight words stay in registers).
template <bool V16>
__device__ __forceinline__ Raw thr_load(const uint8_t *p, bool vec, int nb, bool ok) {
    Raw r;
    r.a = make_uint4(0, 0, 0, 0);
    r.b = r.a;
    if (!ok) return r;
    if (V16 && vec) {
        r.a = __ldg(reinterpret_cast<const uint4 *>(p));
        r.b = __ldg(reinterpret_cast<const uint4 *>(p) + 1);
    } else {
        uint32_t v[8];
#pragma unroll
        for (int k = 0; k < 8; ++k) {
            uint32_t x = 0;
#pragma unroll
            for (int i = 0; i < 4; ++i)
                if (4 * k + i < nb) x |= (uint32_t)__ldg(p + 4 * k + i) << (8 * i);
            v[k] = x;
        }
        r.a = make_uint4(v[0], v[1], v[2], v[3]);
        r.b = make_uint4(v[4], v[5], v[6], v[7]);
    }
    return r;
}

// 32 bytes to one word: bit k = byte k >= t, for 1 <= t <= 255.  With
// c = 256 - t in every byte, a >= t exactly when a + c carries out of the
// byte's bit 7.  Adding the low 7 bits of a and c never crosses a byte and
// leaves the carry into bit 7 there; the carry out of bit 7 is the majority
// of a's bit 7, c's bit 7 and that carry, and c's bit 7 is the same in every
// byte (C7: t <= 128), so it is (a | s) or (a & s) at bits 7, 15, 23, 31:
// one three-input logic op per 4 bytes.  The product with 0x00204081 moves
// those four bits to bits 28..31 (every other partial product falls below
// bit 28, at distinct positions, or beyond bit 31), and a funnel shift
// appends them below the nibbles already gathered.
// MODE: 0 compare with c's bit 7 clear, 1 with it set, 2 all white (t <= 0),
// 3 all black (t > 255).
template <int MODE>
__device__ __forceinline__ uint32_t thr_pack(uint32_t c4_low, const Raw &r) {
    if constexpr (MODE == 2) return kAllOnes;
    if constexpr (MODE == 3) return 0u;
    const uint32_t c[8] = {r.a.x, r.a.y, r.a.z, r.a.w, r.b.x, r.b.y, r.b.z, r.b.w};
    uint32_t out = 0;
#pragma unroll
    for (int k = 7; k >= 0; --k) {
        const uint32_t s = (c[k] & 0x7F7F7F7Fu) + c4_low;
        const uint32_t carry = MODE == 1 ? ((c[k] | s) & 0x80808080u) : (c[k] & s & 0x80808080u);
        out = __funnelshift_l(carry * 0x00204081u, out, 4);     // (out << 4) | bits 28..31
    }
    return out;
}

// What a lane needs for one task: its word, its masks, the band's rows.
struct Lane {
    int wi, y0, y1;                     // word; rows y0 .. y1-1 are written
    bool loads, writes;
    uint32_t keep;
};

__device__ __forceinline__ Lane thr_lane(const TGeo &g, int t, int lane) {
    Lane L;
    const int cb = t % g.ncb;
    L.y0 = (t / g.ncb) * g.band;
    L.y1 = min(L.y0 + g.band, g.h);
    L.wi = cb * kWideLanes + lane - 1;
    L.loads = L.wi >= 0 && L.wi < g.nw;
    L.writes = lane >= 1 && lane <= kWideLanes && L.wi < g.stride;
    L.keep = !L.loads ? 0u : (L.wi < g.nw - 1 ? kAllOnes : g.lastmask);
    return L;
}

template <int MODE>
__device__ __forceinline__ uint32_t thr_word(const TGeo &g, const Lane &L, uint32_t c4_low,
                                             const Raw &raw, int r) {
    if ((unsigned)r >= (unsigned)g.h) return g.fill;
    return (thr_pack<MODE>(c4_low, raw) & L.keep) | (g.fill & ~L.keep);
}

// The band walk from the words of rows y0 - 1 and y0, over the words that
// take(r, i) makes for rows r = y0 + 1, y0 + 2, ... in order (i = the row's
// place in its step, a constant once unrolled): each output row y gets
// ~I & (L | R | U | D) from the words of rows y - 1, y, y + 1 and its
// neighbours' words by shuffle.
template <class Take>
__device__ __forceinline__ void thr_walk(const TGeo &g, const Lane &L, uint32_t up, uint32_t cur,
                                         Take &&take) {
    uint32_t *edge = g.edge + (ptrdiff_t)L.y0 * g.stride + L.wi;
    uint32_t *bin = g.binary == nullptr ? nullptr : g.binary + (ptrdiff_t)L.y0 * g.stride + L.wi;
    for (int y = L.y0; y < L.y1; y += kThrRows) {
        uint32_t dn[kThrRows];
#pragma unroll
        for (int i = 0; i < kThrRows; ++i) dn[i] = take(y + 1 + i, i);
#pragma unroll
        for (int i = 0; i < kThrRows; ++i) {
            if (y + i < L.y1) {
                const uint32_t prev = __shfl_up_sync(0xFFFFFFFFu, cur, 1);
                const uint32_t next = __shfl_down_sync(0xFFFFFFFFu, cur, 1);
                if (L.writes) {
                    const uint32_t Lw = __funnelshift_l(prev, cur, 1);  // I(x-1, y)
                    const uint32_t Rw = __funnelshift_r(cur, next, 1);  // I(x+1, y)
                    __stcs(edge, ~cur & (Lw | Rw | up | dn[i]) & L.keep);
                    if (bin != nullptr) __stcs(bin, cur & L.keep);
                }
                edge += g.stride;
                if (bin != nullptr) bin += g.stride;
            }
            up = cur;
            cur = dn[i];
        }
    }
}

template <bool V16, int MODE>
__device__ __forceinline__ void thr_run(const TGeo &g, int ntasks) {
    const int lane = threadIdx.x & 31;
    const int warp = (int)((blockIdx.x * (unsigned)blockDim.x + threadIdx.x) >> 5);
    const int nwarps = (int)((gridDim.x * (unsigned)blockDim.x) >> 5);
    const uint32_t c4_low = g.t4 & 0x7F7F7F7Fu;
    const ptrdiff_t pitch = g.pitch;
    for (int t = warp; t < ntasks; t += nwarps) {
        const Lane L = thr_lane(g, t, lane);
        const bool vec = (L.wi + 1) * 32 <= g.pitch;
        const int nb = min(32, g.w - L.wi * 32);
        // rows y0 - 1 .. y1 are read (y1: the row below the band's last),
        // one at a time from the top; rp points at the next one's bytes
        int next = L.y0 - 1;
        const uint8_t *rp = g.grey + (ptrdiff_t)next * pitch + (ptrdiff_t)L.wi * 32;
        auto fetch = [&]() {
            const Raw raw = thr_load<V16>(
                rp, vec, nb, L.loads && (unsigned)next < (unsigned)g.h && next <= L.y1);
            ++next;
            rp += pitch;
            return raw;
        };
        const Raw r_up = fetch();
        const Raw r_cur = fetch();
        Raw ahead[kThrRows];
#pragma unroll
        for (int i = 0; i < kThrRows; ++i) ahead[i] = fetch();
        auto take = [&](int r, int i) {
            const uint32_t w = thr_word<MODE>(g, L, c4_low, ahead[i], r);
            ahead[i] = fetch();                             // row r + kThrRows
            return w;
        };
        thr_walk(g, L, thr_word<MODE>(g, L, c4_low, r_up, L.y0 - 1),
                 thr_word<MODE>(g, L, c4_low, r_cur, L.y0), take);
    }
}

template <bool V16, int MODE>
__global__ void __launch_bounds__(32 * kThrWarps, 3)
k_threshold(TGeo g, int ntasks) {
    pdl_enter();
    thr_run<V16, MODE>(g, ntasks);
}

// The same with the threshold read from device memory (written there by
// k_otsu earlier on the stream): the compare form is chosen per launch.
template <bool V16>
__global__ void __launch_bounds__(32 * kThrWarps, 3)
k_threshold_dev(TGeo g, int ntasks, const int32_t *__restrict__ t_dev) {
    // launched while k_otsu may still run: wait for it before reading t
    asm volatile("griddepcontrol.wait;" ::: "memory");
    const int t = *t_dev;
    const uint32_t tc = (uint32_t)min(max(t, 1), 255);
    g.t4 = (256u - tc) * 0x01010101u;
    if (t <= 0)
        thr_run<V16, 2>(g, ntasks);
    else if (t > 255)
        thr_run<V16, 3>(g, ntasks);
    else if (t <= 128)
        thr_run<V16, 1>(g, ntasks);
    else
        thr_run<V16, 0>(g, ntasks);
}

// ---- Otsu's threshold (N. Otsu, IEEE Trans. SMC 9(1), 1979) ----

constexpr int kHistWarps = 8;
constexpr int kHistGroups = 4;  // 16-byte groups per lane in flight

// The grey histogram: one warp per row (rows strided over the grid), lanes
// over 16-byte groups of the row (bytes one by one otherwise), counts in a
// histogram per warp in shared memory, added into hist (256 counters) at
// the end.  Only the w pixels of a row count, not its padding.  Shared
// atomics bound it: about nine updates of distinct counters per clock per
// SM, i.e. about 2.7 TB/s of grey on varied images (updates of one counter
// within a warp merge, so a flat image reads at the copy rate).  A counter
// column per lane (no bank conflicts at all) measured no faster on varied
// images and slower on flat ones; plain read-modify-write in such columns
// was slower still.
template <bool V16>
__global__ void __launch_bounds__(32 * kHistWarps)
k_grey_hist(const uint8_t *__restrict__ grey, int32_t w, int32_t h, int32_t pitch,
            unsigned long long *__restrict__ hist) {
    // k_otsu may be placed now; it waits for this grid before reading
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
    __shared__ uint32_t sh[kHistWarps][256];
    for (int i = threadIdx.x; i < kHistWarps * 256; i += blockDim.x) (&sh[0][0])[i] = 0;
    __syncthreads();
    const int lane = threadIdx.x & 31;
    uint32_t *mine = sh[threadIdx.x >> 5];
    const int nwarps = gridDim.x * kHistWarps;
    for (int y = blockIdx.x * kHistWarps + (threadIdx.x >> 5); y < h; y += nwarps) {
        const uint8_t *row = grey + (size_t)y * (size_t)pitch;
        if constexpr (V16) {
            // four 16-byte groups per lane requested before any is counted
            for (int x0 = lane * 16; x0 < w; x0 += kHistGroups * 32 * 16) {
                uint4 v[kHistGroups];
#pragma unroll
                for (int j = 0; j < kHistGroups; ++j) {
                    const int x = x0 + j * 32 * 16;
                    v[j] = x < w ? __ldcs(reinterpret_cast<const uint4 *>(row + x))
                                 : make_uint4(0, 0, 0, 0);
                }
#pragma unroll
                for (int j = 0; j < kHistGroups; ++j) {
                    const int x = x0 + j * 32 * 16;
                    const uint32_t b[4] = {v[j].x, v[j].y, v[j].z, v[j].w};
                    if (x + 16 <= w) {
#pragma unroll
                        for (int k = 0; k < 16; ++k)
                            atomicAdd(&mine[(b[k >> 2] >> (8 * (k & 3))) & 0xFF], 1u);
                    } else {
#pragma unroll
                        for (int k = 0; k < 16; ++k)
                            if (x + k < w) atomicAdd(&mine[(b[k >> 2] >> (8 * (k & 3))) & 0xFF], 1u);
                    }
                }
            }
        } else {
            for (int x = lane; x < w; x += 32) atomicAdd(&mine[row[x]], 1u);
        }
    }
    __syncthreads();
    for (int bin = threadIdx.x; bin < 256; bin += blockDim.x) {
        unsigned long long c = 0;
#pragma unroll
        for (int k = 0; k < kHistWarps; ++k) c += sh[k][bin];
        if (c != 0) atomicAdd(&hist[bin], c);
    }
}

// The threshold from the histogram, by one CTA of 256 threads: thread i
// takes t = i + 1 (1..255).  With n0, s0 the pixels and grey sum below t
// (prefix sums of the histogram), N and S their totals, t is scored by
// D(t) = x^2 / (n0 (N - n0)), x = S n0 - s0 N: the between-class variance
// times N^2.  Every operation is an explicitly rounded double operation in
// that order (no fused multiply-add), so the scores and their comparison
// are those of the same formula evaluated in IEEE double arithmetic
// anywhere.  The first largest t wins; with one grey value v, t = v.
__global__ void __launch_bounds__(256)
k_otsu(const unsigned long long *__restrict__ hist, int32_t *__restrict__ t_out) {
    asm volatile("griddepcontrol.wait;" ::: "memory");
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
    __shared__ unsigned long long n_s[256], s_s[256];
    __shared__ double best_d[256];
    __shared__ int best_t[256];
    __shared__ int single;
    const int i = threadIdx.x;
    const unsigned long long c = hist[i];
    n_s[i] = c;
    s_s[i] = c * (unsigned long long)i;
    if (i == 0) single = -1;
    __syncthreads();
    for (int off = 1; off < 256; off <<= 1) {               // inclusive prefix sums
        const unsigned long long a = i >= off ? n_s[i - off] : 0;
        const unsigned long long b = i >= off ? s_s[i - off] : 0;
        __syncthreads();
        n_s[i] += a;
        s_s[i] += b;
        __syncthreads();
    }
    const unsigned long long N = n_s[255], S = s_s[255];
    if (c == N) single = i;                                 // one grey value (N > 0)
    const unsigned long long n0 = n_s[i], s0 = s_s[i];      // below t = i + 1
    double d = -1.0;
    if (i < 255 && n0 > 0 && n0 < N) {
        const double x = __dsub_rn(__dmul_rn(__ull2double_rn(S), __ull2double_rn(n0)),
                                   __dmul_rn(__ull2double_rn(s0), __ull2double_rn(N)));
        d = __ddiv_rn(__dmul_rn(x, x), __dmul_rn(__ull2double_rn(n0), __ull2double_rn(N - n0)));
    }
    best_d[i] = d;
    best_t[i] = i + 1;
    __syncthreads();
    for (int half = 128; half > 0; half >>= 1) {            // first largest
        if (i < half) {
            const double od = best_d[i + half];
            const int ot = best_t[i + half];
            if (od > best_d[i] || (od == best_d[i] && ot < best_t[i])) {
                best_d[i] = od;
                best_t[i] = ot;
            }
        }
        __syncthreads();
    }
    if (i == 0) *t_out = best_d[0] < 0.0 ? single : best_t[0];
}


}  // namespace

}  // namespace me

using namespace me;

namespace me {
namespace {

// Argument checks and the geometry shared by both entry points (t4 and the
// band are filled in later).
int thr_setup(const uint8_t *grey, int32_t w, int32_t h, int32_t pitch_bytes, uint32_t *edge,
              int32_t stride_words, uint32_t *binary, int32_t boundary, TGeo *g, bool *v16) {
    if (grey == nullptr || edge == nullptr || w <= 0 || h <= 0 || pitch_bytes < w ||
        stride_words < (int32_t)(((int64_t)w + 31) / 32) ||
        (boundary != ME_BOUNDARY_WHITE && boundary != ME_BOUNDARY_BLACK) ||
        ((uintptr_t)edge & 3) || ((uintptr_t)binary & 3))
        return ME_ERR_ARG;
    const size_t in_bytes = (size_t)h * (size_t)pitch_bytes;
    const size_t out_bytes = (size_t)h * (size_t)stride_words * 4;
    if (ranges_overlap(grey, in_bytes, edge, out_bytes) ||
        (binary != nullptr && (ranges_overlap(grey, in_bytes, binary, out_bytes) ||
                               ranges_overlap(edge, out_bytes, binary, out_bytes))))
        return ME_ERR_ALIAS;
    int rc = check_device_ptr(grey);
    if (rc == ME_OK) rc = check_device_ptr(edge);
    if (rc == ME_OK && binary != nullptr) rc = check_device_ptr(binary);
    if (rc != ME_OK) return rc;
    g->grey = grey;
    g->edge = edge;
    g->binary = binary;
    g->w = w;
    g->h = h;
    g->pitch = pitch_bytes;
    g->stride = stride_words;
    g->nw = (int32_t)(((int64_t)w + 31) / 32);
    // in 64 bits: stride_words + 29 overflows int32 for the widest strides
    g->ncb = (int32_t)(((int64_t)stride_words + kWideLanes - 1) / kWideLanes);
    g->lastmask = (w & 31) ? ((1u << (w & 31)) - 1u) : kAllOnes;
    g->fill = boundary == ME_BOUNDARY_WHITE ? kAllOnes : 0u;
    g->t4 = 0;
    g->band = kThrRows;
    *v16 = ((uintptr_t)grey & 15) == 0 && (pitch_bytes & 15) == 0;
    return ME_OK;
}

// Band height, task count and grid for kernel fn on this device.
int thr_grid(const void *fn, TGeo *g, int *ntasks, unsigned *grid) {
    DevInfo di;
    int rc = device_info(&di);
    if (rc != ME_OK) return rc;
    int occ = 0;
    if ((rc = cached_occupancy(fn, 32 * kThrWarps, 0, &occ)) != ME_OK) return rc;
    const int64_t resident = (int64_t)std::max(1, occ) * di.sm_count * kThrWarps;
    g->band = threshold_band(g->ncb, g->h, resident);
    const int64_t n = (int64_t)g->ncb * (((int64_t)g->h + g->band - 1) / g->band);
    if (n > INT32_MAX) return ME_ERR_ARG;
    *ntasks = (int)n;
    *grid = (unsigned)std::max<int64_t>(1, (std::min(n, resident) + kThrWarps - 1) / kThrWarps);
    return ME_OK;
}

}  // namespace
}  // namespace me

extern "C" int me_threshold_edges(const uint8_t *grey, int32_t w, int32_t h, int32_t pitch_bytes,
                                  int32_t threshold, uint32_t *edge, int32_t stride_words,
                                  uint32_t *binary, int32_t boundary, me_stream_t stream) {
    TGeo g;
    bool v16 = false;
    int rc = thr_setup(grey, w, h, pitch_bytes, edge, stride_words, binary, boundary, &g, &v16);
    if (rc != ME_OK) return rc;
    const uint32_t t = (uint32_t)std::min(std::max(threshold, 1), 255);
    g.t4 = (256u - t) * 0x01010101u;
    const int mode = threshold <= 0 ? 2 : threshold > 255 ? 3 : (t <= 128 ? 1 : 0);
    using Fn = void (*)(TGeo, int);
    static constexpr Fn kFns[2][4] = {
        {k_threshold<false, 0>, k_threshold<false, 1>, k_threshold<false, 2>, k_threshold<false, 3>},
        {k_threshold<true, 0>, k_threshold<true, 1>, k_threshold<true, 2>, k_threshold<true, 3>}};
    const Fn fn = kFns[v16 ? 1 : 0][mode];
    int ntasks = 0;
    unsigned grid = 0;
    if ((rc = thr_grid(reinterpret_cast<const void *>(fn), &g, &ntasks, &grid)) != ME_OK) return rc;
    const cudaError_t e = launch_pdl(fn, dim3(grid), dim3(32 * kThrWarps), 0,
                                     (cudaStream_t)stream, g, ntasks);
    if (e != cudaSuccess) cudaGetLastError();
    return e == cudaSuccess ? ME_OK : record_cuda(e);
}

extern "C" int me_threshold_edges_otsu(const uint8_t *grey, int32_t w, int32_t h,
                                       int32_t pitch_bytes, uint32_t *edge,
                                       int32_t stride_words, uint32_t *binary, int32_t boundary,
                                       int32_t *threshold_out, me_stream_t stream) {
    TGeo g;
    bool v16 = false;
    int rc = thr_setup(grey, w, h, pitch_bytes, edge, stride_words, binary, boundary, &g, &v16);
    if (rc != ME_OK) return rc;
    if (threshold_out != nullptr) {
        if ((uintptr_t)threshold_out & 3) return ME_ERR_ARG;
        const size_t in_bytes = (size_t)h * (size_t)pitch_bytes;
        const size_t out_bytes = (size_t)h * (size_t)stride_words * 4;
        if (ranges_overlap(threshold_out, 4, grey, in_bytes) ||
            ranges_overlap(threshold_out, 4, edge, out_bytes) ||
            (binary != nullptr && ranges_overlap(threshold_out, 4, binary, out_bytes)))
            return ME_ERR_ALIAS;
        if ((rc = check_device_ptr(threshold_out)) != ME_OK) return rc;
    }
    const auto fn = v16 ? k_threshold_dev<true> : k_threshold_dev<false>;
    int ntasks = 0;
    unsigned grid = 0;
    if ((rc = thr_grid(reinterpret_cast<const void *>(fn), &g, &ntasks, &grid)) != ME_OK) return rc;
    DevInfo di;
    if ((rc = device_info(&di)) != ME_OK) return rc;
    const cudaStream_t s = (cudaStream_t)stream;
    // scratch: the histogram (256 counters) and, if the caller gave no
    // place for it, the threshold
    unsigned long long *hist = nullptr;
    cudaError_t e = scratch_alloc(reinterpret_cast<void **>(&hist), 256 * 8 + 16, s);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return record_cuda(e);
    }
    int32_t *t_dev = threshold_out != nullptr ? threshold_out : reinterpret_cast<int32_t *>(hist + 256);
    e = cudaMemsetAsync(hist, 0, 256 * 8, s);
    if (e == cudaSuccess) {
        const unsigned hgrid = (unsigned)std::max<int64_t>(
            1, std::min<int64_t>(((int64_t)h + kHistWarps - 1) / kHistWarps, (int64_t)di.sm_count * 4));
        if (v16)
            k_grey_hist<true><<<hgrid, 32 * kHistWarps, 0, s>>>(grey, w, h, pitch_bytes, hist);
        else
            k_grey_hist<false><<<hgrid, 32 * kHistWarps, 0, s>>>(grey, w, h, pitch_bytes, hist);
        // the choice of t and the threshold pass by programmatic dependent
        // launch: each is placed while the kernel before it runs, and waits
        // for it (griddepcontrol.wait) before reading its result
        cudaLaunchAttribute attr[1];
        attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
        attr[0].val.programmaticStreamSerializationAllowed = 1;
        cudaLaunchConfig_t lc = {};
        lc.gridDim = dim3(1);
        lc.blockDim = dim3(256);
        lc.stream = s;
        lc.attrs = attr;
        lc.numAttrs = 1;
        e = cudaGetLastError();
        if (e == cudaSuccess)
            e = cudaLaunchKernelEx(&lc, k_otsu, (const unsigned long long *)hist, t_dev);
        lc.gridDim = dim3(grid);
        lc.blockDim = dim3(32 * kThrWarps);
        if (e == cudaSuccess)
            e = cudaLaunchKernelEx(&lc, fn, g, ntasks, (const int32_t *)t_dev);
    }
    const cudaError_t f = scratch_free(hist, s);
    if (e == cudaSuccess) e = f;
    if (e != cudaSuccess) {
        cudaGetLastError();
        return record_cuda(e);
    }
    return ME_OK;
}
