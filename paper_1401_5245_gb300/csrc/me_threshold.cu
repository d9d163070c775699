// Thresholding ahead of the method of masks, fused (Section 7: a grey
// photograph is made binary, then its edges are found).  One pass reads the
// 8-bit image, makes each 32-pixel word on the fly (white where grey >= t),
// and writes the edge map (and, if asked, the binary image) packed.
//
// A warp works on a tile of kThrRows rows of a column block of kWideLanes
// packed words: lanes 1..30 produce those words, lanes 0 and 31 make the
// words just left and right of the block, so every neighbour word comes
// from a shuffle.  All rows of the tile, with the row above and below, are
// requested before any is thresholded: one memory round trip per tile, and
// many tiles in flight per SM.
#include <algorithm>

#include "me_internal.h"

namespace me {

namespace {

constexpr int kThrRows = 4;     // rows per warp task

struct TGeo {
    const uint8_t *grey;
    uint32_t *edge, *binary;            // binary may be null
    int32_t w, h, pitch;                // pitch: bytes per grey row
    int32_t stride, nw, ncb;            // output words per row, words with pixels, blocks
    uint32_t lastmask, fill;
    uint32_t t4;                        // 256 - threshold in every byte
};

struct Raw {
    uint4 a, b;                         // 32 grey bytes
};

// The 32 grey bytes of packed word wi of row y (zero where absent).
template <bool V16>
__device__ __forceinline__ Raw thr_load(const TGeo &g, int y, int wi, bool ok) {
    Raw r;
    r.a = make_uint4(0, 0, 0, 0);
    r.b = r.a;
    if (!ok || (unsigned)y >= (unsigned)g.h) return r;
    const uint8_t *p = g.grey + (size_t)y * (size_t)g.pitch + (size_t)wi * 32;
    if (V16 && wi * 32 + 32 <= g.pitch) {
        r.a = __ldg(reinterpret_cast<const uint4 *>(p));
        r.b = __ldg(reinterpret_cast<const uint4 *>(p) + 1);
    } else {
        // byte by byte, the bytes of the row only (fully unrolled, so the
        // eight words stay in registers)
        const int n = min(32, g.w - wi * 32);
        uint32_t v[8];
#pragma unroll
        for (int k = 0; k < 8; ++k) {
            uint32_t x = 0;
#pragma unroll
            for (int i = 0; i < 4; ++i)
                if (4 * k + i < n) x |= (uint32_t)__ldg(p + 4 * k + i) << (8 * i);
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
// bit 28, at distinct positions, or beyond bit 31).
// MODE: 0 compare with c's bit 7 clear, 1 with it set, 2 all white (t <= 0),
// 3 all black (t > 255).
template <int MODE>
__device__ __forceinline__ uint32_t thr_pack(const TGeo &g, const Raw &r) {
    if constexpr (MODE == 2) return kAllOnes;
    if constexpr (MODE == 3) return 0u;
    const uint32_t c[8] = {r.a.x, r.a.y, r.a.z, r.a.w, r.b.x, r.b.y, r.b.z, r.b.w};
    const uint32_t c4_low = g.t4 & 0x7F7F7F7Fu;
    uint32_t out = 0;
#pragma unroll
    for (int k = 0; k < 8; ++k) {
        const uint32_t s = (c[k] & 0x7F7F7F7Fu) + c4_low;
        const uint32_t carry = MODE == 1 ? ((c[k] | s) & 0x80808080u) : (c[k] & s & 0x80808080u);
        // bits 28..31 of the product, placed at bits 4k..4k+3
        out |= ((carry * 0x00204081u) >> (28 - 4 * k)) & (0xFu << (4 * k));
    }
    return out;
}

template <bool V16, int MODE>
__global__ void __launch_bounds__(256)
k_threshold(TGeo g, int ntasks) {
    const int lane = threadIdx.x & 31;
    const int warp = (int)((blockIdx.x * (unsigned)blockDim.x + threadIdx.x) >> 5);
    const int nwarps = (int)((gridDim.x * (unsigned)blockDim.x) >> 5);
    for (int t = warp; t < ntasks; t += nwarps) {
        const int cb = t % g.ncb;
        const int rb = t / g.ncb;
        const int wi = cb * kWideLanes + lane - 1;          // this lane's word
        const bool loads = wi >= 0 && wi < g.nw;
        const bool writes = lane >= 1 && lane <= kWideLanes && wi < g.stride;
        const uint32_t keep = !loads ? 0u : (wi < g.nw - 1 ? kAllOnes : g.lastmask);
        const int y0 = rb * kThrRows;
        auto word = [&](const Raw &r, int y) {
            if ((unsigned)y >= (unsigned)g.h) return g.fill;
            return (thr_pack<MODE>(g, r) & keep) | (g.fill & ~keep);
        };
        // rows y0 - 1 .. y0 + kThrRows, all requested before any is used
        Raw raw[kThrRows + 2];
#pragma unroll
        for (int i = 0; i < kThrRows + 2; ++i) raw[i] = thr_load<V16>(g, y0 - 1 + i, wi, loads);
        uint32_t up = word(raw[0], y0 - 1);
        uint32_t cur = word(raw[1], y0);
#pragma unroll
        for (int j = 0; j < kThrRows; ++j) {
            const int y = y0 + j;
            const uint32_t dn = word(raw[j + 2], y + 1);
            const uint32_t prev = __shfl_up_sync(0xFFFFFFFFu, cur, 1);
            const uint32_t next = __shfl_down_sync(0xFFFFFFFFu, cur, 1);
            if (writes && y < g.h) {
                const uint32_t L = __funnelshift_l(prev, cur, 1);   // I(x-1, y)
                const uint32_t R = __funnelshift_r(cur, next, 1);   // I(x+1, y)
                const size_t at = (size_t)y * (size_t)g.stride + wi;
                __stcs(g.edge + at, ~cur & (L | R | up | dn) & keep);
                if (g.binary != nullptr) __stcs(g.binary + at, cur & keep);
            }
            up = cur;
            cur = dn;
        }
    }
}

}  // namespace

}  // namespace me

using namespace me;

extern "C" int me_threshold_edges(const uint8_t *grey, int32_t w, int32_t h, int32_t pitch_bytes,
                                  int32_t threshold, uint32_t *edge, int32_t stride_words,
                                  uint32_t *binary, int32_t boundary, me_stream_t stream) {
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
    DevInfo di;
    if ((rc = device_info(&di)) != ME_OK) return rc;

    TGeo g;
    g.grey = grey;
    g.edge = edge;
    g.binary = binary;
    g.w = w;
    g.h = h;
    g.pitch = pitch_bytes;
    g.stride = stride_words;
    g.nw = (int32_t)(((int64_t)w + 31) / 32);
    g.ncb = (stride_words + kWideLanes - 1) / kWideLanes;
    g.lastmask = (w & 31) ? ((1u << (w & 31)) - 1u) : kAllOnes;
    g.fill = boundary == ME_BOUNDARY_WHITE ? kAllOnes : 0u;
    const uint32_t t = (uint32_t)std::min(std::max(threshold, 1), 255);
    g.t4 = (256u - t) * 0x01010101u;
    const int mode = threshold <= 0 ? 2 : threshold > 255 ? 3 : (t <= 128 ? 1 : 0);

    const int64_t ntasks = (int64_t)g.ncb * ((h + kThrRows - 1) / kThrRows);
    if (ntasks > INT32_MAX) return ME_ERR_ARG;
    const int warps_per_cta = 8;
    const int64_t grid = std::max<int64_t>(1, std::min<int64_t>((ntasks + warps_per_cta - 1) / warps_per_cta,
                                                                 (int64_t)di.sm_count * 64));
    const bool v16 = ((uintptr_t)grey & 15) == 0 && (pitch_bytes & 15) == 0;
    using Fn = void (*)(TGeo, int);
    static constexpr Fn kFns[2][4] = {
        {k_threshold<false, 0>, k_threshold<false, 1>, k_threshold<false, 2>, k_threshold<false, 3>},
        {k_threshold<true, 0>, k_threshold<true, 1>, k_threshold<true, 2>, k_threshold<true, 3>}};
    kFns[v16 ? 1 : 0][mode]<<<(unsigned)grid, 32 * warps_per_cta, 0, (cudaStream_t)stream>>>(
        g, (int)ntasks);
    const cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? ME_OK : record_cuda(e);
}
