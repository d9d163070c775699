// Register-window tile body of the fused method of masks.
//
// One warp tile covers RPT rows of up to 32 vector columns of VW words
// (VW = 4: one 128-bit load per lane and row; VW = 1: one 32-bit load).
// Narrow images fold the warp: a row segment uses nvp = 2^seg_log2 lanes
// and the warp stacks 32 / nvp segments vertically, so every lane has work
// whatever the width.  Each lane loads its rows y0-1 .. y0+RPT once into
// registers, takes the horizontal neighbour words from the lanes beside it
// with shuffles (lanes at a segment end load the one word beyond, or use
// the outside colour), and writes RPT output words.
//
// Word form of the paper's steps, least significant bit = leftmost pixel:
//   mask          M = ~I                                    (Section 3)
//   image moved right (left neighbour)  I(x-1) = (cur << 1) | (prev >> 31)
//   image moved left (right neighbour)  I(x+1) = (cur >> 1) | (next << 31)
//   image moved down / up               I(y-1), I(y+1) = the words above/below
//   fundamental edges = M AND each moved image             (Section 4)
//   edge = OR of the four                                   (Section 5)
#pragma once

#include <cstdint>

#include "me_internal.h"

namespace me {

template <int VW>
struct Words {
    uint32_t v[VW];
};

// Word c of row y with the outside colour applied: rows and words outside
// the image read as `fill`, the padding bits of word nw-1 as well.
__device__ __forceinline__ uint32_t fix_word(const Geo &g, int c, uint32_t x) {
    if (c >= g.nw) return g.fill;
    if (c == g.nw - 1) return (x & g.lastmask) | (g.fill & ~g.lastmask);
    return x;
}

template <int VW>
__device__ __forceinline__ Words<VW> load_row(const Geo &g, int y, int c0) {
    Words<VW> r;
    if ((unsigned)y < (unsigned)g.h && c0 < g.nw) {
        const uint32_t *p = g.img + (size_t)y * (size_t)g.stride + c0;
        if constexpr (VW == 4) {
            // 16-byte aligned: img is, stride % 4 == 0 and c0 % 4 == 0; the
            // four words stay inside the row's stride.
            uint4 q = __ldg(reinterpret_cast<const uint4 *>(p));
            r.v[0] = fix_word(g, c0 + 0, q.x);
            r.v[1] = fix_word(g, c0 + 1, q.y);
            r.v[2] = fix_word(g, c0 + 2, q.z);
            r.v[3] = fix_word(g, c0 + 3, q.w);
        } else {
            r.v[0] = fix_word(g, c0, __ldg(p));
        }
    } else {
#pragma unroll
        for (int k = 0; k < VW; ++k) r.v[k] = g.fill;
    }
    return r;
}

// Single word c of row y (outside colour applied); for the halo lanes.
__device__ __forceinline__ uint32_t load_word(const Geo &g, int y, int c) {
    if ((unsigned)y < (unsigned)g.h && c >= 0 && c < g.nw)
        return fix_word(g, c, __ldg(g.img + (size_t)y * (size_t)g.stride + c));
    return g.fill;
}

template <int VW>
__device__ __forceinline__ void store_row(const Geo &g, uint32_t *out, int y,
                                          int c0, const Words<VW> &e) {
    if (y >= g.h || c0 >= g.nw || out == nullptr) return;
    uint32_t *p = out + (size_t)y * (size_t)g.stride + c0;
    if constexpr (VW == 4) {
        if (c0 + 3 < g.nw) {
            __stcs(reinterpret_cast<uint4 *>(p), make_uint4(e.v[0], e.v[1], e.v[2], e.v[3]));
            return;
        }
#pragma unroll
        for (int k = 0; k < 4; ++k)
            if (c0 + k < g.nw) __stcs(p + k, e.v[k]);
    } else {
        __stcs(p, e.v[0]);
    }
}

// Image moved one pixel right: bit x holds pixel x-1.
__device__ __forceinline__ uint32_t from_left(uint32_t prev, uint32_t cur) {
    return __funnelshift_l(prev, cur, 1);
}
// Image moved one pixel left: bit x holds pixel x+1.
__device__ __forceinline__ uint32_t from_right(uint32_t cur, uint32_t next) {
    return __funnelshift_r(cur, next, 1);
}

// Rows loaded ahead of the one being computed.
constexpr int kPrefetch = 4;

// One warp tile: column block cb, row block rb of image g.  Rows stream
// through a register window: row r+kPrefetch is requested while row r is
// computed, so at most kPrefetch + 2 rows are live per lane.
template <int VW, int RPT, int MODE>
__device__ __forceinline__ void window_tile(const Geo &g, const Outs &o, int cb,
                                            int rb, int lane) {
    const int nvp = 1 << g.seg_log2;
    const int col = lane & (nvp - 1);
    const int seg = lane >> g.seg_log2;
    const int v = cb * 32 + col;
    const int c0 = v * VW;
    const int y0 = ((rb << (5 - g.seg_log2)) + seg) * RPT;
    const bool seg_first = (col == 0);
    const bool seg_last = (col == nvp - 1);

    // window index r holds row y0 - 1 + r, r = 0 .. RPT + 1
    Words<VW> win[RPT + 2];
    uint32_t hl[RPT + 2], hr[RPT + 2];      // raw halo words of segment-end lanes
    uint32_t prevw[RPT + 2], nextw[RPT + 2];

    auto fetch = [&](int r) {
        const int y = y0 - 1 + r;
        win[r] = load_row<VW>(g, y, c0);
        hl[r] = seg_first ? load_word(g, y, c0 - 1) : 0u;
        hr[r] = seg_last ? load_word(g, y, c0 + VW) : 0u;
    };
    // words just left and right of this lane's columns in window row r
    auto neighbours = [&](int r) {
        uint32_t a = __shfl_up_sync(0xFFFFFFFFu, win[r].v[VW - 1], 1, nvp);
        uint32_t b = __shfl_down_sync(0xFFFFFFFFu, win[r].v[0], 1, nvp);
        prevw[r] = seg_first ? hl[r] : a;
        nextw[r] = seg_last ? hr[r] : b;
    };

#pragma unroll
    for (int r = 0; r <= kPrefetch && r < RPT + 2; ++r) fetch(r);
    if constexpr (MODE == MODE_END) neighbours(0);

#pragma unroll
    for (int r = 1; r <= RPT; ++r) {
        if (r + kPrefetch < RPT + 2) fetch(r + kPrefetch);
        if constexpr (MODE == MODE_END) {
            if (r == 1) neighbours(1);
            neighbours(r + 1);
        } else {
            neighbours(r);
        }
        const int y = y0 - 1 + r;
        Words<VW> e0, e1, e2, e3;
#pragma unroll
        for (int k = 0; k < VW; ++k) {
            const uint32_t cur = win[r].v[k];
            const uint32_t pv = (k == 0) ? prevw[r] : win[r].v[k - 1];
            const uint32_t nx = (k == VW - 1) ? nextw[r] : win[r].v[k + 1];
            const uint32_t L = from_left(pv, cur);      // I(x-1, y)
            const uint32_t R = from_right(cur, nx);     // I(x+1, y)
            const uint32_t U = win[r - 1].v[k];         // I(x, y-1)
            const uint32_t D = win[r + 1].v[k];         // I(x, y+1)
            const uint32_t M = ~cur;                    // the mask
            const uint32_t valid = (c0 + k == g.nw - 1) ? g.lastmask : kAllOnes;
            if constexpr (MODE == MODE_EDGE) {
                e0.v[k] = M & (L | R | U | D) & valid;
            } else if constexpr (MODE == MODE_DISPLAY) {
                e0.v[k] = ~(M & (L | R | U | D)) & valid;
            } else if constexpr (MODE == MODE_FUND) {
                e0.v[k] = M & L & valid;
                e1.v[k] = M & R & valid;
                e2.v[k] = M & U & valid;
                e3.v[k] = M & D & valid;
            } else {
                // Fig. 1 neighbours 1..8 of every pixel of the word, as
                // "is white" planes; count the black ones bit-sliced and
                // keep pixels with at most one.
                const uint32_t pu = (k == 0) ? prevw[r - 1] : win[r - 1].v[k - 1];
                const uint32_t nu = (k == VW - 1) ? nextw[r - 1] : win[r - 1].v[k + 1];
                const uint32_t pd = (k == 0) ? prevw[r + 1] : win[r + 1].v[k - 1];
                const uint32_t nd = (k == VW - 1) ? nextw[r + 1] : win[r + 1].v[k + 1];
                const uint32_t nb[8] = {
                    from_right(U, nu),   // 1: up-right
                    U,                   // 2: up
                    from_left(pu, U),    // 3: up-left
                    L,                   // 4: left
                    from_left(pd, D),    // 5: down-left
                    D,                   // 6: down
                    from_right(D, nd),   // 7: down-right
                    R                    // 8: right
                };
                uint32_t one = 0, two = 0;
#pragma unroll
                for (int j = 0; j < 8; ++j) {
                    const uint32_t black = ~nb[j];
                    two |= one & black;
                    one |= black;
                }
                e0.v[k] = M & ~two & valid;
            }
        }
        store_row<VW>(g, o.p[0], y, c0, e0);
        if constexpr (MODE == MODE_FUND) {
            store_row<VW>(g, o.p[1], y, c0, e1);
            store_row<VW>(g, o.p[2], y, c0, e2);
            store_row<VW>(g, o.p[3], y, c0, e3);
        }
    }
}

}  // namespace me
