// Register-window tile body of the fused method of masks.
//
// One warp tile covers RPT rows of up to 32 vector columns of VW words
// (VW = 4: one 128-bit load per lane and row where the buffers are 16-byte
// aligned and rows hold whole 16-byte groups, else four 32-bit loads;
// VW = 1: one 32-bit load).
// Narrow rows (at most 32 vector columns) fold the warp: a row segment uses
// exactly as many lanes as the row has vector columns and the warp stacks
// 32 / seg_w segments vertically, so nearly every lane has work whatever
// the width, and the words beyond a segment's ends are outside the image.  Wider rows are cut into column
// blocks of kWideLanes columns: lanes 1..30 produce output while lanes 0 and
// 31 only load the column just left and right of the block, so every
// neighbour word comes from a shuffle and no lane needs extra loads.
//
// Each lane streams its RPT rows top to bottom: the rows above, at and below
// the output row sit in registers and the next prefetch_rows(RPT) rows are already
// requested, so each input word is loaded once per tile.  Outside the image
// (rows, words, padding bits) reads as the boundary colour: per lane a mask
// `keep` of its VW words' pixel bits is precomputed and each loaded word is
// fixed with one three-input logic op, (raw & keep) | (fill & ~keep).
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

// Rows requested ahead of the one being computed: all of a tile's rows up
// to 8 rows per lane (one memory round trip per tile), else 4 at a time.
__host__ __device__ constexpr int prefetch_rows(int rpt) { return rpt <= 8 ? rpt : 4; }

template <int VW>
struct Words {
    uint32_t v[VW];
};

// Image moved one pixel right: bit x holds pixel x-1.
__device__ __forceinline__ uint32_t from_left(uint32_t prev, uint32_t cur) {
    return __funnelshift_l(prev, cur, 1);
}
// Image moved one pixel left: bit x holds pixel x+1.
__device__ __forceinline__ uint32_t from_right(uint32_t cur, uint32_t next) {
    return __funnelshift_r(cur, next, 1);
}

// Pixel bits of image word c (0 outside the row and for padding).
__device__ __forceinline__ uint32_t col_keep(const Geo &g, int c) {
    return (c >= 0 && c < g.nw - 1) ? kAllOnes : (c == g.nw - 1 ? g.lastmask : 0u);
}

// Per-lane constants of one tile.
template <int VW>
struct Lane {
    const uint32_t *base;      // image word c0 of row 0 (used only when loads)
    uint32_t *out[4];          // output word c0 of row 0, per output
    int stride, h, nvp;
    uint32_t fill;
    uint32_t keep[VW];         // fixed = (raw & keep) | (fill & ~keep)
    int nst;                   // of the VW words, those inside the stride
    bool loads;                // 0 <= c0 < nw: the lane's words hold pixels
    bool writes;               // the lane owns output words of this tile
    bool seg_first, seg_last;  // lanes whose outer neighbour is outside
};

template <int VW>
__device__ __forceinline__ Lane<VW> make_lane(const Geo &g, const Outs &o, int c0, int col,
                                              int nvp, bool owner) {
    Lane<VW> L;
    L.loads = c0 >= 0 && c0 < g.nw;
    L.writes = owner && c0 >= 0 && c0 < g.stride;
    const int cs = c0 < 0 ? 0 : c0;            // keep pointers inside the image
    L.base = g.img + cs;
#pragma unroll
    for (int k = 0; k < 4; ++k) L.out[k] = o.p[k] ? o.p[k] + cs : nullptr;
    L.stride = g.stride;
    L.h = g.h;
    L.nvp = nvp;
    L.fill = g.fill;
#pragma unroll
    for (int k = 0; k < VW; ++k) L.keep[k] = col_keep(g, c0 + k);
    L.nst = min(max(g.stride - c0, 0), VW);
    L.seg_first = (col == 0);
    L.seg_last = (col == nvp - 1);
    return L;
}

// Row y into registers.  CHECK: y may lie outside [0, h).  VEC (VW == 4):
// the bytes per access -- 16: one 128-bit load; 8: two 64-bit loads; 4: four
// 32-bit loads.
template <int VW, bool CHECK, int VEC>
__device__ __forceinline__ Words<VW> load_row(const Lane<VW> &L, int y) {
    Words<VW> r;
    const bool rowok = !CHECK || (unsigned)y < (unsigned)L.h;
    const bool ok = L.loads && rowok;
    const uint32_t *p = L.base + (size_t)(CHECK && !rowok ? 0 : y) * (size_t)L.stride;
    uint32_t raw[VW];
    if constexpr (VW == 4) {
        uint4 q = make_uint4(0, 0, 0, 0);
        if constexpr (VEC == 16) {
            // 16-byte aligned: img is, stride % 4 == 0 and c0 % 4 == 0; the
            // four words stay inside the row's stride.
            if (ok) q = __ldg(reinterpret_cast<const uint4 *>(p));
        } else if constexpr (VEC == 8) {
            // 8-byte aligned: img is, stride and c0 are even.  A pair that
            // starts at a word with pixels (below nw <= stride) ends inside
            // the stride; pairs without pixels are not read.
            if (ok) {
                if (L.keep[0]) {
                    const uint2 a = __ldg(reinterpret_cast<const uint2 *>(p));
                    q.x = a.x;
                    q.y = a.y;
                }
                if (L.keep[2]) {
                    const uint2 b = __ldg(reinterpret_cast<const uint2 *>(p) + 1);
                    q.z = b.x;
                    q.w = b.y;
                }
            }
        } else if (ok) {
            // one word at a time; words without pixels are not read
            if (L.keep[0]) q.x = __ldg(p);
            if (L.keep[1]) q.y = __ldg(p + 1);
            if (L.keep[2]) q.z = __ldg(p + 2);
            if (L.keep[3]) q.w = __ldg(p + 3);
        }
    raw[0] = q.x; raw[1] = q.y; raw[2] = q.z; raw[3] = q.w;
    } else {
        raw[0] = ok ? __ldg(p) : 0u;
    }
#pragma unroll
    for (int k = 0; k < VW; ++k) {
        const uint32_t f = (raw[k] & L.keep[k]) | (L.fill & ~L.keep[k]);
        r.v[k] = (!CHECK || rowok) ? f : L.fill;
    }
    return r;
}

// Words just left and right of the lane's VW words.  Segments sit side by
// side in the warp, so the lane before / after is in the same segment
// unless this lane is a segment end, whose outer neighbour is outside.
template <int VW>
__device__ __forceinline__ void side_words(const Lane<VW> &L, const Words<VW> &r,
                                           uint32_t &prev, uint32_t &next) {
    const uint32_t a = __shfl_up_sync(0xFFFFFFFFu, r.v[VW - 1], 1);
    const uint32_t b = __shfl_down_sync(0xFFFFFFFFu, r.v[0], 1);
    prev = L.seg_first ? L.fill : a;
    next = L.seg_last ? L.fill : b;
}

template <int VW, int VEC>
__device__ __forceinline__ void store_words(const Lane<VW> &L, uint32_t *out, int y,
                                            const uint32_t (&e)[VW]) {
    // Padding words (nw .. stride-1) are written too, as 0, so every 32-byte
    // sector of an output row is written whole and never read back.
    uint32_t *p = out + (size_t)y * (size_t)L.stride;
    if constexpr (VW == 4) {
        if constexpr (VEC == 16) {
            // stride % 4 == 0: the group lies inside the row
            __stcs(reinterpret_cast<uint4 *>(p), make_uint4(e[0], e[1], e[2], e[3]));
        } else if constexpr (VEC == 8) {
            // stride and c0 even: the group's words inside the stride are
            // whole pairs, at least one
            __stcs(reinterpret_cast<uint2 *>(p), make_uint2(e[0], e[1]));
            if (L.nst > 2) __stcs(reinterpret_cast<uint2 *>(p) + 1, make_uint2(e[2], e[3]));
        } else {
            // the words of the group inside the stride, one at a time
            __stcs(p, e[0]);
            if (L.nst > 1) __stcs(p + 1, e[1]);
            if (L.nst > 2) __stcs(p + 2, e[2]);
            if (L.nst > 3) __stcs(p + 3, e[3]);
        }
    } else {
        __stcs(p, e[0]);
    }
}

// One output row from the rows above (u), at (c) and below (d); cp/cn are
// the words beside c, up_*/dn_* beside u and d (end points only).
template <int VW, int MODE, int VEC>
__device__ __forceinline__ void emit_row(const Lane<VW> &L, int y, const Words<VW> &u,
                                         const Words<VW> &c, const Words<VW> &d, uint32_t cp,
                                         uint32_t cn, uint32_t up_p, uint32_t up_n,
                                         uint32_t dn_p, uint32_t dn_n) {
    uint32_t e0[VW], e1[VW], e2[VW], e3[VW];
#pragma unroll
    for (int k = 0; k < VW; ++k) {
        const uint32_t cur = c.v[k];
        const uint32_t pv = (k == 0) ? cp : c.v[k - 1];
        const uint32_t nx = (k == VW - 1) ? cn : c.v[k + 1];
        const uint32_t Lw = from_left(pv, cur);         // I(x-1, y)
        const uint32_t Rw = from_right(cur, nx);        // I(x+1, y)
        const uint32_t U = u.v[k];                      // I(x, y-1)
        const uint32_t D = d.v[k];                      // I(x, y+1)
        const uint32_t M = ~cur;                        // the mask
        const uint32_t valid = L.keep[k];
        if constexpr (MODE == MODE_EDGE) {
            e0[k] = M & (Lw | Rw | U | D) & valid;
        } else if constexpr (MODE == MODE_DISPLAY) {
            e0[k] = ~(M & (Lw | Rw | U | D)) & valid;
        } else if constexpr (MODE == MODE_FUND) {
            e0[k] = M & Lw & valid;
            e1[k] = M & Rw & valid;
            e2[k] = M & U & valid;
            e3[k] = M & D & valid;
        } else {
            // Fig. 1 neighbours 1..8 of every pixel of the word, as "is
            // white" planes; count the black ones bit-sliced and keep
            // pixels with at most one.
            const uint32_t pu = (k == 0) ? up_p : u.v[k - 1];
            const uint32_t nu = (k == VW - 1) ? up_n : u.v[k + 1];
            const uint32_t pd = (k == 0) ? dn_p : d.v[k - 1];
            const uint32_t nd = (k == VW - 1) ? dn_n : d.v[k + 1];
            const uint32_t nb[8] = {
                from_right(U, nu),   // 1: up-right
                U,                   // 2: up
                from_left(pu, U),    // 3: up-left
                Lw,                  // 4: left
                from_left(pd, D),    // 5: down-left
                D,                   // 6: down
                from_right(D, nd),   // 7: down-right
                Rw                   // 8: right
            };
            uint32_t one = 0, two = 0;
#pragma unroll
            for (int j = 0; j < 8; ++j) {
                const uint32_t black = ~nb[j];
                two |= one & black;
                one |= black;
            }
            e0[k] = M & ~two & valid;
        }
    }
    store_words<VW, VEC>(L, L.out[0], y, e0);
    if constexpr (MODE == MODE_FUND) {
        store_words<VW, VEC>(L, L.out[1], y, e1);
        store_words<VW, VEC>(L, L.out[2], y, e2);
        store_words<VW, VEC>(L, L.out[3], y, e3);
    }
}

// One warp tile: column block cb, row block rb of image g.  CHECK: the
// tile's rows, with one halo row above and below, may leave the image.
template <int VW, int RPT, int MODE, bool CHECK, int VEC>
__device__ __forceinline__ void window_tile_rows(const Geo &g, const Outs &o, int cb, int rb,
                                                 int lane) {
    constexpr int PF = prefetch_rows(RPT);
    static_assert(RPT % PF == 0, "rows per lane is a multiple of the prefetch");
    // lane -> (segment, column): (lane + 0.5) / seg_w is never within float
    // rounding of an integer, so truncation gives the exact quotient
    const int seg = (int)(((float)lane + 0.5f) * __frcp_rn((float)g.seg_w));
    const int col = lane - seg * g.seg_w;
    const bool wide = g.nv > 32;
    const int v = wide ? cb * kWideLanes + lane - 1 : col;
    const bool owner = seg < g.segs && (!wide || (lane >= 1 && lane <= kWideLanes));
    const int y0 = (rb * g.segs + seg) * RPT;
    const Lane<VW> L = make_lane<VW>(g, o, seg < g.segs ? v * VW : -VW, col, g.seg_w, owner);
    const bool rows_left = !CHECK || y0 < g.h;    // the segment has rows

    Words<VW> up = load_row<VW, CHECK, VEC>(L, y0 - 1);
    Words<VW> cur = load_row<VW, CHECK, VEC>(L, y0);
    Words<VW> q[PF];
#pragma unroll
    for (int i = 0; i < PF; ++i) q[i] = load_row<VW, CHECK, VEC>(L, y0 + 1 + i);
    uint32_t up_p = 0, up_n = 0, cur_p, cur_n;
    if constexpr (MODE == MODE_END) side_words<VW>(L, up, up_p, up_n);
    side_words<VW>(L, cur, cur_p, cur_n);

#pragma unroll 1
    for (int r0 = 0; r0 < RPT; r0 += PF) {
#pragma unroll
        for (int j = 0; j < PF; ++j) {
            const int y = y0 + r0 + j;
            const Words<VW> dn = q[j];
            if (r0 + j + 1 + PF <= RPT) q[j] = load_row<VW, CHECK, VEC>(L, y + 1 + PF);
            uint32_t dn_p, dn_n;
            side_words<VW>(L, dn, dn_p, dn_n);
            if (L.writes && rows_left && (!CHECK || y < g.h))
                emit_row<VW, MODE, VEC>(L, y, up, cur, dn, cur_p, cur_n, up_p, up_n, dn_p, dn_n);
            up = cur;
            cur = dn;
            up_p = cur_p;
            up_n = cur_n;
            cur_p = dn_p;
            cur_n = dn_n;
        }
    }
}

template <int VW, int RPT, int MODE, int VEC>
__device__ __forceinline__ void window_tile(const Geo &g, const Outs &o, int cb, int rb,
                                            int lane) {
    const int rows_per_task = RPT * g.segs;
    const int top = rb * rows_per_task;
    if (top >= 1 && top + rows_per_task < g.h)
        window_tile_rows<VW, RPT, MODE, false, VEC>(g, o, cb, rb, lane);
    else
        window_tile_rows<VW, RPT, MODE, true, VEC>(g, o, cb, rb, lane);
}

}  // namespace me
