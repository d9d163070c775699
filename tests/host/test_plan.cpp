// The batch plan on the host (me::plan_batch, linked from the library; it
// touches no device): which kernel form a batch takes, the access-width
// flags packed into each descriptor, and the table of tile -> image that
// the persistent kernel searches.  Addresses are made up (never
// dereferenced): images 16 MiB apart, offset from the 16-byte grid as each
// case needs.
#include <algorithm>
#include <cstdint>
#include <cstdio>
#include <random>
#include <vector>

#include "me_internal.h"

namespace {

me_tile_cfg batch_cfg(int vec_words, int rows_per_lane, int chunk) {
    me_tile_cfg c{};
    c.engine = ME_ENGINE_REGS;
    c.rows_per_lane = rows_per_lane;
    c.vec_words = vec_words;
    c.cta_threads = 512;
    c.ctas_per_sm = 8;
    c.stage_kb = 32;
    c.stages = 4;
    c.chunk_tiles = chunk;
    return c;
}

struct Img {
    int off_bytes;      // past the 16-byte grid
    int stride, w, h;
};

std::vector<me_desc> make(const std::vector<Img> &imgs) {
    std::vector<me_desc> d;
    for (size_t k = 0; k < imgs.size(); ++k) {
        const uintptr_t in = ((uintptr_t)1 << 40) + (uintptr_t)k * (16u << 20) + imgs[k].off_bytes;
        const uintptr_t out = ((uintptr_t)2 << 40) + (uintptr_t)k * (16u << 20) + imgs[k].off_bytes;
        d.push_back({reinterpret_cast<const uint32_t *>(in), reinterpret_cast<uint32_t *>(out),
                     imgs[k].w, imgs[k].h, imgs[k].stride, (int)(k & 1)});
    }
    return d;
}

struct Plan {
    std::vector<char> arena;
    int64_t total = 0;
    bool any = false;
    const me::BatchHeader *hdr() const { return reinterpret_cast<const me::BatchHeader *>(arena.data()); }
    const me::BDesc *bd() const { return reinterpret_cast<const me::BDesc *>(hdr() + 1); }
    const int32_t *table() const { return reinterpret_cast<const int32_t *>(bd() + hdr()->n); }
};

bool plan(const std::vector<me_desc> &d, const me_tile_cfg &cfg, Plan *p) {
    p->arena.assign(me::arena_bytes((int)d.size()), 0);
    int bad = -1;
    const int rc = me::plan_batch(d.data(), (int)d.size(), cfg, p->arena.data(), &p->total, &p->any,
                                  &bad);
    if (rc != ME_OK) std::printf("plan_batch returned %d (image %d)\n", rc, bad);
    return rc == ME_OK;
}

// The persistent kernel's search for the image of tile t (a chunk's first
// tile): the table entry of t's block and the next bracket it, bisect on
// task_base, then step forward while t lies past the image.
int find(const Plan &p, int64_t t) {
    const int shift = p.hdr()->block_shift;
    int i = p.table()[t >> shift];
    int hi = p.table()[(t >> shift) + 1];
    while (i < hi) {
        const int mid = (i + hi + 1) >> 1;
        if (p.bd()[mid].task_base <= t) i = mid; else hi = mid - 1;
    }
    while (t >= p.bd()[i].task_base + p.bd()[i].ntasks) ++i;
    return i;
}

int fails = 0;
void expect(bool ok, const char *what) {
    if (!ok) {
        std::printf("FAIL: %s\n", what);
        ++fails;
    }
}

}  // namespace

int main() {
    // 1. the kernel form: the all-aligned one only when every image takes
    // 128-bit accesses (bit 8); 64-bit (bit 9) and 32-bit images need the
    // form carrying the narrower tiles
    struct Case {
        const char *name;
        std::vector<Img> imgs;
        int vec_words;
        bool want_any;
        std::vector<int> want_bits;     // per image: 1 = 128-bit, 2 = 64-bit, 0 = 32-bit
    };
    const std::vector<Case> cases = {
        {"all 128-bit", {{0, 4, 120, 37}, {0, 8, 250, 5}}, 4, false, {1, 1}},
        {"128-bit and 64-bit only", {{0, 4, 120, 37}, {8, 4, 100, 9}}, 4, true, {1, 2}},
        {"64-bit only (offset, even stride)", {{8, 4, 120, 37}, {0, 6, 190, 3}}, 4, true, {2, 2}},
        {"a 32-bit image (4-byte offset)", {{0, 4, 120, 37}, {4, 4, 128, 2}}, 4, true, {1, 0}},
        {"a 32-bit image (odd stride)", {{0, 5, 150, 11}}, 4, true, {0}},
        {"32-bit accesses asked for", {{0, 4, 120, 37}}, 1, true, {0}},
    };
    for (const Case &c : cases) {
        Plan p;
        if (!plan(make(c.imgs), batch_cfg(c.vec_words, 4, 4), &p)) {
            expect(false, c.name);
            continue;
        }
        if (p.any != c.want_any) std::printf("case '%s': any = %d\n", c.name, (int)p.any);
        expect(p.any == c.want_any, c.name);
        // the batch kind, which picks the tile configuration, agrees with
        // the plan's choice of kernel form wherever the access width is free
        if (c.vec_words == 4) {
            const std::vector<me_desc> d = make(c.imgs);
            expect(me::batch_any(d.data(), (int)d.size()) == c.want_any, "batch kind");
        }
        for (size_t k = 0; k < c.imgs.size(); ++k) {
            const int bits = (p.bd()[k].vw >> 8) & 3;
            expect((p.bd()[k].vw & 0xff) == 4, "4 words per lane");
            if (bits != c.want_bits[k]) std::printf("case '%s' image %zu: bits %d\n", c.name, k, bits);
            expect(bits == c.want_bits[k], c.name);
        }
    }

    // 2. the tile table on random batches: every tile's image found by the
    // kernel's search, task bases contiguous, totals consistent
    std::mt19937_64 rng(11);
    for (int round = 0; round < 60; ++round) {
        const int n = 1 + (int)(rng() % (round < 20 ? 8 : 300));
        std::vector<Img> imgs;
        for (int k = 0; k < n; ++k) {
            const int w = 1 + (int)(rng() % (rng() % 4 == 0 ? 20000 : 600));
            const int h = 1 + (int)(rng() % (rng() % 10 == 0 ? 30000 : 300));
            const int words = (w + 31) / 32;
            const int stride = words + (int)(rng() % 5);
            const int offs[] = {0, 4, 8, 12};
            imgs.push_back({offs[rng() % 4], stride, w, h});
        }
        const int rpts[] = {4, 8, 16, 32};
        const int chunks[] = {1, 3, 4, 64};
        Plan p;
        if (!plan(make(imgs), batch_cfg(4, rpts[rng() % 4], chunks[rng() % 4]), &p)) {
            expect(false, "random batch planned");
            continue;
        }
        expect(p.hdr()->n == n, "header n");
        expect(p.hdr()->total_tasks == p.total, "header total");
        int64_t base = 0, bytes = 0;
        for (int k = 0; k < n; ++k) {
            expect(p.bd()[k].task_base == base && p.bd()[k].ntasks >= 1, "contiguous task bases");
            base += p.bd()[k].ntasks;
            bytes += 2 * (int64_t)imgs[k].h * imgs[k].stride * 4;
        }
        expect(base == p.total, "tasks add up");
        expect(p.hdr()->bytes == bytes, "algorithmic bytes");
        expect(((p.total - 1) >> p.hdr()->block_shift) + 2 <= me::task_table_entries(n),
               "table fits its entries");
        for (int64_t t = 0; t < p.total; ++t) {
            const int i = find(p, t);
            if (!(i >= 0 && i < n && p.bd()[i].task_base <= t &&
                  t < p.bd()[i].task_base + p.bd()[i].ntasks)) {
                std::printf("round %d: tile %lld found image %d\n", round, (long long)t, i);
                expect(false, "tile -> image");
                break;
            }
        }
        if (fails) break;
    }

    // 3. the work items of a launch (me::batch_args for its grid, walked
    // with the persistent kernel's own arithmetic for every warp): every
    // tile taken exactly once, chunks only below `chunked`, and the warps'
    // tile counts at most one chunk apart
    for (int round = 0; round < 200 && fails == 0; ++round) {
        const int n = 1 + (int)(rng() % 400);
        std::vector<Img> imgs;
        for (int k = 0; k < n; ++k) {
            const int w = 1 + (int)(rng() % 3000);
            const int h = 1 + (int)(rng() % (rng() % 8 == 0 ? 5000 : 200));
            imgs.push_back({0, ((w + 31) / 32 + 3) / 4 * 4, w, h});
        }
        const int chunks[] = {1, 2, 3, 4, 8};
        Plan p;
        if (!plan(make(imgs), batch_cfg(4, 4, chunks[rng() % 5]), &p)) {
            expect(false, "random batch planned");
            break;
        }
        const int grids[] = {1, 7, 152, 304, 1216};
        const int threads[] = {128, 256, 512};
        const int grid = grids[rng() % 5], thr = threads[rng() % 3];
        const me::BatchArgs a = me::batch_args(p.arena.data(), grid, thr);
        const unsigned W = (unsigned)grid * (unsigned)thr / 32;
        const int64_t T = p.total;
        expect(a.total == T && a.chunk == p.hdr()->chunk_tiles, "arguments from the header");
        expect(a.chunked % a.chunk == 0 && a.nchunks * a.chunk == a.chunked && a.chunked <= T,
               "chunks cover a prefix");
        std::vector<int> seen((size_t)T, 0);
        int64_t lo = INT64_MAX, hi = 0;
        for (unsigned warp = 0; warp < W; ++warp) {
            int64_t mine = 0;
            for (unsigned k = warp;; k += W) {
                const bool chunk = k < (unsigned)a.nchunks;
                const unsigned c0 = chunk ? k * (unsigned)a.chunk
                                          : k + (unsigned)(a.chunked - a.nchunks);
                if (c0 >= (unsigned)a.total) break;
                const unsigned t1 = c0 + (chunk ? (unsigned)a.chunk : 1u);
                if (chunk && t1 > (unsigned)a.chunked) expect(false, "chunk inside the prefix");
                for (unsigned t = c0; t < t1 && t < (unsigned)T; ++t) ++seen[t];
                mine += t1 - c0;
            }
            lo = std::min(lo, mine);
            hi = std::max(hi, mine);
        }
        for (int64_t t = 0; t < T; ++t)
            if (seen[(size_t)t] != 1) {
                std::printf("round %d: tile %lld taken %d times (T %lld, W %u, C %d)\n", round,
                            (long long)t, seen[(size_t)t], (long long)T, W, a.chunk);
                expect(false, "every tile once");
                break;
            }
        if (hi - lo > a.chunk)
            std::printf("round %d: warps take %lld to %lld tiles (C %d)\n", round, (long long)lo,
                        (long long)hi, a.chunk);
        expect(hi - lo <= a.chunk, "warps' work at most one chunk apart");
    }

    if (fails == 0) std::printf("ok\n");
    return fails == 0 ? 0 : 1;
}
