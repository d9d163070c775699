// Host-side image geometry: the segment table, column blocks, and the
// multiply-shift that replaces t / ncb in the single-image kernel, checked
// against plain integer division; the threshold kernel's band height,
// checked against a search over every band height.
#include <cstdio>
#include <random>

#include "me_internal.h"

int main() {
    std::mt19937_64 rng(7);
    for (int stride = 1; stride <= 70000; stride += (stride < 2000 ? 1 : 97)) {
        for (int vw : {1, 4}) {
            const int w = stride * 32 - (int)(rng() % 32);
            const me::Geo g = me::make_geo(nullptr, w, 1, stride, 0, vw, false);
            const int nv = vw == 4 ? (stride + 3) / 4 : stride;
            if (g.nv != nv) { std::printf("nv %d %d\n", stride, vw); return 1; }
            const int seg_w = nv > 32 ? 32 : nv;
            if (g.seg_w != seg_w || g.segs != 32 / seg_w) { std::printf("segs %d\n", stride); return 1; }
            const int ncb = nv > 32 ? (nv + me::kWideLanes - 1) / me::kWideLanes : 1;
            if (g.ncb != ncb) { std::printf("ncb %d\n", stride); return 1; }
            // t / ncb for task indices up to 2^31 - 1
            const uint32_t probes[] = {0u, 1u, (uint32_t)ncb - 1, (uint32_t)ncb, (uint32_t)ncb + 1,
                                       0x7FFFFFFFu, 0x7FFFFFFEu,
                                       0x7FFFFFFFu / (uint32_t)ncb * (uint32_t)ncb,
                                       0x7FFFFFFFu / (uint32_t)ncb * (uint32_t)ncb - 1};
            for (int k = 0; k < 64 + 9; ++k) {
                const uint32_t t = k < 9 ? probes[k] : (uint32_t)(rng() & 0x7FFFFFFFu);
                if (t > 0x7FFFFFFFu) continue;
                const uint32_t q = (uint32_t)(((uint64_t)t * g.ncb_m) >> g.ncb_s);
                if (q != t / (uint32_t)ncb) {
                    std::printf("t / ncb: t %u ncb %d got %u\n", t, ncb, q);
                    return 1;
                }
            }
        }
    }
    // threshold_band: a multiple of kThrRows, at least kThrRows, no taller
    // than h rounded up, and as cheap as the best of every band height
    auto cost = [](int64_t ncb, int64_t h, int64_t W, int64_t b) {
        const int64_t tasks = ncb * ((h + b - 1) / b);
        return (tasks + W - 1) / W * (b + 2 + 4);
    };
    for (int c = 0; c < 3000 + 4; ++c) {
        int64_t ncb, h, W;
        if (c < 4) {
            const int64_t shapes[4][3] = {{18, 16384, 3648}, {9, 8192, 3648}, {1, 1000000, 3648},
                                          {60, 3, 7}};   // the benchmark's 16384² and 8192², a tall narrow image, a flat one
            ncb = shapes[c][0], h = shapes[c][1], W = shapes[c][2];
        } else {
            ncb = 1 + (int64_t)(rng() % 200);
            h = 1 + (int64_t)(rng() % (c % 3 == 0 ? 60000 : 5000));
            const int64_t Ws[] = {3648, 2432, 1216, 456, 8, 7, 1};
            W = Ws[rng() % 7];
        }
        const int b = me::threshold_band(ncb, (int32_t)h, W);
        const int64_t top = (h + me::kThrRows - 1) / me::kThrRows * me::kThrRows;
        if (b < me::kThrRows || b % me::kThrRows != 0 || b > top) {
            std::printf("band %d for ncb %lld h %lld W %lld\n", b, (long long)ncb, (long long)h,
                        (long long)W);
            return 1;
        }
        int64_t best = INT64_MAX;
        for (int64_t x = me::kThrRows; x <= top; x += me::kThrRows) best = std::min(best, cost(ncb, h, W, x));
        if (cost(ncb, h, W, b) != best) {
            std::printf("band %d costs %lld, best %lld (ncb %lld h %lld W %lld)\n", b,
                        (long long)cost(ncb, h, W, b), (long long)best, (long long)ncb,
                        (long long)h, (long long)W);
            return 1;
        }
    }
    std::printf("ok\n");
    return 0;
}
