// Host-side image geometry: the segment table, column blocks, and the
// multiply-shift that replaces t / ncb in the single-image kernel, checked
// against plain integer division.
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
    std::printf("ok\n");
    return 0;
}
