// Randomised check of the server's range allocator against a byte map.
#include <cstdio>
#include <cstdlib>
#include <random>
#include <vector>

#include "me_alloc.h"

int main() {
    const size_t cap = 1 << 20, align = 256;
    me::RangeAlloc a(cap, align);
    std::vector<unsigned char> owner(cap / align, 0);   // 1 = in use
    std::vector<std::pair<size_t, size_t>> live;
    std::mt19937_64 rng(1);
    for (int step = 0; step < 200000; ++step) {
        if (live.empty() || rng() % 3) {
            const size_t n = 1 + rng() % (cap / 16);
            size_t off;
            // first fit: the lowest run of free units that fits
            const size_t units = (n + align - 1) / align;
            size_t want = SIZE_MAX, run = 0;
            for (size_t u = 0; u < owner.size(); ++u) {
                run = owner[u] ? 0 : run + 1;
                if (run == units) { want = u + 1 - units; break; }
            }
            const bool ok = a.alloc(n, &off);
            if (ok != (want != SIZE_MAX)) { std::printf("fit mismatch at %d\n", step); return 1; }
            if (!ok) continue;
            if (off != want * align) { std::printf("not first fit at %d\n", step); return 1; }
            for (size_t u = 0; u < units; ++u) owner[want + u] = 1;
            live.push_back({off, n});
        } else {
            const size_t i = rng() % live.size();
            a.release(live[i].first, live[i].second);
            const size_t units = (live[i].second + align - 1) / align;
            for (size_t u = 0; u < units; ++u) owner[live[i].first / align + u] = 0;
            live[i] = live.back();
            live.pop_back();
        }
        size_t used = 0;
        for (unsigned char o : owner) used += o;
        if (used * align != a.used()) { std::printf("used mismatch at %d\n", step); return 1; }
    }
    for (auto &l : live) a.release(l.first, l.second);
    if (a.used() != 0 || a.free_ranges() != 1 || a.largest_free() != cap) {
        std::printf("did not coalesce back to one range\n");
        return 1;
    }
    if (a.peak() == 0 || a.peak() > cap) { std::printf("bad peak\n"); return 1; }
    std::printf("ok\n");
    return 0;
}
