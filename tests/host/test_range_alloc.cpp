// Randomised check of the server's range allocator against a byte map.
#include <cstdio>
#include <cstdlib>
#include <random>
#include <vector>

#include "me_alloc.h"

// Next fit against a byte map: the allocation goes at the rover (the end of
// the previous one) when the units from there are free, else at the start
// of the first maximal free run after the rover that fits, else at the
// start of the lowest one that fits.  Lifetimes are mostly first-in
// first-out, as the server's are, with some random frees mixed in.
static int next_fit() {
    const size_t cap = 1 << 20, align = 256, nu = cap / align;
    me::RangeAlloc a(cap, align);
    std::vector<unsigned char> owner(nu, 0);
    std::vector<std::pair<size_t, size_t>> live;       // in allocation order
    std::mt19937_64 rng(2);
    size_t rover = 0;
    int consecutive = 0, allocs = 0;
    for (int step = 0; step < 200000; ++step) {
        if (live.empty() || rng() % 2) {
            const size_t n = 1 + rng() % (cap / 64);
            const size_t units = (n + align - 1) / align;
            auto free_from = [&](size_t p) {
                if (p + units > nu) return false;
                for (size_t u = p; u < p + units; ++u)
                    if (owner[u]) return false;
                return true;
            };
            size_t want = SIZE_MAX;
            if (free_from(rover)) want = rover;
            for (int pass = 0; pass < 2 && want == SIZE_MAX; ++pass) {
                for (size_t u = 0; u < nu && want == SIZE_MAX; ++u) {
                    const bool start = !owner[u] && (u == 0 || owner[u - 1]);
                    if (!start || (pass == 0 ? u <= rover : u > rover)) continue;
                    if (free_from(u)) want = u;
                }
            }
            size_t off;
            const bool ok = a.alloc_next(n, &off);
            if (ok != (want != SIZE_MAX)) { std::printf("next fit mismatch at %d\n", step); return 1; }
            if (!ok) continue;
            if (off != want * align) { std::printf("not next fit at %d\n", step); return 1; }
            consecutive += off / align == rover;
            ++allocs;
            for (size_t u = 0; u < units; ++u) owner[want + u] = 1;
            rover = want + units >= nu ? 0 : want + units;
            live.push_back({off, n});
        } else {
            // the oldest most of the time, otherwise any
            const size_t i = rng() % 8 ? 0 : rng() % live.size();
            a.release(live[i].first, live[i].second);
            const size_t units = (live[i].second + align - 1) / align;
            for (size_t u = 0; u < units; ++u) owner[live[i].first / align + u] = 0;
            live.erase(live.begin() + (long)i);
        }
        size_t used = 0;
        for (unsigned char o : owner) used += o;
        if (used * align != a.used()) { std::printf("used mismatch at %d\n", step); return 1; }
    }
    // first-in first-out lifetimes keep most allocations back to back
    if (consecutive * 10 < allocs * 8) {
        std::printf("only %d of %d next-fit allocations at the rover\n", consecutive, allocs);
        return 1;
    }
    std::printf("ok\n");
    return 0;
}

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
    return next_fit() ? 1 : 0;
}
