// First-fit range allocator with coalescing, used by the server to hand out
// pieces of its device pool and its pinned staging pool.  Pure host code
// (no CUDA), unit-tested on its own.
#pragma once

#include <cstddef>
#include <iterator>
#include <map>

namespace me {

class RangeAlloc {
   public:
    RangeAlloc() = default;
    RangeAlloc(size_t capacity, size_t align) { reset(capacity, align); }

    void reset(size_t capacity, size_t align) {
        align_ = align ? align : 1;
        cap_ = capacity / align_ * align_;
        free_.clear();
        if (cap_) free_[0] = cap_;
        used_ = peak_ = 0;
    }

    size_t round(size_t n) const { return (n + align_ - 1) / align_ * align_; }

    // Lowest free range that fits n bytes (rounded to the alignment).
    bool alloc(size_t n, size_t *off) {
        n = round(n);
        if (n == 0 || n > cap_) return false;
        for (auto it = free_.begin(); it != free_.end(); ++it) {
            if (it->second < n) continue;
            *off = it->first;
            const size_t rest = it->second - n;
            const size_t at = it->first + n;
            free_.erase(it);
            if (rest) free_[at] = rest;
            used_ += n;
            if (used_ > peak_) peak_ = used_;
            return true;
        }
        return false;
    }

    // Return [off, off + n); merges with free neighbours.
    void release(size_t off, size_t n) {
        n = round(n);
        if (n == 0) return;
        used_ -= n;
        auto next = free_.lower_bound(off);
        if (next != free_.begin()) {
            auto prev = std::prev(next);
            if (prev->first + prev->second == off) {
                off = prev->first;
                n += prev->second;
                free_.erase(prev);
            }
        }
        next = free_.lower_bound(off);
        if (next != free_.end() && off + n == next->first) {
            n += next->second;
            free_.erase(next);
        }
        free_[off] = n;
    }

    size_t capacity() const { return cap_; }
    size_t peak() const { return peak_; }
    size_t free_ranges() const { return free_.size(); }
    size_t largest_free() const {
        size_t m = 0;
        for (auto &kv : free_)
            if (kv.second > m) m = kv.second;
        return m;
    }
    size_t free_bytes() const {
        size_t s = 0;
        for (auto &kv : free_) s += kv.second;
        return s;
    }
    size_t used() const { return used_; }

   private:
    size_t align_ = 1, cap_ = 0, used_ = 0, peak_ = 0;
    std::map<size_t, size_t> free_;   // offset -> length, non-adjacent
};

}  // namespace me
