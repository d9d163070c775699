// Range allocator with coalescing, used by the server to hand out pieces of
// its device pool and its pinned staging pool.  Two placement rules: first
// fit (the lowest free range that fits) and next fit (the first free range
// that fits starting at or after the end of the previous next-fit
// allocation, wrapping round to the lowest).  Requests that live and die
// roughly in arrival order get consecutive addresses under next fit, so the
// server can move a batch's requests with a few large copies.  Pure host
// code (no CUDA), unit-tested on its own.
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
        used_ = peak_ = rover_ = 0;
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

    // Next fit: at the rover (the end of the previous next-fit allocation)
    // if the free range holding it has room from there; else at the start
    // of the first free range after the rover that fits; else at the start
    // of the lowest free range that fits.
    bool alloc_next(size_t n, size_t *off) {
        n = round(n);
        if (n == 0 || n > cap_) return false;
        auto it = free_.upper_bound(rover_);             // first start > rover
        if (it != free_.begin()) {
            auto c = std::prev(it);                      // start <= rover
            const size_t end = c->first + c->second;
            if (end >= rover_ + n) {
                const size_t head = rover_ - c->first;
                if (head) c->second = head; else free_.erase(c);
                if (end > rover_ + n) free_[rover_ + n] = end - (rover_ + n);
                return took(rover_, n, off);
            }
        }
        for (auto j = it; j != free_.end(); ++j)
            if (j->second >= n) return take_front(j, n, off);
        for (auto j = free_.begin(); j != it; ++j)
            if (j->second >= n) return take_front(j, n, off);
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
    bool take_front(std::map<size_t, size_t>::iterator it, size_t n, size_t *off) {
        const size_t at = it->first, rest = it->second - n;
        free_.erase(it);
        if (rest) free_[at + n] = rest;
        return took(at, n, off);
    }
    bool took(size_t at, size_t n, size_t *off) {
        *off = at;
        used_ += n;
        if (used_ > peak_) peak_ = used_;
        rover_ = at + n >= cap_ ? 0 : at + n;
        return true;
    }

    size_t align_ = 1, cap_ = 0, used_ = 0, peak_ = 0, rover_ = 0;
    std::map<size_t, size_t> free_;   // offset -> length, non-adjacent
};

}  // namespace me
