// First-fit allocator over one contiguous range of device memory, used by the
// serving loop to admit requests by their device footprint.  Host-only C++
// (no CUDA), so it is also compiled into a CPU test.
#pragma once

#include <cstddef>
#include <iterator>
#include <map>

namespace glcm_arena {

class Arena {
 public:
    static constexpr size_t kAlign = 256;

    static size_t round_up(size_t b) { return (b + kAlign - 1) & ~(kAlign - 1); }

    void reset(size_t capacity)
    {
        cap_ = capacity & ~(kAlign - 1);
        free_.clear();
        if (cap_)
            free_[0] = cap_;
        used_ = peak_ = 0;
    }

    // Lowest-addressed free block that holds `bytes` (rounded up to kAlign);
    // false when none does.
    bool alloc(size_t bytes, size_t* offset)
    {
        const size_t need = round_up(bytes ? bytes : 1);
        for (auto it = free_.begin(); it != free_.end(); ++it) {
            if (it->second < need)
                continue;
            *offset = it->first;
            const size_t rest = it->second - need;
            const size_t next = it->first + need;
            free_.erase(it);
            if (rest)
                free_[next] = rest;
            used_ += need;
            if (used_ > peak_)
                peak_ = used_;
            return true;
        }
        return false;
    }

    // Return a block from alloc(bytes) to the free list, merging neighbours.
    void release(size_t offset, size_t bytes)
    {
        const size_t sz = round_up(bytes ? bytes : 1);
        used_ -= sz;
        auto it = free_.emplace(offset, sz).first;
        auto nx = std::next(it);
        if (nx != free_.end() && it->first + it->second == nx->first) {
            it->second += nx->second;
            free_.erase(nx);
        }
        if (it != free_.begin()) {
            auto pv = std::prev(it);
            if (pv->first + pv->second == it->first) {
                pv->second += it->second;
                free_.erase(it);
            }
        }
    }

    size_t capacity() const { return cap_; }
    size_t used() const { return used_; }
    size_t peak() const { return peak_; }
    size_t free_blocks() const { return free_.size(); }
    size_t largest_free() const
    {
        size_t m = 0;
        for (const auto& kv : free_)
            m = kv.second > m ? kv.second : m;
        return m;
    }

 private:
    size_t cap_ = 0, used_ = 0, peak_ = 0;
    std::map<size_t, size_t> free_;  // offset -> size, non-adjacent blocks
};

}  // namespace glcm_arena
