// fwi_arena.h -- first-fit sub-allocator of the batching engine's arena (host only).
//
// Offsets and sizes are multiples of `align`; freed blocks merge with free neighbours, so an
// arena whose jobs have all retired is one free block again.
#pragma once
#include <algorithm>
#include <cstddef>
#include <iterator>
#include <map>

namespace fwi {

class Arena {
public:
    explicit Arena(size_t align = 256) : align_(align) {}
    void init(size_t bytes)
    {
        free_.clear();
        if (bytes) free_[0] = bytes / align_ * align_;
        used_ = 0;
    }
    size_t largest() const
    {
        size_t m = 0;
        for (auto &kv : free_) m = std::max(m, kv.second);
        return m;
    }
    // first fit: the lowest free offset that holds `bytes`
    bool alloc(size_t bytes, size_t &off)
    {
        bytes = up(bytes);
        for (auto it = free_.begin(); it != free_.end(); ++it) {
            if (it->second < bytes) continue;
            off = it->first;
            const size_t rest = it->second - bytes;
            free_.erase(it);
            if (rest) free_[off + bytes] = rest;
            used_ += bytes;
            return true;
        }
        return false;
    }
    void release(size_t off, size_t bytes)
    {
        bytes = up(bytes);
        used_ -= bytes;
        auto it = free_.emplace(off, bytes).first;
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
    size_t used() const { return used_; }
    size_t free_blocks() const { return free_.size(); }

private:
    size_t up(size_t v) const { return (v + align_ - 1) / align_ * align_; }
    size_t align_;
    std::map<size_t, size_t> free_;   // offset -> size
    size_t used_ = 0;
};

}  // namespace fwi
