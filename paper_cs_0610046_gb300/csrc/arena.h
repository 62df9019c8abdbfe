// First-fit allocator of a fixed device-memory budget, used by the streaming
// service for stream halos, chunk staging and outputs.  Host code only (plain
// C++, no CUDA): it hands out byte offsets into one device allocation.
#pragma once
#include <algorithm>
#include <cstddef>
#include <cstdint>
#include <iterator>
#include <map>

namespace mmf {

// First-fit allocator over [0, size) with coalescing; offsets 256-aligned.
class Arena {
  public:
    void init(size_t size) {
        size_ = size;
        free_.clear();
        if (size) free_[0] = size;
    }
    int64_t alloc(size_t bytes) {
        bytes = round(bytes);
        for (auto it = free_.begin(); it != free_.end(); ++it) {
            if (it->second >= bytes) {
                const size_t off = it->first, sz = it->second;
                free_.erase(it);
                if (sz > bytes) free_[off + bytes] = sz - bytes;
                used_ += bytes;
                return (int64_t)off;
            }
        }
        return -1;
    }
    void release(int64_t off, size_t bytes) {
        bytes = round(bytes);
        used_ -= bytes;
        auto it = free_.emplace((size_t)off, bytes).first;
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
    size_t size() const { return size_; }
    size_t used() const { return used_; }
    static size_t round(size_t b) { return (std::max<size_t>(b, 1) + 255) & ~size_t(255); }

  private:
    size_t size_ = 0, used_ = 0;
    std::map<size_t, size_t> free_;
};

}  // namespace mmf
