// First-fit range allocator over [0, size): the serving engine's device and
// pinned-host arenas.  Offsets only (no memory is touched), so the same code
// manages device memory and is unit-tested on the host.  Not thread-safe: the
// owner serializes calls.
#pragma once

#include <cstdint>
#include <map>
#include <unordered_map>

namespace lg {

class RangeArena {
 public:
  void init(uint64_t size, uint64_t align) {
    align_ = align ? align : 1;
    size_ = size / align_ * align_;
    free_.clear();
    live_.clear();
    if (size_) free_[0] = size_;
    used_ = peak_ = 0;
  }

  // first free range that fits `bytes` (rounded up to the alignment); false if none
  bool alloc(uint64_t bytes, uint64_t* off) {
    const uint64_t need = round_up(bytes ? bytes : 1);
    for (auto it = free_.begin(); it != free_.end(); ++it) {
      if (it->second < need) continue;
      const uint64_t o = it->first, rest = it->second - need;
      free_.erase(it);
      if (rest) free_[o + need] = rest;
      live_[o] = need;
      used_ += need;
      if (used_ > peak_) peak_ = used_;
      *off = o;
      return true;
    }
    return false;
  }

  // returns false for an offset that is not live (nothing changes)
  bool release(uint64_t off) {
    auto it = live_.find(off);
    if (it == live_.end()) return false;
    uint64_t o = off, len = it->second;
    live_.erase(it);
    used_ -= len;
    auto next = free_.lower_bound(o);
    if (next != free_.end() && next->first == o + len) {  // merge with the range after
      len += next->second;
      next = free_.erase(next);
    }
    if (next != free_.begin()) {  // merge with the range before
      auto prev = std::prev(next);
      if (prev->first + prev->second == o) {
        prev->second += len;
        return true;
      }
    }
    free_[o] = len;
    return true;
  }

  uint64_t size() const { return size_; }
  uint64_t used() const { return used_; }
  uint64_t peak() const { return peak_; }
  uint64_t free_ranges() const { return free_.size(); }
  uint64_t largest_free() const {
    uint64_t m = 0;
    for (const auto& f : free_) m = f.second > m ? f.second : m;
    return m;
  }

 private:
  uint64_t round_up(uint64_t x) const { return (x + align_ - 1) / align_ * align_; }
  std::map<uint64_t, uint64_t> free_;            // offset -> length, disjoint, merged
  std::unordered_map<uint64_t, uint64_t> live_;  // offset -> length
  uint64_t size_ = 0, align_ = 1, used_ = 0, peak_ = 0;
};

}  // namespace lg
