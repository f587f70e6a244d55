// fw_arena.h -- the device-memory arena of the serving worker (host code
// only: it hands out byte offsets into one allocation made elsewhere).
#pragma once

#include <cstddef>
#include <iterator>
#include <map>

namespace fw {

// Allocator over [0, size) with byte offsets.  Rows are placed next-fit
// (right after the previously admitted query's rows when that space is free,
// else first-fit from the bottom) and staged starts last-fit from the top, so
// the rows of queries admitted one after another lie back to back and their
// copies to back-to-back host buffers merge into one.  Zero-byte requests
// take nothing.
class Arena {
 public:
  explicit Arena(size_t size) { free_[0] = size; }
  bool alloc(size_t bytes, size_t* off) {
    if (bytes == 0) {
      *off = 0;
      return true;
    }
    for (auto it = free_.begin(); it != free_.end(); ++it) {
      if (it->second >= bytes) {
        *off = it->first;
        const size_t rest = it->second - bytes, start = it->first + bytes;
        free_.erase(it);
        if (rest) free_[start] = rest;
        used_ += bytes;
        return true;
      }
    }
    return false;
  }
  // [off, off + bytes) if it lies inside one free block
  bool alloc_at(size_t off, size_t bytes) {
    if (bytes == 0) return true;
    auto it = free_.upper_bound(off);
    if (it == free_.begin()) return false;
    --it;
    const size_t start = it->first, end = it->first + it->second;
    if (off + bytes > end) return false;
    if (off > start) it->second = off - start;
    else free_.erase(it);
    if (off + bytes < end) free_[off + bytes] = end - (off + bytes);
    used_ += bytes;
    return true;
  }
  bool alloc_top(size_t bytes, size_t* off) {
    if (bytes == 0) {
      *off = 0;
      return true;
    }
    for (auto it = free_.rbegin(); it != free_.rend(); ++it) {
      if (it->second >= bytes) {
        it->second -= bytes;
        *off = it->first + it->second;
        if (it->second == 0) free_.erase(std::next(it).base());
        used_ += bytes;
        return true;
      }
    }
    return false;
  }
  void release(size_t off, size_t bytes) {
    if (bytes == 0) return;
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
    used_ -= bytes;
  }
  size_t used() const { return used_; }

 private:
  std::map<size_t, size_t> free_;
  size_t used_ = 0;
};

}  // namespace fw
