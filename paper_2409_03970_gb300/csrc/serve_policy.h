// Host-side policy of the sort server: the scratch arena allocator and the
// admission / co-batching decision.  Pure C++ with no CUDA calls, so that it
// can be tested on a machine without a GPU (nsort_serve_policy_selftest).
#pragma once

#include <cstddef>
#include <cstdint>
#include <deque>
#include <map>
#include <vector>

namespace nsort {
namespace serve {

// First-fit allocator over [0, capacity) with coalescing of free ranges.
// Offsets are multiples of `align`.
class Arena {
 public:
  Arena(size_t capacity = 0, size_t align = 256) { reset(capacity, align); }

  void reset(size_t capacity, size_t align) {
    cap_ = capacity;
    align_ = align;
    free_.clear();
    if (capacity) free_[0] = capacity;
    used_ = 0;
  }

  // Returns true and the offset of a block of `bytes`, or false when no
  // free range is large enough.
  bool alloc(size_t bytes, size_t *off) {
    bytes = round(bytes ? bytes : 1);
    for (auto it = free_.begin(); it != free_.end(); ++it) {
      if (it->second >= bytes) {
        *off = it->first;
        const size_t rest = it->second - bytes;
        const size_t next = it->first + bytes;
        free_.erase(it);
        if (rest) free_[next] = rest;
        used_ += bytes;
        return true;
      }
    }
    return false;
  }

  void release(size_t off, size_t bytes) {
    bytes = round(bytes ? bytes : 1);
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

  size_t capacity() const { return cap_; }
  size_t used() const { return used_; }
  size_t largest_free() const {
    size_t m = 0;
    for (auto &kv : free_) m = kv.second > m ? kv.second : m;
    return m;
  }
  size_t round(size_t b) const { return (b + align_ - 1) / align_ * align_; }

 private:
  size_t cap_ = 0, align_ = 256, used_ = 0;
  std::map<size_t, size_t> free_;   // offset -> length
};

// What the scheduler knows about a waiting request.
struct Pending {
  uint64_t ticket;
  int kind;        // NSORT_KIND_KEYS or NSORT_KIND_PAIRS
  int dtype;
  uint64_t n;
};

// The admission decision for one free stream slot.  The batch starts at the
// first waiting request it may take: the queue's head, unless a large
// request (n >= large_min) is already running, in which case large requests
// wait and the first request below large_min goes ahead of them.  If that
// request is small (n <= batch_max_keys), every later waiting small request
// of the same kind and dtype joins it, in arrival order, up to max_batch
// requests and max_batch_keys keys.  Returns the queue positions of the
// requests to run together (empty when nothing may start); the caller
// removes them with take() once it has found memory for them.  Larger
// requests run alone.  A large sort fills the GPU by itself (its persistent
// merge grids take every SM), so two at once only share it and both finish
// late; one at a time, the first finishes at its own speed.
inline std::vector<size_t> pick_batch(const std::deque<Pending> &queue, uint64_t batch_max_keys,
                                      size_t max_batch, uint64_t max_batch_keys,
                                      uint64_t large_min = ~uint64_t(0),
                                      bool large_running = false) {
  std::vector<size_t> out;
  size_t h = 0;
  if (large_running)
    while (h < queue.size() && queue[h].n >= large_min) ++h;
  if (h >= queue.size()) return out;
  const Pending &head = queue[h];
  out.push_back(h);
  if (batch_max_keys == 0 || head.n > batch_max_keys) return out;
  uint64_t keys = head.n;
  for (size_t i = h + 1; i < queue.size() && out.size() < max_batch; ++i) {
    const Pending &q = queue[i];
    if (q.kind == head.kind && q.dtype == head.dtype && q.n <= batch_max_keys &&
        keys + q.n <= max_batch_keys) {
      keys += q.n;
      out.push_back(i);
    }
  }
  return out;
}

// Removes the entries at `pos` (ascending) from the queue and returns them
// in that order.
inline std::vector<Pending> take(std::deque<Pending> &queue, const std::vector<size_t> &pos) {
  std::vector<Pending> out;
  out.reserve(pos.size());
  for (size_t i : pos) out.push_back(queue[i]);
  for (size_t k = pos.size(); k-- > 0;) queue.erase(queue.begin() + (std::ptrdiff_t)pos[k]);
  return out;
}

}  // namespace serve
}  // namespace nsort
