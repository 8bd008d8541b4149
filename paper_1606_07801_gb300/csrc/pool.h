// First-fit allocator of byte ranges inside [0, capacity), with coalescing
// of freed neighbours.  Host code only: the server carves its device arena
// (resident simulation states) and its host result staging out of one
// allocation each with it, so admitting and retiring simulations never calls
// cudaMalloc or cudaFree.
#pragma once

#include <stdint.h>

#include <map>

namespace lbfd {

class RangePool {
 public:
  RangePool(int64_t capacity, int64_t align);

  // Offset of a free range of `size` bytes (rounded up to the alignment),
  // or -1 when no free range is large enough.
  int64_t alloc(int64_t size);
  // Returns the range starting at `offset`; false if no range starts there.
  bool release(int64_t offset);

  int64_t capacity() const { return capacity_; }
  int64_t used() const { return used_; }
  int64_t largest_free() const;
  int free_ranges() const { return static_cast<int>(free_.size()); }
  int64_t rounded(int64_t size) const { return (size + align_ - 1) / align_ * align_; }

 private:
  int64_t capacity_, align_, used_ = 0;
  std::map<int64_t, int64_t> free_;  // offset -> size, disjoint, never adjacent
  std::map<int64_t, int64_t> live_;  // offset -> size
};

}  // namespace lbfd
