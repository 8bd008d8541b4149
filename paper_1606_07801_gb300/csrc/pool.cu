// First-fit range allocator (pool.h) and its C ABI (lbfd_pool_*), which the
// tests use to check the allocator on the host.
#include <algorithm>
#include <new>

#include "internal.h"
#include "lbfd.h"
#include "pool.h"

namespace lbfd {

RangePool::RangePool(int64_t capacity, int64_t align) : capacity_(capacity), align_(align < 1 ? 1 : align) {
  capacity_ = capacity_ / align_ * align_;
  if (capacity_ > 0) free_[0] = capacity_;
}

int64_t RangePool::alloc(int64_t size) {
  if (size <= 0) size = 1;
  size = rounded(size);
  for (auto it = free_.begin(); it != free_.end(); ++it) {
    if (it->second < size) continue;
    const int64_t off = it->first, rest = it->second - size;
    free_.erase(it);
    if (rest > 0) free_[off + size] = rest;
    live_[off] = size;
    used_ += size;
    return off;
  }
  return -1;
}

bool RangePool::release(int64_t offset) {
  auto lv = live_.find(offset);
  if (lv == live_.end()) return false;
  int64_t off = offset, size = lv->second;
  live_.erase(lv);
  used_ -= size;
  // merge with the free neighbour after, then the one before
  auto next = free_.lower_bound(off);
  if (next != free_.end() && next->first == off + size) {
    size += next->second;
    next = free_.erase(next);
  }
  if (next != free_.begin()) {
    auto prev = std::prev(next);
    if (prev->first + prev->second == off) {
      off = prev->first;
      size += prev->second;
      free_.erase(prev);
    }
  }
  free_[off] = size;
  return true;
}

int64_t RangePool::largest_free() const {
  int64_t best = 0;
  for (const auto &kv : free_) best = std::max(best, kv.second);
  return best;
}

}  // namespace lbfd

struct lbfd_pool {
  lbfd::RangePool pool;
  lbfd_pool(int64_t c, int64_t a) : pool(c, a) {}
};

extern "C" {

int lbfd_pool_create(lbfd_pool_t *out, int64_t capacity, int64_t align) {
  if (!out || capacity < 0 || align < 1 || (align & (align - 1)) != 0)
    return lbfd::set_last_error(LBFD_EINVAL, "lbfd_pool_create: capacity >= 0 and a power-of-two alignment needed");
  *out = new (std::nothrow) lbfd_pool(capacity, align);
  return *out ? LBFD_OK : lbfd::set_last_error(LBFD_ENOMEM, "lbfd_pool_create: host allocation failed");
}

int lbfd_pool_destroy(lbfd_pool_t p) {
  delete p;
  return LBFD_OK;
}

int lbfd_pool_alloc(lbfd_pool_t p, int64_t size, int64_t *offset) {
  if (!p || !offset || size < 0) return lbfd::set_last_error(LBFD_EINVAL, "lbfd_pool_alloc: bad argument");
  *offset = p->pool.alloc(size);
  return *offset < 0 ? lbfd::set_last_error(LBFD_EBUSY, "lbfd_pool_alloc: no free range is large enough") : LBFD_OK;
}

int lbfd_pool_free(lbfd_pool_t p, int64_t offset) {
  if (!p) return lbfd::set_last_error(LBFD_EINVAL, "lbfd_pool_free: null pool");
  return p->pool.release(offset) ? LBFD_OK
                                 : lbfd::set_last_error(LBFD_EINVAL, "lbfd_pool_free: no range starts at that offset");
}

int lbfd_pool_stats(lbfd_pool_t p, int64_t *used, int64_t *largest_free, int32_t *free_ranges) {
  if (!p) return lbfd::set_last_error(LBFD_EINVAL, "lbfd_pool_stats: null pool");
  if (used) *used = p->pool.used();
  if (largest_free) *largest_free = p->pool.largest_free();
  if (free_ranges) *free_ranges = p->pool.free_ranges();
  return LBFD_OK;
}

}  // extern "C"
