// Division by a fixed divisor by multiply and shift (host and device).
#pragma once

#include <stdint.h>

namespace lbfd {

// Division by a fixed divisor d in [1, 2^31) by multiply and shift
// (Granlund & Montgomery, PLDI 1994): with l = ceil(log2 d) and
// m = floor(2^(32+l) / d) + 1 = 2^32 + mlo, floor(n / d) equals
// floor(m n / 2^(32+l)) = (mulhi(mlo, n) + n) >> l for 0 <= n < 2^31 (the
// rounding error of m contributes less than n 2^-(32+l) < 1/d, and the sum
// cannot overflow 32 bits).  The work-item indices of a tile are split into
// row, column and plane with it.
struct FastDiv {
  uint32_t mlo, l;
};

__host__ __device__ inline FastDiv make_fastdiv(uint32_t d) {
  uint32_t l = 0;
  while ((uint64_t(1) << l) < d) ++l;
  FastDiv f;
  f.mlo = static_cast<uint32_t>(((uint64_t((uint64_t(1) << l) - d)) << 32) / d + 1);
  f.l = l;
  return f;
}

__host__ __device__ __forceinline__ uint32_t fastdiv(uint32_t n, FastDiv f) {
#ifdef __CUDA_ARCH__
  const uint32_t hi = __umulhi(f.mlo, n);
#else
  const uint32_t hi = static_cast<uint32_t>((uint64_t(f.mlo) * n) >> 32);
#endif
  return (hi + n) >> f.l;
}

}  // namespace lbfd
