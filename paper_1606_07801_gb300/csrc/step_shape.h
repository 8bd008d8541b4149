// Launch shape of the one-launch-per-step register-pull kernels (k_step,
// k_step_vec): sites per thread and the block/grid over the lattice.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include <cstdlib>

#include "device.cuh"

namespace lbfd {

// Sites per thread of the register-pull step kernel (k_step_vec; 1 is
// k_step): 4 (16-byte loads and stores of FP32) where that measured faster on
// GB300 and Lx allows, else 2 where Lx is even, else 1.  Four sites won for
// D2Q9 in every FP32-arithmetic format (84.5 against 83.9 GLUPS at 2048^2)
// and for D3Q19 with 16-bit storage (37.9 against 37.6 at 256^3); D3Q19 in
// FP32 needs too many registers for four (31.7 against 38.9), and FP64 keeps
// two.  A tuning knob only; results do not depend on it.  LBFD_STEP_VX = 1,
// 2 or 4 overrides the choice where Lx allows.
inline int step_vec_width(int lattice, int precision, int32_t Lx) {
  static int forced = [] {
    const char *e = getenv("LBFD_STEP_VX");
    const int r = e ? atoi(e) : 0;
    return (r == 1 || r == 2 || r == 4) ? r : 0;
  }();
  int vx = forced;
  if (vx == 0) {
    const bool four = precision != kStoreF64 && (lattice == kD2Q9 || (lattice == kD3Q19 && precision != kStoreF32));
    vx = four ? 4 : 2;
  }
  if (vx == 4 && precision == kStoreF64) vx = 2;
  if (Lx % vx == 0) return vx;
  return Lx % 2 == 0 ? 2 : 1;
}

// Block and grid of the one-launch-per-step kernels for vx sites per thread:
// 256-thread blocks, x fastest (at least one warp along x), one grid plane
// per z.
inline void step_shape(int32_t Lx, int32_t Ly, int32_t Lz, dim3 &grid, dim3 &block, int vx = 1) {
  const int cols = Lx / vx;
  int bx = 256;
  while (bx > 32 && bx / 2 >= cols) bx /= 2;
  int by = 256 / bx;
  while (by > 1 && by / 2 >= Ly) by /= 2;
  block = dim3(bx, by, 1);
  grid = dim3((cols + bx - 1) / bx, (Ly + by - 1) / by, Lz);
}

}  // namespace lbfd
