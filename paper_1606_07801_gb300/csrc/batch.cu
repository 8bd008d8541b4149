// Host side of the batched step (kernels in batch_kernels.cuh): the
// per-launch argument kernel, lattice dispatch, and the tile assignment that
// the ensemble and the server share.
#include <cuda_runtime.h>

#include "batch.h"

namespace lbfd {

__global__ void k_batch_prep(const BatchMember *__restrict__ members, int n, const uint64_t *__restrict__ clock_dev,
                             uint64_t clock, int noise_mode, int noise_dist, BatchStep *__restrict__ out) {
  const uint64_t now = clock_dev ? *clock_dev : clock;
  for (int m = blockIdx.x * blockDim.x + threadIdx.x; m < n; m += gridDim.x * blockDim.x) {
    const BatchMember mb = members[m];
    BatchStep s{};
    s.a.Lx = mb.Lx;
    s.a.Ly = mb.Ly;
    s.a.Lz = mb.Lz;
    s.a.N = mb.N;
    fill_step_params(s.a, mb.tau, mb.rho_mean);
    s.a.noise_mode = noise_mode;
    s.a.noise_dist = noise_dist;
    const uint64_t t = now - mb.t0;  // the member's own step counter
    s.a.ph = make_philox_step(mb.seed, mb.lattice_id, t);
    const int p = static_cast<int>(t & 1);
    s.src = mb.off[p];
    s.dst = mb.off[p ^ 1];
    s.tile0 = mb.tile0;
    s.vx = mb.vx;
    s.cols = mb.Lx / mb.vx;
    s.items = static_cast<int32_t>(static_cast<int64_t>(s.cols) * mb.Ly * mb.Lz);
    s.div_cols = make_fastdiv(static_cast<uint32_t>(s.cols));
    s.div_Ly = make_fastdiv(static_cast<uint32_t>(mb.Ly));
    out[m] = s;
  }
}

__global__ void k_clock_advance(uint64_t *clock_dev) {
  if (threadIdx.x == 0 && blockIdx.x == 0) *clock_dev += 1;
}

cudaError_t launch_batch_prep(const BatchMember *members, int n, const uint64_t *clock_dev, uint64_t clock,
                              int noise_mode, int noise_dist, BatchStep *out, cudaStream_t stream) {
  if (n <= 0) return cudaSuccess;
  const int grid = (n + 127) / 128;
  k_batch_prep<<<grid, 128, 0, stream>>>(members, n, clock_dev, clock, noise_mode, noise_dist, out);
  return cudaGetLastError();
}

cudaError_t launch_clock_advance(uint64_t *clock_dev, cudaStream_t stream) {
  k_clock_advance<<<1, 32, 0, stream>>>(clock_dev);
  return cudaGetLastError();
}

cudaError_t launch_batch_step(int lattice, int precision, void *base, const BatchStep *steps, const int64_t *tile_start,
                              int nmembers, int64_t ntiles, int passes, int occ, int walk, int vx_max, int noise_mode,
                              int noise_dist, int grid, cudaStream_t stream) {
  switch (lattice) {
    case kD1Q3:
      return launch_batch_step_d1q3(precision, base, steps, tile_start, nmembers, ntiles, passes, occ, walk, vx_max, noise_mode,
                                    noise_dist, grid, stream);
    case kD2Q9:
      return launch_batch_step_d2q9(precision, base, steps, tile_start, nmembers, ntiles, passes, occ, walk, vx_max, noise_mode,
                                    noise_dist, grid, stream);
    case kD3Q19:
      return launch_batch_step_d3q19(precision, base, steps, tile_start, nmembers, ntiles, passes, occ, walk, vx_max, noise_mode,
                                     noise_dist, grid, stream);
  }
  return cudaErrorInvalidValue;
}

int batch_blocks_per_sm(int lattice, int precision, int occ, int vx_max, int walk, int noise_mode, int noise_dist) {
  switch (lattice) {
    case kD1Q3: return batch_blocks_per_sm_d1q3(precision, occ, vx_max, walk, noise_mode, noise_dist);
    case kD2Q9: return batch_blocks_per_sm_d2q9(precision, occ, vx_max, walk, noise_mode, noise_dist);
    case kD3Q19: return batch_blocks_per_sm_d3q19(precision, occ, vx_max, walk, noise_mode, noise_dist);
  }
  return 1;
}

BatchMember make_batch_member(const int64_t dims[3], double tau, double rho_mean, uint64_t seed, uint32_t lattice_id,
                              int64_t off0, int64_t off1, uint64_t t0, int vx_max) {
  BatchMember m{};
  m.Lx = static_cast<int32_t>(dims[0]);
  m.Ly = static_cast<int32_t>(dims[1]);
  m.Lz = static_cast<int32_t>(dims[2]);
  m.vx = (vx_max >= 2 && m.Lx % 2 == 0) ? 2 : 1;
  m.N = dims[0] * dims[1] * dims[2];
  m.off[0] = off0;
  m.off[1] = off1;
  m.t0 = t0;
  m.seed = seed;
  m.lattice_id = lattice_id;
  m.tau = tau;
  m.rho_mean = rho_mean;
  return m;
}

int64_t batch_assign_tiles(BatchMember *members, int n, int passes, int64_t *tile_start) {
  const int64_t per_tile = int64_t(passes) * kBatchThreads;
  int64_t next = 0;
  for (int m = 0; m < n; ++m) {
    BatchMember &mb = members[m];
    const int64_t items = int64_t(mb.Lx / mb.vx) * mb.Ly * mb.Lz;
    mb.tile0 = next;
    tile_start[m] = next;
    next += (items + per_tile - 1) / per_tile;
  }
  return next;
}

}  // namespace lbfd
