// Host side of the batched step (kernels in batch_kernels.cuh): the
// per-launch argument kernel, lattice dispatch, and the tile assignment that
// the ensemble and the server share.
#include <cuda_runtime.h>

#include <algorithm>
#include <vector>

#include "batch.h"

namespace lbfd {

__global__ void k_batch_prep(const BatchMember *__restrict__ members, int n, const uint64_t *__restrict__ clock_dev,
                             uint64_t clock, int noise_mode, int noise_dist, BatchStep *__restrict__ out) {
  const uint64_t now = clock_dev ? *clock_dev : clock;
  for (int m = blockIdx.x * blockDim.x + threadIdx.x; m < n; m += gridDim.x * blockDim.x)
    out[m] = batch_step_of(members[m], now, noise_mode, noise_dist);
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
      return launch_batch_step_d1q3(precision, base, steps, tile_start, nmembers, ntiles, passes, occ, walk, vx_max,
                                    noise_mode, noise_dist, grid, stream);
    case kD2Q9:
      return launch_batch_step_d2q9(precision, base, steps, tile_start, nmembers, ntiles, passes, occ, walk, vx_max,
                                    noise_mode, noise_dist, grid, stream);
    case kD3Q19:
      return launch_batch_step_d3q19(precision, base, steps, tile_start, nmembers, ntiles, passes, occ, walk, vx_max,
                                     noise_mode, noise_dist, grid, stream);
  }
  return cudaErrorInvalidValue;
}

cudaError_t launch_batch_param(int lattice, int precision, void *base, const BatchParams *groups, int ngroups,
                               const BatchStep *steps, int passes, int occ, int vx_max, int noise_mode, int noise_dist,
                               cudaStream_t stream) {
  switch (lattice) {
    case kD1Q3:
      return launch_batch_param_d1q3(precision, base, groups, ngroups, steps, passes, occ, vx_max, noise_mode,
                                     noise_dist, stream);
    case kD2Q9:
      return launch_batch_param_d2q9(precision, base, groups, ngroups, steps, passes, occ, vx_max, noise_mode,
                                     noise_dist, stream);
    case kD3Q19:
      return launch_batch_param_d3q19(precision, base, groups, ngroups, steps, passes, occ, vx_max, noise_mode,
                                      noise_dist, stream);
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

int batch_build_params(const BatchMember *members, int n, int64_t ntiles, int noise_mode, int noise_dist,
                       std::vector<BatchParams> &groups) {
  groups.clear();
  for (int first = 0; first < n; first += kParamMembers) {
    BatchParams p{};
    p.first = first;
    p.n = std::min(kParamMembers, n - first);
    const int64_t base = members[first].tile0;
    for (int k = 0; k < p.n; ++k) {
      const BatchMember &mb = members[first + k];
      p.tile_start[k] = static_cast<int32_t>(mb.tile0 - base);
      p.mem[k] = batch_step_of(mb, mb.t0, noise_mode, noise_dist);
    }
    const int64_t end = first + p.n < n ? members[first + p.n].tile0 : ntiles;
    p.tile_start[p.n] = static_cast<int32_t>(end - base);
    groups.push_back(p);
  }
  return static_cast<int>(groups.size());
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
