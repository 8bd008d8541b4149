// Ensemble step: many independent lattices of one lattice type, with their
// own sizes, relaxation times, mean densities, seeds and Philox lattice ids,
// advanced by one launch per time step.
//
// Work is a flat list of tiles.  A tile is up to 256 consecutive work items
// of one member, where an item is VX sites of a row.  A persistent grid walks
// the tiles.  For each tile, thread 0 builds the member's step parameters
// and Philox words in shared memory.  Each item then runs the same per-site
// code as the single-lattice kernels, so a member evolves bit-identically to
// the same lattice stepped alone.
#pragma once

#include "step_kernels.cuh"

namespace lbfd {

struct EnsMember {
  int32_t Lx, Ly, Lz, pad0;
  int64_t N;       // sites
  int64_t offset;  // first value of this member in the ensemble buffers
  double tau, rho_mean;
  uint64_t seed;
  uint32_t lattice_id, pad1;
};

struct EnsTile {
  int32_t member, pad;
  int64_t item0;  // first work item (items are row-major: row * (Lx / VX) + column)
};

constexpr int kEnsThreads = 256;

template <int LAT, typename S, int VX>
constexpr int ens_min_blocks() {
  return step_min_blocks<LAT, S>();
}

template <int LAT, typename S, int VX, int NOISE>
__global__ void __launch_bounds__(kEnsThreads, ens_min_blocks<LAT, S, VX>())
    k_ens_step(const S *__restrict__ src, S *__restrict__ dst, const EnsMember *__restrict__ members,
               const EnsTile *__restrict__ tiles, int ntiles, const uint64_t *__restrict__ t_dev, int noise_mode,
               int noise_dist) {
  __shared__ StepArgs sa;
  const uint64_t t = *t_dev;
  for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    const EnsTile tl = tiles[tile];
    const EnsMember &m = members[tl.member];
    if (threadIdx.x == 0) {
      sa.Lx = m.Lx;
      sa.Ly = m.Ly;
      sa.Lz = m.Lz;
      sa.N = m.N;
      fill_step_params(sa, m.tau, m.rho_mean);
      sa.noise_mode = noise_mode;
      sa.noise_dist = noise_dist;
      sa.ph = make_philox_step(m.seed, m.lattice_id, t);
    }
    __syncthreads();
    const int cols = m.Lx / VX;
    const int64_t items = static_cast<int64_t>(cols) * m.Ly * m.Lz;
    const int64_t item = tl.item0 + threadIdx.x;
    if (item < items) {
      const int64_t row = item / cols;
      const int col = static_cast<int>(item - row * cols);
      const int y = static_cast<int>(row % m.Ly), z = static_cast<int>(row / m.Ly);
      const S *s = src + m.offset;
      S *d = dst + m.offset;
      if constexpr (VX == 1)
        step_scalar_body<LAT, S, NOISE>(s, d, sa, col, y, z);
      else
        step_vec_body<LAT, S, VX, NOISE>(s, d, sa, col * VX, y, z);
    }
    __syncthreads();
  }
}

template <int LAT, typename S, int VX>
cudaError_t ens_step_t(const void *src, void *dst, const EnsMember *members, const EnsTile *tiles, int ntiles,
                       const uint64_t *t_dev, int noise_mode, int noise_dist, int grid, cudaStream_t stream) {
  const S *s = static_cast<const S *>(src);
  S *d = static_cast<S *>(dst);
  if (noise_mode == kNoiseOff)
    k_ens_step<LAT, S, VX, kStepNoiseOff><<<grid, kEnsThreads, 0, stream>>>(s, d, members, tiles, ntiles, t_dev,
                                                                           noise_mode, noise_dist);
  else if (noise_dist == kGaussian)
    k_ens_step<LAT, S, VX, kStepNoiseGauss><<<grid, kEnsThreads, 0, stream>>>(s, d, members, tiles, ntiles, t_dev,
                                                                             noise_mode, noise_dist);
  else
    k_ens_step<LAT, S, VX, kStepNoiseFlat><<<grid, kEnsThreads, 0, stream>>>(s, d, members, tiles, ntiles, t_dev,
                                                                            noise_mode, noise_dist);
  return cudaGetLastError();
}

// Resident blocks per SM of the ensemble kernel (for sizing the persistent grid).
template <int LAT, typename S, int VX>
int ens_blocks_per_sm(int noise_mode, int noise_dist) {
  int nb = 0;
  cudaError_t e;
  if (noise_mode == kNoiseOff)
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_ens_step<LAT, S, VX, kStepNoiseOff>, kEnsThreads, 0);
  else if (noise_dist == kGaussian)
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_ens_step<LAT, S, VX, kStepNoiseGauss>, kEnsThreads, 0);
  else
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_ens_step<LAT, S, VX, kStepNoiseFlat>, kEnsThreads, 0);
  return e == cudaSuccess && nb > 0 ? nb : 1;
}

}  // namespace lbfd
