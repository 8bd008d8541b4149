// Batched step: many independent lattices of one lattice type, each with its
// own size, relaxation time, mean density, seed, Philox lattice id and step
// counter, advanced by one launch per time step.  Used by the ensemble
// (members that start together) and by the server (members admitted at
// different times).
//
// Memory.  All members live in one device buffer `base`; member m keeps its
// two population blocks at value offsets off[0] and off[1].  Its own step
// counter is t = clock - t0, where clock counts the launches of the batch;
// the stored state is in block t & 1 and the step writes block (t & 1) ^ 1.
//
// Work.  A launch walks a flat list of tiles with a persistent grid.  Member m
// owns tiles [tile_start[m], tile_start[m + 1]); a tile is `passes` x 256
// consecutive work items of one member, and an item is vx sites of a row
// (vx = 2 for even Lx, else 1).  Per tile, warp 0 finds the member by a
// 32-way search of tile_start and copies that member's step arguments into
// shared memory; every item then runs the per-site code of the single-lattice
// kernels, so a member evolves bit-identically to the same lattice stepped
// alone.  The step arguments (relaxation constants and the Philox words of
// the member's t) are written once per launch and member by k_batch_prep.
#pragma once

#include "fastdiv.cuh"
#include "step_kernels.cuh"

namespace lbfd {

constexpr int kBatchThreads = 256;
// Order in which blocks take tiles: a persistent grid whose blocks take every
// grid-th tile (strided) or one run of consecutive tiles (contiguous), or one
// block per tile.
constexpr int kWalkStrided = 0, kWalkContiguous = 1, kWalkPerTile = 2;

// One member, as the host builds it (constant while the member is listed).
struct BatchMember {
  int32_t Lx, Ly, Lz, vx;  // vx: sites per work item, 1 or 2 (2 needs Lx even)
  int64_t N;               // sites
  int64_t off[2];          // first value of population block 0 / 1 in the batch buffer
  int64_t tile0;           // first tile of the member in the launch's tile list
  uint64_t t0;             // clock value at which the member's own step counter is 0
  uint64_t seed;
  uint32_t lattice_id, pad;
  double tau, rho_mean;
};

// What one launch needs of one member (written by k_batch_prep).
struct alignas(16) BatchStep {
  StepArgs a;          // sizes, relaxation and noise constants, Philox words of this step
  int64_t src, dst;    // value offsets of the blocks read and written
  int64_t tile0;
  int32_t items, cols; // work items and items per row
  int32_t vx, pad;
  FastDiv div_cols, div_Ly;  // division by cols and by Ly
};
static_assert(sizeof(BatchStep) % 16 == 0, "BatchStep is copied as int4 words");

// Step arguments of every member for the clock value *clock_dev (or `clock`
// when clock_dev is null).
__global__ void k_batch_prep(const BatchMember *__restrict__ members, int n, const uint64_t *__restrict__ clock_dev,
                             uint64_t clock, int noise_mode, int noise_dist, BatchStep *__restrict__ out);

// Index m with tile_start[m] <= tile < tile_start[m + 1] (tile_start strictly
// increasing, tile_start[0] = 0 <= tile), found by warp 0: each round tests
// 32 evenly spaced splitters and keeps the segment of the last one passed.
__device__ __forceinline__ int batch_find_member(const int64_t *__restrict__ tile_start, int n, int64_t tile) {
  const int lane = threadIdx.x & 31;
  int lo = 0, len = n;
  while (len > 1) {
    const int stride = (len + 31) >> 5;
    const int idx = lo + lane * stride;
    const bool pass = idx < lo + len && __ldg(tile_start + idx) <= tile;
    const unsigned b = __ballot_sync(0xffffffffu, pass);
    const int k = 31 - __clz(b);
    const int nlo = lo + k * stride;
    len = min(stride, lo + len - nlo);
    lo = nlo;
  }
  return lo;
}

// Minimum resident blocks per SM asked of the register allocator: occupancy
// variant 0 is the single-lattice kernel's choice, variant 1 one block fewer
// (more registers per thread, no spills); the tuner picks between them.
template <int LAT, typename S, int OCC>
constexpr int batch_min_blocks() {
  return OCC == 0 ? step_min_blocks<LAT, S>() : (step_min_blocks<LAT, S>() > 1 ? step_min_blocks<LAT, S>() - 1 : 1);
}

// The work items of one tile of member b (rel: the tile's index within the
// member).  VXMAX = 1: every member takes one site per item (the two-site
// path, with its larger register footprint, is not compiled in); VXMAX = 2:
// members with even Lx take two.
template <int LAT, typename S, int NOISE, int VXMAX>
__device__ __forceinline__ void batch_tile_items(S *__restrict__ base, const BatchStep &b, int rel, int passes) {
  const S *src = base + b.src;
  S *dst = base + b.dst;
  const int first = rel * passes * kBatchThreads + threadIdx.x;
  for (int p = 0; p < passes; ++p) {
    const int item = first + p * kBatchThreads;
    if (item < b.items) {
      const int row = static_cast<int>(fastdiv(static_cast<uint32_t>(item), b.div_cols));
      const int col = item - row * b.cols;
      const int z = static_cast<int>(fastdiv(static_cast<uint32_t>(row), b.div_Ly));
      const int y = row - z * b.a.Ly;
      // a member's value offsets fit 32 bits (checked when it is listed)
      using C = SrtCollide<LAT, typename Store<S>::R, NOISE>;
      if (VXMAX == 2 && b.vx == 2)
        step_vec_body<LAT, S, 2, NOISE, C, uint32_t>(src, dst, b.a, col * 2, y, z);
      else
        step_scalar_body<LAT, S, NOISE, C, uint32_t>(src, dst, b.a, col, y, z);
    }
  }
}

// Warp 0 finds the member of `tile`, copies its arguments to *sb and its
// first tile to *lo (and the end of its tiles to *hi when hi is not null).
__device__ __forceinline__ void batch_load_member(const BatchStep *__restrict__ steps,
                                                  const int64_t *__restrict__ tile_start, int nmembers, int ntiles,
                                                  int tile, BatchStep *sb, int *lo, int *hi) {
  if (threadIdx.x < 32) {
    const int m = batch_find_member(tile_start, nmembers, tile);
    const int4 *g = reinterpret_cast<const int4 *>(steps + m);
    int4 *s = reinterpret_cast<int4 *>(sb);
    for (int k = threadIdx.x; k < int(sizeof(BatchStep) / 16); k += 32) s[k] = g[k];
    if (threadIdx.x == 0) {
      *lo = static_cast<int>(__ldg(tile_start + m));
      if (hi) *hi = m + 1 < nmembers ? static_cast<int>(__ldg(tile_start + m + 1)) : ntiles;
    }
  }
}

// Persistent grid: the tiles of this block are every gridDim.x-th tile from
// blockIdx.x (strided walk) or one run of consecutive tiles (contiguous
// walk), in which the member changes only where the run crosses a member
// boundary.
template <int LAT, typename S, int NOISE, int OCC, int VXMAX>
__global__ void __launch_bounds__(kBatchThreads, batch_min_blocks<LAT, S, OCC>())
    k_batch_step(S *__restrict__ base, const BatchStep *__restrict__ steps, const int64_t *__restrict__ tile_start,
                 int nmembers, int ntiles, int passes, int walk) {
  int tile, stop, stride;
  if (walk == kWalkContiguous) {
    tile = static_cast<int>(int64_t(blockIdx.x) * ntiles / gridDim.x);
    stop = static_cast<int>(int64_t(blockIdx.x + 1) * ntiles / gridDim.x);
    stride = 1;
  } else {
    tile = blockIdx.x;
    stop = ntiles;
    stride = gridDim.x;
  }
  // two copies of the member's arguments and tile range: the copy for the
  // next member is written while no thread reads the copy before the current
  // one any more (one barrier per change of member)
  __shared__ BatchStep sb[2];
  __shared__ int srange[2][2];
  int buf = 1, lo = 0, hi = 0;
  for (; tile < stop; tile += stride) {
    if (tile < lo || tile >= hi) {
      buf ^= 1;
      batch_load_member(steps, tile_start, nmembers, ntiles, tile, &sb[buf], &srange[buf][0], &srange[buf][1]);
      __syncthreads();
      lo = srange[buf][0];
      hi = srange[buf][1];
    }
    batch_tile_items<LAT, S, NOISE, VXMAX>(base, sb[buf], tile - lo, passes);
  }
}

// One tile per block (grid = number of tiles): no loop state is carried
// across tiles, which leaves the per-site code the registers it has in the
// single-lattice kernels.
template <int LAT, typename S, int NOISE, int OCC, int VXMAX>
__global__ void __launch_bounds__(kBatchThreads, batch_min_blocks<LAT, S, OCC>())
    k_batch_tile(S *__restrict__ base, const BatchStep *__restrict__ steps, const int64_t *__restrict__ tile_start,
                 int nmembers, int ntiles, int passes) {
  __shared__ BatchStep sb;
  __shared__ int lo;
  batch_load_member(steps, tile_start, nmembers, ntiles, static_cast<int>(blockIdx.x), &sb, &lo, nullptr);
  __syncthreads();
  batch_tile_items<LAT, S, NOISE, VXMAX>(base, sb, static_cast<int>(blockIdx.x) - lo, passes);
}

template <int LAT, typename S, int NOISE, int OCC, int VXMAX>
cudaError_t batch_step_k(S *b, const BatchStep *steps, const int64_t *tile_start, int nmembers, int ntiles, int passes,
                         int walk, int grid, cudaStream_t stream) {
  if (walk == kWalkPerTile)
    k_batch_tile<LAT, S, NOISE, OCC, VXMAX><<<ntiles, kBatchThreads, 0, stream>>>(b, steps, tile_start, nmembers, ntiles,
                                                                                  passes);
  else
    k_batch_step<LAT, S, NOISE, OCC, VXMAX><<<grid, kBatchThreads, 0, stream>>>(b, steps, tile_start, nmembers, ntiles,
                                                                                passes, walk);
  return cudaGetLastError();
}

template <int LAT, typename S, int OCC, int VXMAX>
cudaError_t batch_step_occ(S *b, const BatchStep *steps, const int64_t *tile_start, int nmembers, int ntiles,
                           int passes, int walk, int noise_mode, int noise_dist, int grid, cudaStream_t stream) {
  if (noise_mode == kNoiseOff)
    return batch_step_k<LAT, S, kStepNoiseOff, OCC, VXMAX>(b, steps, tile_start, nmembers, ntiles, passes, walk, grid,
                                                           stream);
  if (noise_dist == kGaussian)
    return batch_step_k<LAT, S, kStepNoiseGauss, OCC, VXMAX>(b, steps, tile_start, nmembers, ntiles, passes, walk, grid,
                                                             stream);
  return batch_step_k<LAT, S, kStepNoiseFlat, OCC, VXMAX>(b, steps, tile_start, nmembers, ntiles, passes, walk, grid,
                                                          stream);
}

// vx_max: the largest sites per item of any member (1 or 2).
template <int LAT, typename S>
cudaError_t batch_step_t(void *base, const BatchStep *steps, const int64_t *tile_start, int nmembers, int64_t ntiles,
                         int passes, int occ, int walk, int vx_max, int noise_mode, int noise_dist, int grid,
                         cudaStream_t stream) {
  S *b = static_cast<S *>(base);
  if (ntiles >= (int64_t(1) << 31)) return cudaErrorInvalidValue;
  const int nt = static_cast<int>(ntiles);
  if (vx_max == 1) {
    if (occ == 1)
      return batch_step_occ<LAT, S, 1, 1>(b, steps, tile_start, nmembers, nt, passes, walk, noise_mode, noise_dist,
                                          grid, stream);
    return batch_step_occ<LAT, S, 0, 1>(b, steps, tile_start, nmembers, nt, passes, walk, noise_mode, noise_dist, grid,
                                        stream);
  }
  if (occ == 1)
    return batch_step_occ<LAT, S, 1, 2>(b, steps, tile_start, nmembers, nt, passes, walk, noise_mode, noise_dist, grid,
                                        stream);
  return batch_step_occ<LAT, S, 0, 2>(b, steps, tile_start, nmembers, nt, passes, walk, noise_mode, noise_dist, grid,
                                      stream);
}

template <int LAT, typename S, int NOISE, int OCC, int VXMAX>
int batch_blocks_k(int walk) {
  int nb = 0;
  const cudaError_t e =
      walk == kWalkPerTile
          ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_batch_tile<LAT, S, NOISE, OCC, VXMAX>, kBatchThreads, 0)
          : cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_batch_step<LAT, S, NOISE, OCC, VXMAX>, kBatchThreads, 0);
  return e == cudaSuccess && nb > 0 ? nb : 1;
}

template <int LAT, typename S, int OCC, int VXMAX>
int batch_blocks_occ(int walk, int noise_mode, int noise_dist) {
  if (noise_mode == kNoiseOff) return batch_blocks_k<LAT, S, kStepNoiseOff, OCC, VXMAX>(walk);
  if (noise_dist == kGaussian) return batch_blocks_k<LAT, S, kStepNoiseGauss, OCC, VXMAX>(walk);
  return batch_blocks_k<LAT, S, kStepNoiseFlat, OCC, VXMAX>(walk);
}

// Resident blocks per SM of the batch kernel (sizes the persistent grid).
template <int LAT, typename S>
int batch_blocks_per_sm(int occ, int vx_max, int walk, int noise_mode, int noise_dist) {
  if (vx_max == 1)
    return occ == 1 ? batch_blocks_occ<LAT, S, 1, 1>(walk, noise_mode, noise_dist)
                    : batch_blocks_occ<LAT, S, 0, 1>(walk, noise_mode, noise_dist);
  return occ == 1 ? batch_blocks_occ<LAT, S, 1, 2>(walk, noise_mode, noise_dist)
                  : batch_blocks_occ<LAT, S, 0, 2>(walk, noise_mode, noise_dist);
}

}  // namespace lbfd
