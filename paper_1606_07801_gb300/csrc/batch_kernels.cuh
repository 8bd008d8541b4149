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
// Work.  Member m owns tiles [tile_start[m], tile_start[m + 1]) of a flat
// tile list; a tile is `passes` x 256 consecutive work items of one member,
// and an item is vx sites of a row (vx = 2 for even Lx, else 1).  Every item
// runs the per-site code of the single-lattice kernels, so a member evolves
// bit-identically to the same lattice stepped alone.  The step arguments
// (relaxation constants and the Philox words of the member's t) are written
// once per launch and member by k_batch_prep.  Three kernels take the tiles:
//   k_batch_tile   one block per tile; warp 0 finds the member by a 32-way
//                  search of tile_start and copies its arguments to shared
//                  memory;
//   k_batch_param  one block per tile, one launch per group of up to
//                  kParamMembers members whose t-independent arguments are a
//                  kernel parameter (uniform operands, fewer registers); only
//                  the t words come from k_batch_prep's output;
//   k_batch_step   a persistent grid whose blocks take every grid-th tile or
//                  one run of consecutive tiles, reloading the arguments when
//                  the member changes.
#pragma once

#include "fastdiv.cuh"
#include "step_kernels.cuh"

namespace lbfd {

constexpr int kBatchThreads = 256;
// Order in which blocks take tiles: a persistent grid whose blocks take every
// grid-th tile (strided) or one run of consecutive tiles (contiguous), one
// block per tile, or one block per tile with the members' arguments in the
// kernel parameters (one launch per group of members).
constexpr int kWalkStrided = 0, kWalkContiguous = 1, kWalkPerTile = 2, kWalkParam = 3;

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

// What one launch needs of member mb at clock value `now` (its own step
// counter is now - t0).  Host and device share it, so the arguments a launch
// takes from kernel parameters and the ones k_batch_prep writes agree bit for
// bit.
__host__ __device__ inline BatchStep batch_step_of(const BatchMember &mb, uint64_t now, int noise_mode,
                                                   int noise_dist) {
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
  return s;
}

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

// The collision of the batched kernels: one site at a time.  With the
// one-site and two-site item paths in one kernel, colliding two sites at once
// on the packed instructions measured slower (D2Q9 ensemble of 4096
// lattices: 78.6 against 81.2 GLUPS); the results are the same either way.
template <int LAT, typename S, int NOISE>
struct BatchCollide : SrtCollideFor<LAT, S, NOISE> {
  static constexpr bool kPairs = false;
};

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
      using C = BatchCollide<LAT, S, NOISE>;
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

// Members of one parameter-space launch (tile order LBFD_WALK_PARAM): the
// t-independent arguments of at most kParamMembers consecutive members travel
// as a kernel parameter (30.9 KB of the 32 KB parameter space), so the
// per-site code reads them as uniform operands, as the single-lattice kernels
// read theirs.  Only the Philox words of the member's t and the parity of its
// blocks come from the BatchStep that k_batch_prep writes for the launch.
constexpr int kParamMembers = 112;
struct BatchParams {
  int32_t n, first;                      // members first .. first + n - 1 of the batch
  int32_t tile_start[kParamMembers + 1];  // first tile of each, relative to the launch; [n] = tiles
  BatchStep mem[kParamMembers];          // arguments at t = 0 (the t words are replaced)
};
static_assert(sizeof(BatchParams) + 64 <= 32764, "kernel parameters are limited to 32764 bytes");

template <int LAT, typename S, int NOISE, int OCC, int VXMAX>
__global__ void __launch_bounds__(kBatchThreads, batch_min_blocks<LAT, S, OCC>())
    k_batch_param(S *__restrict__ base, const __grid_constant__ BatchParams p, const BatchStep *__restrict__ steps,
                  int passes) {
  const int tile = static_cast<int>(blockIdx.x);
  // the member of this block: a search of uniform (parameter) words
  int lo = 0, hi = p.n;
  while (hi - lo > 1) {
    const int mid = (lo + hi) >> 1;
    if (p.tile_start[mid] <= tile)
      lo = mid;
    else
      hi = mid;
  }
  BatchStep b = p.mem[lo];
  const BatchStep &s = steps[p.first + lo];
  // the t words: e[j] = ((t_hi << 3) | j) ^ K1[0] = e[0] ^ j for j < 8
  const uint32_t e0 = s.a.ph.e[0];
#pragma unroll
  for (int j = 0; j < 8; ++j) b.a.ph.e[j] = e0 ^ static_cast<uint32_t>(j);
  b.a.ph.f = s.a.ph.f;
  b.a.ph.g = s.a.ph.g;
  b.a.ph.q = s.a.ph.q;
  b.src = s.src;
  b.dst = s.dst;
  batch_tile_items<LAT, S, NOISE, VXMAX>(base, b, tile - p.tile_start[lo], passes);
}

template <int LAT, typename S, int NOISE, int OCC, int VXMAX>
cudaError_t batch_param_k(S *b, const BatchParams *groups, int ngroups, const BatchStep *steps, int passes,
                          cudaStream_t stream) {
  for (int g = 0; g < ngroups; ++g) {
    const int tiles = groups[g].tile_start[groups[g].n];
    if (tiles > 0)
      k_batch_param<LAT, S, NOISE, OCC, VXMAX><<<tiles, kBatchThreads, 0, stream>>>(b, groups[g], steps, passes);
  }
  return cudaGetLastError();
}

template <int LAT, typename S, int OCC, int VXMAX>
cudaError_t batch_param_occ(S *b, const BatchParams *groups, int ngroups, const BatchStep *steps, int passes,
                            int noise_mode, int noise_dist, cudaStream_t stream) {
  if (noise_mode == kNoiseOff)
    return batch_param_k<LAT, S, kStepNoiseOff, OCC, VXMAX>(b, groups, ngroups, steps, passes, stream);
  if (noise_dist == kGaussian)
    return batch_param_k<LAT, S, kStepNoiseGauss, OCC, VXMAX>(b, groups, ngroups, steps, passes, stream);
  return batch_param_k<LAT, S, kStepNoiseFlat, OCC, VXMAX>(b, groups, ngroups, steps, passes, stream);
}

// One launch per group of at most kParamMembers members.
template <int LAT, typename S>
cudaError_t batch_param_t(void *base, const BatchParams *groups, int ngroups, const BatchStep *steps, int passes,
                          int occ, int vx_max, int noise_mode, int noise_dist, cudaStream_t stream) {
  S *b = static_cast<S *>(base);
  if (vx_max == 1)
    return occ == 1 ? batch_param_occ<LAT, S, 1, 1>(b, groups, ngroups, steps, passes, noise_mode, noise_dist, stream)
                    : batch_param_occ<LAT, S, 0, 1>(b, groups, ngroups, steps, passes, noise_mode, noise_dist, stream);
  return occ == 1 ? batch_param_occ<LAT, S, 1, 2>(b, groups, ngroups, steps, passes, noise_mode, noise_dist, stream)
                  : batch_param_occ<LAT, S, 0, 2>(b, groups, ngroups, steps, passes, noise_mode, noise_dist, stream);
}

template <int LAT, typename S, int NOISE, int OCC, int VXMAX>
cudaError_t batch_step_k(S *b, const BatchStep *steps, const int64_t *tile_start, int nmembers, int ntiles, int passes,
                         int walk, int grid, cudaStream_t stream) {
  if (walk == kWalkPerTile)
    k_batch_tile<LAT, S, NOISE, OCC, VXMAX><<<ntiles, kBatchThreads, 0, stream>>>(b, steps, tile_start, nmembers,
                                                                                  ntiles, passes);
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
  cudaError_t e;
  if (walk == kWalkParam)
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_batch_param<LAT, S, NOISE, OCC, VXMAX>, kBatchThreads, 0);
  else if (walk == kWalkPerTile)
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_batch_tile<LAT, S, NOISE, OCC, VXMAX>, kBatchThreads, 0);
  else
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_batch_step<LAT, S, NOISE, OCC, VXMAX>, kBatchThreads, 0);
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
