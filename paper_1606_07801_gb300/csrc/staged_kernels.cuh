// The fused fluctuating lattice-Boltzmann step with the pull staged through
// shared memory by the tensor-memory-access (TMA) unit.  Included by one
// translation unit per lattice.
//
// The site update is the one of step_kernels.cuh (collide_site: density,
// relaxation, Philox noise in the non-conserved moments, back-transform), so
// the result is bit-identical to the register-pull kernels.  What differs is
// how the populations move (paper Sec. II, eq. LB, pull form):
//   - A tile is W consecutive sites of one row (y, z).  For each population
//     i, its source is the same W columns of row (y - v_iy, z - v_iz), plus,
//     where v_ix != 0, the one column left or right of them (periodic).  One
//     thread issues, per population, a bulk copy of the W columns and, where
//     needed, a 16-byte copy holding the neighbour column
//     (cp.async.bulk ... mbarrier::complete_tx), into a stage buffer of
//     shared memory; an mbarrier completes when all bytes have landed.
//   - The consumer warps pull f_i(x, t) for their sites from the stage
//     buffer (the x shift is an index offset; the y/z shift was done by the
//     choice of source row), release the buffer, collide in registers and
//     store f*_i straight to global memory (VX-wide stores per population).
//   - A producer warp keeps the copies NS tiles ahead: the grid is
//     persistent, CTA b takes tiles b, b + G, b + 2G, ..., its local tile k
//     lives in stage k mod NS (NS = 3), and a stage is refilled as soon as
//     every consumer warp has pulled from it.  Memory latency is hidden by
//     the copy engine instead of by more resident warps, no consumer spends
//     issue slots on load addresses, and no warp waits on a block-wide
//     barrier.
// Every mbarrier wait is bounded (about one second of wall time).  A wait
// that gives up records a non-zero status in *status (the host reports
// LBFD_ETIMEOUT) and its warp leaves the tile loop; the other warps' waits
// then run out in turn, so the kernel ends within a few seconds.
//
// Requirements (checked by the host): every population row starts on a
// 16-byte boundary (Lx * sizeof(S) a multiple of 16, both buffers 16-byte
// aligned) and the lattice has fewer than 2^31 sites.
#pragma once

#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>

#include "sample_kernels.cuh"
#include "step_kernels.cuh"

namespace lbfd {

// ---------------------------------------------------------------------------
// PTX wrappers: mbarrier, bulk asynchronous copies, proxy fences
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint32_t smem_u32(const void *p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

// Makes the initialised barriers visible to the asynchronous proxy (the copy
// engine) before any copy signals them.
__device__ __forceinline__ void fence_mbar_init() { asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory"); }

// Raises the number of bytes the current phase waits for.
__device__ __forceinline__ void mbar_expect_tx(uint64_t *bar, uint32_t bytes) {
  asm volatile("mbarrier.expect_tx.relaxed.cta.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
               : "memory");
}

__device__ __forceinline__ void mbar_arrive(uint64_t *bar) {
  uint64_t state;
  asm volatile("mbarrier.arrive.shared::cta.b64 %0, [%1];" : "=l"(state) : "r"(smem_u32(bar)) : "memory");
  (void)state;
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t parity) {
  uint32_t done;
  asm volatile(
      "{\n"
      " .reg .pred p;\n"
      " mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
      " selp.u32 %0, 1, 0, p;\n"
      "}\n"
      : "=r"(done)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return done != 0;
}

__device__ __forceinline__ uint64_t global_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// Wall-time limit of one mbarrier wait, and a cap on its polls.
constexpr uint64_t kStagedWaitNs = 1000000000ull;
constexpr uint32_t kStagedWaitPolls = 1u << 26;

// Waits for the phase of the given parity; false when it did not complete
// within the limits.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t *bar, uint32_t parity) {
  if (mbar_try_wait(bar, parity)) return true;
  const uint64_t t0 = global_ns();
  for (uint32_t k = 1; k < kStagedWaitPolls; ++k) {
    if (mbar_try_wait(bar, parity)) return true;
    if ((k & 255u) == 0 && global_ns() - t0 > kStagedWaitNs) return false;
  }
  return false;
}

// Global -> shared bulk copy (both addresses and the size multiples of 16
// bytes) that completes `bytes` transactions on bar.
__device__ __forceinline__ void bulk_load(void *dst_smem, const void *src_gmem, uint32_t bytes, uint64_t *bar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                   smem_u32(dst_smem)),
               "l"(src_gmem), "r"(bytes), "r"(smem_u32(bar))
               : "memory");
}

// Orders this thread's generic-proxy shared-memory writes before later
// async-proxy (bulk copy) reads of them.
__device__ __forceinline__ void fence_proxy_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

// ---------------------------------------------------------------------------
// Tile shapes
// ---------------------------------------------------------------------------
// kW sites per tile (a multiple of the 16-byte chunk), kVX sites per
// consumer thread, kStages stage buffers, kMinBlocks resident blocks per SM
// asked of the register allocator.  A block is kW / kVX consumer threads and
// one producer warp.
template <int LAT, typename S>
struct StagedShape {
  static constexpr bool kF64 = sizeof(typename Store<S>::R) == 8;
  static constexpr int kW = LAT == kD3Q19 ? (kF64 ? 128 : 256) : (kF64 ? 256 : 512);
  static constexpr int kVX = LAT == kD3Q19 ? 1 : 2;
  static constexpr int kConsumers = kW / kVX;
  static constexpr int kConsumerWarps = kConsumers / 32;
  static constexpr int kThreads = kConsumers + 32;
  static constexpr int kStages = 3;
  static constexpr int kMinBlocks = kF64 ? 2 : (LAT == kD3Q19 ? 3 : 4);
  static constexpr int kChunk = 16 / static_cast<int>(sizeof(S));  // elements of one 16-byte chunk
  static constexpr int kRow = kW + 2 * kChunk;                       // elements of a population row of a stage
  static constexpr int kStage = Lattice<LAT>::Q * kRow;              // elements of a stage buffer
  static constexpr size_t kSmemBytes = size_t(kStages) * kStage * sizeof(S);
  static_assert(kW % kChunk == 0 && kChunk % kVX == 0, "tile width and sites per thread must fit the chunk");
  static_assert(kConsumers % 32 == 0, "consumers are whole warps");
};

// Tile coordinates, written by the producer with the copies and read by the
// consumers once the stage's full barrier has completed.
struct StagedTile {
  int32_t row;  // y + Ly z
  int32_t x0;   // first column
  int32_t wt;   // columns in this tile (kW, or less at the end of a row)
  int32_t pad;
};

// Issues the copies of tile `tile` into stage buffer st; bar completes when
// every byte has landed.  Population i's row in the stage holds, at
// [kChunk, kChunk + wt), columns x0 .. x0 + wt - 1 of its source row
// (y - v_iy, z - v_iz); for v_ix = +1 the chunk before it ends with column
// x0 - 1, for v_ix = -1 the chunk after it starts with column x0 + wt
// (periodic in x).  Each copy raises the barrier's byte count by its own
// size before it is issued, and the one arrival comes last, so the phase
// cannot complete early.
template <int LAT, typename S>
__device__ __forceinline__ void staged_issue(const S *__restrict__ src, S *st, uint64_t *bar, StagedTile *meta,
                                             uint32_t tile, uint32_t ntx, uint32_t row_begin, const StepArgs &a) {
  using L = Lattice<LAT>;
  using SH = StagedShape<LAT, S>;
  constexpr int Q = L::Q, H = SH::kChunk, ROW = SH::kRow;
  const uint32_t tr = tile / ntx, xt = tile - tr * ntx;
  const uint32_t row = row_begin + tr;
  const int x0 = static_cast<int>(xt) * SH::kW;
  const int wt = min(SH::kW, a.Lx - x0);
  const int y = static_cast<int>(row % static_cast<uint32_t>(a.Ly)), z = static_cast<int>(row / static_cast<uint32_t>(a.Ly));
  meta->row = static_cast<int32_t>(row);
  meta->x0 = x0;
  meta->wt = wt;
  const int ym = (y == 0 ? a.Ly : y) - 1, yp = (y + 1 == a.Ly) ? 0 : y + 1;
  const int zm = (z == 0 ? a.Lz : z) - 1, zp = (z + 1 == a.Lz) ? 0 : z + 1;
  const int xl = (x0 == 0 ? a.Lx : x0) - H;         // chunk ending with column x0 - 1
  const int xr = (x0 + wt == a.Lx) ? 0 : x0 + wt;   // chunk starting with column x0 + wt
  const uint32_t main_bytes = static_cast<uint32_t>(wt) * sizeof(S);
  static_for<Q>([&](auto I) {
    constexpr int i = decltype(I)::value;
    constexpr int vx = L::v(i, 0), vy = L::v(i, 1), vz = L::v(i, 2);
    const int ys = vy == 0 ? y : (vy > 0 ? ym : yp);
    const int zs = vz == 0 ? z : (vz > 0 ? zm : zp);
    const S *g = src + (static_cast<size_t>(i) * static_cast<size_t>(a.N) +
                        static_cast<size_t>(a.Lx) * (static_cast<size_t>(ys) + static_cast<size_t>(a.Ly) * zs));
    S *r = st + i * ROW;
    mbar_expect_tx(bar, main_bytes);
    bulk_load(r + H, g + x0, main_bytes, bar);
    if constexpr (vx > 0) {
      mbar_expect_tx(bar, 16u);
      bulk_load(r, g + xl, 16u, bar);
    } else if constexpr (vx < 0) {
      mbar_expect_tx(bar, 16u);
      bulk_load(r + H + wt, g + xr, 16u, bar);
    }
  });
  mbar_arrive(bar);
}

// Populations f_i(x, t) of sites k0 .. k0 + VX - 1 of the tile in stage st
// (site k pulls column k - v_ix of population i's stage row).
template <int LAT, typename S, int VX>
__device__ __forceinline__ void staged_pull(const S *st, int k0, typename Store<S>::R (&f)[VX][Lattice<LAT>::Q],
                                            const StepArgs &a) {
  using L = Lattice<LAT>;
  using SH = StagedShape<LAT, S>;
  using P = Pack<S, VX>;
  constexpr int Q = L::Q, H = SH::kChunk, ROW = SH::kRow;
  static_for<Q>([&](auto I) {
    constexpr int i = decltype(I)::value;
    constexpr int vx = L::v(i, 0);
    const S *r = st + i * ROW + H + k0;
    typename Store<S>::R v[VX];
    PackCvt<S, VX>::load(*reinterpret_cast<const P *>(r), v);
    if constexpr (vx == 0) {
#pragma unroll
      for (int k = 0; k < VX; ++k) f[k][i] = v[k];
    } else if constexpr (vx > 0) {
      f[0][i] = Store<S>::load(r[-1]);
#pragma unroll
      for (int k = 1; k < VX; ++k) f[k][i] = v[k - 1];
    } else {
#pragma unroll
      for (int k = 0; k < VX - 1; ++k) f[k][i] = v[k + 1];
      f[VX - 1][i] = Store<S>::load(r[VX]);
    }
  });
}

// Stores f*_i of sites (x, .. x + VX - 1) of a row to global memory: one
// VX-wide store per population at value offset i N + off.
template <int LAT, typename S, int VX>
__device__ __forceinline__ void staged_store_regs(S *__restrict__ dst, uint32_t off,
                                                  const typename Store<S>::R (&f)[VX][Lattice<LAT>::Q],
                                                  const StepArgs &a) {
  using P = Pack<S, VX>;
  constexpr int Q = Lattice<LAT>::Q;
  S *p = dst + off;
  static_for<Q>([&](auto I) {
    constexpr int i = decltype(I)::value;
    typename Store<S>::R v[VX];
#pragma unroll
    for (int k = 0; k < VX; ++k) v[k] = f[k][i];
    *reinterpret_cast<P *>(p + static_cast<size_t>(i) * static_cast<size_t>(a.N)) = PackCvt<S, VX>::store(v);
  });
}

// Status codes a staged kernel leaves in *status (0 = fine).
constexpr int kStagedTimeout = 1;

// StagedRows (internal.h): the rows a launch updates and how their sites
// are keyed: rows row_begin .. row_begin + nrows - 1 of the stored lattice
// (row = y + Ly z), and site x of row r draws the noise of global site
// (r + row_key) Lx + x (modulo 2^32).  A whole lattice is {0, Ly Lz, 0}; a
// slab with one halo plane on each side skips the first and last planes and
// keys its rows by their global position.
//
// Roles.  The last warp of the block is the producer: its first lane issues
// the copies of the CTA's tiles into the stage buffers, local tile k into
// stage k mod NS, and before reusing a stage waits until every consumer warp
// has released it.  The other warps are consumers: for each tile they wait
// for its stage to fill, pull their sites' populations into registers,
// release the stage (one arrival per warp), collide and store to global
// memory.  No thread ever waits on a block-wide barrier after set-up, so a
// warp's progress depends only on its own work and on the copies.
//
// SAMPLE: the step also adds the observables of the state it reads
// (sample_kernels.cuh): each consumer warp feeds its pulled sites to a warp
// sampler, and at the end the consumers write the block's partial sums to
// partials[blockIdx.x] (the grid is at most kObsBlocks).
// Resident blocks per SM the sampled kernel is compiled for: two, whose
// 4.5-warp share of each scheduler's 16384 registers allows 96 per thread.
constexpr int kStagedSampleMinBlocks = 2;

// Whether the staged kernel collides its sites two at a time (collide_pair):
// as the register-pull kernel does.
template <int LAT, typename S, int VX, bool SAMPLE>
__host__ __device__ constexpr bool staged_pairs() {
  return step_pairs<LAT, S, VX>();
}

template <int LAT, typename S, int NOISE, bool SAMPLE = false>
__global__ void __launch_bounds__(StagedShape<LAT, S>::kThreads,
                                  SAMPLE ? kStagedSampleMinBlocks : StagedShape<LAT, S>::kMinBlocks)
    k_step_staged(const S *__restrict__ src, S *__restrict__ dst, const StepArgs a, uint32_t ntiles, uint32_t ntx,
                  const StagedRows rows, int *status, uint32_t wait_test_bytes, const SampleArgs sa,
                  double *__restrict__ partials) {
  using SH = StagedShape<LAT, S>;
  using R = typename Store<S>::R;
  using WS = SamplerFor<LAT, SH::kVX>;
  constexpr int Q = Lattice<LAT>::Q, NS = SH::kStages, VX = SH::kVX;
  extern __shared__ __align__(128) unsigned char staged_smem[];
  S *stages = reinterpret_cast<S *>(staged_smem);
  typename WS::Smem *wsm = reinterpret_cast<typename WS::Smem *>(staged_smem + SH::kSmemBytes);
  __shared__ __align__(8) uint64_t full[NS], empty[NS];
  __shared__ StagedTile meta[NS];

  if constexpr (!SAMPLE) pdl_launch_dependents();  // the sampled form is launched plainly (as k_step_sample)
  const uint32_t G = gridDim.x;
  const int warp = static_cast<int>(threadIdx.x) >> 5, lane = static_cast<int>(threadIdx.x) & 31;
  if (threadIdx.x == 0) {
#pragma unroll
    for (int s = 0; s < NS; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], SH::kConsumerWarps);
    }
    fence_mbar_init();
    fence_proxy_async_smem();
  }
  __syncthreads();
  // the previous step's grid has finished reading this step's destination
  // and writing its source
  pdl_wait();

  if (warp == SH::kConsumerWarps) {  // producer
    if (lane != 0) return;
    // tests of the bounded wait only: bytes that no copy delivers, so the
    // first tile's wait runs out (every issued copy still lands)
    if (wait_test_bytes) mbar_expect_tx(&full[0], wait_test_bytes);
    uint32_t k = 0;
    bool ok = true;
    for (uint32_t tile = blockIdx.x; tile < ntiles; tile += G, ++k) {
      const uint32_t s = k % NS;
      // stage s last held local tile k - NS: all consumer warps must have
      // pulled from it (its release is the (k / NS - 1)-th phase of empty[s])
      if (k >= NS && !mbar_wait_bounded(&empty[s], ((k / NS) - 1) & 1u)) {
        ok = false;
        break;
      }
      staged_issue<LAT, S>(src, stages + s * SH::kStage, &full[s], &meta[s], tile, ntx, rows.row_begin, a);
    }
    if (!ok) {
      // let the copies still in flight land before the CTA's shared memory
      // is released: the last NS issued tiles hold distinct stages
      for (uint32_t j = k > NS ? k - NS : 0; j < k; ++j) (void)mbar_wait_bounded(&full[j % NS], (j / NS) & 1u);
      *reinterpret_cast<volatile int *>(status) = kStagedTimeout;
    }
    return;
  }

  // consumers
  const int k0 = static_cast<int>(threadIdx.x) * VX;
  WS ws;
  if constexpr (SAMPLE) ws.init(&wsm[warp], lane);
  uint32_t it = 0;
  for (uint32_t tile = blockIdx.x; tile < ntiles; tile += G, ++it) {
    const uint32_t s = it % NS;
    // every lane waits (each needs the barrier's acquire of the copied
    // data); the warp gives up together if any lane's wait ran out
    const bool landed = mbar_wait_bounded(&full[s], (it / NS) & 1u);
    if (!__all_sync(0xffffffffu, landed)) {
      if (lane == 0) *reinterpret_cast<volatile int *>(status) = kStagedTimeout;
      break;
    }
    const StagedTile m = meta[s];
    const bool mine = k0 < m.wt;
    R f[VX][Q];
    if (mine) staged_pull<LAT, S, VX>(stages + s * SH::kStage, k0, f, a);
    __syncwarp();
    if (lane == 0) mbar_arrive(&empty[s]);  // this warp is done with stage s
    if constexpr (SAMPLE) {
      const int y = m.row % a.Ly, z = m.row / a.Ly;
      ws.template add<S>(f, mine, m.x0 + k0, y, z, a.Lx, a.Ly, a.Lz, sa);
    }
    if (mine) {
      const uint32_t off = static_cast<uint32_t>(m.row) * static_cast<uint32_t>(a.Lx) + static_cast<uint32_t>(m.x0 + k0);
      const uint32_t key = off + rows.row_key * static_cast<uint32_t>(a.Lx);
      collide_sites<LAT, S, VX, NOISE, staged_pairs<LAT, S, VX, SAMPLE>()>(f, key, a);
      staged_store_regs<LAT, S, VX>(dst, off, f, a);
    }
  }
  if constexpr (SAMPLE) {
    ws.flush(sa.K);
    // the consumers only (the producer warp has left): named barrier 1
    auto sync = [] { asm volatile("bar.sync 1, %0;" ::"r"(SH::kConsumers) : "memory"); };
    sync();
    const int nq = 2 + Q + 2 * sa.K + Q * (Q + 1) / 2;
    WS::block_partials(wsm, SH::kConsumerWarps, sa.K, partials + static_cast<size_t>(blockIdx.x) * nq,
                       static_cast<int>(threadIdx.x), SH::kConsumers, sync);
  }
}

// Tiles along x and in total for nrows rows.
template <int LAT, typename S>
inline void staged_tiles(const StepArgs &a, uint32_t nrows, uint32_t &ntx, uint32_t &ntiles) {
  ntx = static_cast<uint32_t>((a.Lx + StagedShape<LAT, S>::kW - 1) / StagedShape<LAT, S>::kW);
  ntiles = ntx * nrows;
}

// Whether the staged kernel can run a lattice stored in S: every row must
// start on a 16-byte boundary (the buffers themselves are checked by the
// caller), and the tile count must fit 32 bits.
template <typename S>
inline bool staged_fits_t(int32_t Lx, int64_t N) {
  return (static_cast<int64_t>(Lx) * static_cast<int64_t>(sizeof(S))) % 16 == 0 && N < (int64_t(1) << 31);
}

template <int LAT, typename S, int NOISE, bool SAMPLE = false>
cudaError_t staged_noise(const void *src, void *dst, const StepArgs &a, const StagedRows &rows, int *status,
                         uint32_t wait_test_bytes, cudaStream_t stream, const SampleArgs &sa = SampleArgs{},
                         double *partials = nullptr, int *nblocks = nullptr) {
  using SH = StagedShape<LAT, S>;
  auto kern = k_step_staged<LAT, S, NOISE, SAMPLE>;
  const size_t smem =
      SH::kSmemBytes + (SAMPLE ? SH::kConsumerWarps * sizeof(typename SamplerFor<LAT, SH::kVX>::Smem) : 0);
  // resident CTAs per SM times SMs, found once (after a successful query)
  static std::atomic<int> slots{0};
  int g = slots.load(std::memory_order_relaxed);
  if (g == 0) {
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem));
    int dev = 0, sms = 0, occ = 0;
    if (e == cudaSuccess) e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, SH::kThreads, smem);
    if (e != cudaSuccess) return e;
    if (occ < 1 || sms < 1) return cudaErrorInvalidConfiguration;
    g = occ * sms;
    if (SAMPLE) g = std::min(g, kObsBlocks);  // one partial set per block
    slots.store(g, std::memory_order_relaxed);
  }
  uint32_t ntx = 0, ntiles = 0;
  staged_tiles<LAT, S>(a, rows.nrows, ntx, ntiles);
  if (ntiles == 0) return cudaSuccess;
  const uint32_t grid = static_cast<uint32_t>(std::min<int64_t>(ntiles, g));
  if (nblocks) *nblocks = static_cast<int>(grid);
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(grid, 1, 1);
  cfg.blockDim = dim3(SH::kThreads, 1, 1);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = stream;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = step_pdl() && !SAMPLE ? 1 : 0;
  return cudaLaunchKernelEx(&cfg, kern, static_cast<const S *>(src), static_cast<S *>(dst), a, ntiles, ntx, rows,
                            status, wait_test_bytes, sa, partials);
}

template <int LAT, typename S>
cudaError_t staged_t(const void *src, void *dst, const StepArgs &a, const StagedRows &rows, int *status,
                     uint32_t wait_test_bytes, cudaStream_t stream) {
  if (a.noise_mode == kNoiseOff)
    return staged_noise<LAT, S, kStepNoiseOff>(src, dst, a, rows, status, wait_test_bytes, stream);
  if (a.noise_dist == kGaussian)
    return staged_noise<LAT, S, kStepNoiseGauss>(src, dst, a, rows, status, wait_test_bytes, stream);
  return staged_noise<LAT, S, kStepNoiseFlat>(src, dst, a, rows, status, wait_test_bytes, stream);
}

// The fused step-and-sample launch (FP32 arithmetic): the register-pull
// kernel on a persistent grid, with the per-lane register sampler for D1Q3
// and D2Q9 and the tensor-core sampler for D3Q19 (measured on GB300, the
// staged kernel with the same samplers was no faster: for D2Q9 at the one
// block per SM its registers allow; for D3Q19 16-bit 256^3 at a sample every
// 10 steps 36.8 against 37.7 GLUPS).  LBFD_SAMPLE_STAGED = 1 takes the
// staged kernel for D3Q19 where the lattice meets its requirements and two
// of its blocks fit the 228 KB of shared memory of an SM (a tuning knob; the
// results agree within FP32 rounding of the sums, and the state bit for bit).
inline bool sample_staged_default() {
  static const bool v = [] {
    const char *e = getenv("LBFD_SAMPLE_STAGED");
    return e && atoi(e) == 1;
  }();
  return v;
}

template <int LAT, typename S>
cudaError_t step_sample_t(const void *src, void *dst, const StepArgs &a, int n_modes, const void *phase,
                          double *partials, int *nblocks, bool staged_ok, int *status, cudaStream_t stream) {
  if constexpr (sizeof(typename Store<S>::R) != 4) {
    return cudaErrorInvalidValue;  // FP64 storage samples in FP64 by its own pass
  } else if constexpr (Lattice<LAT>::Q <= 9) {
    if (n_modes < 0 || n_modes > kFusedModes || (n_modes > 0 && !phase)) return cudaErrorInvalidValue;
    return sample_vec_t<LAT, S>(src, dst, a, n_modes, phase, partials, nblocks, stream);
  } else {
    if (n_modes < 0 || n_modes > kFusedModes || (n_modes > 0 && !phase)) return cudaErrorInvalidValue;
    using SH = StagedShape<LAT, S>;
    using WS = WarpSampler<LAT, SH::kVX>;
    constexpr bool fits = kStagedSampleMinBlocks * (SH::kSmemBytes + SH::kConsumerWarps * sizeof(typename WS::Smem) +
                                                    1024) <= 228 * 1024;
    if (!(fits && staged_ok && sample_staged_default()))
      return sample_vec_t<LAT, S>(src, dst, a, n_modes, phase, partials, nblocks, stream);
    const SampleArgs sa = make_sample_args<LAT>(a, n_modes, phase, dim3(1, 1, 1));
    const StagedRows rows{0, static_cast<uint32_t>(a.Ly) * static_cast<uint32_t>(a.Lz), 0};
    if (a.noise_mode == kNoiseOff)
      return staged_noise<LAT, S, kStepNoiseOff, true>(src, dst, a, rows, status, 0, stream, sa, partials, nblocks);
    if (a.noise_dist == kGaussian)
      return staged_noise<LAT, S, kStepNoiseGauss, true>(src, dst, a, rows, status, 0, stream, sa, partials, nblocks);
    return staged_noise<LAT, S, kStepNoiseFlat, true>(src, dst, a, rows, status, 0, stream, sa, partials, nblocks);
  }
}

}  // namespace lbfd
