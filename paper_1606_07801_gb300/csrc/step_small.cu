// Many steps of a small lattice in one launch.  a.ph must hold the Philox
// words of (seed, lattice id, t0): the kernel keeps its round keys and
// advances the t-dependent words each step.
//
// A lattice whose two population buffers fit in one block's shared memory
// (for example the D1Q3 FP64 line of 256 sites, 12 KB) is otherwise bound by
// launch latency: one launch per step for a few hundred sites.  Here one
// block loads the stored state into shared memory, runs the steps with a
// block barrier between them, and writes the final state back.  Every site
// update is the single-lattice kernels' site-update body (same arithmetic,
// same Philox keys), so the result is bit-identical to one launch per step.
//
// A lattice too large for one block, or one whose arithmetic is too slow for
// one SM (FP64), runs on a thread-block cluster of up to 8 CTAs instead:
// CTA r owns a contiguous slice of the sites and keeps that slice of both
// buffers in its own shared memory; a site's pull reads each neighbour from
// the shared memory of the CTA that owns it (distributed shared memory), and
// one cluster barrier separates the steps.
#include <algorithm>
#include <cooperative_groups.h>
#include <cuda_runtime.h>

#include "step_kernels.cuh"

namespace cg = cooperative_groups;

namespace lbfd {

namespace {

constexpr int kSmallThreads = 512;

// src and dst may be the same buffer (lbfd_step runs an even number of steps
// in place), so neither is __restrict__: every read of src happens before the
// first barrier and every write of dst after the last one.
template <int LAT, typename S, int NOISE>
__global__ void __launch_bounds__(kSmallThreads)
    k_step_small(const S *src, S *dst, const StepArgs a, uint32_t lattice_id, uint64_t t0, int nsteps) {
  extern __shared__ __align__(16) unsigned char smem[];
  const int Q = Lattice<LAT>::Q;
  const int64_t n = static_cast<int64_t>(Q) * a.N;
  S *buf0 = reinterpret_cast<S *>(smem);
  S *buf1 = buf0 + n;
  __shared__ StepArgs sa;
  for (int64_t k = threadIdx.x; k < n; k += blockDim.x) buf0[k] = src[k];
  if (threadIdx.x == 0) sa = a;
  for (int step = 0; step < nsteps; ++step) {
    // a carries the round keys of seed; only the t-dependent words change
    if (threadIdx.x == 0) philox_step_set_t(sa.ph, lattice_id, t0 + static_cast<uint64_t>(step));
    __syncthreads();
    const S *from = (step & 1) ? buf1 : buf0;
    S *to = (step & 1) ? buf0 : buf1;
    for (int s = threadIdx.x; s < a.N; s += blockDim.x) {
      const int x = s % a.Lx, r = s / a.Lx;
      const int y = r % a.Ly, z = r / a.Ly;
      step_scalar_body<LAT, S, NOISE, SrtCollideFor<LAT, S, NOISE>, uint32_t>(from, to, sa, x, y, z);
    }
    __syncthreads();
  }
  const S *last = (nsteps & 1) ? buf1 : buf0;
  for (int64_t k = threadIdx.x; k < n; k += blockDim.x) dst[k] = last[k];
}

template <int LAT, typename S, int NOISE>
cudaError_t small_t(const void *src, void *dst, const StepArgs &a, uint64_t seed, uint32_t lattice_id, uint64_t t0,
                    int nsteps, cudaStream_t stream) {
  const size_t bytes = 2 * size_t(Lattice<LAT>::Q) * size_t(a.N) * sizeof(S);
  // the opt-in above 48 KB of dynamic shared memory, on the current device
  cudaError_t e = cudaFuncSetAttribute(k_step_small<LAT, S, NOISE>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       int(kSmallMaxBytes));
  if (e != cudaSuccess) return e;
  int threads = kSmallThreads;
  while (threads > 32 && threads / 2 >= a.N) threads /= 2;
  k_step_small<LAT, S, NOISE><<<1, threads, bytes, stream>>>(static_cast<const S *>(src), static_cast<S *>(dst), a,
                                                            lattice_id, t0, nsteps);
  return cudaGetLastError();
}

constexpr int kClusterMax = 8;       // portable cluster size
constexpr int kClusterThreads = 256;

// Sites of CTA `rank`: [rank * chunk, min(N, (rank + 1) * chunk)).  As in
// k_step_small, src and dst may be the same buffer: all reads of src come
// before the first cluster barrier and all writes of dst after the last.
template <int LAT, typename S, int NOISE>
__global__ void __launch_bounds__(kClusterThreads)
    k_step_cluster(const S *src, S *dst, const StepArgs a, uint32_t lattice_id, uint64_t t0, int nsteps, int chunk) {
  using L = Lattice<LAT>;
  using R = typename Store<S>::R;
  constexpr int Q = L::Q;
  cg::cluster_group cl = cg::this_cluster();
  const int rank = static_cast<int>(cl.block_rank());
  const int nblk = static_cast<int>(cl.num_blocks());
  extern __shared__ __align__(16) unsigned char smem[];
  S *own[2] = {reinterpret_cast<S *>(smem), reinterpret_cast<S *>(smem) + static_cast<int64_t>(Q) * chunk};
  // step arguments for even and odd steps (Philox words of t0 + step)
  __shared__ StepArgs sa[2];
  __shared__ S *remote[2][kClusterMax];
  const int N = static_cast<int>(a.N);
  const int s0 = rank * chunk, cnt = min(chunk, N - s0);
  for (int k = threadIdx.x; k < Q * cnt; k += blockDim.x) {
    const int i = k / cnt, l = k - i * cnt;
    own[0][i * chunk + l] = src[static_cast<int64_t>(i) * N + s0 + l];
  }
  if (threadIdx.x == 0) {
    sa[0] = a;
    sa[1] = a;
    philox_step_set_t(sa[1].ph, lattice_id, t0 + 1);
  }
  if (threadIdx.x < nblk) {
    remote[0][threadIdx.x] = cl.map_shared_rank(own[0], threadIdx.x);
    remote[1][threadIdx.x] = cl.map_shared_rank(own[1], threadIdx.x);
  }
  cl.sync();  // every slice loaded, pointers and arguments in place
  const uint32_t Lx = static_cast<uint32_t>(a.Lx), Lxy = Lx * static_cast<uint32_t>(a.Ly);
  for (int step = 0; step < nsteps; ++step) {
    const int from = step & 1;
    // the copy for the next step is the one the previous step read, which
    // every thread of the cluster has finished with at the last barrier
    if (threadIdx.x == 0 && step >= 1 && step + 1 < nsteps)
      philox_step_set_t(sa[from ^ 1].ph, lattice_id, t0 + static_cast<uint64_t>(step + 1));
    const StepArgs &args = sa[from];
    for (int l = threadIdx.x; l < cnt; l += blockDim.x) {
      const int s = s0 + l;
      const int x = s % a.Lx, r = s / a.Lx;
      const int y = r % a.Ly, z = r / a.Ly;
      const int xm = (x == 0 ? a.Lx : x) - 1, xp = (x + 1 == a.Lx) ? 0 : x + 1;
      const int ym = (y == 0 ? a.Ly : y) - 1, yp = (y + 1 == a.Ly) ? 0 : y + 1;
      const int zm = (z == 0 ? a.Lz : z) - 1, zp = (z + 1 == a.Lz) ? 0 : z + 1;
      R f[Q];
      static_for<Q>([&](auto I) {
        constexpr int i = decltype(I)::value;
        constexpr int vx = L::v(i, 0), vy = L::v(i, 1), vz = L::v(i, 2);
        const int xs = vx == 0 ? x : (vx > 0 ? xm : xp);
        const int ys = vy == 0 ? y : (vy > 0 ? ym : yp);
        const int zs = vz == 0 ? z : (vz > 0 ? zm : zp);
        const int so = static_cast<int>(static_cast<uint32_t>(xs) + Lx * static_cast<uint32_t>(ys) +
                                        Lxy * static_cast<uint32_t>(zs));
        const int owner = so / chunk;
        f[i] = Store<S>::load(remote[from][owner][i * chunk + (so - owner * chunk)]);
      });
      collide_site<LAT, R, NOISE, Store<S>::kDeviation>(f, static_cast<uint32_t>(s), args);
      static_for<Q>([&](auto I) {
        constexpr int i = decltype(I)::value;
        own[from ^ 1][i * chunk + l] = Store<S>::store(f[i]);
      });
    }
    cl.sync();  // the step's writes are visible cluster-wide before the next reads
  }
  const S *last = own[nsteps & 1];
  for (int k = threadIdx.x; k < Q * cnt; k += blockDim.x) {
    const int i = k / cnt, l = k - i * cnt;
    dst[static_cast<int64_t>(i) * N + s0 + l] = last[i * chunk + l];
  }
}

// CTAs of the cluster for a lattice: enough that each slice of both buffers
// fits kSmallMaxBytes, and for FP64 arithmetic (slow on this GPU) one per 32
// sites; 1 means a single block (k_step_small); 0 means too large.
int small_ctas(int Q, int64_t N, int elem, bool f64) {
  const uint64_t bytes = 2ull * uint64_t(Q) * uint64_t(N) * uint64_t(elem);
  int c = int((bytes + kSmallMaxBytes - 1) / kSmallMaxBytes);
  if (f64) c = std::max<int>(c, int(std::min<int64_t>(kClusterMax, (N + 31) / 32)));
  if (c > kClusterMax) return 0;
  return std::max(c, 1);
}

template <int LAT, typename S, int NOISE>
cudaError_t cluster_t(const void *src, void *dst, const StepArgs &a, uint32_t lattice_id, uint64_t t0, int nsteps,
                      int ctas, cudaStream_t stream) {
  const int chunk = int((a.N + ctas - 1) / ctas);
  const size_t bytes = 2 * size_t(Lattice<LAT>::Q) * size_t(chunk) * sizeof(S);
  cudaError_t e = cudaFuncSetAttribute(k_step_cluster<LAT, S, NOISE>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       int(kSmallMaxBytes));
  if (e != cudaSuccess) return e;
  int threads = kClusterThreads;
  while (threads > 32 && threads / 2 >= chunk) threads /= 2;
  cudaLaunchConfig_t cfg{};
  cfg.gridDim = dim3(ctas, 1, 1);
  cfg.blockDim = dim3(threads, 1, 1);
  cfg.dynamicSmemBytes = bytes;
  cfg.stream = stream;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = ctas;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  // a cluster that the GPU cannot place is reported, not launched
  int placeable = 0;
  e = cudaOccupancyMaxActiveClusters(&placeable, k_step_cluster<LAT, S, NOISE>, &cfg);
  if (e != cudaSuccess) return e;
  if (placeable < 1) return cudaErrorNotSupported;
  return cudaLaunchKernelEx(&cfg, k_step_cluster<LAT, S, NOISE>, static_cast<const S *>(src), static_cast<S *>(dst), a,
                            lattice_id, t0, nsteps, chunk);
}

template <int LAT, typename S, int NOISE>
cudaError_t small_or_cluster(const void *src, void *dst, const StepArgs &a, uint64_t seed, uint32_t lattice_id,
                             uint64_t t0, int nsteps, cudaStream_t stream) {
  const int ctas = small_ctas(Lattice<LAT>::Q, a.N, sizeof(S), sizeof(typename Store<S>::R) == 8);
  if (ctas == 0) return cudaErrorInvalidValue;
  if (ctas == 1) return small_t<LAT, S, NOISE>(src, dst, a, seed, lattice_id, t0, nsteps, stream);
  return cluster_t<LAT, S, NOISE>(src, dst, a, lattice_id, t0, nsteps, ctas, stream);
}

}  // namespace

int small_path_ctas(int lattice, int precision, int64_t N) {
  if (lattice != kD1Q3 && lattice != kD2Q9 && lattice != kD3Q19) return 0;
  if (N < 1) return 0;
  const int Q = lattice == kD1Q3 ? 3 : (lattice == kD2Q9 ? 9 : 19);
  return small_ctas(Q, N, storage_bytes(precision), precision == kStoreF64);
}

bool small_path_fits(int lattice, int precision, int64_t N) { return small_path_ctas(lattice, precision, N) > 0; }

template <int LAT>
cudaError_t small_lat(int precision, const void *src, void *dst, const StepArgs &a, uint64_t seed,
                      uint32_t lattice_id, uint64_t t0, int nsteps, cudaStream_t stream) {
  return dispatch_storage(precision, [&](auto tag) -> cudaError_t {
    using S = typename decltype(tag)::type;
    if (a.noise_mode == kNoiseOff)
      return small_or_cluster<LAT, S, kStepNoiseOff>(src, dst, a, seed, lattice_id, t0, nsteps, stream);
    if (a.noise_dist == kGaussian)
      return small_or_cluster<LAT, S, kStepNoiseGauss>(src, dst, a, seed, lattice_id, t0, nsteps, stream);
    return small_or_cluster<LAT, S, kStepNoiseFlat>(src, dst, a, seed, lattice_id, t0, nsteps, stream);
  });
}

// Single-relaxation lattices only (D2Q5 and moment-space runs take their own kernel).
cudaError_t launch_step_small(int lattice, int precision, const void *src, void *dst, const StepArgs &a, uint64_t seed,
                              uint32_t lattice_id, uint64_t t0, int nsteps, cudaStream_t stream) {
  if (nsteps < 1 || a.N < 1) return cudaErrorInvalidValue;
  switch (lattice) {
    case kD1Q3: return small_lat<kD1Q3>(precision, src, dst, a, seed, lattice_id, t0, nsteps, stream);
    case kD2Q9: return small_lat<kD2Q9>(precision, src, dst, a, seed, lattice_id, t0, nsteps, stream);
    case kD3Q19: return small_lat<kD3Q19>(precision, src, dst, a, seed, lattice_id, t0, nsteps, stream);
  }
  return cudaErrorInvalidValue;
}

}  // namespace lbfd
