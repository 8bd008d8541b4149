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
#include <cuda_runtime.h>

#include "step_kernels.cuh"

namespace lbfd {

namespace {

constexpr int kSmallThreads = 512;

template <int LAT, typename S, int NOISE>
__global__ void __launch_bounds__(kSmallThreads)
    k_step_small(const S *__restrict__ src, S *__restrict__ dst, const StepArgs a, uint32_t lattice_id, uint64_t t0,
                 int nsteps) {
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
      step_scalar_body<LAT, S, NOISE, SrtCollide<LAT, typename Store<S>::R, NOISE>, uint32_t>(from, to, sa, x, y, z);
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

}  // namespace

template <int LAT>
cudaError_t small_lat(int precision, const void *src, void *dst, const StepArgs &a, uint64_t seed,
                      uint32_t lattice_id, uint64_t t0, int nsteps, cudaStream_t stream) {
  return dispatch_storage(precision, [&](auto tag) -> cudaError_t {
    using S = typename decltype(tag)::type;
    if (!small_fits(Lattice<LAT>::Q, a.N, sizeof(S))) return cudaErrorInvalidValue;
    if (a.noise_mode == kNoiseOff) return small_t<LAT, S, kStepNoiseOff>(src, dst, a, seed, lattice_id, t0, nsteps, stream);
    if (a.noise_dist == kGaussian)
      return small_t<LAT, S, kStepNoiseGauss>(src, dst, a, seed, lattice_id, t0, nsteps, stream);
    return small_t<LAT, S, kStepNoiseFlat>(src, dst, a, seed, lattice_id, t0, nsteps, stream);
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
