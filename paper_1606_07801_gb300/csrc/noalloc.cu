// lbfd_mass_noalloc: the FP64 mass reduction for callers that may not
// allocate device memory.
//
// Some callers cannot call cudaMalloc where they need the mass: a host
// framework that reserved the whole GPU for its own caching allocator and
// forbids other libraries to allocate, a service that runs under a fixed
// device-memory budget, or a time-critical loop that must not pay for
// cudaMalloc/cudaFree (which can synchronise the device).  This entry point
// takes the caller's population array and a caller-owned output slot, and
// keeps its per-block partial sums in a file-scope device array instead of
// allocating scratch.  The first call on each device looks up that array's
// device address; make that first call before any stream capture.  A lookup
// that fails is not remembered: the next call on that device tries again.
//
// The scratch array is kNoAllocMaxBlocks doubles (128 KiB).  Every GPU that
// loads this library holds it until the process exits.  One block reduces
// kSitesPerBlock sites, so a call accepts at most
// kNoAllocMaxBlocks * kSitesPerBlock = 16,777,216 sites.  Every call writes
// all the slots it reads, so nothing has to start at zero; the array keeps
// the last call's partials.  All calls share the one array: two calls whose
// kernels overlap on the GPU (different streams, no ordering between them)
// race on it and may return wrong sums.  Order such calls on one stream.
#include <cuda_runtime.h>

#include <mutex>
#include <string>

#include "device.cuh"
#include "internal.h"
#include "lbfd.h"

namespace lbfd {

constexpr int kNoAllocThreads = 256;
constexpr int kSitesPerThread = 4;
constexpr int64_t kSitesPerBlock = int64_t(kNoAllocThreads) * kSitesPerThread;
constexpr int kNoAllocMaxBlocks = 16384;
constexpr int kNoAllocMaxDevices = 64;

static __device__ __align__(256) double g_noalloc_partials[kNoAllocMaxBlocks];

// Stage 1: block b sums sites [b * kSitesPerBlock, (b + 1) * kSitesPerBlock)
// in a fixed order and writes partials[b].
template <int LAT, typename R>
__global__ void __launch_bounds__(kNoAllocThreads) k_mass_tile_partials(const R *__restrict__ f, int64_t N,
                                                                       double *__restrict__ partials) {
  using L = Lattice<LAT>;
  __shared__ double warp_tot[kNoAllocThreads / 32];
  const int64_t base = blockIdx.x * kSitesPerBlock;
  double acc = 0.0;
#pragma unroll
  for (int k = 0; k < kSitesPerThread; ++k) {
    const int64_t s = base + int64_t(k) * kNoAllocThreads + threadIdx.x;
    if (s < N) {
      double r = 0.0;
      static_for<L::Q>([&](auto I) { r += static_cast<double>(f[decltype(I)::value * N + s]); });
      acc += r;
    }
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
  if ((threadIdx.x & 31) == 0) warp_tot[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < kNoAllocThreads / 32; ++w) t += warp_tot[w];
    partials[blockIdx.x] = t;
  }
}

// Stage 2: one block adds the partials in a fixed order into *out.
__global__ void __launch_bounds__(kNoAllocThreads) k_mass_tile_total(const double *__restrict__ partials, int nblocks,
                                                                    double *__restrict__ out) {
  __shared__ double lane_tot[kNoAllocThreads];
  double t = 0.0;
  for (int b = threadIdx.x; b < nblocks; b += kNoAllocThreads) t += partials[b];
  lane_tot[threadIdx.x] = t;
  __syncthreads();
  for (int half = kNoAllocThreads / 2; half > 0; half >>= 1) {
    if (threadIdx.x < half) lane_tot[threadIdx.x] += lane_tot[threadIdx.x + half];
    __syncthreads();
  }
  if (threadIdx.x == 0) *out = lane_tot[0];
}

// Launches both stages.  The caller has cleared the thread's last runtime
// error, so the check after each launch sees only that launch's own error.
template <int LAT, typename R>
static cudaError_t mass_tiles(const void *f, int64_t N, double *scratch, double *out, cudaStream_t stream) {
  const int nblocks = static_cast<int>((N + kSitesPerBlock - 1) / kSitesPerBlock);
  k_mass_tile_partials<LAT, R><<<nblocks, kNoAllocThreads, 0, stream>>>(static_cast<const R *>(f), N, scratch);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  k_mass_tile_total<<<1, kNoAllocThreads, 0, stream>>>(scratch, nblocks, out);
  return cudaGetLastError();
}

// Device address of the scratch array, looked up with the device current
// and cached per device once the lookup has succeeded.  A failed lookup (for
// example one made during a stream capture) is not cached, so a later call
// tries again.
static double *g_scratch_addr[kNoAllocMaxDevices] = {};
static std::mutex g_scratch_mutex;

static cudaError_t scratch_for_current_device(double **ptr) {
  int dev = -1;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kNoAllocMaxDevices) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(g_scratch_mutex);
  if (!g_scratch_addr[dev]) {
    void *p = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_partials);
    if (e != cudaSuccess) return e;
    g_scratch_addr[dev] = static_cast<double *>(p);
  }
  *ptr = g_scratch_addr[dev];
  return cudaSuccess;
}

// Records a failed CUDA call as the thread's lbfd_last_error() and clears the
// runtime's per-thread last error, so that the next launch check elsewhere
// does not report it again.
static int noalloc_cuda_fail(const char *what, cudaError_t e) {
  (void)cudaGetLastError();
  return set_last_error(LBFD_ECUDA, std::string("lbfd_mass_noalloc: ") + what + ": " + cudaGetErrorName(e) + " (" +
                                        cudaGetErrorString(e) + ")");
}

}  // namespace lbfd

using namespace lbfd;

extern "C" int lbfd_mass_noalloc(int32_t lattice, int32_t precision, const void *f_dev, int64_t n_sites,
                                 double *mass_dev, void *stream) {
  if (!f_dev || !mass_dev) return set_last_error(LBFD_EINVAL, "lbfd_mass_noalloc: null pointer");
  if (lattice < LBFD_D1Q3 || lattice > LBFD_D3Q19 || (precision != LBFD_F32 && precision != LBFD_F64))
    return set_last_error(LBFD_EINVAL, "lbfd_mass_noalloc: unknown lattice or precision");
  if (n_sites < 1 || n_sites > int64_t(kNoAllocMaxBlocks) * kSitesPerBlock)
    return set_last_error(LBFD_EINVAL,
                          "lbfd_mass_noalloc: n_sites must be between 1 and 16777216, the capacity of its fixed scratch");
  double *scratch = nullptr;
  cudaError_t e = scratch_for_current_device(&scratch);
  if (e != cudaSuccess) return noalloc_cuda_fail("cudaGetSymbolAddress", e);
  // an error left on this thread by earlier, unrelated work is not this
  // call's: report it as such before launching anything
  e = cudaGetLastError();
  if (e != cudaSuccess) return noalloc_cuda_fail("earlier CUDA error pending on this thread", e);
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const bool f64 = precision == LBFD_F64;
  switch (lattice) {
    case LBFD_D1Q3:
      e = f64 ? mass_tiles<kD1Q3, double>(f_dev, n_sites, scratch, mass_dev, s)
              : mass_tiles<kD1Q3, float>(f_dev, n_sites, scratch, mass_dev, s);
      break;
    case LBFD_D2Q9:
      e = f64 ? mass_tiles<kD2Q9, double>(f_dev, n_sites, scratch, mass_dev, s)
              : mass_tiles<kD2Q9, float>(f_dev, n_sites, scratch, mass_dev, s);
      break;
    default:
      e = f64 ? mass_tiles<kD3Q19, double>(f_dev, n_sites, scratch, mass_dev, s)
              : mass_tiles<kD3Q19, float>(f_dev, n_sites, scratch, mass_dev, s);
      break;
  }
  if (e != cudaSuccess) return noalloc_cuda_fail("launch", e);
  return LBFD_OK;
}
