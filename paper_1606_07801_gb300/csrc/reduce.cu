// Deterministic FP64 reductions over the lattice: the total mass and the
// sampled observables of the paper's equilibrium tests (Sec. IV):
//   sum_x rho, sum_x rho^2              (density variance, eq. rhoth)
//   sum_x f_i, sum_x f_i f_j            (<f_i>, d_ij of eqs. dij / dijexp)
//   |sum_x (rho - rho_mean) e^{-2 pi i k.x / L}|^2 for chosen k
//                                       (structure factor, eq. fkfk)
// Stage 1: a fixed grid of kReduceBlocks x kReduceThreads threads walks the
// sites in a fixed order, reduces in registers, by warp shuffles and through
// shared memory, and writes one partial per block.  Stage 2: one block adds
// the partials in block order.  The result does not depend on timing.
#include <cuda_runtime.h>

#include "device.cuh"
#include "internal.h"

namespace lbfd {

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  return v;
}

// ---------------------------------------------------------------------------
// Mass
// ---------------------------------------------------------------------------
template <int LAT, typename S>
__global__ void __launch_bounds__(kReduceThreads) k_mass_partials(const S *__restrict__ f, int64_t N, double rho_mean,
                                                                 double *__restrict__ partials) {
  using L = Lattice<LAT>;
  __shared__ double warp_tot[kReduceThreads / 32];
  double acc = 0.0;
  for (int64_t s = blockIdx.x * static_cast<int64_t>(kReduceThreads) + threadIdx.x; s < N;
       s += static_cast<int64_t>(gridDim.x) * kReduceThreads) {
    double r = 0.0;
    static_for<L::Q>([&](auto I) {
      constexpr int i = decltype(I)::value;
      r += Store<S>::getd(f[i * N + s], L::w(i) * rho_mean);
    });
    acc += r;
  }
  acc = warp_sum(acc);
  if ((threadIdx.x & 31) == 0) warp_tot[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < kReduceThreads / 32; ++w) t += warp_tot[w];
    partials[blockIdx.x] = t;
  }
}

__global__ void k_sum_partials(const double *__restrict__ partials, int nblocks, double *__restrict__ out) {
  if (threadIdx.x == 0 && blockIdx.x == 0) {
    double t = 0.0;
    for (int b = 0; b < nblocks; ++b) t += partials[b];
    *out = t;
  }
}

cudaError_t launch_mass(int lattice, int precision, const void *f, int64_t N, double rho_mean, double *partials,
                        double *out, cudaStream_t stream) {
  return dispatch_lattice_storage(lattice, precision, [&](auto lat, auto tag) {
    constexpr int LAT = decltype(lat)::value;
    using S = typename decltype(tag)::type;
    k_mass_partials<LAT, S><<<kReduceBlocks, kReduceThreads, 0, stream>>>(static_cast<const S *>(f), N, rho_mean,
                                                                          partials);
    k_sum_partials<<<1, 32, 0, stream>>>(partials, kReduceBlocks, out);
    return cudaGetLastError();
  });
}

// ---------------------------------------------------------------------------
// Observables
// ---------------------------------------------------------------------------
struct ModeArgs {
  int32_t n;
  int32_t k[LBFD_MAX_MODES_DEV][3];
};

// partial layout per block: [rho, rho2, f_0..f_{Q-1}, re_0, im_0, .., re_{K-1}, im_{K-1}, ff pairs (i <= j)]
int obs_quantities(int Q, int n_modes) { return 2 + Q + 2 * n_modes + Q * (Q + 1) / 2; }

template <int LAT, typename S>
__global__ void __launch_bounds__(kReduceThreads) k_obs_partials(const S *__restrict__ f, int32_t Lx, int32_t Ly,
                                                                int32_t Lz, double rho_mean, const ModeArgs modes,
                                                                double *__restrict__ partials) {
  using L = Lattice<LAT>;
  constexpr int Q = L::Q;
  constexpr int NPAIR = Q * (Q + 1) / 2;
  constexpr int TILE = kReduceThreads;
  __shared__ double tile[Q][TILE + 1];
  __shared__ double warp_tot[kReduceThreads / 32][2 + Q + 2 * LBFD_MAX_MODES_DEV];
  const int64_t N = static_cast<int64_t>(Lx) * Ly * Lz;
  const int K = modes.n;
  const int nq1 = 2 + Q + 2 * K;

  double a_rho = 0.0, a_rho2 = 0.0;
  double a_f[Q];
  double a_re[LBFD_MAX_MODES_DEV], a_im[LBFD_MAX_MODES_DEV];
#pragma unroll
  for (int i = 0; i < Q; ++i) a_f[i] = 0.0;
#pragma unroll
  for (int m = 0; m < LBFD_MAX_MODES_DEV; ++m) a_re[m] = a_im[m] = 0.0;
  // this thread's pair (i, j), i <= j, for the f_i f_j sums
  int pi = 0, pj = 0;
  {
    int p = threadIdx.x, i = 0;
    while (p >= Q - i && i < Q) { p -= Q - i; ++i; }
    pi = i; pj = i + p;
  }
  double a_ff = 0.0;

  for (int64_t base = blockIdx.x * static_cast<int64_t>(TILE); base < N; base += static_cast<int64_t>(gridDim.x) * TILE) {
    const int64_t s = base + threadIdx.x;
    if (s < N) {
      double r = 0.0;
#pragma unroll
      for (int i = 0; i < Q; ++i) {
        const double fi = Store<S>::getd(f[i * N + s], L::w(i) * rho_mean);
        tile[i][threadIdx.x] = fi;
        a_f[i] += fi;
        r += fi;
      }
      a_rho += r;
      a_rho2 += r * r;
      if (K > 0) {
        const int64_t x = s % Lx, y = (s / Lx) % Ly, z = s / (static_cast<int64_t>(Lx) * Ly);
        const double d = r - rho_mean;
        for (int m = 0; m < K; ++m) {
          const int64_t px = ((modes.k[m][0] * x) % Lx + Lx) % Lx;
          const int64_t py = ((modes.k[m][1] * y) % Ly + Ly) % Ly;
          const int64_t pz = ((modes.k[m][2] * z) % Lz + Lz) % Lz;
          const float frac = static_cast<float>(double(px) / Lx + double(py) / Ly + double(pz) / Lz);
          float sn, cs;
          sincospif(2.0f * frac, &sn, &cs);
          a_re[m] += d * static_cast<double>(cs);
          a_im[m] -= d * static_cast<double>(sn);
        }
      }
    } else {
#pragma unroll
      for (int i = 0; i < Q; ++i) tile[i][threadIdx.x] = 0.0;
    }
    __syncthreads();
    if (threadIdx.x < NPAIR) {
      double acc = 0.0;
      for (int k = 0; k < TILE; ++k) acc += tile[pi][k] * tile[pj][k];
      a_ff += acc;
    }
    __syncthreads();
  }

  // block reduction of the per-site quantities
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  auto put = [&](int q, double v) {
    v = warp_sum(v);
    if (lane == 0) warp_tot[warp][q] = v;
  };
  put(0, a_rho);
  put(1, a_rho2);
#pragma unroll
  for (int i = 0; i < Q; ++i) put(2 + i, a_f[i]);
  for (int m = 0; m < K; ++m) {
    put(2 + Q + 2 * m, a_re[m]);
    put(3 + Q + 2 * m, a_im[m]);
  }
  __syncthreads();
  double *out = partials + static_cast<int64_t>(blockIdx.x) * (nq1 + NPAIR);
  if (threadIdx.x < nq1) {
    double t = 0.0;
    for (int w = 0; w < kReduceThreads / 32; ++w) t += warp_tot[w][threadIdx.x];
    out[threadIdx.x] = t;
  }
  if (threadIdx.x < NPAIR) out[nq1 + threadIdx.x] = a_ff;
}

// acc layout: [sum_rho, sum_rho2, sum_f[Q], sum_ff[Q*Q] (full, symmetric), sum_sk[K]]
__global__ void k_obs_finalize(const double *__restrict__ partials, int nblocks, int Q, int K, double *__restrict__ acc) {
  extern __shared__ double tot[];
  const int nq1 = 2 + Q + 2 * K, npair = Q * (Q + 1) / 2, nq = nq1 + npair;
  for (int q = threadIdx.x; q < nq; q += blockDim.x) {
    double t = 0.0;
    for (int b = 0; b < nblocks; ++b) t += partials[static_cast<int64_t>(b) * nq + q];
    tot[q] = t;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    acc[0] += tot[0];
    acc[1] += tot[1];
    for (int i = 0; i < Q; ++i) acc[2 + i] += tot[2 + i];
    int p = 0;
    for (int i = 0; i < Q; ++i)
      for (int j = i; j < Q; ++j, ++p) {
        const double v = tot[nq1 + p];
        acc[2 + Q + i * Q + j] += v;
        if (j != i) acc[2 + Q + j * Q + i] += v;
      }
    for (int m = 0; m < K; ++m) {
      const double re = tot[2 + Q + 2 * m], im = tot[3 + Q + 2 * m];
      acc[2 + Q + Q * Q + m] += re * re + im * im;
    }
  }
}

template <int LAT, typename S>
static cudaError_t obs_t(const void *f, int32_t Lx, int32_t Ly, int32_t Lz, double rho_mean, const ModeArgs &ma,
                         double *partials, double *acc, cudaStream_t stream) {
  constexpr int Q = Lattice<LAT>::Q;
  k_obs_partials<LAT, S><<<kReduceBlocks, kReduceThreads, 0, stream>>>(static_cast<const S *>(f), Lx, Ly, Lz, rho_mean,
                                                                       ma, partials);
  const int nq = obs_quantities(Q, ma.n);
  k_obs_finalize<<<1, 256, nq * sizeof(double), stream>>>(partials, kReduceBlocks, Q, ma.n, acc);
  return cudaGetLastError();
}

cudaError_t launch_observables(int lattice, int precision, const void *f, int32_t Lx, int32_t Ly, int32_t Lz,
                               double rho_mean, int n_modes, const int32_t *modes, double *partials, double *acc,
                               cudaStream_t stream) {
  if (n_modes < 0 || n_modes > LBFD_MAX_MODES_DEV) return cudaErrorInvalidValue;
  ModeArgs ma{};
  ma.n = n_modes;
  for (int m = 0; m < n_modes; ++m)
    for (int k = 0; k < 3; ++k) ma.k[m][k] = modes[3 * m + k];
  return dispatch_lattice_storage(lattice, precision, [&](auto lat, auto tag) {
    constexpr int LAT = decltype(lat)::value;
    using S = typename decltype(tag)::type;
    return obs_t<LAT, S>(f, Lx, Ly, Lz, rho_mean, ma, partials, acc, stream);
  });
}

}  // namespace lbfd
