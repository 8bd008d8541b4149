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

#include <algorithm>
#include <cmath>
#include <type_traits>

#include "device.cuh"
#include "fastdiv.cuh"
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
__global__ void __launch_bounds__(kReduceThreads) k_mass_partials(const S *__restrict__ f, int64_t N, int64_t stride,
                                                                 double rho_mean, double *__restrict__ partials) {
  using L = Lattice<LAT>;
  __shared__ double warp_tot[kReduceThreads / 32];
  double acc = 0.0;
  for (int64_t s = blockIdx.x * static_cast<int64_t>(kReduceThreads) + threadIdx.x; s < N;
       s += static_cast<int64_t>(gridDim.x) * kReduceThreads) {
    double r = 0.0;
    static_for<L::Q>([&](auto I) {
      constexpr int i = decltype(I)::value;
      r += Store<S>::getd(f[i * stride + s], L::w(i) * rho_mean);
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
                        double *out, cudaStream_t stream, int64_t stride) {
  if (stride == 0) stride = N;
  return dispatch_lattice_storage(lattice, precision, [&](auto lat, auto tag) {
    constexpr int LAT = decltype(lat)::value;
    using S = typename decltype(tag)::type;
    k_mass_partials<LAT, S><<<kReduceBlocks, kReduceThreads, 0, stream>>>(static_cast<const S *>(f), N, stride,
                                                                          rho_mean, partials);
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

// Stage-2 sum of per-block partials[b][q] (b < nblocks, q < nq) in a fixed
// order, by kFinalThreads threads: warp w adds the blocks w, w + W, ... of 32
// quantities at a time (coalesced rows; all its loads issued before the
// adds), then thread q adds the W warp sums.  tot needs nq + W * nq doubles
// of shared memory.
constexpr int kFinalThreads = 512;
constexpr int kFinalWarps = kFinalThreads / 32;
constexpr int kFinalPer = ((kObsBlocks > kReduceBlocks ? kObsBlocks : kReduceBlocks) + kFinalWarps - 1) / kFinalWarps;
__device__ __forceinline__ void sum_partials_ordered(const double *__restrict__ partials, int nblocks, int nq,
                                                     double *tot) {
  double *part = tot + nq;  // [W][nq]
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int q0 = 0; q0 < nq; q0 += 32) {
    const int q = q0 + lane;
    if (q < nq) {
      double v[kFinalPer];
#pragma unroll
      for (int j = 0; j < kFinalPer; ++j) {
        const int b = warp + j * kFinalWarps;
        v[j] = b < nblocks ? partials[static_cast<int64_t>(b) * nq + q] : 0.0;
      }
      double t = 0.0;
#pragma unroll
      for (int j = 0; j < kFinalPer; ++j) t += v[j];
      part[warp * nq + q] = t;
    }
  }
  __syncthreads();
  for (int q = threadIdx.x; q < nq; q += blockDim.x) {
    double t = 0.0;
    for (int w = 0; w < kFinalWarps; ++w) t += part[w * nq + q];
    tot[q] = t;
  }
  __syncthreads();
}

inline size_t final_smem(int nq) { return sizeof(double) * size_t(nq) * (1 + kFinalWarps); }

// acc layout: [sum_rho, sum_rho2, sum_f[Q], sum_ff[Q*Q] (full, symmetric), sum_sk[K]]
__global__ void k_obs_finalize(const double *__restrict__ partials, int nblocks, int Q, int K, double *__restrict__ acc) {
  extern __shared__ double tot[];
  const int nq1 = 2 + Q + 2 * K, npair = Q * (Q + 1) / 2, nq = nq1 + npair;
  sum_partials_ordered(partials, nblocks, nq, tot);
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
  k_obs_finalize<<<1, kFinalThreads, final_smem(nq), stream>>>(partials, kReduceBlocks, Q, ma.n, acc);
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

// ---------------------------------------------------------------------------
// Observables of a lattice in FP32 arithmetic (FP32, FP16 and BF16 storage),
// straight from the stored post-collision state g: population i at site x
// is f_i(x, t) = g_i(x - v_i), pulled as the step pulls it, so no streamed
// copy of the state is made.  The GPU has few FP64 units, so per site the
// kernel works in FP32 on deviations e_i = f_i - c_i from the constants
// c_i = w_i rho_mean (what the 16-bit formats store), delta = sum_i e_i, and
// d = rho - rho_mean; each block reduces a tile of 256 sites in FP32 and adds
// the tile totals to FP64 accumulators.  A tile total has at most 256 terms
// of one sign-mixed quantity, so its relative error is at most 256 x 2^-24 of
// the sum of the terms' magnitudes; everything after it is FP64.  The final
// pass restores the sums of f and rho from the deviations in FP64.
// ---------------------------------------------------------------------------
constexpr int kObsThreads = 256;


__device__ __forceinline__ float warp_sum_f(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Sizes of the lattice with their fast divisions and FP32 inverses.
struct ObsDims {
  int32_t Lx, Ly, Lz;
  uint32_t s0, count;           // the sites sampled: s0 .. s0 + count - 1
  FastDiv div_x, div_y, div_z;  // exact for numerators below 2^31
  float inv_x, inv_y, inv_z;
  int32_t big;                  // some side >= 46341: k x may not fit 31 bits
};

// (k x) mod L for 0 <= k, x < L
__device__ __forceinline__ uint32_t obs_mulmod(uint32_t k, uint32_t x, uint32_t L, FastDiv dv, bool big) {
  if (big) return static_cast<uint32_t>((static_cast<uint64_t>(k) * x) % L);
  const uint32_t n = k * x;
  return n - fastdiv(n, dv) * L;
}

// Pair sums sum_x e_i e_j by register blocks: the rows i are padded to QP =
// 4 G and grouped by four; a thread owns one block (I, J), I <= J, of 4 x 4
// pairs and one slice of the tile's sites (sites sl, sl + SL, ...), and reads
// each site's two row groups as two 16-byte shared loads for 16 FMAs.  Its
// FP32 block sums cover SL tiles (256 products each) before they go to FP64.
// Row Q (always padding) holds 1 at every site, so the pairs (i, Q) give
// sum_x e_i, and sum delta = sum_i sum_x e_i, sum delta^2 = sum_ij sum_x e_i e_j
// follow without per-site reductions.
template <int Q>
struct ObsPairPlan {
  static constexpr int QP = (Q / 4 + 1) * 4;
  static constexpr int G = QP / 4;
  static constexpr int NB = G * (G + 1) / 2;
  static constexpr int SL = NB <= 1 ? 256 : NB <= 2 ? 128 : NB <= 4 ? 64 : NB <= 8 ? 32 : NB <= 16 ? 16 : 8;
  static constexpr int SPS = kObsThreads / SL;  // sites of a slice in one tile
  static_assert(NB * SL <= kObsThreads && NB * 16 <= kObsThreads, "pair plan exceeds the block");
};

template <int LAT, typename S>
__global__ void __launch_bounds__(kObsThreads) k_obs_pull(const S *__restrict__ g, const ObsDims dm, float rho_f,
                                                         float d_off, const ModeArgs modes,
                                                         const float2 *__restrict__ phase,
                                                         double *__restrict__ partials) {
  using L = Lattice<LAT>;
  constexpr int Q = L::Q;
  constexpr int NPAIR = Q * (Q + 1) / 2;
  constexpr int NW = kObsThreads / 32;
  using P = ObsPairPlan<Q>;
  constexpr int QP = P::QP, SL = P::SL, SPS = P::SPS;
  __shared__ __align__(16) float tile[kObsThreads][QP];
  __shared__ float red[P::NB * SL][16];
  __shared__ float wsum[NW][2 * LBFD_MAX_MODES_DEV];
  __shared__ double slot_sum[P::NB * 16];
  const int32_t Lx = dm.Lx, Ly = dm.Ly, Lz = dm.Lz;
  const uint32_t N = static_cast<uint32_t>(Lx) * static_cast<uint32_t>(Ly) * static_cast<uint32_t>(Lz);
  const int K = modes.n;
  const int nq1 = 2 + Q + 2 * K;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  // this thread's pair block (I, J) and slice, when it has one
  const bool has_block = threadIdx.x < P::NB * SL;
  const int blk = threadIdx.x / SL, sl = threadIdx.x % SL;
  int bI = 0, bJ = 0;
  {
    int b = has_block ? blk : 0, i = 0;
    while (b >= P::G - i) {
      b -= P::G - i;
      ++i;
    }
    bI = i;
    bJ = i + b;
  }
  float pa[16];
#pragma unroll
  for (int e = 0; e < 16; ++e) pa[e] = 0.0f;
  double acc_q = 0.0, acc_pair = 0.0;  // mode sum threadIdx.x (< 2 K), pair slot threadIdx.x (< NB * 16)
  int tiles = 0;

  // FP32 block sums of the last tiles into the FP64 slot sums (in slice order)
  auto flush_pairs = [&]() {
    if (has_block) {
#pragma unroll
      for (int e = 0; e < 16; ++e) {
        red[threadIdx.x][e] = pa[e];
        pa[e] = 0.0f;
      }
    }
    __syncthreads();
    if (threadIdx.x < P::NB * 16) {
      const int b = threadIdx.x >> 4, e = threadIdx.x & 15;
      double t = 0.0;
      for (int k = 0; k < SL; ++k) t += static_cast<double>(red[b * SL + k][e]);
      acc_pair += t;
    }
    __syncthreads();
  };

  for (uint32_t base = blockIdx.x * kObsThreads; base < dm.count; base += gridDim.x * kObsThreads) {
    const bool valid = base + threadIdx.x < dm.count;
    const uint32_t s = dm.s0 + base + threadIdx.x;
    float e[QP];
#pragma unroll
    for (int i = 0; i < QP; ++i) e[i] = 0.0f;
    float delta = 0.0f;
    uint32_t x = 0, y = 0, z = 0;
    if (valid) {
      const uint32_t r = fastdiv(s, dm.div_x);
      x = s - r * static_cast<uint32_t>(Lx);
      z = fastdiv(r, dm.div_y);
      y = r - z * static_cast<uint32_t>(Ly);
      const uint32_t xm = (x == 0 ? Lx : x) - 1, xp = (x + 1 == static_cast<uint32_t>(Lx)) ? 0 : x + 1;
      const uint32_t ym = (y == 0 ? Ly : y) - 1, yp = (y + 1 == static_cast<uint32_t>(Ly)) ? 0 : y + 1;
      const uint32_t zm = (z == 0 ? Lz : z) - 1, zp = (z + 1 == static_cast<uint32_t>(Lz)) ? 0 : z + 1;
      const uint32_t Lxu = static_cast<uint32_t>(Lx), Lxy = Lxu * static_cast<uint32_t>(Ly);
      static_for<Q>([&](auto I) {
        constexpr int i = decltype(I)::value;
        constexpr int vx = L::v(i, 0), vy = L::v(i, 1), vz = L::v(i, 2);
        const uint32_t xs = vx == 0 ? x : (vx > 0 ? xm : xp);
        const uint32_t ys = vy == 0 ? y : (vy > 0 ? ym : yp);
        const uint32_t zs = vz == 0 ? z : (vz > 0 ? zm : zp);
        const S v = g[static_cast<size_t>(i) * N + xs + Lxu * ys + Lxy * zs];
        // 16-bit formats store the deviation itself; FP32 stores f
        e[i] = Store<S>::kDeviation ? Store<S>::get(v, 0.0f)
                                    : sub_rn(Store<S>::get(v, 0.0f), obs_offset<LAT>(i, rho_f));
        delta += e[i];
      });
      e[Q] = 1.0f;
    }
#pragma unroll
    for (int i = 0; i < QP; i += 4)
      *reinterpret_cast<float4 *>(&tile[threadIdx.x][i]) = make_float4(e[i], e[i + 1], e[i + 2], e[i + 3]);
    // per-tile FP32 sums of the mode quantities, one warp total each
    auto put = [&](int q, float v) {
      v = warp_sum_f(v);
      if (lane == 0) wsum[warp][q] = v;
    };
    if (K > 0) {
      const float d = valid ? delta + d_off : 0.0f;
      for (int m = 0; m < K; ++m) {
        float cs, sn;
        if (phase) {
          // e^{-2 pi i k.x / L} as the product of its three per-axis factors
          const float2 fx = phase[m * Lx + x];
          const float2 fy = phase[K * Lx + m * Ly + y];
          const float2 fz = phase[K * (Lx + Ly) + m * Lz + z];
          const float ar = fx.x * fy.x - fx.y * fy.y, ai = fx.x * fy.y + fx.y * fy.x;
          cs = ar * fz.x - ai * fz.y;
          sn = -(ar * fz.y + ai * fz.x);
        } else {
          const uint32_t px = obs_mulmod(static_cast<uint32_t>(modes.k[m][0]), x, Lx, dm.div_x, dm.big);
          const uint32_t py = obs_mulmod(static_cast<uint32_t>(modes.k[m][1]), y, Ly, dm.div_y, dm.big);
          const uint32_t pz = obs_mulmod(static_cast<uint32_t>(modes.k[m][2]), z, Lz, dm.div_z, dm.big);
          // each term is below 1 and exact to FP32 rounding; sincospif reduces exactly
          const float frac = fmaf(static_cast<float>(px), dm.inv_x,
                                  fmaf(static_cast<float>(py), dm.inv_y, static_cast<float>(pz) * dm.inv_z));
          sincospif(2.0f * frac, &sn, &cs);
        }
        put(2 * m, d * cs);
        put(2 * m + 1, -d * sn);
      }
    }
    __syncthreads();
    if (threadIdx.x < 2 * K) {
      float t = 0.0f;
#pragma unroll
      for (int w = 0; w < NW; ++w) t += wsum[w][threadIdx.x];
      acc_q += static_cast<double>(t);
    }
    if (has_block) {
#pragma unroll 4
      for (int kk = 0; kk < SPS; ++kk) {
        const int k = sl + kk * SL;
        const float4 u = *reinterpret_cast<const float4 *>(&tile[k][4 * bI]);
        const float4 v = *reinterpret_cast<const float4 *>(&tile[k][4 * bJ]);
        const float uu[4] = {u.x, u.y, u.z, u.w}, vv[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
        for (int a = 0; a < 4; ++a)
#pragma unroll
          for (int c = 0; c < 4; ++c) pa[4 * a + c] = fmaf(uu[a], vv[c], pa[4 * a + c]);
      }
    }
    __syncthreads();
    if (++tiles == SL) {
      flush_pairs();
      tiles = 0;
    }
  }
  if (tiles > 0) flush_pairs();
  // gather the slot sums, then write the block's partials in the layout of
  // k_obs_partials: [sum delta, sum delta^2, sum e_i, modes, pairs i <= j]
  if (threadIdx.x < P::NB * 16) slot_sum[threadIdx.x] = acc_pair;
  __syncthreads();
  auto slot_of = [](int i, int j) {  // i <= j < QP
    const int I = i >> 2, J = j >> 2;
    return (I * P::G - I * (I - 1) / 2 + (J - I)) * 16 + (i & 3) * 4 + (j & 3);
  };
  double *out = partials + static_cast<size_t>(blockIdx.x) * (nq1 + NPAIR);
  if (threadIdx.x < NPAIR) {
    int p = threadIdx.x, i = 0;
    while (p >= Q - i) {
      p -= Q - i;
      ++i;
    }
    out[nq1 + threadIdx.x] = slot_sum[slot_of(i, i + p)];
  }
  if (threadIdx.x < Q) out[2 + threadIdx.x] = slot_sum[slot_of(threadIdx.x, Q)];
  if (threadIdx.x < 2 * K) out[2 + Q + threadIdx.x] = acc_q;
  if (threadIdx.x == 0) {
    double sd = 0.0, sd2 = 0.0;
    for (int i = 0; i < Q; ++i) {
      sd += slot_sum[slot_of(i, Q)];
      sd2 += slot_sum[slot_of(i, i)];
      for (int j = i + 1; j < Q; ++j) sd2 += 2.0 * slot_sum[slot_of(i, j)];
    }
    out[0] = sd;
    out[1] = sd2;
  }
}

// Stage 2 of the FP32 pass, spread over the GPU (its FP64 units are few, so
// one block summing every quantity would take ~0.1 ms): warp w sums
// quantity w over the block partials (lane l adds blocks l, l + 32, ... in
// order, then a fixed butterfly), and the last block to finish (a ticket in
// fin[nq_max]) restores the sums of rho, f and f f from the deviation sums
// with c_i = w_i rho_mean (the kernels' own FP32 constants) and adds them to
// acc:
//   sum rho   = S_delta + N C,            C = sum_i c_i
//   sum rho^2 = S_delta2 + 2 C S_delta + N C^2
//   sum f_i   = E_i + N c_i
//   sum f_i f_j = P_ij + c_j E_i + c_i E_j + N c_i c_j
// Every sum has a fixed order, so the result does not depend on timing.
constexpr int kFinWarps = 8;
template <int LAT>
__global__ void __launch_bounds__(kFinWarps * 32)
    k_obs_pull_finalize(const double *__restrict__ partials, int nblocks, int K, double Nd, float rho_f,
                        double *__restrict__ tot, unsigned int *__restrict__ ticket, double *__restrict__ acc) {
  constexpr int Q = Lattice<LAT>::Q;
  const int nq = 2 + Q + 2 * K + Q * (Q + 1) / 2;
  const int lane = threadIdx.x & 31, q = blockIdx.x * kFinWarps + (threadIdx.x >> 5);
  if (q < nq) {
    double t = 0.0;
    for (int b = lane; b < nblocks; b += 32) t += partials[static_cast<size_t>(b) * nq + q];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
    if (lane == 0) tot[q] = t;
  }
  __threadfence();
  __syncthreads();
  __shared__ bool last;
  if (threadIdx.x == 0) last = atomicAdd(ticket, 1u) == gridDim.x - 1;
  __syncthreads();
  if (!last) return;
  // the last block: the totals into shared memory (from L2: the other blocks
  // wrote them), then one accumulator entry per thread
  __threadfence();
  __shared__ double tt[2 + LBFD_MAX_Q_DEV + 2 * LBFD_MAX_MODES_DEV + LBFD_MAX_Q_DEV * (LBFD_MAX_Q_DEV + 1) / 2];
  __shared__ double cs[LBFD_MAX_Q_DEV + 1];
  const volatile double *vt = tot;
  for (int k = threadIdx.x; k < nq; k += blockDim.x) tt[k] = vt[k];
  if (threadIdx.x < Q) cs[threadIdx.x] = static_cast<double>(obs_offset<LAT>(static_cast<int>(threadIdx.x), rho_f));
  __syncthreads();
  if (threadIdx.x == 0) {
    double C = 0.0;
    for (int i = 0; i < Q; ++i) C += cs[i];
    cs[Q] = C;
    *ticket = 0u;  // for the next launch (stream-ordered after this one)
  }
  __syncthreads();
  const double C = cs[Q];
  const int nacc = 2 + Q + Q * Q + K;
  for (int k = threadIdx.x; k < nacc; k += blockDim.x) acc[k] += obs_restore<Q>(k, tt, cs, C, Nd, K);
}

template <int LAT>
static cudaError_t pull_finalize_t(const double *partials, int nblocks, int n_modes, int64_t N, float rho_f,
                                   double *fin, double *acc, cudaStream_t stream) {
  constexpr int Q = Lattice<LAT>::Q;
  const int nq = obs_quantities(Q, n_modes);
  unsigned int *ticket = reinterpret_cast<unsigned int *>(fin + obs_quantities(Q, LBFD_MAX_MODES_DEV));
  // a plain launch: as a dependent launch it let the next step's blocks take
  // the SMs while it still waited for the sampled step, which cost D3Q19
  // 256^3 0.5 ms per sample on GB300
  k_obs_pull_finalize<LAT><<<(nq + kFinWarps - 1) / kFinWarps, kFinWarps * 32, 0, stream>>>(
      partials, nblocks, n_modes, double(N), rho_f, fin, ticket, acc);
  return cudaGetLastError();
}

// Stage 2 of the FP32-arithmetic observables for partials written by a
// fused sampling step (sample_kernels.cuh), in the layout of k_obs_pull.
cudaError_t launch_obs_pull_finalize(int lattice, const double *partials, int nblocks, int n_modes, int64_t N,
                                     double rho_mean, double *fin, double *acc, cudaStream_t stream) {
  const float rho_f = static_cast<float>(rho_mean);
  return dispatch_lattice(lattice, [&](auto lat) -> cudaError_t {
    constexpr int LAT = decltype(lat)::value;
    return pull_finalize_t<LAT>(partials, nblocks, n_modes, N, rho_f, fin, acc, stream);
  });
}

int obs_pull_blocks(int64_t N) {
  return static_cast<int>(std::max<int64_t>(1, std::min<int64_t>(kObsBlocks, (N + kObsThreads - 1) / kObsThreads)));
}

cudaError_t launch_observables_pull_partials(int lattice, int precision, const void *g, int32_t Lx, int32_t Ly,
                                             int32_t Lz, int64_t s0, int64_t count, double rho_mean, int n_modes,
                                             const int32_t *modes, const void *phase, double *partials, int *nblocks,
                                             cudaStream_t stream) {
  if (n_modes < 0 || n_modes > LBFD_MAX_MODES_DEV || precision == kStoreF64) return cudaErrorInvalidValue;
  const int64_t N = int64_t(Lx) * Ly * Lz;
  if (N >= (int64_t(1) << 31) || s0 < 0 || count < 0 || s0 + count > N) return cudaErrorInvalidValue;
  const int32_t L3[3] = {Lx, Ly, Lz};
  ModeArgs ma{};
  ma.n = n_modes;
  for (int m = 0; m < n_modes; ++m)
    for (int k = 0; k < 3; ++k)
      ma.k[m][k] = static_cast<int32_t>(((int64_t(modes[3 * m + k]) % L3[k]) + L3[k]) % L3[k]);
  ObsDims dm{};
  dm.Lx = Lx;
  dm.Ly = Ly;
  dm.Lz = Lz;
  dm.s0 = static_cast<uint32_t>(s0);
  dm.count = static_cast<uint32_t>(count);
  dm.div_x = make_fastdiv(uint32_t(Lx));
  dm.div_y = make_fastdiv(uint32_t(Ly));
  dm.div_z = make_fastdiv(uint32_t(Lz));
  dm.inv_x = 1.0f / float(Lx);
  dm.inv_y = 1.0f / float(Ly);
  dm.inv_z = 1.0f / float(Lz);
  dm.big = (Lx >= 46341 || Ly >= 46341 || Lz >= 46341) ? 1 : 0;
  const float rho_f = static_cast<float>(rho_mean);
  *nblocks = obs_pull_blocks(count);
  return dispatch_lattice_storage(lattice, precision, [&](auto lat, auto tag) {
    constexpr int LAT = decltype(lat)::value;
    using S = typename decltype(tag)::type;
    if constexpr (std::is_same_v<S, double>) {
      return cudaErrorInvalidValue;
    } else {
      constexpr int Q = Lattice<LAT>::Q;
      // d = rho - rho_mean = delta + (C - rho_mean), C from the same FP32 constants
      double C = 0.0;
      for (int i = 0; i < Q; ++i) C += static_cast<double>(static_cast<float>(Lattice<LAT>::w(i)) * rho_f);
      const float d_off = static_cast<float>(C - rho_mean);
      k_obs_pull<LAT, S><<<*nblocks, kObsThreads, 0, stream>>>(static_cast<const S *>(g), dm, rho_f, d_off, ma,
                                                               static_cast<const float2 *>(phase), partials);
      return cudaGetLastError();
    }
  });
}

cudaError_t launch_observables_pull(int lattice, int precision, const void *g, int32_t Lx, int32_t Ly, int32_t Lz,
                                    double rho_mean, int n_modes, const int32_t *modes, const void *phase,
                                    double *partials, double *fin, double *acc, cudaStream_t stream) {
  const int64_t N = int64_t(Lx) * Ly * Lz;
  int nblocks = 0;
  cudaError_t e = launch_observables_pull_partials(lattice, precision, g, Lx, Ly, Lz, 0, N, rho_mean, n_modes, modes,
                                                   phase, partials, &nblocks, stream);
  if (e != cudaSuccess) return e;
  return launch_obs_pull_finalize(lattice, partials, nblocks, n_modes, N, rho_mean, fin, acc, stream);
}

size_t obs_phase_values(int n_modes, int32_t Lx, int32_t Ly, int32_t Lz) {
  return size_t(n_modes) * (size_t(Lx) + size_t(Ly) + size_t(Lz));
}

void obs_phase_fill(int n_modes, const int32_t *modes, int32_t Lx, int32_t Ly, int32_t Lz, float *out,
                    const int64_t *period, const int64_t *offset) {
  // per axis d and mode m: e^{-2 pi i r / P_d}, r = (k_d ((o_d + u) mod P_d)) mod P_d, u < L_d, in FP64 then
  // rounded (P_d = L_d and o_d = 0 unless a slab gives its global period and its first stored plane)
  const int32_t L3[3] = {Lx, Ly, Lz};
  size_t at = 0;
  for (int d = 0; d < 3; ++d)
    for (int m = 0; m < n_modes; ++m) {
      const int64_t P = period ? period[d] : L3[d], o = offset ? offset[d] : 0;
      const int64_t k = ((int64_t(modes[3 * m + d]) % P) + P) % P;
      for (int64_t u = 0; u < L3[d]; ++u, ++at) {
        const int64_t x = ((o + u) % P + P) % P;
        const double a = 2.0 * 3.14159265358979323846 * double((k * x) % P) / double(P);
        out[2 * at] = static_cast<float>(std::cos(a));
        out[2 * at + 1] = static_cast<float>(-std::sin(a));
      }
    }
}

}  // namespace lbfd
