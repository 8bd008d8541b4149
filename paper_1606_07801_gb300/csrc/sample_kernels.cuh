// A step fused with the sampled observables of the state it reads (paper
// Sec. IV: the equilibrium statistics of eqs. dijexp, fkfk and rhoth are
// sums over sites of rho, rho^2, f_i, f_i f_j and |rho(k)|^2).  Included by
// one translation unit per lattice.
//
// The kernel is the register-pull vector kernel on a persistent grid: block
// b takes the work blocks b, b + G, ... of the one-launch-per-step kernel's
// grid.  Between the pull and the collision every warp, whose 32 lanes hold
// 32 VX consecutive sites of one row, adds the observables of those sites:
//   - each lane writes its sites' deviations e_i = f_i - c_i (c_i =
//     w_i rho_mean in FP32; the 16-bit formats hold e_i already) as rows of
//     a per-warp shared tile, with a 1 in column Q and zeros beyond;
//   - lane (block (I, J), slice sl) adds, for the tile's sites sl,
//     sl + NSL, ..., the 4 x 4 products of row groups I and J into FP32
//     registers; column Q turns the pairs (i, Q) into sum_x e_i, so
//     sum delta and sum delta^2 (delta = sum_i e_i) follow from the pair
//     sums without per-site reductions;
//   - the structure-factor terms d e^{-2 pi i k.x/L}, d = delta + d_off =
//     rho - rho_mean, accumulate per lane in FP32;
//   - after at most 256 terms a lane's FP32 sums go, summed over the
//     slices in slice order, into the warp's FP64 slots.
// At the end the block adds its warps' slots in warp order and writes one
// partial set in the layout of the separate FP32 observable pass, whose
// stage 2 (launch_obs_pull_finalize) restores the sums of rho, f and f f.
// No step sees another's data and every sum has a fixed order, so the
// result does not depend on timing.  The site update itself is the one of
// k_step_vec (vec_pull, collide_site, vec_store): bit-identical.
#pragma once

#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>

#include "step_kernels.cuh"

namespace lbfd {

// Pair blocking of one warp's tile: rows padded to QP (a multiple of 4 with
// at least one spare column, the constant 1 at column Q), G groups of four,
// NB blocks (I, J), I <= J, and NSL site slices per block.
template <int LAT>
struct WarpPairPlan {
  static constexpr int Q = Lattice<LAT>::Q;
  static constexpr int QP = (Q / 4 + 1) * 4;
  static constexpr int G = QP / 4;
  static constexpr int NB = G * (G + 1) / 2;
  static constexpr int NSL = 32 / NB;
  static constexpr int LANES = NB * NSL;
  static_assert(NSL >= 1, "pair blocks exceed a warp");
};

constexpr int kSampleThreads = 256;
constexpr int kSampleWarps = kSampleThreads / 32;
constexpr int kSampleFlushTerms = 256;  // FP32 terms of a block sum before it goes to FP64

struct SampleArgs {
  const float2 *phase;  // per-axis e^{-2 pi i k_d u / L_d} tables (obs_phase_fill)
  int32_t K;            // modes, <= kFusedModes
  float rho_f;          // rho_mean in FP32 (the c_i)
  float d_off;          // rho - rho_mean = delta + d_off
  int32_t gx, gy, gz;   // the work-block grid of the one-launch-per-step kernel
  int32_t nvb;          // gx gy gz
};

// Slot of the pair (i, j), i <= j < QP, in a warp's FP64 slots.
template <int LAT>
__host__ __device__ __forceinline__ int pair_slot(int i, int j) {
  using P = WarpPairPlan<LAT>;
  const int I = i >> 2, J = j >> 2;
  return (I * P::G - I * (I - 1) / 2 + (J - I)) * 16 + (i & 3) * 4 + (j & 3);
}

// The observables of the sites one warp holds: each lane holds VX
// consecutive sites of one row (the warp 32 VX of them, or fewer at the end
// of a row).  Every lane of the warp calls add() for each group of sites,
// then flush() once at the end.
template <int LAT, int VX>
struct WarpSampler {
  using P = WarpPairPlan<LAT>;
  static constexpr int Q = P::Q, QP = P::QP, ROWS = 32 * VX;
  static constexpr int kTermsPerTile = (ROWS + P::NSL - 1) / P::NSL;
  struct Smem {  // one warp's
    float tile[ROWS][QP];
    double slots[P::NB * 16];
    double modes[2 * kFusedModes];
  };
  Smem *sm;
  int lane, blk, sl, bI, bJ, terms;
  bool pair_lane;
  float pa[16];
  float mre[kFusedModes], mim[kFusedModes];

  __device__ __forceinline__ void init(Smem *s, int lane_) {
    sm = s;
    lane = lane_;
    for (int k = lane; k < P::NB * 16; k += 32) sm->slots[k] = 0.0;
    if (lane < 2 * kFusedModes) sm->modes[lane] = 0.0;
    pair_lane = lane < P::LANES;
    blk = pair_lane ? lane / P::NSL : 0;
    sl = lane % P::NSL;
    int b = blk, i = 0;
    while (b >= P::G - i) {
      b -= P::G - i;
      ++i;
    }
    bI = i;
    bJ = i + b;
#pragma unroll
    for (int e = 0; e < 16; ++e) pa[e] = 0.0f;
#pragma unroll
    for (int m = 0; m < kFusedModes; ++m) mre[m] = mim[m] = 0.0f;
    terms = 0;
    __syncwarp();
  }

  // FP32 sums into the warp's FP64 slots: the slices of a pair block are
  // added in slice order by the block's first lane; the mode sums by a
  // butterfly over the warp, then lane 0.
  __device__ __forceinline__ void flush(int K) {
#pragma unroll
    for (int e = 0; e < 16; ++e) {
      const double v = static_cast<double>(pa[e]);
      double t = v;
      for (int j = 1; j < P::NSL; ++j) t += __shfl_sync(0xffffffffu, v, (lane + j) & 31);
      if (pair_lane && sl == 0) sm->slots[blk * 16 + e] += t;
      pa[e] = 0.0f;
    }
#pragma unroll
    for (int m = 0; m < kFusedModes; ++m) {
      double re = static_cast<double>(mre[m]), im = static_cast<double>(mim[m]);
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        re += __shfl_xor_sync(0xffffffffu, re, o);
        im += __shfl_xor_sync(0xffffffffu, im, o);
      }
      if (lane == 0 && m < K) {
        sm->modes[2 * m] += re;
        sm->modes[2 * m + 1] += im;
      }
      mre[m] = mim[m] = 0.0f;
    }
    terms = 0;
  }

  // Sites x0 .. x0 + VX - 1 of row (y, z) with pulled populations f (their
  // deviations for the 16-bit formats); inactive lanes add nothing.
  template <typename S>
  __device__ __forceinline__ void add(const typename Store<S>::R (&f)[VX][Q], bool active, int x0, int y, int z,
                                      int Lx, int Ly, int Lz, const SampleArgs &sa) {
    float tre[kFusedModes], tim[kFusedModes];
#pragma unroll
    for (int m = 0; m < kFusedModes; ++m) tre[m] = tim[m] = 0.0f;
#pragma unroll
    for (int k = 0; k < VX; ++k) {
      float e[QP];
#pragma unroll
      for (int i = 0; i < QP; ++i) e[i] = 0.0f;
      if (active) {
        float delta = 0.0f;
#pragma unroll
        for (int i = 0; i < Q; ++i) {
          e[i] = Store<S>::kDeviation ? static_cast<float>(f[k][i])
                                      : sub_rn(static_cast<float>(f[k][i]), obs_offset<LAT>(i, sa.rho_f));
          delta += e[i];
        }
        e[Q] = 1.0f;
        // structure factor, x part: sum_k d_k e^{-2 pi i k_x x / Lx}
        const float d = delta + sa.d_off;
#pragma unroll
        for (int m = 0; m < kFusedModes; ++m)
          if (m < sa.K) {
            const float2 fx = sa.phase[m * Lx + x0 + k];
            tre[m] = fmaf(d, fx.x, tre[m]);
            tim[m] = fmaf(d, fx.y, tim[m]);
          }
      }
#pragma unroll
      for (int i = 0; i < QP; i += 4)
        *reinterpret_cast<float4 *>(&sm->tile[lane * VX + k][i]) = make_float4(e[i], e[i + 1], e[i + 2], e[i + 3]);
    }
    if (active) {
      // times the row's y and z factors (the same for all of this lane's sites)
#pragma unroll
      for (int m = 0; m < kFusedModes; ++m)
        if (m < sa.K) {
          const float2 fy = sa.phase[sa.K * Lx + m * Ly + y];
          const float2 fz = sa.phase[sa.K * (Lx + Ly) + m * Lz + z];
          const float gr = fy.x * fz.x - fy.y * fz.y, gi = fy.x * fz.y + fy.y * fz.x;
          mre[m] += tre[m] * gr - tim[m] * gi;
          mim[m] += tre[m] * gi + tim[m] * gr;
        }
    }
    __syncwarp();
    if (pair_lane) {
#pragma unroll 4
      for (int kk = sl; kk < ROWS; kk += P::NSL) {
        const float4 u = *reinterpret_cast<const float4 *>(&sm->tile[kk][4 * bI]);
        const float4 v = *reinterpret_cast<const float4 *>(&sm->tile[kk][4 * bJ]);
        const float uu[4] = {u.x, u.y, u.z, u.w}, vv[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
        for (int p = 0; p < 4; ++p)
#pragma unroll
          for (int c = 0; c < 4; ++c) pa[4 * p + c] = fmaf(uu[p], vv[c], pa[4 * p + c]);
      }
    }
    __syncwarp();  // the tile is read before the next call writes it
    terms += kTermsPerTile;
    if (terms + kTermsPerTile > kSampleFlushTerms) flush(sa.K);
  }
};

// The block's partial sums from its warps' slots (warps added in warp
// order), in the layout of the FP32 observable pass: [sum delta,
// sum delta^2, sum e_i, modes, pairs i <= j].  Called by `nthreads` threads
// (tid < nthreads) after a barrier among them that follows every warp's
// flush; `sync` is that barrier.
template <int LAT, int VX, class Sync>
__device__ __forceinline__ void sample_block_partials(typename WarpSampler<LAT, VX>::Smem *w, int nwarps, int K,
                                                      double *out, int tid, int nthreads, Sync sync) {
  using P = WarpPairPlan<LAT>;
  constexpr int Q = P::Q;
  for (int k = tid; k < P::NB * 16; k += nthreads) {
    double t = 0.0;
    for (int j = 0; j < nwarps; ++j) t += w[j].slots[k];
    w[0].slots[k] = t;
  }
  if (tid < 2 * kFusedModes) {
    double t = 0.0;
    for (int j = 0; j < nwarps; ++j) t += w[j].modes[tid];
    w[0].modes[tid] = t;
  }
  sync();
  const int nq1 = 2 + Q + 2 * K, npair = Q * (Q + 1) / 2;
  const double *sl0 = w[0].slots;
  for (int p0 = tid; p0 < npair; p0 += nthreads) {
    int p = p0, i = 0;
    while (p >= Q - i) {
      p -= Q - i;
      ++i;
    }
    out[nq1 + p0] = sl0[pair_slot<LAT>(i, i + p)];
  }
  if (tid < Q) out[2 + tid] = sl0[pair_slot<LAT>(tid, Q)];
  if (tid < 2 * K) out[2 + Q + tid] = w[0].modes[tid];
  if (tid == 0) {
    double sd = 0.0, sd2 = 0.0;
    for (int i = 0; i < Q; ++i) {
      sd += sl0[pair_slot<LAT>(i, Q)];
      sd2 += sl0[pair_slot<LAT>(i, i)];
      for (int j = i + 1; j < Q; ++j) sd2 += 2.0 * sl0[pair_slot<LAT>(i, j)];
    }
    out[0] = sd;
    out[1] = sd2;
  }
}

template <int LAT, typename S, int VX, int NOISE, typename Idx>
__global__ void __launch_bounds__(kSampleThreads, 2)
    k_step_sample(const S *__restrict__ src, S *__restrict__ dst, const StepArgs a, const SampleArgs sa,
                  double *__restrict__ partials) {
  using L = Lattice<LAT>;
  using R = typename Store<S>::R;
  using WS = WarpSampler<LAT, VX>;
  constexpr int Q = L::Q;
  extern __shared__ __align__(16) unsigned char sample_smem[];
  typename WS::Smem *wsm = reinterpret_cast<typename WS::Smem *>(sample_smem);
  const int tid = static_cast<int>(threadIdx.x + blockDim.x * threadIdx.y);
  const int warp = tid >> 5;
  WS ws;
  ws.init(&wsm[warp], tid & 31);

  pdl_launch_dependents();
  pdl_wait();
  for (int vb = blockIdx.x; vb < sa.nvb; vb += gridDim.x) {
    const int vbx = vb % sa.gx, vr = vb / sa.gx;
    const int vby = vr % sa.gy, vbz = vr / sa.gy;
    const int x0 = (vbx * static_cast<int>(blockDim.x) + static_cast<int>(threadIdx.x)) * VX;
    const int y = vby * static_cast<int>(blockDim.y) + static_cast<int>(threadIdx.y);
    const int z = vbz;
    const bool active = x0 < a.Lx && y < a.Ly;
    R f[VX][Q];
    uint32_t row = 0;
    if (active) row = vec_pull<LAT, S, VX, Idx>(src, a, x0, y, z, f);
    ws.template add<S>(f, active, x0, y, z, a.Lx, a.Ly, a.Lz, sa);
    // the step: the collision and store of k_step_vec
    if (active) {
#pragma unroll
      for (int k = 0; k < VX; ++k)
        collide_site<LAT, R, NOISE, Store<S>::kDeviation>(f[k], row + static_cast<uint32_t>(x0 + k), a);
      vec_store<LAT, S, VX, Idx>(dst, a, row, x0, f);
    }
  }
  ws.flush(sa.K);
  __syncthreads();
  const int nq = 2 + Q + 2 * sa.K + Q * (Q + 1) / 2;
  sample_block_partials<LAT, VX>(wsm, kSampleWarps, sa.K, partials + static_cast<size_t>(blockIdx.x) * nq, tid,
                                 kSampleThreads, [] { __syncthreads(); });
}

template <int LAT, typename S, int VX, int NOISE, typename Idx>
cudaError_t sample_launch(const void *src, void *dst, const StepArgs &a, const SampleArgs &sa_in, dim3 block,
                          double *partials, int *nblocks, cudaStream_t stream) {
  auto kern = k_step_sample<LAT, S, VX, NOISE, Idx>;
  constexpr size_t smem = kSampleWarps * sizeof(typename WarpSampler<LAT, VX>::Smem);
  static std::atomic<int> slots{0};  // resident blocks per SM times SMs, found once
  int g = slots.load(std::memory_order_relaxed);
  if (g == 0) {
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem));
    int dev = 0, sms = 0, occ = 0;
    if (e == cudaSuccess) e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, kSampleThreads, smem);
    if (e != cudaSuccess) return e;
    if (occ < 1 || sms < 1) return cudaErrorInvalidConfiguration;
    g = std::min(occ * sms, kObsBlocks);
    slots.store(g, std::memory_order_relaxed);
  }
  const int grid = std::max(1, std::min(sa_in.nvb, g));
  *nblocks = grid;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(grid, 1, 1);
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = stream;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = step_pdl() ? 1 : 0;
  return cudaLaunchKernelEx(&cfg, kern, static_cast<const S *>(src), static_cast<S *>(dst), a, sa_in, partials);
}

// Arguments of a fused sampled step for a lattice in FP32 arithmetic.
template <int LAT>
inline SampleArgs make_sample_args(const StepArgs &a, int n_modes, const void *phase, const dim3 &grid) {
  SampleArgs sa{};
  sa.phase = static_cast<const float2 *>(phase);
  sa.K = n_modes;
  sa.rho_f = static_cast<float>(a.rho_eq);
  double C = 0.0;
  for (int i = 0; i < Lattice<LAT>::Q; ++i) C += static_cast<double>(obs_offset<LAT>(i, sa.rho_f));
  sa.d_off = static_cast<float>(C - a.rho_eq);
  sa.gx = int(grid.x);
  sa.gy = int(grid.y);
  sa.gz = int(grid.z);
  sa.nvb = sa.gx * sa.gy * sa.gz;
  return sa;
}

// The fused step-and-sample launch on the register-pull kernel's blocks.
template <int LAT, typename S>
cudaError_t sample_vec_t(const void *src, void *dst, const StepArgs &a, int n_modes, const void *phase,
                         double *partials, int *nblocks, cudaStream_t stream) {
  const int vx = step_vec_width(LAT, Store<S>::kDeviation ? kStoreF16 : kStoreF32, a.Lx) >= 2 ? 2 : 1;
  dim3 grid, block;
  step_shape(a.Lx, a.Ly, a.Lz, grid, block, vx);
  if (block.x * block.y != kSampleThreads || block.x % 32 != 0) return cudaErrorInvalidValue;
  const SampleArgs sa = make_sample_args<LAT>(a, n_modes, phase, grid);
  const bool fit32 = offsets_fit_32(Lattice<LAT>::Q, a.N);
  auto go = [&](auto noise) -> cudaError_t {
    constexpr int NZ = decltype(noise)::value;
    if (vx == 2)
      return fit32 ? sample_launch<LAT, S, 2, NZ, uint32_t>(src, dst, a, sa, block, partials, nblocks, stream)
                   : sample_launch<LAT, S, 2, NZ, size_t>(src, dst, a, sa, block, partials, nblocks, stream);
    return fit32 ? sample_launch<LAT, S, 1, NZ, uint32_t>(src, dst, a, sa, block, partials, nblocks, stream)
                 : sample_launch<LAT, S, 1, NZ, size_t>(src, dst, a, sa, block, partials, nblocks, stream);
  };
  if (a.noise_mode == kNoiseOff) return go(std::integral_constant<int, kStepNoiseOff>{});
  if (a.noise_dist == kGaussian) return go(std::integral_constant<int, kStepNoiseGauss>{});
  return go(std::integral_constant<int, kStepNoiseFlat>{});
}

}  // namespace lbfd
