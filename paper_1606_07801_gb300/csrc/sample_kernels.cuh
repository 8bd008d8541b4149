// A step fused with the sampled observables of the state it reads (paper
// Sec. IV: the equilibrium statistics of eqs. dijexp, fkfk and rhoth are
// sums over sites of rho, rho^2, f_i, f_i f_j and |rho(k)|^2).  Included by
// one translation unit per lattice.
//
// The kernel is the register-pull vector kernel on a persistent grid: block
// b takes the work blocks b, b + G, ... of the one-launch-per-step kernel's
// grid.  Between the pull and the collision every warp, whose 32 lanes hold
// 32 VX consecutive sites of one row, adds the observables of those sites
// (WarpSampler):
//   - each lane writes its sites' deviations e_i = f_i - c_i (c_i =
//     w_i rho_mean in FP32; the 16-bit formats hold e_i already), and a 1,
//     as columns of a per-warp shared tile;
//   - the warp's tensor cores add the tile's pair sums sum_x e_i e_j, the
//     1 giving sum_x e_i, so sum delta and sum delta^2 (delta = sum_i e_i)
//     follow from the pair sums without per-site reductions;
//   - the structure-factor terms d e^{-2 pi i k.x/L}, d = delta + d_off =
//     rho - rho_mean, accumulate per lane in FP32;
//   - FP32 sums of at most kSampleFlushTerms sites go to the warp's FP64
//     slots.
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
#include <type_traits>

#include "step_kernels.cuh"

namespace lbfd {

constexpr int kSampleThreads = 256;
constexpr int kSampleWarps = kSampleThreads / 32;
constexpr int kSampleInnerTerms = 256;   // sites in the tensor cores' FP32 accumulators before they are folded
constexpr int kSampleFlushTerms = 2048;  // sites in the folded FP32 sums before they go to FP64

struct SampleArgs {
  const float2 *phase;    // per-axis e^{-2 pi i k_d u / L_d} tables (obs_phase_fill)
  int32_t K;              // modes, <= kFusedModes
  float rho_f;            // rho_mean in FP32 (the c_i)
  float d_off;            // rho - rho_mean = delta + d_off
  int32_t gx, gy, gz;     // the work-block grid of the one-launch-per-step kernel
  int32_t nvb;            // gx gy gz
};

// One warp-level tensor-core step: D += A B, A 16 x 8 and B 8 x 8 in TF32,
// D in FP32 (m16n8k8; fragments as the PTX ISA lays them out).
__device__ __forceinline__ void mma_tf32(float (&d)[4], uint32_t a0, uint32_t a1, uint32_t a2, uint32_t a3,
                                         uint32_t b0, uint32_t b1) {
  asm volatile(
      "mma.sync.aligned.m16n8k8.row.col.f32.tf32.tf32.f32 {%0, %1, %2, %3}, {%4, %5, %6, %7}, {%8, %9}, "
      "{%0, %1, %2, %3};\n"
      : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
      : "r"(a0), "r"(a1), "r"(a2), "r"(a3), "r"(b0), "r"(b1));
}

// The TF32 value nearest to x (cvt.rna.tf32.f32), as its bit pattern.
__device__ __forceinline__ uint32_t to_tf32(float x) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
  return r;
}

// The observables of the sites one warp holds: each lane holds VX
// consecutive sites of one row (the warp 32 VX of them, or fewer at the end
// of a row).  Every lane of the warp calls add() for each group of sites,
// then flush() once at the end.
//
// Pair sums.  With E the (sites x QL) matrix of a tile's rows (e_0 ..
// e_{Q-1} and a constant 1 for a site that is there, so the pairs (i, Q)
// give sum_x e_i), the sums are the upper triangle of E^T E: a dense
// contraction, taken on the tensor cores by warp-level m16n8k8 TF32 steps
// over 8 sites at a time.  E^T is kept transposed in shared memory (row r =
// quantity r, one column per site), so fragment element (row, k) of A = E^T
// and element (k, column) of B = E are the same shared values.  The sum over
// sites does not depend on their order, so k = t and k = t + 4 of a step
// are the adjacent columns 2t and 2t + 1: one 8-byte load gives a lane both.
// Each value is split into TF32 parts hi + lo (hi the nearest TF32, lo =
// e - hi, exact), so that C += H^T H + H^T L + L^T H keeps the products to
// FP32 accuracy, on the m16n8 tiles of the upper triangle: D1Q3 (0,0); D2Q9
// (0,0) (0,1); D3Q19 (0,0) (0,1) (0,2) (1,2).
// The tensor cores add in FP32; after at most kSampleInnerTerms sites a
// lane adds its accumulators into a second FP32 set (in its own column of
// shared memory, to spare registers), and after at most
// kSampleFlushTerms sites that set goes to the warp's FP64 slots (FP64
// arithmetic is slow on this part, so it runs rarely).  Every slot is
// written by one lane at a time, in a fixed order.
template <int LAT, int VX>
struct WarpSampler {
  static constexpr int Q = Lattice<LAT>::Q;
  static constexpr int QL = Q + 1;              // live quantities: e_0 .. e_{Q-1}, 1
  static constexpr int NRB = (QL + 7) / 8;      // row blocks of 8 quantities (rows beyond QL read as 0)
  static constexpr int SITES = 32 * VX;
  static constexpr int KSTEPS = SITES / 8;
  static constexpr int NSLOT = QL * (QL + 1) / 2;
  struct Smem {  // one warp's
    float hi[QL][SITES], lo[QL][SITES];         // columns swizzled (col)
    float outer[(NRB == 1 ? 1 : (NRB == 2 ? 2 : 4)) * 4][32];  // each lane's folded FP32 sums
    double slots[NSLOT];                        // upper triangle of E^T E, row-major
    double modes[2 * kFusedModes];
  };
  // the m16n8 tiles: (m, n) with rows 16m.. and columns 8n..
  static constexpr int NMMA = NRB == 1 ? 1 : (NRB == 2 ? 2 : 4);
  __device__ static constexpr int tile_m(int k) { return NRB == 3 && k == 3 ? 1 : 0; }
  __device__ static constexpr int tile_n(int k) { return NRB == 3 && k == 3 ? 2 : k; }
  static constexpr int kInnerTiles = kSampleInnerTerms / SITES;
  static constexpr int kOuterFlushes = kSampleFlushTerms / kSampleInnerTerms;
  static_assert(kInnerTiles >= 1 && kOuterFlushes >= 1, "flush intervals");

  Smem *sm;
  int lane, tiles, inners;
  float acc[NMMA][4];
  float mre[kFusedModes], mim[kFusedModes];

  __device__ static __forceinline__ int slot(int r, int c) { return r * QL - r * (r - 1) / 2 + (c - r); }
  // the block's partial set (warp_sampler_partials)
  template <class Sync>
  __device__ static void block_partials(Smem *w, int nwarps, int K, double *out, int tid, int nthreads, Sync sync);
  // Shared column of site column c in row r: bits 3-4 of c flipped by r mod
  // 4, so that the 8-byte fragment loads of rows g = 0..3 (columns 8 ks ..
  // 8 ks + 7) fall in distinct banks without padding; pairs (2u, 2u + 1)
  // stay adjacent.
  __device__ static __forceinline__ int col(int r, int c) { return c ^ ((r & 3) << 3); }

  __device__ __forceinline__ void init(Smem *s, int lane_) {
    sm = s;
    lane = lane_;
    for (int k = lane; k < NSLOT; k += 32) sm->slots[k] = 0.0;
    if (lane < 2 * kFusedModes) sm->modes[lane] = 0.0;
#pragma unroll
    for (int t = 0; t < NMMA; ++t)
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        acc[t][e] = 0.0f;
        sm->outer[4 * t + e][lane] = 0.0f;
      }
#pragma unroll
    for (int m = 0; m < kFusedModes; ++m) mre[m] = mim[m] = 0.0f;
    tiles = inners = 0;
    __syncwarp();
  }

  // the accumulators into this lane's folded sums (its own shared column)
  __device__ __forceinline__ void fold_inner() {
#pragma unroll
    for (int k = 0; k < NMMA; ++k)
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        sm->outer[4 * k + e][lane] += acc[k][e];
        acc[k][e] = 0.0f;
      }
  }

  // FP32 sums into the warp's FP64 slots; the mode sums over the warp by an
  // FP32 butterfly, then lane 0.  Called by all lanes between tiles.
  __device__ __forceinline__ void flush(int K) {
    fold_inner();
    const int g = lane >> 2, t = lane & 3;
#pragma unroll
    for (int k = 0; k < NMMA; ++k)
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        const int r = 16 * tile_m(k) + g + (e >= 2 ? 8 : 0), c = 8 * tile_n(k) + 2 * t + (e & 1);
        if (r <= c && c < QL) sm->slots[slot(r, c)] += static_cast<double>(sm->outer[4 * k + e][lane]);
      }
#pragma unroll
    for (int k = 0; k < NMMA; ++k)
#pragma unroll
      for (int e = 0; e < 4; ++e) sm->outer[4 * k + e][lane] = 0.0f;
#pragma unroll
    for (int m = 0; m < kFusedModes; ++m) {
      float re = mre[m], im = mim[m];
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        re += __shfl_xor_sync(0xffffffffu, re, o);
        im += __shfl_xor_sync(0xffffffffu, im, o);
      }
      if (lane == 0 && m < K) {
        sm->modes[2 * m] += static_cast<double>(re);
        sm->modes[2 * m + 1] += static_cast<double>(im);
      }
      mre[m] = mim[m] = 0.0f;
    }
    tiles = inners = 0;
  }

  // Sites x0 .. x0 + VX - 1 of row (y, z) with pulled populations f (their
  // deviations for the 16-bit formats); inactive lanes add nothing.
  template <typename S>
  __device__ __forceinline__ void add(const typename Store<S>::R (&f)[VX][Q], bool active, int x0, int y, int z,
                                      int Lx, int Ly, int Lz, const SampleArgs &sa) {
    float tre[kFusedModes], tim[kFusedModes];
#pragma unroll
    for (int m = 0; m < kFusedModes; ++m) tre[m] = tim[m] = 0.0f;
    // this lane's columns of the transposed tile, hi and lo parts
    float e[VX][QL];
#pragma unroll
    for (int k = 0; k < VX; ++k) {
      float delta = 0.0f;
#pragma unroll
      for (int i = 0; i < Q; ++i) {
        e[k][i] = !active ? 0.0f
                          : (Store<S>::kDeviation ? static_cast<float>(f[k][i])
                                                  : sub_rn(static_cast<float>(f[k][i]), obs_offset<LAT>(i, sa.rho_f)));
        delta += e[k][i];
      }
      e[k][Q] = active ? 1.0f : 0.0f;
      if (active) {
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
    }
#pragma unroll
    for (int r = 0; r < QL; ++r) {
      float vh[VX], vl[VX];
#pragma unroll
      for (int k = 0; k < VX; ++k) {
        vh[k] = __uint_as_float(to_tf32(e[k][r]));
        vl[k] = e[k][r] - vh[k];
      }
      if constexpr (VX == 2) {
        *reinterpret_cast<float2 *>(&sm->hi[r][col(r, 2 * lane)]) = make_float2(vh[0], vh[1]);
        *reinterpret_cast<float2 *>(&sm->lo[r][col(r, 2 * lane)]) = make_float2(vl[0], vl[1]);
      } else {
        sm->hi[r][col(r, lane)] = vh[0];
        sm->lo[r][col(r, lane)] = vl[0];
      }
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
    // E^T E over the tile's sites, 8 at a time
    const int g = lane >> 2, t = lane & 3;
#pragma unroll
    for (int ks = 0; ks < KSTEPS; ++ks) {
      const int c0 = 8 * ks + 2 * t;  // columns of k = t and k = t + 4
      uint32_t h0[NRB], h1[NRB], l0[NRB], l1[NRB];  // row block j: (row 8j + g; k = t, t + 4)
#pragma unroll
      for (int j = 0; j < NRB; ++j) {
        const int r = 8 * j + g;
        float2 hv = make_float2(0.0f, 0.0f), lv = make_float2(0.0f, 0.0f);
        if (r < QL) {
          hv = *reinterpret_cast<const float2 *>(&sm->hi[r][col(r, c0)]);
          lv = *reinterpret_cast<const float2 *>(&sm->lo[r][col(r, c0)]);
        }
        h0[j] = __float_as_uint(hv.x);
        h1[j] = __float_as_uint(hv.y);
        l0[j] = __float_as_uint(lv.x);
        l1[j] = __float_as_uint(lv.y);
      }
#pragma unroll
      for (int k = 0; k < NMMA; ++k) {
        const int am = 2 * tile_m(k), bn = tile_n(k);
        const uint32_t ah0 = h0[am], ah2 = h1[am], al0 = l0[am], al2 = l1[am];
        const uint32_t ah1 = am + 1 < NRB ? h0[am + 1] : 0u, ah3 = am + 1 < NRB ? h1[am + 1] : 0u;
        const uint32_t al1 = am + 1 < NRB ? l0[am + 1] : 0u, al3 = am + 1 < NRB ? l1[am + 1] : 0u;
        mma_tf32(acc[k], ah0, ah1, ah2, ah3, h0[bn], h1[bn]);
        mma_tf32(acc[k], ah0, ah1, ah2, ah3, l0[bn], l1[bn]);
        mma_tf32(acc[k], al0, al1, al2, al3, h0[bn], h1[bn]);
      }
    }
    __syncwarp();  // the tile is read before the next call writes it
    if (++tiles == kInnerTiles) {
      fold_inner();
      tiles = 0;
      if (++inners == kOuterFlushes) flush(sa.K);
    }
  }
};

// The observables of the sites one warp holds, for lattices with few
// populations (D1Q3, D2Q9): every lane adds its own sites' products into
// FP32 registers (the Q(Q+1)/2 pair sums e_i e_j, i <= j, the Q sums e_i and
// the mode sums), with no shared memory and no exchange per site.  After at
// most kThreadFoldSites sites a butterfly adds each value over the warp in
// FP32 (5 more roundings), and the lanes add the totals, two per lane, to the
// warp's FP64 values.  Same interface as WarpSampler.
constexpr int kThreadFoldSites = 128;

template <int LAT, int VX>
struct ThreadSampler {
  static constexpr int Q = Lattice<LAT>::Q;
  static constexpr int NP = Q * (Q + 1) / 2;        // pairs i <= j, row-major
  static constexpr int NV = NP + Q + 2 * kFusedModes;  // values a lane accumulates
  static_assert(NV <= 64, "two totals per lane");
  static constexpr int kFoldIters = kThreadFoldSites / VX;
  struct Smem {  // one warp's: [pairs | sum e_i | modes re, im]
    double v[NV];
  };

  Smem *sm;
  int lane, iters;
  float acc[NV];

  __device__ __forceinline__ void init(Smem *s, int lane_) {
    sm = s;
    lane = lane_;
    for (int k = lane; k < NV; k += 32) sm->v[k] = 0.0;
#pragma unroll
    for (int k = 0; k < NV; ++k) acc[k] = 0.0f;
    iters = 0;
    __syncwarp();
  }

  // FP32 sums over the warp (butterfly), then into the FP64 values: lane l
  // adds totals l and l + 32.  Called by all lanes.
  __device__ __forceinline__ void flush(int) {
    float t0 = 0.0f, t1 = 0.0f;
#pragma unroll
    for (int k = 0; k < NV; ++k) {
      float t = acc[k];
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
      if (k == lane) t0 = t;
      if (k == lane + 32) t1 = t;
      acc[k] = 0.0f;
    }
    if (lane < NV) sm->v[lane] += static_cast<double>(t0);
    if (lane + 32 < NV) sm->v[lane + 32] += static_cast<double>(t1);
    iters = 0;
  }

  template <typename S>
  __device__ __forceinline__ void add(const typename Store<S>::R (&f)[VX][Q], bool active, int x0, int y, int z,
                                      int Lx, int Ly, int Lz, const SampleArgs &sa) {
    if (active) {
      float tre[kFusedModes], tim[kFusedModes];
#pragma unroll
      for (int m = 0; m < kFusedModes; ++m) tre[m] = tim[m] = 0.0f;
#pragma unroll
      for (int k = 0; k < VX; ++k) {
        float e[Q], delta = 0.0f;
#pragma unroll
        for (int i = 0; i < Q; ++i) {
          e[i] = Store<S>::kDeviation ? static_cast<float>(f[k][i])
                                      : sub_rn(static_cast<float>(f[k][i]), obs_offset<LAT>(i, sa.rho_f));
          delta += e[i];
        }
        int p = 0;
#pragma unroll
        for (int i = 0; i < Q; ++i) {
#pragma unroll
          for (int j = i; j < Q; ++j, ++p) acc[p] = fmaf(e[i], e[j], acc[p]);
          acc[NP + i] += e[i];
        }
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
      // times the row's y and z factors
#pragma unroll
      for (int m = 0; m < kFusedModes; ++m)
        if (m < sa.K) {
          const float2 fy = sa.phase[sa.K * Lx + m * Ly + y];
          const float2 fz = sa.phase[sa.K * (Lx + Ly) + m * Lz + z];
          const float gr = fy.x * fz.x - fy.y * fz.y, gi = fy.x * fz.y + fy.y * fz.x;
          acc[NP + Q + 2 * m] += tre[m] * gr - tim[m] * gi;
          acc[NP + Q + 2 * m + 1] += tre[m] * gi + tim[m] * gr;
        }
    }
    if (++iters == kFoldIters) flush(sa.K);
  }

  // The block's partial set from its warps' values (warps in order), in the
  // layout of the FP32 observable pass: [sum delta, sum delta^2, sum e_i,
  // modes, pairs i <= j].  Called by `nthreads` threads after a barrier that
  // follows every warp's flush.
  template <class Sync>
  __device__ static __forceinline__ void block_partials(Smem *w, int nwarps, int K, double *out, int tid,
                                                        int nthreads, Sync sync) {
    for (int k = tid; k < NV; k += nthreads) {
      double t = 0.0;
      for (int j = 0; j < nwarps; ++j) t += w[j].v[k];
      w[0].v[k] = t;
    }
    sync();
    const int nq1 = 2 + Q + 2 * K;
    const double *v = w[0].v;
    for (int p = tid; p < NP; p += nthreads) out[nq1 + p] = v[p];
    if (tid < Q) out[2 + tid] = v[NP + tid];
    if (tid < 2 * K) out[2 + Q + tid] = v[NP + Q + tid];
    if (tid == 0) {
      double sd = 0.0, sd2 = 0.0;
      int p = 0;
      for (int i = 0; i < Q; ++i) {
        sd += v[NP + i];
        for (int j = i; j < Q; ++j, ++p) sd2 += (i == j ? 1.0 : 2.0) * v[p];
      }
      out[0] = sd;
      out[1] = sd2;
    }
  }
};

// The block's partial sums from its warps' slots (warps added in warp
// order), in the layout of the FP32 observable pass: [sum delta,
// sum delta^2, sum e_i, modes, pairs i <= j].  Called by `nthreads` threads
// (tid < nthreads) after a barrier among them that follows every warp's
// flush; `sync` is that barrier.
template <int LAT, int VX, class Sync>
__device__ __forceinline__ void warp_sampler_partials(typename WarpSampler<LAT, VX>::Smem *w, int nwarps, int K,
                                                      double *out, int tid, int nthreads, Sync sync) {
  using WS = WarpSampler<LAT, VX>;
  constexpr int Q = WS::Q;
  for (int k = tid; k < WS::NSLOT; k += nthreads) {
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
    out[nq1 + p0] = sl0[WS::slot(i, i + p)];
  }
  if (tid < Q) out[2 + tid] = sl0[WS::slot(tid, Q)];
  if (tid < 2 * K) out[2 + Q + tid] = w[0].modes[tid];
  if (tid == 0) {
    double sd = 0.0, sd2 = 0.0;
    for (int i = 0; i < Q; ++i) {
      sd += sl0[WS::slot(i, Q)];
      sd2 += sl0[WS::slot(i, i)];
      for (int j = i + 1; j < Q; ++j) sd2 += 2.0 * sl0[WS::slot(i, j)];
    }
    out[0] = sd;
    out[1] = sd2;
  }
}

template <int LAT, int VX>
template <class Sync>
__device__ __forceinline__ void WarpSampler<LAT, VX>::block_partials(Smem *w, int nwarps, int K, double *out, int tid,
                                                                     int nthreads, Sync sync) {
  warp_sampler_partials<LAT, VX>(w, nwarps, K, out, tid, nthreads, sync);
}

// The sampler of the register-pull kernel: per-lane registers where the
// pair sums fit them (D1Q3: 6, D2Q9: 45), else the tensor cores (D3Q19: 190).
template <int LAT, int VX>
using SamplerFor = std::conditional_t<(Lattice<LAT>::Q <= 9), ThreadSampler<LAT, VX>, WarpSampler<LAT, VX>>;

// Whether the sampled register-pull kernel collides its sites two at a time
// (collide_pair): as the unsampled kernel does, and for D3Q19 at two sites
// per thread too, where the sampled kernel's 128 registers hold both sites'
// variates (256^3 at a sample every 10 steps: 16-bit 37.7 against 37.4
// GLUPS, FP32 35.8 against 35.2).
template <int LAT, typename S, int VX>
__host__ __device__ constexpr bool sample_pairs() {
  return step_pairs<LAT, S, VX>() || LAT == kD3Q19;
}

template <int LAT, typename S, int VX, int NOISE, typename Idx>
__global__ void __launch_bounds__(kSampleThreads, 2)
    k_step_sample(const S *__restrict__ src, S *__restrict__ dst, const StepArgs a, const SampleArgs sa,
                  double *__restrict__ partials) {
  using L = Lattice<LAT>;
  using R = typename Store<S>::R;
  using WS = SamplerFor<LAT, VX>;
  constexpr int Q = L::Q;
  extern __shared__ __align__(16) unsigned char sample_smem[];
  typename WS::Smem *wsm = reinterpret_cast<typename WS::Smem *>(sample_smem);
  const int tid = static_cast<int>(threadIdx.x + blockDim.x * threadIdx.y);
  const int warp = tid >> 5;
  WS ws;
  ws.init(&wsm[warp], tid & 31);

  // a plain launch (no programmatic dependent launch either way): as a
  // dependent of a multi-wave step its persistent blocks cost D3Q19 256^3
  // 0.5 ms per sample on GB300
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
      collide_sites<LAT, S, VX, NOISE, sample_pairs<LAT, S, VX>()>(f, row + static_cast<uint32_t>(x0), a);
      vec_store<LAT, S, VX, Idx>(dst, a, row, x0, f);
    }
  }
  ws.flush(sa.K);
  __syncthreads();
  const int nq = 2 + Q + 2 * sa.K + Q * (Q + 1) / 2;
  WS::block_partials(wsm, kSampleWarps, sa.K, partials + static_cast<size_t>(blockIdx.x) * nq, tid, kSampleThreads,
                     [] { __syncthreads(); });
}

template <int LAT, typename S, int VX, int NOISE, typename Idx>
cudaError_t sample_launch(const void *src, void *dst, const StepArgs &a, const SampleArgs &sa_in, dim3 block,
                          double *partials, int *nblocks, cudaStream_t stream) {
  auto kern = k_step_sample<LAT, S, VX, NOISE, Idx>;
  constexpr size_t smem = kSampleWarps * sizeof(typename SamplerFor<LAT, VX>::Smem);
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
  kern<<<grid, block, smem, stream>>>(static_cast<const S *>(src), static_cast<S *>(dst), a, sa_in, partials);
  return cudaGetLastError();
}

// The sampled observables of a state alone, without the step: the pull and
// the sampler of k_step_sample on a persistent grid.  The separate sampling
// pass of the register-sampler lattices (D1Q3, D2Q9), in the partials
// layout of k_obs_pull.
template <int LAT, typename S, int VX, typename Idx>
__global__ void __launch_bounds__(kSampleThreads, 2)
    k_obs_sample(const S *__restrict__ src, const StepArgs a, const SampleArgs sa, double *__restrict__ partials) {
  using L = Lattice<LAT>;
  using R = typename Store<S>::R;
  using WS = SamplerFor<LAT, VX>;
  constexpr int Q = L::Q;
  extern __shared__ __align__(16) unsigned char sample_smem[];
  typename WS::Smem *wsm = reinterpret_cast<typename WS::Smem *>(sample_smem);
  const int tid = static_cast<int>(threadIdx.x + blockDim.x * threadIdx.y);
  const int warp = tid >> 5;
  WS ws;
  ws.init(&wsm[warp], tid & 31);
  for (int vb = blockIdx.x; vb < sa.nvb; vb += gridDim.x) {
    const int vbx = vb % sa.gx, vr = vb / sa.gx;
    const int vby = vr % sa.gy, vbz = vr / sa.gy;
    const int x0 = (vbx * static_cast<int>(blockDim.x) + static_cast<int>(threadIdx.x)) * VX;
    const int y = vby * static_cast<int>(blockDim.y) + static_cast<int>(threadIdx.y);
    const int z = vbz;
    const bool active = x0 < a.Lx && y < a.Ly;
    R f[VX][Q];
    if (active) (void)vec_pull<LAT, S, VX, Idx>(src, a, x0, y, z, f);
    ws.template add<S>(f, active, x0, y, z, a.Lx, a.Ly, a.Lz, sa);
  }
  ws.flush(sa.K);
  __syncthreads();
  const int nq = 2 + Q + 2 * sa.K + Q * (Q + 1) / 2;
  WS::block_partials(wsm, kSampleWarps, sa.K, partials + static_cast<size_t>(blockIdx.x) * nq, tid, kSampleThreads,
                     [] { __syncthreads(); });
}

template <int LAT, typename S, int VX, typename Idx>
cudaError_t obs_sample_launch(const void *src, const StepArgs &a, const SampleArgs &sa_in, dim3 block,
                              double *partials, int *nblocks, cudaStream_t stream) {
  auto kern = k_obs_sample<LAT, S, VX, Idx>;
  constexpr size_t smem = kSampleWarps * sizeof(typename SamplerFor<LAT, VX>::Smem);
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
  kern<<<grid, block, smem, stream>>>(static_cast<const S *>(src), a, sa_in, partials);
  return cudaGetLastError();
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

// The separate sampling pass on the register-pull kernel's blocks (D1Q3,
// D2Q9, FP32 arithmetic, the shape sample_fusable accepts).
template <int LAT, typename S>
cudaError_t obs_sample_t(const void *src, const StepArgs &a, int n_modes, const void *phase, double *partials,
                         int *nblocks, cudaStream_t stream) {
  if constexpr (sizeof(typename Store<S>::R) != 4 || Lattice<LAT>::Q > 9) {
    return cudaErrorInvalidValue;
  } else {
    if (n_modes < 0 || n_modes > kFusedModes || (n_modes > 0 && !phase)) return cudaErrorInvalidValue;
    const int vx = step_vec_width(LAT, Store<S>::kDeviation ? kStoreF16 : kStoreF32, a.Lx) >= 2 ? 2 : 1;
    dim3 grid, block;
    step_shape(a.Lx, a.Ly, a.Lz, grid, block, vx);
    if (block.x * block.y != kSampleThreads || block.x % 32 != 0) return cudaErrorInvalidValue;
    const SampleArgs sa = make_sample_args<LAT>(a, n_modes, phase, grid);
    const bool fit32 = offsets_fit_32(Lattice<LAT>::Q, a.N);
    if (vx == 2)
      return fit32 ? obs_sample_launch<LAT, S, 2, uint32_t>(src, a, sa, block, partials, nblocks, stream)
                   : obs_sample_launch<LAT, S, 2, size_t>(src, a, sa, block, partials, nblocks, stream);
    return fit32 ? obs_sample_launch<LAT, S, 1, uint32_t>(src, a, sa, block, partials, nblocks, stream)
                 : obs_sample_launch<LAT, S, 1, size_t>(src, a, sa, block, partials, nblocks, stream);
  }
}

}  // namespace lbfd
