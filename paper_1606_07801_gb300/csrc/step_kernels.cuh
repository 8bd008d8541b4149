// Kernels of the fused fluctuating lattice-Boltzmann step (see step.cu for
// the method).  Included by one translation unit per lattice.
#pragma once

#include <cuda_runtime.h>

#include <cstdlib>

#include "device.cuh"
#include "internal.h"

namespace lbfd {

enum StepNoise : int { kStepNoiseOff = 0, kStepNoiseGauss = 1, kStepNoiseFlat = 2 };

// The collision (collide_site below) written once over the value type V of
// device.cuh's lane arithmetic: V = R for one site, V = float2 (R = float)
// for sites s and s + 1 in the two lanes.  Every floating-point operation is
// an explicit add_rn / sub_rn / mul_rn / fma_rn, so both forms round alike.
template <int LAT, typename R, int NOISE, bool DEV, typename V>
__device__ __forceinline__ void collide_lanes(V (&f)[Lattice<LAT>::Q], uint32_t s, const StepArgs &a) {
  using L = Lattice<LAT>;
  constexpr int Q = L::Q;
  V rho = f[0];  // drho for DEV
  static_for<Q - 1>([&](auto I) { rho = add_rn(rho, f[decltype(I)::value + 1]); });

  V sigma = splat<V>(R(0));
  V T[Q];
  static_for<Q>([&](auto I) { T[decltype(I)::value] = splat<V>(R(0)); });
  if constexpr (NOISE != kStepNoiseOff) {
    // local noise: max(rho, 0); global noise: rho^eq (a select, not a branch)
    const V rho_eq = splat<V>(step_param<R>(a.rho_eq, a.rho_eq_f));
    const V rho_loc = positive_part(DEV ? add_rn(rho_eq, rho) : rho);
    const V rho_n = a.noise_mode == kNoiseLocal ? rho_loc : rho_eq;
    sigma = noise_amplitude<V>(mul_rn(rho_n, splat<V>(step_param<R>(a.noise_var, a.noise_var_f))));
    V zz[Q - 1];
    if constexpr (LaneOf<V>::kLanes == 2)
      draw_variates_pair<Q - 1, NOISE == kStepNoiseGauss>(zz, s, a.ph);
    else
      draw_variates_t<R, Q - 1, NOISE == kStepNoiseGauss>(zz, s, a.ph);
    NoiseTransform<LAT, R>::apply(zz, T);
  }

  const V omega = splat<V>(step_param<R>(a.omega, a.omega_f));
  const V relaxed = mul_rn(rho, splat<V>(step_param<R>(a.inv_tau, a.inv_tau_f)));
  // f*_i = (1 - 1/tau) f_i + w_i rho/tau + w_i sigma T_i, with w_i rho/tau and
  // w_i sigma formed once per distinct weight.  The moving populations are
  // written first; the rest population takes what mass conservation leaves,
  // so the rounding of sum_i w_i = 1 cannot make the mass drift.
  V wrel[Q], wsig[Q];
  V moved = splat<V>(R(0));
  static_for<Q - 1>([&](auto I) {
    constexpr int i = decltype(I)::value + 1;
    constexpr int k = first_of_weight<LAT>(i);
    if constexpr (k == i) {
      wrel[i] = mul_rn(cst<V>(L::w(i)), relaxed);
      if constexpr (!NoiseTransform<LAT, R>::kWeighted) wsig[i] = mul_rn(cst<V>(L::w(i)), sigma);
    }
    if constexpr (NoiseTransform<LAT, R>::kWeighted) {
      f[i] = fma_rn(omega, f[i], fma_rn(sigma, T[i], wrel[k]));
    } else {
      f[i] = fma_rn(omega, f[i], fma_rn(wsig[k], T[i], wrel[k]));
    }
    moved = add_rn(moved, f[i]);
  });
  f[0] = sub_rn(rho, moved);
}

// Collision of one site in registers: f holds the pulled populations
// f_i(x, t) on entry and the post-collision f*_i(x) on exit; s is the site
// index that keys the noise.
//
// DEV: f holds the deviations d_i = f_i - w_i rho_mean instead (the 16-bit
// storage formats).  With rho = rho_mean + drho, drho = sum_i d_i, and
// 1 - 1/tau = omega, the update f*_i = omega f_i + w_i rho/tau + w_i sigma T_i
// is d*_i = omega d_i + w_i drho/tau + w_i sigma T_i in exact arithmetic (the
// w_i rho_mean terms cancel), so the same code runs on the deviations with
// drho in place of rho; only the noise amplitude needs rho itself.
template <int LAT, typename R, int NOISE, bool DEV = false>
__device__ __forceinline__ void collide_site(R (&f)[Lattice<LAT>::Q], uint32_t s, const StepArgs &a) {
  collide_lanes<LAT, R, NOISE, DEV, R>(f, s, a);
}

// Collision of sites s (fa) and s + 1 (fb) at once on the packed FP32
// instructions: bit for bit the same as collide_site on each.
template <int LAT, int NOISE, bool DEV = false>
__device__ __forceinline__ void collide_pair(float (&fa)[Lattice<LAT>::Q], float (&fb)[Lattice<LAT>::Q], uint32_t s,
                                             const StepArgs &a) {
  constexpr int Q = Lattice<LAT>::Q;
  float2 f[Q];
#pragma unroll
  for (int i = 0; i < Q; ++i) f[i] = make_float2(fa[i], fb[i]);
  collide_lanes<LAT, float, NOISE, DEV, float2>(f, s, a);
#pragma unroll
  for (int i = 0; i < Q; ++i) {
    fa[i] = f[i].x;
    fb[i] = f[i].y;
  }
}

// The single-relaxation-time collision as a function object, the default
// collision of the site-update bodies below (DEV for the deviation formats).
// kPairs: FP32 arithmetic, so pair() updates two neighbouring sites on the
// packed instructions.
template <int LAT, typename R, int NOISE, bool DEV = false>
struct SrtCollide {
  static constexpr bool kPairs = std::is_same<R, float>::value;
  __device__ __forceinline__ void operator()(R (&f)[Lattice<LAT>::Q], uint32_t s, const StepArgs &a) const {
    collide_site<LAT, R, NOISE, DEV>(f, s, a);
  }
  __device__ __forceinline__ void pair(R (&fa)[Lattice<LAT>::Q], R (&fb)[Lattice<LAT>::Q], uint32_t s,
                                       const StepArgs &a) const {
    if constexpr (kPairs) {
      collide_pair<LAT, NOISE, DEV>(fa, fb, s, a);
    } else {
      collide_site<LAT, R, NOISE, DEV>(fa, s, a);
      collide_site<LAT, R, NOISE, DEV>(fb, s + 1u, a);
    }
  }
};
// The default collision for storage S.
template <int LAT, typename S, int NOISE>
using SrtCollideFor = SrtCollide<LAT, typename Store<S>::R, NOISE, Store<S>::kDeviation>;

// Whether collision C has a paired form (SrtCollide with FP32 arithmetic).
template <class C, class = void>
struct CollidePairs : std::false_type {};
template <class C>
struct CollidePairs<C, std::void_t<decltype(C::kPairs)>> : std::bool_constant<C::kPairs> {};

// The work block of this CTA: its own index, or for sweep = 1 the mirror
// image, so that a step launched after a forward one starts on the rows the
// previous step wrote last, which are still in L2.  The hardware dispatches
// CTAs in index order either way; which CTA takes which block changes
// nothing else.
__device__ __forceinline__ uint3 sweep_block(int32_t sweep) {
  if (!sweep) return blockIdx;
  return make_uint3(gridDim.x - 1 - blockIdx.x, gridDim.y - 1 - blockIdx.y, gridDim.z - 1 - blockIdx.z);
}

// Update of site (x, y, z) of one lattice (any shape).  S is the storage
// type (float, double, or a 16-bit deviation format with FP32 arithmetic).
// Idx is the type of the value offsets i N + site: uint32_t when Q N < 2^32
// (fewer address instructions), size_t otherwise.
template <int LAT, typename S, int NOISE, class C = SrtCollideFor<LAT, S, NOISE>, typename Idx = size_t>
__device__ __forceinline__ void step_scalar_body(const S *__restrict__ src, S *__restrict__ dst, const StepArgs &a,
                                                 int x, int y, int z, const C &collide = C()) {
  using L = Lattice<LAT>;
  using R = typename Store<S>::R;
  constexpr int Q = L::Q;
  const uint32_t Lx = static_cast<uint32_t>(a.Lx), Lxy = Lx * static_cast<uint32_t>(a.Ly);
  const uint32_t Lxyz = Lxy * static_cast<uint32_t>(a.Lz);
  const uint32_t s = static_cast<uint32_t>(x) + Lx * static_cast<uint32_t>(y) + Lxy * static_cast<uint32_t>(z);
  // periodic neighbours as offsets from s (modulo 2^32): to x - 1 and x + 1,
  // y - 1 and y + 1, z - 1 and z + 1
  const uint32_t dxm = x == 0 ? Lx - 1u : 0u - 1u, dxp = x + 1 == a.Lx ? 1u - Lx : 1u;
  const uint32_t dym = y == 0 ? Lxy - Lx : 0u - Lx, dyp = y + 1 == a.Ly ? Lx - Lxy : Lx;
  const uint32_t dzm = z == 0 ? Lxyz - Lxy : 0u - Lxy, dzp = z + 1 == a.Lz ? Lxy - Lxyz : Lxy;

  // pull: population i arrives from x - v_i
  R f[Q];
  static_for<Q>([&](auto I) {
    constexpr int i = decltype(I)::value;
    constexpr int vx = L::v(i, 0), vy = L::v(i, 1), vz = L::v(i, 2);
    const uint32_t ox = vx == 0 ? 0u : (vx > 0 ? dxm : dxp);
    const uint32_t oy = vy == 0 ? 0u : (vy > 0 ? dym : dyp);
    const uint32_t oz = vz == 0 ? 0u : (vz > 0 ? dzm : dzp);
    const uint32_t so = s + ox + oy + oz;
    f[i] = Store<S>::load(src[static_cast<Idx>(i) * static_cast<Idx>(a.N) + so]);
  });
  collide(f, s, a);
  static_for<Q>([&](auto I) {
    constexpr int i = decltype(I)::value;
    dst[static_cast<Idx>(i) * static_cast<Idx>(a.N) + s] = Store<S>::store(f[i]);
  });
}

// Programmatic dependent launch.  A step kernel lets the next kernel of its
// stream launch once all of its own blocks have started, so the next step's
// blocks take the SM slots that this step's last blocks free; each block then
// waits for the previous grid's completion (and memory) before its first
// load.  Without the launch attribute both instructions do nothing.
__device__ __forceinline__ void pdl_launch_dependents() {
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }

// Scalar kernel: one site per thread, any lattice shape.
template <int LAT, typename S, int NOISE, typename Idx>
__global__ void __launch_bounds__(256) k_step(const S *__restrict__ src, S *__restrict__ dst, const StepArgs a) {
  pdl_launch_dependents();
  const uint3 b = sweep_block(a.sweep);
  const int x = b.x * blockDim.x + threadIdx.x;
  const int y = b.y * blockDim.y + threadIdx.y;
  const int z = b.z;
  pdl_wait();
  if (x >= a.Lx || y >= a.Ly) return;
  step_scalar_body<LAT, S, NOISE, SrtCollideFor<LAT, S, NOISE>, Idx>(src, dst, a, x, y, z);
}

// Vector kernel: VX consecutive sites of a row per thread (needs Lx % VX == 0).
// Each population is one aligned VX-wide load at x0 (populations with
// v_x = 0), plus, for v_x = +1 / -1, one scalar load of the column left of
// x0 / right of x0 + VX - 1 (wrapped); stores are VX-wide.  This cuts the
// address arithmetic and memory instructions per site by about VX.
template <typename S, int VX>
struct alignas(sizeof(S) * VX) Pack {
  S v[VX];
};

// Conversions of a VX-wide pack of stored values to and from the compute
// type (format only, see Store<S>::load/store).  Two 16-bit values go
// through one paired conversion each way (cvt.rn.f16x2.f32 /
// cvt.rn.bf16x2.f32 for the encode); every element rounds as the scalar
// conversion would, so packed and single-value kernels agree bit for bit.
template <typename S, int VX>
struct PackCvt {
  using R = typename Store<S>::R;
  __device__ static __forceinline__ void load(const Pack<S, VX> &p, R (&v)[VX]) {
#pragma unroll
    for (int k = 0; k < VX; ++k) v[k] = Store<S>::load(p.v[k]);
  }
  __device__ static __forceinline__ Pack<S, VX> store(const R (&v)[VX]) {
    Pack<S, VX> p;
#pragma unroll
    for (int k = 0; k < VX; ++k) p.v[k] = Store<S>::store(v[k]);
    return p;
  }
};
template <>
struct PackCvt<__half, 2> {
  __device__ static __forceinline__ void load(const Pack<__half, 2> &p, float (&v)[2]) {
    const float2 f = __half22float2(*reinterpret_cast<const __half2 *>(&p));
    v[0] = f.x;
    v[1] = f.y;
  }
  __device__ static __forceinline__ Pack<__half, 2> store(const float (&v)[2]) {
    const __half2 h = __floats2half2_rn(v[0], v[1]);  // .x (low half, v[0]) first in memory
    return *reinterpret_cast<const Pack<__half, 2> *>(&h);
  }
};
template <>
struct PackCvt<__nv_bfloat16, 2> {
  __device__ static __forceinline__ void load(const Pack<__nv_bfloat16, 2> &p, float (&v)[2]) {
    const float2 f = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162 *>(&p));
    v[0] = f.x;
    v[1] = f.y;
  }
  __device__ static __forceinline__ Pack<__nv_bfloat16, 2> store(const float (&v)[2]) {
    const __nv_bfloat162 h = __floats2bfloat162_rn(v[0], v[1]);
    return *reinterpret_cast<const Pack<__nv_bfloat16, 2> *>(&h);
  }
};

// Minimum resident 256-thread blocks per SM asked of the register allocator
// for the vector kernel.  Measured on GB300 (FP32, local Gaussian noise):
// D2Q9 2048^2 is fastest at 4 blocks (<= 64 registers, no spills with two
// or four sites per thread; four sites: 47.9 against 48.9 us per step at 3
// blocks), D3Q19 256^3 at 3 (<= 85 registers); the unconstrained allocation
// leaves D3Q19 one block per SM, and tighter caps spill.  D3Q19 with four
// sites per thread (16-bit storage) and FP64 kernels need more registers: 2.
template <int LAT, typename S, int VX = 2>
constexpr int step_min_blocks() {
  if (VX == 4) return (sizeof(typename Store<S>::R) != 4 || LAT == kD3Q19) ? 2 : 4;
  if (sizeof(typename Store<S>::R) != 4) return 2;
  return LAT == kD3Q19 ? 3 : 4;
}

// Whether the vector kernel collides its sites two at a time on the packed
// FP32 instructions (collide_pair; a tuning choice, results are the same bit
// for bit).  Pairs cut the instructions per site (D3Q19 FP32: 590 against 695,
// D2Q9: 244 against 277) but hold two sites' noise variates at once, and pay
// only where the registers allow.  On GB300, microseconds per step:
//   D2Q9 FP32 at 2048^2, 2 sites per thread:    46.5 paired, 47.8 not
//   D2Q9 FP32 at 2048^2, 4 sites per thread:    48.2 paired (spills), 46.3 not
//   D3Q19 FP32 at 256^3, 2 sites per thread:   472.7 paired (spills), 412.5 not
//   D3Q19 16-bit at 256^3, 4 sites per thread: 400.6 paired, 419.1 not
//   D2Q9 16-bit at 2048^2, 4 sites per thread:   41.4 paired, 42.5 not
//   D1Q3 FP32 at 2^24, 2 sites per thread:       68.1 paired, 72.3 not
template <int LAT, typename S, int VX>
__host__ __device__ constexpr bool step_pairs() {
  if (LAT == kD3Q19) return Store<S>::kDeviation && VX == 4;
  return VX == 2 || (LAT == kD2Q9 && Store<S>::kDeviation);
}

// The SRT collision of sites s0 .. s0 + VX - 1 (f[k] holds site s0 + k), two
// at a time where PAIRS (FP32 arithmetic only).
template <int LAT, typename S, int VX, int NOISE, bool PAIRS>
__device__ __forceinline__ void collide_sites(typename Store<S>::R (&f)[VX][Lattice<LAT>::Q], uint32_t s0,
                                              const StepArgs &a) {
  using R = typename Store<S>::R;
  constexpr bool DEV = Store<S>::kDeviation;
  if constexpr (PAIRS && VX % 2 == 0 && std::is_same<R, float>::value) {
#pragma unroll
    for (int k = 0; k < VX; k += 2) collide_pair<LAT, NOISE, DEV>(f[k], f[k + 1], s0 + static_cast<uint32_t>(k), a);
  } else {
#pragma unroll
    for (int k = 0; k < VX; ++k) collide_site<LAT, R, NOISE, DEV>(f[k], s0 + static_cast<uint32_t>(k), a);
  }
}

// Update of sites (x0 .. x0 + VX - 1, y, z) of one lattice (Lx % VX == 0).
// Pull of sites (x0 .. x0 + VX - 1, y, z) into f[k][i] = f_i(x0 + k, t):
// the first half of step_vec_body (Lx % VX == 0).  Returns the row offset
// Lx (y + Ly z) of the sites.
template <int LAT, typename S, int VX, typename Idx>
__device__ __forceinline__ uint32_t vec_pull(const S *__restrict__ src, const StepArgs &a, int x0, int y, int z,
                                             typename Store<S>::R (&f)[VX][Lattice<LAT>::Q]) {
  using L = Lattice<LAT>;
  using R = typename Store<S>::R;
  using P = Pack<S, VX>;
  constexpr int Q = L::Q;
  const int xl = (x0 == 0 ? a.Lx : x0) - 1;        // column left of the vector
  const int xr = (x0 + VX == a.Lx) ? 0 : x0 + VX;  // column right of the vector
  const int ym = (y == 0 ? a.Ly : y) - 1, yp = (y + 1 == a.Ly) ? 0 : y + 1;
  const int zm = (z == 0 ? a.Lz : z) - 1, zp = (z + 1 == a.Lz) ? 0 : z + 1;
  const uint32_t Lx = static_cast<uint32_t>(a.Lx), Lxy = Lx * static_cast<uint32_t>(a.Ly);
  static_for<Q>([&](auto I) {
    constexpr int i = decltype(I)::value;
    constexpr int vx = L::v(i, 0), vy = L::v(i, 1), vz = L::v(i, 2);
    const int ys = vy == 0 ? y : (vy > 0 ? ym : yp);
    const int zs = vz == 0 ? z : (vz > 0 ? zm : zp);
    const uint32_t srow = Lx * static_cast<uint32_t>(ys) + Lxy * static_cast<uint32_t>(zs);
    const S *pop = src + (static_cast<Idx>(i) * static_cast<Idx>(a.N) + static_cast<Idx>(srow));
    const P pk = *reinterpret_cast<const P *>(pop + x0);
    R v[VX];
    PackCvt<S, VX>::load(pk, v);
    if constexpr (vx == 0) {
#pragma unroll
      for (int k = 0; k < VX; ++k) f[k][i] = v[k];
    } else if constexpr (vx > 0) {  // site x0 + k pulls from x0 + k - 1
      f[0][i] = Store<S>::load(pop[xl]);
#pragma unroll
      for (int k = 1; k < VX; ++k) f[k][i] = v[k - 1];
    } else {  // site x0 + k pulls from x0 + k + 1
#pragma unroll
      for (int k = 0; k < VX - 1; ++k) f[k][i] = v[k + 1];
      f[VX - 1][i] = Store<S>::load(pop[xr]);
    }
  });
  return Lx * static_cast<uint32_t>(y) + Lxy * static_cast<uint32_t>(z);
}

// Store of f*_i of sites (x0 .. x0 + VX - 1) of the row at offset `row`:
// the second half of step_vec_body (VX-wide stores).
template <int LAT, typename S, int VX, typename Idx>
__device__ __forceinline__ void vec_store(S *__restrict__ dst, const StepArgs &a, uint32_t row, int x0,
                                          const typename Store<S>::R (&f)[VX][Lattice<LAT>::Q]) {
  using R = typename Store<S>::R;
  using P = Pack<S, VX>;
  static_for<Lattice<LAT>::Q>([&](auto I) {
    constexpr int i = decltype(I)::value;
    R v[VX];
#pragma unroll
    for (int k = 0; k < VX; ++k) v[k] = f[k][i];
    *reinterpret_cast<P *>(dst + (static_cast<Idx>(i) * static_cast<Idx>(a.N) + static_cast<Idx>(row) + static_cast<Idx>(x0))) =
        PackCvt<S, VX>::store(v);
  });
}

template <int LAT, typename S, int VX, int NOISE, class C = SrtCollideFor<LAT, S, NOISE>, typename Idx = size_t>
__device__ __forceinline__ void step_vec_body(const S *__restrict__ src, S *__restrict__ dst, const StepArgs &a, int x0,
                                              int y, int z, const C &collide = C()) {
  typename Store<S>::R f[VX][Lattice<LAT>::Q];
  const uint32_t row = vec_pull<LAT, S, VX, Idx>(src, a, x0, y, z, f);
  if constexpr (CollidePairs<C>::value && VX % 2 == 0 && step_pairs<LAT, S, VX>()) {
#pragma unroll
    for (int k = 0; k < VX; k += 2) collide.pair(f[k], f[k + 1], row + static_cast<uint32_t>(x0 + k), a);
  } else {
#pragma unroll
    for (int k = 0; k < VX; ++k) collide(f[k], row + static_cast<uint32_t>(x0 + k), a);
  }
  vec_store<LAT, S, VX, Idx>(dst, a, row, x0, f);
}

template <int LAT, typename S, int VX, int NOISE, typename Idx>
__global__ void __launch_bounds__(256, step_min_blocks<LAT, S, VX>())
    k_step_vec(const S *__restrict__ src, S *__restrict__ dst, const StepArgs a) {
  pdl_launch_dependents();
  const uint3 b = sweep_block(a.sweep);
  const int x0 = (b.x * blockDim.x + threadIdx.x) * VX;
  const int y = b.y * blockDim.y + threadIdx.y;
  const int z = b.z;
  pdl_wait();
  if (x0 >= a.Lx || y >= a.Ly) return;
  step_vec_body<LAT, S, VX, NOISE, SrtCollideFor<LAT, S, NOISE>, Idx>(src, dst, a, x0, y, z);
}

// True when every value offset i N + site of a lattice fits 32 bits.
inline bool offsets_fit_32(int Q, int64_t N) {
  return static_cast<uint64_t>(Q) * static_cast<uint64_t>(N) <= 0xffffffffull;
}


// Programmatic dependent launch of the step kernels (a tuning knob; results
// do not depend on it).  LBFD_STEP_PDL = 0 launches them plainly.
inline bool step_pdl() {
  static bool v = [] {
    const char *e = getenv("LBFD_STEP_PDL");
    return !(e && atoi(e) == 0);
  }();
  return v;
}

template <int LAT, typename S, int NOISE, typename Idx>
cudaError_t step_noise_idx(const S *s, S *d, const StepArgs &a, int vx, cudaStream_t stream) {
  dim3 grid, block;
  step_shape(a.Lx, a.Ly, a.Lz, grid, block, vx);
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = 0;
  cfg.stream = stream;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = step_pdl() ? 1 : 0;
  if (vx == 2) return cudaLaunchKernelEx(&cfg, k_step_vec<LAT, S, 2, NOISE, Idx>, s, d, a);
  if constexpr (sizeof(typename Store<S>::R) == 4)
    if (vx == 4) return cudaLaunchKernelEx(&cfg, k_step_vec<LAT, S, 4, NOISE, Idx>, s, d, a);
  return cudaLaunchKernelEx(&cfg, k_step<LAT, S, NOISE, Idx>, s, d, a);
}

template <int LAT, typename S, int NOISE>
cudaError_t step_noise(const void *src, void *dst, const StepArgs &a, cudaStream_t stream, int vx) {
  const S *s = static_cast<const S *>(src);
  S *d = static_cast<S *>(dst);
  if (offsets_fit_32(Lattice<LAT>::Q, a.N)) return step_noise_idx<LAT, S, NOISE, uint32_t>(s, d, a, vx, stream);
  return step_noise_idx<LAT, S, NOISE, size_t>(s, d, a, vx, stream);
}

// Kernel selection by noise configuration: each variant is branch-free in
// its per-site code, so the compiler can interleave the sites of a thread.
template <int LAT, typename S>
cudaError_t step_t(const void *src, void *dst, const StepArgs &a, cudaStream_t stream, int vx) {
  if (a.noise_mode == kNoiseOff) return step_noise<LAT, S, kStepNoiseOff>(src, dst, a, stream, vx);
  if (a.noise_dist == kGaussian) return step_noise<LAT, S, kStepNoiseGauss>(src, dst, a, stream, vx);
  return step_noise<LAT, S, kStepNoiseFlat>(src, dst, a, stream, vx);
}

}  // namespace lbfd
