// Kernels of the fused fluctuating lattice-Boltzmann step (see step.cu for
// the method).  Included by one translation unit per lattice.
#pragma once

#include <cuda_runtime.h>

#include <cstdlib>

#include "device.cuh"
#include "internal.h"

namespace lbfd {

enum StepNoise : int { kStepNoiseOff = 0, kStepNoiseGauss = 1, kStepNoiseFlat = 2 };

// Collision of one site in registers: f holds the pulled populations
// f_i(x, t) on entry and the post-collision f*_i(x) on exit; s is the site
// index that keys the noise.
template <int LAT, typename R, int NOISE>
__device__ __forceinline__ void collide_site(R (&f)[Lattice<LAT>::Q], uint32_t s, const StepArgs &a) {
  using L = Lattice<LAT>;
  constexpr int Q = L::Q;
  R rho = f[0];
  static_for<Q - 1>([&](auto I) { rho += f[decltype(I)::value + 1]; });

  R sigma = R(0);
  R T[Q];
  static_for<Q>([&](auto I) { T[decltype(I)::value] = R(0); });
  if constexpr (NOISE != kStepNoiseOff) {
    // local noise: max(rho, 0); global noise: rho^eq (a select, not a branch)
    const R rho_loc = rho > R(0) ? rho : R(0);
    const R rho_n = a.noise_mode == kNoiseLocal ? rho_loc : step_param<R>(a.rho_eq, a.rho_eq_f);
    sigma = noise_amplitude<R>(rho_n * step_param<R>(a.noise_var, a.noise_var_f));
    R zz[Q - 1];
    draw_variates_t<R, Q - 1, NOISE == kStepNoiseGauss>(zz, s, a.ph);
    NoiseTransform<LAT, R>::apply(zz, T);
  }

  const R omega = step_param<R>(a.omega, a.omega_f);
  const R relaxed = rho * step_param<R>(a.inv_tau, a.inv_tau_f);
  // f*_i = (1 - 1/tau) f_i + w_i rho/tau + w_i sigma T_i, with w_i rho/tau and
  // w_i sigma formed once per distinct weight.  The moving populations are
  // written first; the rest population takes what mass conservation leaves,
  // so the rounding of sum_i w_i = 1 cannot make the mass drift.
  R moved = R(0);
  static_for<Q - 1>([&](auto I) {
    constexpr int i = decltype(I)::value + 1;
    const R w = static_cast<R>(L::w(i));
    const R wrel = w * relaxed;
    if constexpr (NoiseTransform<LAT, R>::kWeighted) {
      f[i] = fma(omega, f[i], fma(sigma, T[i], wrel));
    } else {
      f[i] = fma(omega, f[i], fma(w * sigma, T[i], wrel));
    }
    moved += f[i];
  });
  f[0] = rho - moved;
}

// Scalar kernel: one site per thread, any lattice shape.
template <int LAT, typename R, int NOISE>
__global__ void __launch_bounds__(256) k_step(const R *__restrict__ src, R *__restrict__ dst, const StepArgs a) {
  using L = Lattice<LAT>;
  constexpr int Q = L::Q;
  const int x = blockIdx.x * blockDim.x + threadIdx.x;
  const int y = blockIdx.y * blockDim.y + threadIdx.y;
  const int z = blockIdx.z;
  if (x >= a.Lx || y >= a.Ly) return;
  // periodic neighbours
  const int xm = (x == 0 ? a.Lx : x) - 1, xp = (x + 1 == a.Lx) ? 0 : x + 1;
  const int ym = (y == 0 ? a.Ly : y) - 1, yp = (y + 1 == a.Ly) ? 0 : y + 1;
  const int zm = (z == 0 ? a.Lz : z) - 1, zp = (z + 1 == a.Lz) ? 0 : z + 1;
  const uint32_t Lx = static_cast<uint32_t>(a.Lx), Lxy = Lx * static_cast<uint32_t>(a.Ly);
  const uint32_t s = static_cast<uint32_t>(x) + Lx * static_cast<uint32_t>(y) + Lxy * static_cast<uint32_t>(z);

  // pull: population i arrives from x - v_i
  R f[Q];
  static_for<Q>([&](auto I) {
    constexpr int i = decltype(I)::value;
    constexpr int vx = L::v(i, 0), vy = L::v(i, 1), vz = L::v(i, 2);
    const int xs = vx == 0 ? x : (vx > 0 ? xm : xp);
    const int ys = vy == 0 ? y : (vy > 0 ? ym : yp);
    const int zs = vz == 0 ? z : (vz > 0 ? zm : zp);
    const uint32_t so = static_cast<uint32_t>(xs) + Lx * static_cast<uint32_t>(ys) + Lxy * static_cast<uint32_t>(zs);
    f[i] = __ldg(src + static_cast<size_t>(i) * static_cast<size_t>(a.N) + so);
  });
  collide_site<LAT, R, NOISE>(f, s, a);
  static_for<Q>([&](auto I) {
    constexpr int i = decltype(I)::value;
    dst[static_cast<size_t>(i) * static_cast<size_t>(a.N) + s] = f[i];
  });
}

// Vector kernel: VX consecutive sites of a row per thread (needs Lx % VX == 0).
// Each population is one aligned VX-wide load at x0 (populations with
// v_x = 0), plus, for v_x = +1 / -1, one scalar load of the column left of
// x0 / right of x0 + VX - 1 (wrapped); stores are VX-wide.  This cuts the
// address arithmetic and memory instructions per site by about VX.
template <typename R, int VX>
struct VecOf;
template <>
struct VecOf<float, 4> {
  using T = float4;
  __device__ static __forceinline__ void get(const T &v, float (&o)[4]) { o[0] = v.x; o[1] = v.y; o[2] = v.z; o[3] = v.w; }
  __device__ static __forceinline__ T make(const float (&o)[4]) { return make_float4(o[0], o[1], o[2], o[3]); }
};
template <>
struct VecOf<float, 2> {
  using T = float2;
  __device__ static __forceinline__ void get(const T &v, float (&o)[2]) { o[0] = v.x; o[1] = v.y; }
  __device__ static __forceinline__ T make(const float (&o)[2]) { return make_float2(o[0], o[1]); }
};
template <>
struct VecOf<double, 2> {
  using T = double2;
  __device__ static __forceinline__ void get(const T &v, double (&o)[2]) { o[0] = v.x; o[1] = v.y; }
  __device__ static __forceinline__ T make(const double (&o)[2]) { return make_double2(o[0], o[1]); }
};

// Minimum resident 256-thread blocks per SM asked of the register allocator
// for the vector kernel.  Measured on GB300 (FP32, local Gaussian noise,
// two sites per thread): D2Q9 2048^2 is fastest at 4 blocks (<= 64
// registers), D3Q19 256^3 at 3 (<= 85 registers); the unconstrained
// allocation leaves D3Q19 one block per SM, and tighter caps spill.  FP64
// kernels need more registers: 2.
template <int LAT, typename R>
constexpr int step_min_blocks() {
  if (sizeof(R) != 4) return 2;
  return LAT == kD3Q19 ? 3 : 4;
}

template <int LAT, typename R, int VX, int NOISE>
__global__ void __launch_bounds__(256, step_min_blocks<LAT, R>()) k_step_vec(const R *__restrict__ src, R *__restrict__ dst, const StepArgs a) {
  using L = Lattice<LAT>;
  using V = VecOf<R, VX>;
  constexpr int Q = L::Q;
  const int x0 = (blockIdx.x * blockDim.x + threadIdx.x) * VX;
  const int y = blockIdx.y * blockDim.y + threadIdx.y;
  const int z = blockIdx.z;
  if (x0 >= a.Lx || y >= a.Ly) return;
  const int xl = (x0 == 0 ? a.Lx : x0) - 1;        // column left of the vector
  const int xr = (x0 + VX == a.Lx) ? 0 : x0 + VX;  // column right of the vector
  const int ym = (y == 0 ? a.Ly : y) - 1, yp = (y + 1 == a.Ly) ? 0 : y + 1;
  const int zm = (z == 0 ? a.Lz : z) - 1, zp = (z + 1 == a.Lz) ? 0 : z + 1;
  const uint32_t Lx = static_cast<uint32_t>(a.Lx), Lxy = Lx * static_cast<uint32_t>(a.Ly);
  const uint32_t row = Lx * static_cast<uint32_t>(y) + Lxy * static_cast<uint32_t>(z);

  R f[VX][Q];
  static_for<Q>([&](auto I) {
    constexpr int i = decltype(I)::value;
    constexpr int vx = L::v(i, 0), vy = L::v(i, 1), vz = L::v(i, 2);
    const int ys = vy == 0 ? y : (vy > 0 ? ym : yp);
    const int zs = vz == 0 ? z : (vz > 0 ? zm : zp);
    const uint32_t srow = Lx * static_cast<uint32_t>(ys) + Lxy * static_cast<uint32_t>(zs);
    const R *pop = src + static_cast<size_t>(i) * static_cast<size_t>(a.N) + srow;
    R v[VX];
    V::get(__ldg(reinterpret_cast<const typename V::T *>(pop + x0)), v);
    if constexpr (vx == 0) {
#pragma unroll
      for (int k = 0; k < VX; ++k) f[k][i] = v[k];
    } else if constexpr (vx > 0) {  // site x0 + k pulls from x0 + k - 1
      f[0][i] = __ldg(pop + xl);
#pragma unroll
      for (int k = 1; k < VX; ++k) f[k][i] = v[k - 1];
    } else {  // site x0 + k pulls from x0 + k + 1
#pragma unroll
      for (int k = 0; k < VX - 1; ++k) f[k][i] = v[k + 1];
      f[VX - 1][i] = __ldg(pop + xr);
    }
  });
#pragma unroll
  for (int k = 0; k < VX; ++k) collide_site<LAT, R, NOISE>(f[k], row + static_cast<uint32_t>(x0 + k), a);
  static_for<Q>([&](auto I) {
    constexpr int i = decltype(I)::value;
    R o[VX];
#pragma unroll
    for (int k = 0; k < VX; ++k) o[k] = f[k][i];
    *reinterpret_cast<typename V::T *>(dst + static_cast<size_t>(i) * static_cast<size_t>(a.N) + row + x0) = V::make(o);
  });
}

inline void step_shape(int32_t Lx, int32_t Ly, int32_t Lz, dim3 &grid, dim3 &block, int vx = 1) {
  const int cols = Lx / vx;
  int bx = 256;
  while (bx > 32 && bx / 2 >= cols) bx /= 2;
  int by = 256 / bx;
  while (by > 1 && by / 2 >= Ly) by /= 2;
  block = dim3(bx, by, 1);
  grid = dim3((cols + bx - 1) / bx, (Ly + by - 1) / by, Lz);
}

// Sites per thread of the step kernel (a tuning knob; results do not depend
// on it).  LBFD_STEP_VX = 1, 2 or 4 overrides the default of 2 when Lx
// allows (else 1).
inline int step_vx_override() {
  static int v = [] {
    const char *e = getenv("LBFD_STEP_VX");
    const int r = e ? atoi(e) : 0;
    return (r == 1 || r == 2 || r == 4) ? r : 0;
  }();
  return v;
}

template <int LAT, typename R, int NOISE>
cudaError_t step_noise(const void *src, void *dst, const StepArgs &a, cudaStream_t stream) {
  int vx = step_vx_override();
  if (vx == 0) vx = 2;
  if (sizeof(R) == 8 && vx == 4) vx = 2;
  while (vx > 1 && a.Lx % vx != 0) vx /= 2;
  dim3 grid, block;
  step_shape(a.Lx, a.Ly, a.Lz, grid, block, vx);
  const R *s = static_cast<const R *>(src);
  R *d = static_cast<R *>(dst);
  if constexpr (sizeof(R) == 4) {
    if (vx == 4) {
      k_step_vec<LAT, R, 4, NOISE><<<grid, block, 0, stream>>>(s, d, a);
      return cudaGetLastError();
    }
  }
  if (vx == 2) {
    k_step_vec<LAT, R, 2, NOISE><<<grid, block, 0, stream>>>(s, d, a);
    return cudaGetLastError();
  }
  k_step<LAT, R, NOISE><<<grid, block, 0, stream>>>(s, d, a);
  return cudaGetLastError();
}

// Kernel selection by noise configuration: each variant is branch-free in
// its per-site code, so the compiler can interleave the sites of a thread.
template <int LAT, typename R>
cudaError_t step_t(const void *src, void *dst, const StepArgs &a, cudaStream_t stream) {
  if (a.noise_mode == kNoiseOff) return step_noise<LAT, R, kStepNoiseOff>(src, dst, a, stream);
  if (a.noise_dist == kGaussian) return step_noise<LAT, R, kStepNoiseGauss>(src, dst, a, stream);
  return step_noise<LAT, R, kStepNoiseFlat>(src, dst, a, stream);
}


}  // namespace lbfd
