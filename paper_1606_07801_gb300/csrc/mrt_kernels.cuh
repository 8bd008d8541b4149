// Multiple-relaxation-time collision and lattices with run-time tables.
//
// The paper relaxes each moment with its own time (Sec. III: the isotropic
// collision matrix is diag(tau^rho, tau^j, tau^j, tau^n, tau^s) in moment
// space for D2Q5) and gives each non-conserved moment the noise variance
// rho (2 tau^a - 1) / (tau^a)^2 (eqs. xiglobal, xilocal).  Per site:
//   M^a   = sum_i m_i^a f_i                      (a >= 1; M^0 = rho)
//   M^a*  = (1 - 1/tau^a) M^a + sqrt(rho_n) amp_a z^a,  amp_a^2 = (2 tau^a - 1)/(tau^a)^2
//   f*_i  = w_i (rho + sum_{a>=1} m_i^a M^a*)     (i >= 1; n_i^a = m_i^a w_i)
//   f*_0  = rho - sum_{i>=1} f*_i                  (mass conservation)
// The basis and weights are compiled in for D1Q3, D2Q9 and D3Q19 (CT = true,
// zero entries skipped) and come from the kernel arguments for D2Q5, whose
// weights w_0 = 1 - 2 theta, w_1..4 = theta/2 depend on theta (Sec. II).
// The pull, the noise keys and the store are those of the single-relaxation
// kernels (the same site-update bodies with another collision).
#pragma once

#include "step_kernels.cuh"

namespace lbfd {

template <typename R, int Q>
struct MrtParams {
  R m[Q][Q];   // m[a][i] = m_i^a (read only when the basis is not compiled in)
  R w[Q];      // weights (likewise)
  R omega[Q];  // 1 - 1/tau^a for a >= 1
  R amp[Q];    // sqrt((2 tau^a - 1) / (tau^a)^2) for a >= 1
};

template <int LAT, typename R, int NOISE, bool CT>
__device__ __forceinline__ void collide_site_mrt(R (&f)[Lattice<LAT>::Q], uint32_t s, const StepArgs &a,
                                                 const MrtParams<R, Lattice<LAT>::Q> &p) {
  using L = Lattice<LAT>;
  constexpr int Q = L::Q;
  R rho = f[0];
  static_for<Q - 1>([&](auto I) { rho += f[decltype(I)::value + 1]; });
  // forward transform of the non-conserved moments
  R M[Q];
  M[0] = rho;
  static_for<Q - 1>([&](auto A) {
    constexpr int am = decltype(A)::value + 1;
    R acc = R(0);
    static_for<Q>([&](auto I) {
      constexpr int i = decltype(I)::value;
      if constexpr (CT) {
        constexpr double c = kBasis<LAT, am, i>;
        if constexpr (c != 0.0) acc = fma(static_cast<R>(c), f[i], acc);
      } else {
        acc = fma(p.m[am][i], f[i], acc);
      }
    });
    M[am] = acc;
  });
  // relaxation and noise, moment by moment
  if constexpr (NOISE != kStepNoiseOff) {
    const R rho_loc = rho > R(0) ? rho : R(0);
    const R rho_n = a.noise_mode == kNoiseLocal ? rho_loc : step_param<R>(a.rho_eq, a.rho_eq_f);
    const R sr = noise_amplitude<R>(rho_n);
    R zz[Q - 1];
    draw_variates_t<R, Q - 1, NOISE == kStepNoiseGauss>(zz, s, a.ph);
    static_for<Q - 1>([&](auto A) {
      constexpr int am = decltype(A)::value + 1;
      M[am] = fma(p.omega[am], M[am], (sr * p.amp[am]) * zz[am - 1]);
    });
  } else {
    static_for<Q - 1>([&](auto A) {
      constexpr int am = decltype(A)::value + 1;
      M[am] = p.omega[am] * M[am];
    });
  }
  // back transform; the rest population from mass conservation
  R moved = R(0);
  static_for<Q - 1>([&](auto I) {
    constexpr int i = decltype(I)::value + 1;
    R acc = rho;
    static_for<Q - 1>([&](auto A) {
      constexpr int am = decltype(A)::value + 1;
      if constexpr (CT) {
        constexpr double c = kBasis<LAT, am, i>;
        if constexpr (c != 0.0) acc = fma(static_cast<R>(c), M[am], acc);
      } else {
        acc = fma(p.m[am][i], M[am], acc);
      }
    });
    R wi;
    if constexpr (CT)
      wi = static_cast<R>(L::w(i));
    else
      wi = p.w[i];
    f[i] = wi * acc;
    moved += f[i];
  });
  f[0] = rho - moved;
}

template <int LAT, typename R, int NOISE, bool CT>
struct MrtCollide {
  const MrtParams<R, Lattice<LAT>::Q> &p;
  __device__ __forceinline__ void operator()(R (&f)[Lattice<LAT>::Q], uint32_t s, const StepArgs &a) const {
    collide_site_mrt<LAT, R, NOISE, CT>(f, s, a, p);
  }
};

template <int LAT, typename S, int VX, int NOISE, bool CT>
__global__ void __launch_bounds__(256)
    k_step_mrt(const S *__restrict__ src, S *__restrict__ dst, const StepArgs a,
               const MrtParams<typename Store<S>::R, Lattice<LAT>::Q> p) {
  using R = typename Store<S>::R;
  const int x0 = (blockIdx.x * blockDim.x + threadIdx.x) * VX;
  const int y = blockIdx.y * blockDim.y + threadIdx.y;
  const int z = blockIdx.z;
  if (x0 >= a.Lx || y >= a.Ly) return;
  // value offsets fit 32 bits (checked by the API)
  const MrtCollide<LAT, R, NOISE, CT> c{p};
  if constexpr (VX == 1)
    step_scalar_body<LAT, S, NOISE, MrtCollide<LAT, R, NOISE, CT>, uint32_t>(src, dst, a, x0, y, z, c);
  else
    step_vec_body<LAT, S, VX, NOISE, MrtCollide<LAT, R, NOISE, CT>, uint32_t>(src, dst, a, x0, y, z, c);
}

// Launch for one lattice and storage type (FP32 or FP64).  m (Q*Q, [a][i])
// and w (Q) are the run-time basis and weights (used when the basis is not
// compiled in); tau holds tau^a for a = 0..Q-1 (entry 0 unused).
template <int LAT, typename S>
cudaError_t step_mrt_t(const void *src, void *dst, const StepArgs &a, const double *m, const double *w,
                       const double *tau, cudaStream_t stream) {
  using R = typename Store<S>::R;
  constexpr int Q = Lattice<LAT>::Q;
  constexpr bool CT = LAT != kD2Q5;
  MrtParams<R, Q> p{};
  for (int b = 0; b < Q; ++b) {
    for (int i = 0; i < Q; ++i) p.m[b][i] = static_cast<R>(m[b * Q + i]);
    p.w[b] = static_cast<R>(w[b]);
    if (b == 0) continue;
    p.omega[b] = static_cast<R>(1.0 - 1.0 / tau[b]);
    p.amp[b] = static_cast<R>(std::sqrt((2.0 * tau[b] - 1.0) / (tau[b] * tau[b])));
  }
  const int vx = a.Lx % 2 == 0 ? 2 : 1;
  dim3 grid, block;
  step_shape(a.Lx, a.Ly, a.Lz, grid, block, vx);
  const S *s = static_cast<const S *>(src);
  S *d = static_cast<S *>(dst);
  auto go = [&](auto noise) {
    constexpr int NOISE = decltype(noise)::value;
    if (vx == 2)
      k_step_mrt<LAT, S, 2, NOISE, CT><<<grid, block, 0, stream>>>(s, d, a, p);
    else
      k_step_mrt<LAT, S, 1, NOISE, CT><<<grid, block, 0, stream>>>(s, d, a, p);
  };
  if (a.noise_mode == kNoiseOff)
    go(std::integral_constant<int, kStepNoiseOff>{});
  else if (a.noise_dist == kGaussian)
    go(std::integral_constant<int, kStepNoiseGauss>{});
  else
    go(std::integral_constant<int, kStepNoiseFlat>{});
  return cudaGetLastError();
}

}  // namespace lbfd
