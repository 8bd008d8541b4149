// The fused fluctuating lattice-Boltzmann step and its helpers.
//
// One thread updates one site x per step (Wagner & Strand, arXiv:1606.07801):
//   pull    f_i <- f*_i(x - v_i, t)            (eq. LB, periodic, two buffers)
//   density rho = sum_i f_i
//   noise   sigma^2 = rho_n (2 tau - 1)/tau^2,  rho_n = max(rho, 0) (local,
//           eq. xilocal; the clamp of Sec. IV) or rho^eq (global, eq. xiglobal)
//           z^a, a = 1..Q-1, from Philox4x32-10 keyed by (seed, site, t)
//   collide f*_i = (1 - 1/tau) f_i + w_i (rho/tau + sigma sum_{a>=1} m_i^a z^a)
//           which is eq. collision with Lambda = 1/tau (eq. coll) written in
//           f-space: M^{a*} = (1 - 1/tau) M^a + sigma z^a for a >= 1,
//           M^{0*} = rho, back-transformed with n_i^a = m_i^a w_i; the rest
//           population is rho - sum_{i>=1} f*_i (the same in exact arithmetic)
//   store   f*_i(x) into the other buffer
// Everything lives in registers; the populations are read and written once.
#include <cuda_runtime.h>

#include <cstdlib>

#include "device.cuh"
#include "internal.h"
#include "step_kernels.cuh"

namespace lbfd {

cudaError_t launch_step(int lattice, int precision, const void *src, void *dst, const StepArgs &a,
                        cudaStream_t stream, int vec_width) {
  if (vec_width == 0) vec_width = step_vec_width(lattice, precision, a.Lx);
  if (vec_width != 1 && ((vec_width != 2 && vec_width != 4) || a.Lx % vec_width != 0)) return cudaErrorInvalidValue;
  if (vec_width == 4 && precision == kStoreF64) return cudaErrorInvalidValue;
  switch (lattice) {
    case kD1Q3: return launch_step_d1q3(precision, src, dst, a, stream, vec_width);
    case kD2Q9: return launch_step_d2q9(precision, src, dst, a, stream, vec_width);
    case kD3Q19: return launch_step_d3q19(precision, src, dst, a, stream, vec_width);
  }
  return cudaErrorInvalidValue;
}

// ---------------------------------------------------------------------------
// Streaming shifts (pure data movement).  The pull kernel keeps the
// post-collision populations g of the last step, which relate to the
// paper's f(x, t) (eq. LB) by one streaming: f_i(x, t) = g_i(x - v_i).
//   dir = +1: dst_i(x) = src_i(x - v_i)   (g -> f)
//   dir = -1: dst_i(x) = src_i(x + v_i)   (f -> g)
// ---------------------------------------------------------------------------
template <int LAT, typename T>
__global__ void k_shift(const T *__restrict__ src, T *__restrict__ dst, int32_t Lx, int32_t Ly, int32_t Lz, int dir) {
  using L = Lattice<LAT>;
  const int x = blockIdx.x * blockDim.x + threadIdx.x;
  const int y = blockIdx.y * blockDim.y + threadIdx.y;
  const int z = blockIdx.z;
  if (x >= Lx || y >= Ly) return;
  const int xm = (x == 0 ? Lx : x) - 1, xp = (x + 1 == Lx) ? 0 : x + 1;
  const int ym = (y == 0 ? Ly : y) - 1, yp = (y + 1 == Ly) ? 0 : y + 1;
  const int zm = (z == 0 ? Lz : z) - 1, zp = (z + 1 == Lz) ? 0 : z + 1;
  const uint32_t ux = static_cast<uint32_t>(Lx), uxy = ux * static_cast<uint32_t>(Ly);
  const size_t N = static_cast<size_t>(uxy) * static_cast<uint32_t>(Lz);
  const uint32_t s = static_cast<uint32_t>(x) + ux * static_cast<uint32_t>(y) + uxy * static_cast<uint32_t>(z);
  static_for<L::Q>([&](auto I) {
    constexpr int i = decltype(I)::value;
    constexpr int vx = L::v(i, 0), vy = L::v(i, 1), vz = L::v(i, 2);
    // source = x - dir * v_i
    const int xs = vx == 0 ? x : ((vx * dir) > 0 ? xm : xp);
    const int ys = vy == 0 ? y : ((vy * dir) > 0 ? ym : yp);
    const int zs = vz == 0 ? z : ((vz * dir) > 0 ? zm : zp);
    const uint32_t so = static_cast<uint32_t>(xs) + ux * static_cast<uint32_t>(ys) + uxy * static_cast<uint32_t>(zs);
    dst[i * N + s] = src[i * N + so];
  });
}

template <int LAT, typename T>
static cudaError_t shift_t(const void *src, void *dst, int32_t Lx, int32_t Ly, int32_t Lz, int dir, cudaStream_t stream) {
  dim3 grid, block;
  step_shape(Lx, Ly, Lz, grid, block);
  k_shift<LAT, T><<<grid, block, 0, stream>>>(static_cast<const T *>(src), static_cast<T *>(dst), Lx, Ly, Lz, dir);
  return cudaGetLastError();
}

cudaError_t launch_shift(int lattice, int value_bytes, const void *src, void *dst, int32_t Lx, int32_t Ly, int32_t Lz,
                         int dir, cudaStream_t stream) {
  return dispatch_lattice(lattice, [&](auto lat) -> cudaError_t {
    constexpr int LAT = decltype(lat)::value;
    if (value_bytes == 8) return shift_t<LAT, uint64_t>(src, dst, Lx, Ly, Lz, dir, stream);
    if (value_bytes == 4) return shift_t<LAT, uint32_t>(src, dst, Lx, Ly, Lz, dir, stream);
    if (value_bytes == 2) return shift_t<LAT, uint16_t>(src, dst, Lx, Ly, Lz, dir, stream);
    return cudaErrorInvalidValue;
  });
}

// ---------------------------------------------------------------------------
// Initial state f_i = w_i rho(x) (local equilibrium, eq. f0def)
// ---------------------------------------------------------------------------
// Weights passed by value (run-time for D2Q5, whose weights depend on theta).
struct WeightArg {
  double w[LBFD_MAX_Q_DEV];
};

// Where a stored lattice sits in the lattice whose sine mode is set up: the
// stored coordinate c of axis a is c + off[a] (mod len[a]) there (a slab
// with a halo plane sits at its first plane minus one).
struct PhaseFrame {
  int32_t off[3], len[3];
};

template <int LAT, typename S>
__global__ void k_init(S *__restrict__ f, int32_t Lx, int32_t Ly, int32_t Lz, double rho_mean, double amp, int32_t kx,
                       int32_t ky, int32_t kz, const WeightArg wt, const PhaseFrame fr) {
  using L = Lattice<LAT>;
  const int64_t N = static_cast<int64_t>(Lx) * Ly * Lz;
  for (int64_t s = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; s < N;
       s += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    const int64_t x = s % Lx, y = (s / Lx) % Ly, z = s / (static_cast<int64_t>(Lx) * Ly);
    double rho = rho_mean;
    if (amp != 0.0) {
      // phase / (2 pi) reduced exactly with integers before the sine
      const int64_t Px = fr.len[0], Py = fr.len[1], Pz = fr.len[2];
      const int64_t gx = ((x + fr.off[0]) % Px + Px) % Px, gy = ((y + fr.off[1]) % Py + Py) % Py;
      const int64_t gz = ((z + fr.off[2]) % Pz + Pz) % Pz;
      const int64_t px = ((static_cast<int64_t>(kx) * gx) % Px + Px) % Px;
      const int64_t py = ((static_cast<int64_t>(ky) * gy) % Py + Py) % Py;
      const int64_t pz = ((static_cast<int64_t>(kz) * gz) % Pz + Pz) % Pz;
      const double frac = double(px) / Px + double(py) / Py + double(pz) / Pz;
      rho += amp * sinpi(2.0 * frac);
    }
    static_for<L::Q>([&](auto I) {
      constexpr int i = decltype(I)::value;
      f[i * N + s] = Store<S>::putd(wt.w[i] * rho, wt.w[i] * rho_mean);
    });
  }
}

cudaError_t launch_init(int lattice, int precision, void *f, int32_t Lx, int32_t Ly, int32_t Lz, double rho_mean,
                        double amp, const int32_t *k, cudaStream_t stream, const double *w, const int32_t *phase_off,
                        const int32_t *phase_len) {
  return dispatch_lattice_storage(lattice, precision, [&](auto lat, auto tag) {
    constexpr int LAT = decltype(lat)::value;
    using S = typename decltype(tag)::type;
    WeightArg wt{};
    for (int i = 0; i < Lattice<LAT>::Q; ++i) wt.w[i] = w ? w[i] : Lattice<LAT>::w(i);
    PhaseFrame fr{{0, 0, 0}, {Lx, Ly, Lz}};
    for (int a = 0; a < 3; ++a) {
      if (phase_off) fr.off[a] = phase_off[a];
      if (phase_len) fr.len[a] = phase_len[a];
    }
    const int64_t N = static_cast<int64_t>(Lx) * Ly * Lz;
    const int64_t blocks = (N + 255) / 256;
    const int grid = static_cast<int>(blocks < 152 * 64 ? blocks : 152 * 64);
    k_init<LAT, S><<<grid, 256, 0, stream>>>(static_cast<S *>(f), Lx, Ly, Lz, rho_mean, amp, k[0], k[1], k[2], wt,
                                             fr);
    return cudaGetLastError();
  });
}

// ---------------------------------------------------------------------------
// Density and flux (FP64 outputs)
// ---------------------------------------------------------------------------
template <int LAT, typename S>
__global__ void k_moments(const S *__restrict__ f, int64_t N, double rho_mean, double *__restrict__ rho,
                          double *__restrict__ j) {
  using L = Lattice<LAT>;
  for (int64_t s = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; s < N;
       s += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    double r = 0.0, jx = 0.0, jy = 0.0, jz = 0.0;
    static_for<L::Q>([&](auto I) {
      constexpr int i = decltype(I)::value;
      const double fi = Store<S>::getd(f[i * N + s], L::w(i) * rho_mean);
      r += fi;
      if constexpr (L::v(i, 0) != 0) jx += L::v(i, 0) * fi;
      if constexpr (L::v(i, 1) != 0) jy += L::v(i, 1) * fi;
      if constexpr (L::v(i, 2) != 0) jz += L::v(i, 2) * fi;
    });
    rho[s] = r;
    if (j) {
      j[s] = jx;
      if (L::D > 1) j[N + s] = jy;
      if (L::D > 2) j[2 * N + s] = jz;
    }
  }
}

cudaError_t launch_moments(int lattice, int precision, const void *f, int32_t Lx, int32_t Ly, int32_t Lz,
                           double rho_mean, double *rho, double *j, cudaStream_t stream) {
  return dispatch_lattice_storage(lattice, precision, [&](auto lat, auto tag) {
    constexpr int LAT = decltype(lat)::value;
    using S = typename decltype(tag)::type;
    const int64_t N = static_cast<int64_t>(Lx) * Ly * Lz;
    const int64_t blocks = (N + 255) / 256;
    const int grid = static_cast<int>(blocks < 152 * 32 ? blocks : 152 * 32);
    k_moments<LAT, S><<<grid, 256, 0, stream>>>(static_cast<const S *>(f), N, rho_mean, rho, j);
    return cudaGetLastError();
  });
}

// rho(x) = sum_i g_i(x - v_i): the density of the paper's f(x, t) computed
// from the stored post-collision state g, summed in FP64 in velocity order
// (the same values and order as a streaming shift followed by k_moments).
template <int LAT, typename S>
__global__ void k_density_of_state(const S *__restrict__ g, int32_t Lx, int32_t Ly, int32_t Lz, double rho_mean,
                                   double *__restrict__ rho) {
  using L = Lattice<LAT>;
  const int64_t N = static_cast<int64_t>(Lx) * Ly * Lz;
  for (int64_t s = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; s < N;
       s += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    const int x = static_cast<int>(s % Lx);
    const int64_t r = s / Lx;
    const int y = static_cast<int>(r % Ly), z = static_cast<int>(r / Ly);
    const int xm = (x == 0 ? Lx : x) - 1, xp = (x + 1 == Lx) ? 0 : x + 1;
    const int ym = (y == 0 ? Ly : y) - 1, yp = (y + 1 == Ly) ? 0 : y + 1;
    const int zm = (z == 0 ? Lz : z) - 1, zp = (z + 1 == Lz) ? 0 : z + 1;
    double acc = 0.0;
    static_for<L::Q>([&](auto I) {
      constexpr int i = decltype(I)::value;
      constexpr int vx = L::v(i, 0), vy = L::v(i, 1), vz = L::v(i, 2);
      const int xs = vx == 0 ? x : (vx > 0 ? xm : xp);
      const int ys = vy == 0 ? y : (vy > 0 ? ym : yp);
      const int zs = vz == 0 ? z : (vz > 0 ? zm : zp);
      const int64_t so = xs + static_cast<int64_t>(Lx) * (ys + static_cast<int64_t>(Ly) * zs);
      acc += Store<S>::getd(g[i * N + so], L::w(i) * rho_mean);
    });
    rho[s] = acc;
  }
}

cudaError_t launch_density_of_state(int lattice, int precision, const void *g, int32_t Lx, int32_t Ly,
                                           int32_t Lz, double rho_mean, double *rho, cudaStream_t stream) {
  return dispatch_lattice_storage(lattice, precision, [&](auto lat, auto tag) {
    constexpr int LAT = decltype(lat)::value;
    using S = typename decltype(tag)::type;
    const int64_t N = static_cast<int64_t>(Lx) * Ly * Lz;
    const int64_t blocks = (N + 255) / 256;
    const int grid = static_cast<int>(blocks < 152 * 16 ? blocks : 152 * 16);
    k_density_of_state<LAT, S><<<grid, 256, 0, stream>>>(static_cast<const S *>(g), Lx, Ly, Lz, rho_mean, rho);
    return cudaGetLastError();
  });
}

// ---------------------------------------------------------------------------
// Noise probe: the variates the step kernel draws, for checks of the RNG
// ---------------------------------------------------------------------------
template <typename R, int NMOM>
__global__ void k_noise_draw(int dist, const PhiloxStep ph, int64_t site0, int64_t nsites, double *__restrict__ out) {
  for (int64_t k = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; k < nsites;
       k += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    R z[NMOM];
    draw_variates<R, NMOM>(z, static_cast<uint32_t>(site0 + k), ph, dist);
#pragma unroll
    for (int a = 0; a < NMOM; ++a) out[k * NMOM + a] = static_cast<double>(z[a]);
  }
}

template <typename R, int NMOM>
static cudaError_t noise_t(int dist, const PhiloxStep &ph, int64_t site0, int64_t nsites, double *z,
                           cudaStream_t stream) {
  const int64_t blocks = (nsites + 255) / 256;
  const int grid = static_cast<int>(blocks < 4096 ? (blocks > 0 ? blocks : 1) : 4096);
  k_noise_draw<R, NMOM><<<grid, 256, 0, stream>>>(dist, ph, site0, nsites, z);
  return cudaGetLastError();
}

template <typename R>
static cudaError_t noise_p(int dist, const PhiloxStep &ph, int64_t site0, int64_t nsites, int nmom, double *z,
                           cudaStream_t stream) {
  switch (nmom) {
    case 2: return noise_t<R, 2>(dist, ph, site0, nsites, z, stream);
    case 4: return noise_t<R, 4>(dist, ph, site0, nsites, z, stream);
    case 8: return noise_t<R, 8>(dist, ph, site0, nsites, z, stream);
    case 18: return noise_t<R, 18>(dist, ph, site0, nsites, z, stream);
  }
  return cudaErrorInvalidValue;
}

cudaError_t launch_noise_draw(int precision, int dist, const PhiloxStep &ph, int64_t site0, int64_t nsites, int nmom,
                              double *z, cudaStream_t stream) {
  return precision == 1 ? noise_p<double>(dist, ph, site0, nsites, nmom, z, stream)
                        : noise_p<float>(dist, ph, site0, nsites, nmom, z, stream);
}

// Box-Muller on given word pairs (edge cases of the uniform grid)
template <typename R>
__global__ void k_box_muller_probe(const uint32_t *__restrict__ words, int64_t npairs, double *__restrict__ z) {
  for (int64_t k = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; k < npairs;
       k += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    R z0, z1;
    BoxMuller<R>::pair(words[2 * k], words[2 * k + 1], z0, z1);
    z[2 * k] = static_cast<double>(z0);
    z[2 * k + 1] = static_cast<double>(z1);
  }
}

// The lane operations of the collision (add_rn, sub_rn, mul_rn, fma_rn) on
// float and on float2: a thread takes values 2p and 2p + 1, computes each
// operation twice per value, one value at a time and both in one packed
// instruction, and stores both forms.
__global__ void k_lane_ops_probe(const float *__restrict__ a, const float *__restrict__ b, const float *__restrict__ c,
                                 int64_t n, float *__restrict__ out) {
  const int64_t npairs = n / 2;
  for (int64_t p = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; p < npairs;
       p += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    const int64_t k = 2 * p;
    const float2 A = make_float2(a[k], a[k + 1]), B = make_float2(b[k], b[k + 1]), C = make_float2(c[k], c[k + 1]);
    float s[6][2];
    float2 v[6];
#pragma unroll
    for (int l = 0; l < 2; ++l) {
      const float x = l ? A.y : A.x, y = l ? B.y : B.x, z = l ? C.y : C.x;
      s[0][l] = add_rn(x, y);
      s[1][l] = sub_rn(x, y);
      s[2][l] = mul_rn(x, y);
      s[3][l] = fma_rn(x, y, z);
      s[4][l] = add_rn(mul_rn(x, y), z);
      s[5][l] = sub_rn(z, mul_rn(x, y));
    }
    v[0] = add_rn(A, B);
    v[1] = sub_rn(A, B);
    v[2] = mul_rn(A, B);
    v[3] = fma_rn(A, B, C);
    v[4] = add_rn(mul_rn(A, B), C);
    v[5] = sub_rn(C, mul_rn(A, B));
#pragma unroll
    for (int op = 0; op < 6; ++op) {
      out[(2 * op) * n + k] = s[op][0];
      out[(2 * op) * n + k + 1] = s[op][1];
      out[(2 * op + 1) * n + k] = v[op].x;
      out[(2 * op + 1) * n + k + 1] = v[op].y;
    }
  }
}

cudaError_t launch_lane_ops_probe(const float *a, const float *b, const float *c, int64_t n, float *out,
                                  cudaStream_t stream) {
  const int64_t blocks = (n / 2 + 255) / 256;
  const int grid = static_cast<int>(blocks < 4096 ? (blocks > 0 ? blocks : 1) : 4096);
  k_lane_ops_probe<<<grid, 256, 0, stream>>>(a, b, c, n, out);
  return cudaGetLastError();
}

cudaError_t launch_box_muller_probe(int precision, const uint32_t *words, int64_t npairs, double *z,
                                    cudaStream_t stream) {
  const int64_t blocks = (npairs + 255) / 256;
  const int grid = static_cast<int>(blocks < 4096 ? (blocks > 0 ? blocks : 1) : 4096);
  if (precision == 1)
    k_box_muller_probe<double><<<grid, 256, 0, stream>>>(words, npairs, z);
  else
    k_box_muller_probe<float><<<grid, 256, 0, stream>>>(words, npairs, z);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Host copies of the tables the kernels are compiled with
// ---------------------------------------------------------------------------
template <int LAT>
static void tables_t(int *Q, int *D, int *v, double *w, double *m) {
  using L = Lattice<LAT>;
  if (Q) *Q = L::Q;
  if (D) *D = L::D;
  for (int i = 0; i < L::Q; ++i) {
    if (v)
      for (int a = 0; a < 3; ++a) v[3 * i + a] = L::v(i, a);
    if (w) w[i] = L::w(i);
  }
  if (m) {
    constexpr BasisTable<L::Q> B = make_basis<LAT>();
    for (int a = 0; a < L::Q; ++a)
      for (int i = 0; i < L::Q; ++i) m[a * L::Q + i] = B.m[a][i];
  }
}

int lattice_table(int lattice, int *Q, int *D, int *v, double *w) {
  switch (lattice) {
    case kD1Q3: tables_t<kD1Q3>(Q, D, v, w, nullptr); return 0;
    case kD2Q9: tables_t<kD2Q9>(Q, D, v, w, nullptr); return 0;
    case kD3Q19: tables_t<kD3Q19>(Q, D, v, w, nullptr); return 0;
    case kD2Q5: {
      // theta = 1/3; lattice_table_theta gives other theta
      using L = Lattice<kD2Q5>;
      if (Q) *Q = 5;
      if (D) *D = 2;
      for (int i = 0; i < 5; ++i) {
        if (v)
          for (int a = 0; a < 3; ++a) v[3 * i + a] = L::v(i, a);
        if (w) w[i] = L::w(i);
      }
      return 0;
    }
  }
  return -1;
}

int basis_table(int lattice, double *m) {
  switch (lattice) {
    case kD1Q3: {
      // the factorised kernel path uses mu^p(v) directly
      const int vs[3] = {0, 1, -1};
      for (int a = 0; a < 3; ++a)
        for (int i = 0; i < 3; ++i) m[a * 3 + i] = d1q3_mu(a, vs[i]);
      return 0;
    }
    case kD2Q9: {
      using L = Lattice<kD2Q9>;
      for (int p = 0; p < 3; ++p)
        for (int q = 0; q < 3; ++q)
          for (int i = 0; i < 9; ++i) m[(3 * p + q) * 9 + i] = d1q3_mu(p, L::v(i, 0)) * d1q3_mu(q, L::v(i, 1));
      return 0;
    }
    case kD3Q19: tables_t<kD3Q19>(nullptr, nullptr, nullptr, nullptr, m); return 0;
    case kD2Q5: {
      double w[5];
      d2q5_tables(1.0 / 3.0, w, m);
      return 0;
    }
  }
  return -1;
}

}  // namespace lbfd
