// Device-side building blocks of the fluctuating lattice-Boltzmann step:
// lattice traits, the moment basis as compile-time constants, Philox4x32-10,
// the noise variates and the noise back-transform.
//
// Method: Wagner & Strand, arXiv:1606.07801.
//   - f^0_i = rho w_i, sum_i w_i v_i v_i = theta (Sec. II, eqs. f0_0-f0_2, f0def)
//   - moments M^a = sum_i m_i^a f_i with n_i^a = m_i^a w_i and
//     sum_i m_i^a w_i m_i^b = delta^{ab} (Sec. II, Gram-Schmidt passage)
//   - noise xi^a, a >= 1, variance rho (2 tau - 1)/tau^2 (eqs. xiglobal, xilocal)
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <stdint.h>

#include <type_traits>
#include <utility>

namespace lbfd {

enum LatticeId : int { kD1Q3 = 0, kD2Q9 = 1, kD3Q19 = 2, kD2Q5 = 3 };
enum NoiseMode : int { kNoiseLocal = 0, kNoiseGlobal = 1, kNoiseOff = 2 };
enum NoiseDist : int { kGaussian = 0, kUniform = 1 };

// ---------------------------------------------------------------------------
// Storage formats of the populations.  FP32 and FP64 store f_i itself.  The
// 16-bit formats store the deviation d_i = f_i - w_i rho_mean (rounded to
// nearest even), and all arithmetic on them is FP32.  load() / store()
// convert the stored value alone (the step kernels collide on the
// deviations themselves); get() / put() (and the FP64 getd() / putd())
// decode to and encode from f_i with wr = w_i rho_mean.
// ---------------------------------------------------------------------------
enum StorageId : int { kStoreF32 = 0, kStoreF64 = 1, kStoreF16 = 2, kStoreBF16 = 3 };

// Rounded adds, subtracts and multiplies that the device compiler may not
// fuse into an FMA with a neighbouring operation: the offset w_i rho_mean and
// its add to a decoded deviation then round the same way in every kernel, so
// a lattice evolves bit-identically whichever kernel steps it.  (The library's
// host code is compiled with FMA contraction off.)
__host__ __device__ __forceinline__ float add_rn(float a, float b) {
#ifdef __CUDA_ARCH__
  return __fadd_rn(a, b);
#else
  return a + b;  // host code is compiled without FMA contraction
#endif
}
__host__ __device__ __forceinline__ float sub_rn(float a, float b) {
#ifdef __CUDA_ARCH__
  return __fsub_rn(a, b);
#else
  return a - b;  // host code is compiled without FMA contraction
#endif
}
__host__ __device__ __forceinline__ float mul_rn(float a, float b) {
#ifdef __CUDA_ARCH__
  return __fmul_rn(a, b);
#else
  return a * b;  // host code is compiled without FMA contraction
#endif
}
__host__ __device__ __forceinline__ double add_rn(double a, double b) {
#ifdef __CUDA_ARCH__
  return __dadd_rn(a, b);
#else
  return a + b;  // host code is compiled without FMA contraction
#endif
}
__host__ __device__ __forceinline__ double sub_rn(double a, double b) {
#ifdef __CUDA_ARCH__
  return __dsub_rn(a, b);
#else
  return a - b;  // host code is compiled without FMA contraction
#endif
}
__host__ __device__ __forceinline__ double mul_rn(double a, double b) {
#ifdef __CUDA_ARCH__
  return __dmul_rn(a, b);
#else
  return a * b;  // host code is compiled without FMA contraction
#endif
}
__host__ __device__ __forceinline__ float fma_rn(float a, float b, float c) {
#ifdef __CUDA_ARCH__
  return __fmaf_rn(a, b, c);
#else
  return fmaf(a, b, c);
#endif
}
__host__ __device__ __forceinline__ double fma_rn(double a, double b, double c) {
#ifdef __CUDA_ARCH__
  return __fma_rn(a, b, c);
#else
  return fma(a, b, c);
#endif
}

// ---------------------------------------------------------------------------
// Two sites at once.  From sm_100 on, an FP32 add, multiply or fused
// multiply-add can act on a pair of registers (add/sub/mul/fma.rn.f32x2), each
// lane rounded exactly as the scalar instruction rounds it.  The collision
// is written once over a value type V -- float or double for one site, float2
// for the same quantity of two neighbouring sites -- with every operation an
// explicit add_rn / sub_rn / mul_rn / fma_rn, so that nothing is fused
// differently in the two forms and a site's update is the same bit pattern
// whether a thread computes it alone or paired with the next site.
// Conversions, comparisons and the special-function unit act lane by lane.
// ---------------------------------------------------------------------------
template <typename V>
struct LaneOf {
  using type = V;
  static constexpr int kLanes = 1;
};
template <>
struct LaneOf<float2> {
  using type = float;
  static constexpr int kLanes = 2;
};
template <typename V>
__host__ __device__ __forceinline__ V splat(typename LaneOf<V>::type s) {
  if constexpr (LaneOf<V>::kLanes == 2)
    return make_float2(s, s);
  else
    return s;
}
// A compile-time constant rounded once to the lane type.
template <typename V>
__host__ __device__ __forceinline__ V cst(double c) {
  return splat<V>(static_cast<typename LaneOf<V>::type>(c));
}
// On the device these are the PTX instructions add/sub/mul/fma.rn.f32x2 in
// inline assembly: an explicit rounding modifier keeps the assembler from
// fusing a multiply into a following add, and the compiler cannot see into
// the assembly to fuse them earlier, so a packed product added to something
// rounds twice, as __fmul_rn and __fadd_rn do.  (Before sm_100, and on the
// host, two scalar operations.)
#if defined(__CUDA_ARCH__) && __CUDA_ARCH__ >= 1000
#define LBFD_F32X2 1
__device__ __forceinline__ uint64_t f32x2_bits(float2 a) {
  uint64_t u;
  asm("mov.b64 %0, {%1, %2};" : "=l"(u) : "f"(a.x), "f"(a.y));
  return u;
}
__device__ __forceinline__ float2 f32x2_value(uint64_t u) {
  float2 a;
  asm("mov.b64 {%0, %1}, %2;" : "=f"(a.x), "=f"(a.y) : "l"(u));
  return a;
}
#endif
__host__ __device__ __forceinline__ float2 add_rn(float2 a, float2 b) {
#ifdef LBFD_F32X2
  uint64_t r;
  asm("add.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(f32x2_bits(a)), "l"(f32x2_bits(b)));
  return f32x2_value(r);
#else
  return make_float2(add_rn(a.x, b.x), add_rn(a.y, b.y));
#endif
}
__host__ __device__ __forceinline__ float2 sub_rn(float2 a, float2 b) {
#ifdef LBFD_F32X2
  uint64_t r;
  asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(f32x2_bits(a)), "l"(f32x2_bits(b)));
  return f32x2_value(r);
#else
  return make_float2(sub_rn(a.x, b.x), sub_rn(a.y, b.y));
#endif
}
__host__ __device__ __forceinline__ float2 mul_rn(float2 a, float2 b) {
#ifdef LBFD_F32X2
  uint64_t r;
  asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(f32x2_bits(a)), "l"(f32x2_bits(b)));
  return f32x2_value(r);
#else
  return make_float2(mul_rn(a.x, b.x), mul_rn(a.y, b.y));
#endif
}
__host__ __device__ __forceinline__ float2 fma_rn(float2 a, float2 b, float2 c) {
#ifdef LBFD_F32X2
  uint64_t r;
  asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(r) : "l"(f32x2_bits(a)), "l"(f32x2_bits(b)), "l"(f32x2_bits(c)));
  return f32x2_value(r);
#else
  return make_float2(fma_rn(a.x, b.x, c.x), fma_rn(a.y, b.y, c.y));
#endif
}
// x where x > 0, else +0 (also for NaN), lane by lane.
template <typename V>
__host__ __device__ __forceinline__ V positive_part(V x) {
  if constexpr (LaneOf<V>::kLanes == 2)
    return make_float2(x.x > 0.0f ? x.x : 0.0f, x.y > 0.0f ? x.y : 0.0f);
  else
    return x > V(0) ? x : V(0);
}
// v < t ? a : b, lane by lane.
template <typename V>
__host__ __device__ __forceinline__ V select_below(V v, typename LaneOf<V>::type t, V a, V b) {
  if constexpr (LaneOf<V>::kLanes == 2)
    return make_float2(v.x < t ? a.x : b.x, v.y < t ? a.y : b.y);
  else
    return v < t ? a : b;
}

template <typename S>
struct Store;
template <>
struct Store<float> {
  using R = float;
  static constexpr bool kDeviation = false;
  __host__ __device__ static __forceinline__ float load(float v) { return v; }
  __host__ __device__ static __forceinline__ float store(float f) { return f; }
  __host__ __device__ static __forceinline__ float get(float v, float) { return v; }
  __host__ __device__ static __forceinline__ float put(float f, float) { return f; }
  __host__ __device__ static __forceinline__ double getd(float v, double) { return v; }
  __host__ __device__ static __forceinline__ float putd(double f, double) { return static_cast<float>(f); }
};
template <>
struct Store<double> {
  using R = double;
  static constexpr bool kDeviation = false;
  __host__ __device__ static __forceinline__ double load(double v) { return v; }
  __host__ __device__ static __forceinline__ double store(double f) { return f; }
  __host__ __device__ static __forceinline__ double get(double v, double) { return v; }
  __host__ __device__ static __forceinline__ double put(double f, double) { return f; }
  __host__ __device__ static __forceinline__ double getd(double v, double) { return v; }
  __host__ __device__ static __forceinline__ double putd(double f, double) { return f; }
};
template <>
struct Store<__half> {
  using R = float;
  static constexpr bool kDeviation = true;
  __host__ __device__ static __forceinline__ float load(__half v) { return __half2float(v); }
  __host__ __device__ static __forceinline__ __half store(float d) { return __float2half_rn(d); }
  __host__ __device__ static __forceinline__ float get(__half v, float wr) { return add_rn(__half2float(v), wr); }
  __host__ __device__ static __forceinline__ __half put(float f, float wr) { return __float2half_rn(sub_rn(f, wr)); }
  __host__ __device__ static __forceinline__ double getd(__half v, double wr) {
    return add_rn(static_cast<double>(__half2float(v)), wr);
  }
  __host__ __device__ static __forceinline__ __half putd(double f, double wr) {
    return __float2half_rn(static_cast<float>(sub_rn(f, wr)));
  }
};
template <>
struct Store<__nv_bfloat16> {
  using R = float;
  static constexpr bool kDeviation = true;
  __host__ __device__ static __forceinline__ float load(__nv_bfloat16 v) { return __bfloat162float(v); }
  __host__ __device__ static __forceinline__ __nv_bfloat16 store(float d) { return __float2bfloat16_rn(d); }
  __host__ __device__ static __forceinline__ float get(__nv_bfloat16 v, float wr) {
    return add_rn(__bfloat162float(v), wr);
  }
  __host__ __device__ static __forceinline__ __nv_bfloat16 put(float f, float wr) {
    return __float2bfloat16_rn(sub_rn(f, wr));
  }
  __host__ __device__ static __forceinline__ double getd(__nv_bfloat16 v, double wr) {
    return add_rn(static_cast<double>(__bfloat162float(v)), wr);
  }
  __host__ __device__ static __forceinline__ __nv_bfloat16 putd(double f, double wr) {
    return __float2bfloat16_rn(static_cast<float>(sub_rn(f, wr)));
  }
};

template <typename T>
struct Tag {
  using type = T;
};

// ---------------------------------------------------------------------------
// Compile-time iteration
// ---------------------------------------------------------------------------
template <int... Is, class F>
__host__ __device__ __forceinline__ constexpr void static_for_impl(std::integer_sequence<int, Is...>, F &&f) {
  (f(std::integral_constant<int, Is>{}), ...);
}
template <int N, class F>
__host__ __device__ __forceinline__ constexpr void static_for(F &&f) {
  static_for_impl(std::make_integer_sequence<int, N>{}, f);
}

// ---------------------------------------------------------------------------
// Lattices.  Velocity order is the storage order of the populations.
// ---------------------------------------------------------------------------
template <int LAT>
struct Lattice;

template <>
struct Lattice<kD1Q3> {
  static constexpr int D = 1, Q = 3;
  __host__ __device__ static constexpr int v(int i, int a) {
    constexpr int t[3] = {0, 1, -1};
    return a == 0 ? t[i] : 0;
  }
  __host__ __device__ static constexpr double w(int i) { return i == 0 ? 2.0 / 3.0 : 1.0 / 6.0; }
  // seed monomial exponents (p, q, r) of v_x^p v_y^q v_z^r, Gram-Schmidt order
  __host__ __device__ static constexpr int mono(int a, int k) { return k == 0 ? a : 0; }
};

template <>
struct Lattice<kD2Q9> {
  static constexpr int D = 2, Q = 9;
  __host__ __device__ static constexpr int v(int i, int a) {
    constexpr int t[9][2] = {{0, 0}, {1, 0}, {0, 1}, {-1, 0}, {0, -1}, {1, 1}, {-1, 1}, {-1, -1}, {1, -1}};
    return a < 2 ? t[i][a] : 0;
  }
  __host__ __device__ static constexpr double w(int i) {
    return i == 0 ? 4.0 / 9.0 : (i <= 4 ? 1.0 / 9.0 : 1.0 / 36.0);
  }
  // v_x^p v_y^q, p-major: a = 3p + q
  __host__ __device__ static constexpr int mono(int a, int k) { return k == 0 ? a / 3 : (k == 1 ? a % 3 : 0); }
};

template <>
struct Lattice<kD3Q19> {
  static constexpr int D = 3, Q = 19;
  __host__ __device__ static constexpr int v(int i, int a) {
    constexpr int t[19][3] = {{0, 0, 0},  {1, 0, 0},  {-1, 0, 0}, {0, 1, 0},   {0, -1, 0}, {0, 0, 1},  {0, 0, -1},
                              {1, 1, 0},  {-1, -1, 0}, {1, -1, 0}, {-1, 1, 0},  {1, 0, 1},  {-1, 0, -1}, {1, 0, -1},
                              {-1, 0, 1}, {0, 1, 1},  {0, -1, -1}, {0, 1, -1}, {0, -1, 1}};
    return t[i][a];
  }
  __host__ __device__ static constexpr double w(int i) {
    return i == 0 ? 1.0 / 3.0 : (i <= 6 ? 1.0 / 18.0 : 1.0 / 36.0);
  }
  // v_x^p v_y^q v_z^r with p, q, r <= 2 and at most two of them non-zero,
  // by total degree, then (p, q, r) descending
  __host__ __device__ static constexpr int mono(int a, int k) {
    constexpr int t[19][3] = {{0, 0, 0}, {1, 0, 0}, {0, 1, 0}, {0, 0, 1}, {2, 0, 0}, {1, 1, 0}, {1, 0, 1},
                              {0, 2, 0}, {0, 1, 1}, {0, 0, 2}, {2, 1, 0}, {2, 0, 1}, {1, 2, 0}, {1, 0, 2},
                              {0, 2, 1}, {0, 1, 2}, {2, 2, 0}, {2, 0, 2}, {0, 2, 2}};
    return t[a][k];
  }
};

// The paper's own lattice (Sec. II), in its velocity order.  Its weights
// w_0 = 1 - 2 theta, w_1..4 = theta / 2 depend on theta, a parameter of the
// simulation, so its step and init kernels take the weights and the moment
// basis at run time.  w() below is the theta = 1/3 case; it only offsets the
// 16-bit storage formats, which D2Q5 does not offer.
template <>
struct Lattice<kD2Q5> {
  static constexpr int D = 2, Q = 5;
  __host__ __device__ static constexpr int v(int i, int a) {
    constexpr int t[5][2] = {{0, 0}, {1, 0}, {-1, 0}, {0, 1}, {0, -1}};
    return a < 2 ? t[i][a] : 0;
  }
  __host__ __device__ static constexpr double w(int i) { return i == 0 ? 1.0 / 3.0 : 1.0 / 6.0; }
};

// The first moving velocity j >= 1 with the weight of velocity i.
template <int LAT>
__host__ __device__ constexpr int first_of_weight(int i) {
  for (int j = 1; j < i; ++j)
    if (Lattice<LAT>::w(j) == Lattice<LAT>::w(i)) return j;
  return i;
}

// ---------------------------------------------------------------------------
// Moment basis by weighted Gram-Schmidt, evaluated by the compiler.
// ---------------------------------------------------------------------------
__host__ __device__ constexpr double ce_sqrt(double x) {
  // Newton's iteration from above; stops when the iterate no longer falls.
  if (!(x > 0.0)) return 0.0;
  double r = x > 1.0 ? x : 1.0;
  for (int k = 0; k < 2000; ++k) {
    double n = 0.5 * (r + x / r);
    if (!(n < r)) break;
    r = n;
  }
  return r;
}

__host__ __device__ constexpr double ce_pow(int x, int p) {
  double r = 1.0;
  for (int k = 0; k < p; ++k) r *= static_cast<double>(x);
  return r;
}

template <int Q>
struct BasisTable {
  double m[Q][Q];  // m[a][i] = m_i^a
};

template <int LAT>
__host__ __device__ constexpr BasisTable<Lattice<LAT>::Q> make_basis() {
  using L = Lattice<LAT>;
  constexpr int Q = L::Q;
  BasisTable<Q> B{};
  for (int a = 0; a < Q; ++a) {
    double u[Q] = {};
    for (int i = 0; i < Q; ++i)
      u[i] = ce_pow(L::v(i, 0), L::mono(a, 0)) * ce_pow(L::v(i, 1), L::mono(a, 1)) *
             ce_pow(L::v(i, 2), L::mono(a, 2));
    for (int b = 0; b < a; ++b) {
      double p = 0.0;
      for (int i = 0; i < Q; ++i) p += u[i] * L::w(i) * B.m[b][i];
      for (int i = 0; i < Q; ++i) u[i] -= p * B.m[b][i];
    }
    double n2 = 0.0;
    for (int i = 0; i < Q; ++i) n2 += u[i] * L::w(i) * u[i];
    const double inv = 1.0 / ce_sqrt(n2);
    for (int i = 0; i < Q; ++i) {
      double x = u[i] * inv;
      // entries that vanish by symmetry come out as exact zeros already;
      // rounding dust below 1e-13 is zeroed so the kernel can skip it
      B.m[a][i] = (x < 1e-13 && x > -1e-13) ? 0.0 : x;
    }
  }
  return B;
}

template <int LAT>
inline constexpr BasisTable<Lattice<LAT>::Q> kBasisTable = make_basis<LAT>();
template <int LAT, int A, int I>
inline constexpr double kBasis = kBasisTable<LAT>.m[A][I];

// D1Q3 basis functions mu^p(v) (p = 0, 1, 2): 1, sqrt3 v, (3 v^2 - 1)/sqrt2.
// D2Q9's basis is their product mu^p(v_x) mu^q(v_y), moment a = 3p + q.
inline constexpr double kSqrt2 = 1.41421356237309504880;
inline constexpr double kSqrt3 = 1.73205080756887729353;
inline constexpr double kInvSqrt2 = 0.70710678118654752440;

// ---------------------------------------------------------------------------
// Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11)
// ---------------------------------------------------------------------------
struct Philox {
  static constexpr uint32_t M0 = 0xD2511F53u, M1 = 0xCD9E8D57u;
  static constexpr uint32_t W0 = 0x9E3779B9u, W1 = 0xBB67AE85u;
};

__host__ __device__ __forceinline__ uint32_t mulhi32(uint32_t a, uint32_t b) {
#ifdef __CUDA_ARCH__
  return __umulhi(a, b);
#else
  return static_cast<uint32_t>((static_cast<uint64_t>(a) * b) >> 32);
#endif
}

__host__ __device__ __forceinline__ uint4 philox4x32_10(uint4 c, uint32_t k0, uint32_t k1) {
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    // one 32x32 -> 64-bit multiply gives both halves of each product
    const uint64_t p0 = static_cast<uint64_t>(c.x) * Philox::M0;
    const uint64_t p1 = static_cast<uint64_t>(c.z) * Philox::M1;
    const uint32_t lo0 = static_cast<uint32_t>(p0), hi0 = static_cast<uint32_t>(p0 >> 32);
    const uint32_t lo1 = static_cast<uint32_t>(p1), hi1 = static_cast<uint32_t>(p1 >> 32);
    c = make_uint4(hi1 ^ c.y ^ k0, lo1, hi0 ^ c.w ^ k1, lo0);
    k0 += Philox::W0;
    k1 += Philox::W1;
  }
  return c;
}

// Top 24 bits of a word as a cell-centred uniform on (0, 1): exact in FP64,
// and in FP32 below 1/2.
template <typename R>
__host__ __device__ __forceinline__ R unit24(uint32_t r) {
  return (static_cast<R>(r >> 8) + R(0.5)) * R(5.9604644775390625e-08);
}

template <typename R>
struct Math;
// Device: CUDA's math library.  Host (unit tests of this header only):
// the C library, with sin/cos of pi x.
template <>
struct Math<double> {
  __host__ __device__ static __forceinline__ double log(double x) { return ::log(x); }
  __host__ __device__ static __forceinline__ double sqrt(double x) { return ::sqrt(x); }
  __host__ __device__ static __forceinline__ void sincospi(double x, double *s, double *c) {
#ifdef __CUDA_ARCH__
    ::sincospi(x, s, c);
#else
    *s = ::sin(3.14159265358979323846 * x);
    *c = ::cos(3.14159265358979323846 * x);
#endif
  }
};
template <>
struct Math<float> {
  __host__ __device__ static __forceinline__ float log(float x) { return ::logf(x); }
  __host__ __device__ static __forceinline__ float sqrt(float x) { return ::sqrtf(x); }
  __host__ __device__ static __forceinline__ void sincospi(float x, float *s, float *c) {
#ifdef __CUDA_ARCH__
    ::sincospif(x, s, c);
#else
    *s = ::sinf(3.14159265f * x);
    *c = ::cosf(3.14159265f * x);
#endif
  }
};

// Square root on the special-function unit: the PTX instruction
// sqrt.approx.ftz.f32 (relative error about 2^-23; subnormal inputs count
// as 0).  Used where the argument is a noise variance or -2 ln u >= 2^-24.
__device__ __forceinline__ float sqrt_sfu(float x) {
  float r;
  asm("sqrt.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
  return r;
}

// Noise amplitude sqrt(x), x = rho_n (2 tau - 1)/tau^2 >= 0.  FP32 on the
// device: sqrt_sfu.
template <typename R>
__host__ __device__ __forceinline__ R noise_amplitude(R x) {
  return Math<R>::sqrt(x);
}
template <>
__host__ __device__ __forceinline__ float noise_amplitude<float>(float x) {
#ifdef __CUDA_ARCH__
  return sqrt_sfu(x);
#else
  return sqrtf(x);
#endif
}
template <>
__host__ __device__ __forceinline__ float2 noise_amplitude<float2>(float2 x) {
  return make_float2(noise_amplitude<float>(x.x), noise_amplitude<float>(x.y));
}

// Box-Muller pair (z0, z1) = sqrt(-2 ln u0) (cos 2 pi u1, sin 2 pi u1) from
// two Philox words, u = ((r >> 8) + 1/2) 2^-24.
// FP64: the uniforms are exact; CUDA's log / sqrt / sincospi.
// FP32 on the device: the special-function unit.  An odd multiple of 2^-25
// above 1/2 has no FP32 representation, so the quantities that need it are
// formed exactly from the integer word instead:
//   v  = 1 - u0 (exact below 1/2); when v < 1/64, -2 ln u0 comes from its
//        Taylor series in v (there the SFU log has only absolute accuracy,
//        which the square root would amplify); otherwise from the SFU log
//        of u0
//   the angle 2 pi u1 is taken to [-pi, pi) by whole turns before the SFU
//        sine and cosine
// Absolute error of the FP32 variates against FP64: about 1e-6.
template <typename R>
struct BoxMuller {
  __host__ __device__ static __forceinline__ void pair(uint32_t r0, uint32_t r1, R &z0, R &z1) {
    const R u0 = unit24<R>(r0), u1 = unit24<R>(r1);
    const R rad = Math<R>::sqrt(R(-2) * Math<R>::log(u0));
    R s, c;
    Math<R>::sincospi(R(2) * u1, &s, &c);
    z0 = rad * c;
    z1 = rad * s;
  }
};

template <>
struct BoxMuller<float> {
  __host__ __device__ static __forceinline__ void pair(uint32_t r0, uint32_t r1, float &z0, float &z1) {
#ifdef __CUDA_ARCH__
    // the arithmetic shift of the angle word is (r1 >> 8) - 2^24 when the top
    // bit is set, an exact turn less
    sfu_pair<float>(static_cast<float>(r0 >> 8), static_cast<float>(static_cast<int32_t>(r1) >> 8), z0, z1);
#else
    const float rad = sqrtf(-2.0f * logf(unit24<float>(r0)));
    float s, c;
    Math<float>::sincospi(2.0f * unit24<float>(r1), &s, &c);
    z0 = rad * c;
    z1 = rad * s;
#endif
  }
#ifdef __CUDACC__
  // The pairs of two sites (words ra0, ra1 and rb0, rb1) in the two lanes:
  // lane by lane the same values as pair().
  __device__ static __forceinline__ void pair2(uint32_t ra0, uint32_t ra1, uint32_t rb0, uint32_t rb1, float2 &z0,
                                               float2 &z1) {
    sfu_pair<float2>(make_float2(static_cast<float>(ra0 >> 8), static_cast<float>(rb0 >> 8)),
                     make_float2(static_cast<float>(static_cast<int32_t>(ra1) >> 8),
                                 static_cast<float>(static_cast<int32_t>(rb1) >> 8)),
                     z0, z1);
  }
#endif

 private:
#ifdef __CUDACC__
  // k0 = r0 >> 8 and k1 = the arithmetic shift r1 >> 8 as floats (exact).
  template <typename V>
  __device__ static __forceinline__ void sfu_pair(V k0, V k1, V &z0, V &z1) {
    // u0 = (k + 1/2) 2^-24 is one rounding of k 2^-24 + 2^-25, and v = 1 - u0
    // = (1 - k 2^-24) - 2^-25: both steps exact wherever v < 1/2 (k 2^-24 has
    // 24 significant bits at most)
    const V u0 = fma_rn(k0, splat<V>(5.9604644775390625e-08f), splat<V>(2.98023223876953125e-08f));
    const V v = sub_rn(fma_rn(k0, splat<V>(-5.9604644775390625e-08f), splat<V>(1.0f)),
                       splat<V>(2.98023223876953125e-08f));
    // -2 ln(1 - v) = v (2 + v (1 + v (2/3 + v/2))) + O(v^5), used below 1/64;
    // above, -2 ln u0 = -2 ln(2) log2(u0)
    const V series = mul_rn(
        v, fma_rn(v, fma_rn(v, fma_rn(v, splat<V>(0.5f), splat<V>(0.6666667f)), splat<V>(1.0f)), splat<V>(2.0f)));
    const V lg = mul_rn(splat<V>(-1.38629436111989061f), log2_sfu(u0));
    const V x = select_below(v, 0.015625f, series, lg);  // x >= 2^-24 > 0
    const V rad = noise_amplitude<V>(x);
    // angle 2 pi u1 taken to [-pi, pi)
    const V angle = fma_rn(k1, splat<V>(3.7450703871400037e-07f) /* 2 pi 2^-24 */,
                           splat<V>(1.8725351935700019e-07f) /* pi 2^-24 */);
    V s, c;
    sincos_sfu(angle, s, c);
    z0 = mul_rn(rad, c);
    z1 = mul_rn(rad, s);
  }
  __device__ static __forceinline__ float log2_sfu(float x) { return __log2f(x); }
  __device__ static __forceinline__ float2 log2_sfu(float2 x) { return make_float2(__log2f(x.x), __log2f(x.y)); }
  __device__ static __forceinline__ void sincos_sfu(float a, float &s, float &c) { __sincosf(a, &s, &c); }
  __device__ static __forceinline__ void sincos_sfu(float2 a, float2 &s, float2 &c) {
    __sincosf(a.x, &s.x, &c.x);
    __sincosf(a.y, &s.y, &c.y);
  }
#endif
};

// Philox4x32-10 for the step kernel.  In one step every thread's counter is
// (site, lattice id, t_lo, t_hi*8 + j): only the site differs between
// threads and only j between the calls of a site.  The parts of rounds 0-2
// that depend on the uniform words alone, and all round keys, are computed
// once per step on the host (make_philox_step); per thread and call the
// first two rounds then cost one 32x32 -> 64-bit multiply and three XORs.
// philox_site(...) equals philox4x32_10(make_uint4(site, lid, t_lo,
// t_hi*8 + j), k0, k1) for every input (checked by the tests).
struct PhiloxStep {
  uint32_t e[8];   // round 0: (t_hi*8 + j) ^ K1[0], per call j
  uint32_t f;      // round 1: lo(t_lo M1) ^ K0[1]
  uint32_t g;      // round 1: hi(a1 M0) ^ K1[1], a1 = hi(t_lo M1) ^ lid ^ K0[0]
  uint32_t q;      // round 2: lo(a1 M0) ^ K1[2]
  uint32_t k0[10], k1[10];  // round keys K0[r] = k0 + r W0, K1[r] = k1 + r W1
};

// The words of P that depend on t (and the lattice id); the round keys stay.
__host__ __device__ inline void philox_step_set_t(PhiloxStep &P, uint32_t lattice_id, uint64_t t) {
  const uint32_t t_lo = static_cast<uint32_t>(t), t_hi8 = static_cast<uint32_t>(t >> 32) << 3;
  for (int j = 0; j < 8; ++j) P.e[j] = (t_hi8 | static_cast<uint32_t>(j)) ^ P.k1[0];
  const uint64_t u = static_cast<uint64_t>(t_lo) * Philox::M1;
  const uint32_t a1 = static_cast<uint32_t>(u >> 32) ^ lattice_id ^ P.k0[0];
  const uint32_t b1 = static_cast<uint32_t>(u);
  const uint64_t v = static_cast<uint64_t>(a1) * Philox::M0;
  P.f = b1 ^ P.k0[1];
  P.g = static_cast<uint32_t>(v >> 32) ^ P.k1[1];
  P.q = static_cast<uint32_t>(v) ^ P.k1[2];
}

__host__ __device__ inline PhiloxStep make_philox_step(uint64_t seed, uint32_t lattice_id, uint64_t t) {
  PhiloxStep P{};
  const uint32_t key0 = static_cast<uint32_t>(seed), key1 = static_cast<uint32_t>(seed >> 32);
  for (int r = 0; r < 10; ++r) {
    P.k0[r] = key0 + static_cast<uint32_t>(r) * Philox::W0;
    P.k1[r] = key1 + static_cast<uint32_t>(r) * Philox::W1;
  }
  philox_step_set_t(P, lattice_id, t);
  return P;
}

// Call j of a site whose product site * M0 is (s_hi, s_lo).
__host__ __device__ __forceinline__ uint4 philox_site(uint32_t s_hi, uint32_t s_lo, const PhiloxStep &P, int j) {
  // rounds 0 and 1
  const uint64_t p = static_cast<uint64_t>(s_hi ^ P.e[j]) * Philox::M1;
  uint4 c = make_uint4(static_cast<uint32_t>(p >> 32) ^ P.f, static_cast<uint32_t>(p), s_lo ^ P.g, 0u);
  // round 2 (its third word takes the uniform q)
  {
    const uint64_t p0 = static_cast<uint64_t>(c.x) * Philox::M0;
    const uint64_t p1 = static_cast<uint64_t>(c.z) * Philox::M1;
    c = make_uint4(static_cast<uint32_t>(p1 >> 32) ^ c.y ^ P.k0[2], static_cast<uint32_t>(p1),
                   static_cast<uint32_t>(p0 >> 32) ^ P.q, static_cast<uint32_t>(p0));
  }
#pragma unroll
  for (int r = 3; r < 10; ++r) {
    const uint64_t p0 = static_cast<uint64_t>(c.x) * Philox::M0;
    const uint64_t p1 = static_cast<uint64_t>(c.z) * Philox::M1;
    c = make_uint4(static_cast<uint32_t>(p1 >> 32) ^ c.y ^ P.k0[r], static_cast<uint32_t>(p1),
                   static_cast<uint32_t>(p0 >> 32) ^ c.w ^ P.k1[r], static_cast<uint32_t>(p0));
  }
  return c;
}

// Unit-variance variates z[0..NMOM-1] (moments a = 1..NMOM) of one site.
// Call j has counter (site, lattice_id, t_lo, t_hi * 8 + j); moment 4j + k + 1
// takes word k.  GAUSS: Box-Muller on the word pairs (0,1) and (2,3);
// otherwise flat variates sqrt(3) (2u - 1).
// Flat variate sqrt3 (2 u - 1) of the uniform u = (k + 1/2) 2^-24, k = r >> 8
// given as a float (exact): in exact arithmetic mean 0 and variance 1 - 2^-48.
template <typename V>
__host__ __device__ __forceinline__ V flat_variate(V k) {
  using R = typename LaneOf<V>::type;
  const V u = mul_rn(add_rn(k, splat<V>(R(0.5))), splat<V>(R(5.9604644775390625e-08)));
  return mul_rn(cst<V>(kSqrt3), fma_rn(splat<V>(R(2)), u, splat<V>(R(-1))));
}

template <typename R, int NMOM, bool GAUSS>
__host__ __device__ __forceinline__ void draw_variates_t(R (&z)[NMOM], uint32_t site, const PhiloxStep &P) {
  constexpr int NCALL = (NMOM + 3) / 4;
  const uint64_t sp = static_cast<uint64_t>(site) * Philox::M0;
  const uint32_t s_hi = static_cast<uint32_t>(sp >> 32), s_lo = static_cast<uint32_t>(sp);
#pragma unroll
  for (int j = 0; j < NCALL; ++j) {
    const uint4 r = philox_site(s_hi, s_lo, P, j);
    const uint32_t w[4] = {r.x, r.y, r.z, r.w};
    if constexpr (GAUSS) {
#pragma unroll
      for (int p = 0; p < 2; ++p) {
        if (4 * j + 2 * p < NMOM) {
          R z0, z1;
          BoxMuller<R>::pair(w[2 * p], w[2 * p + 1], z0, z1);
          z[4 * j + 2 * p] = z0;
          if (4 * j + 2 * p + 1 < NMOM) z[4 * j + 2 * p + 1] = z1;
        }
      }
    } else {
#pragma unroll
      for (int k = 0; k < 4; ++k)
        if (4 * j + k < NMOM) z[4 * j + k] = flat_variate<R>(static_cast<R>(w[k] >> 8));
    }
  }
}

#ifdef __CUDACC__
// The variates of sites (site, site + 1) in the two lanes: lane by lane the
// same values as draw_variates_t<float, NMOM, GAUSS> of each site.
template <int NMOM, bool GAUSS>
__device__ __forceinline__ void draw_variates_pair(float2 (&z)[NMOM], uint32_t site, const PhiloxStep &P) {
  constexpr int NCALL = (NMOM + 3) / 4;
  const uint64_t spa = static_cast<uint64_t>(site) * Philox::M0;
  const uint64_t spb = static_cast<uint64_t>(site + 1u) * Philox::M0;
#pragma unroll
  for (int j = 0; j < NCALL; ++j) {
    const uint4 ra = philox_site(static_cast<uint32_t>(spa >> 32), static_cast<uint32_t>(spa), P, j);
    const uint4 rb = philox_site(static_cast<uint32_t>(spb >> 32), static_cast<uint32_t>(spb), P, j);
    const uint32_t wa[4] = {ra.x, ra.y, ra.z, ra.w}, wb[4] = {rb.x, rb.y, rb.z, rb.w};
    if constexpr (GAUSS) {
#pragma unroll
      for (int p = 0; p < 2; ++p) {
        if (4 * j + 2 * p < NMOM) {
          float2 z0, z1;
          BoxMuller<float>::pair2(wa[2 * p], wa[2 * p + 1], wb[2 * p], wb[2 * p + 1], z0, z1);
          z[4 * j + 2 * p] = z0;
          if (4 * j + 2 * p + 1 < NMOM) z[4 * j + 2 * p + 1] = z1;
        }
      }
    } else {
#pragma unroll
      for (int k = 0; k < 4; ++k)
        if (4 * j + k < NMOM)
          z[4 * j + k] =
              flat_variate<float2>(make_float2(static_cast<float>(wa[k] >> 8), static_cast<float>(wb[k] >> 8)));
    }
  }
}
#endif

template <typename R, int NMOM>
__host__ __device__ __forceinline__ void draw_variates(R (&z)[NMOM], uint32_t site, const PhiloxStep &P, int dist) {
  if (dist == kGaussian)
    draw_variates_t<R, NMOM, true>(z, site, P);
  else
    draw_variates_t<R, NMOM, false>(z, site, P);
}

// ---------------------------------------------------------------------------
// Noise back-transform T_i = sum_{a >= 1} m_i^a z^a (the f-space noise is
// xi_i = w_i sigma T_i).  kWeighted tells whether apply() returns w_i T_i.
// ---------------------------------------------------------------------------
// Index of the velocity -v_i, and the parity of basis row a under v -> -v
// (the parity of its seed monomial's degree; Gram-Schmidt over a symmetric
// velocity set never mixes the two parities, which make_basis's table obeys
// exactly: checked below).
template <int LAT>
__host__ __device__ constexpr int partner(int i) {
  using L = Lattice<LAT>;
  for (int j = 0; j < L::Q; ++j)
    if (L::v(j, 0) == -L::v(i, 0) && L::v(j, 1) == -L::v(i, 1) && L::v(j, 2) == -L::v(i, 2)) return j;
  return -1;
}
template <int LAT>
__host__ __device__ constexpr int row_parity(int a) {
  using L = Lattice<LAT>;
  return (L::mono(a, 0) + L::mono(a, 1) + L::mono(a, 2)) & 1;
}
template <int LAT>
constexpr bool basis_has_parity() {
  constexpr int Q = Lattice<LAT>::Q;
  for (int a = 0; a < Q; ++a)
    for (int i = 0; i < Q; ++i) {
      const double m = kBasisTable<LAT>.m[a][i], mp = kBasisTable<LAT>.m[a][partner<LAT>(i)];
      if (partner<LAT>(i) < 0 || mp != (row_parity<LAT>(a) ? -m : m)) return false;
    }
  return true;
}

// Generic transform, weighted: wT_i = w_i sum_{a>=1} m_i^a z^a.  The
// constants w_i m_i^a are folded at compile time and zeros skipped; each pair
// (i, -i) shares its even part E and odd part O: wT_i = E + O, wT_-i = E - O,
// or, when O is a single term c z, wT_+-i = fma(+-c, z, E).  apply() takes z
// and returns wT as R (one site) or, for R = float, float2 (two sites).
template <int LAT, typename R>
struct NoiseTransform {
  static constexpr bool kWeighted = true;
  static_assert(basis_has_parity<LAT>(), "basis rows must have definite parity");
  // number of terms of part<I, PAR>
  template <int I, int PAR>
  static constexpr int terms() {
    constexpr int Q = Lattice<LAT>::Q;
    int n = 0;
    for (int a = 1; a < Q; ++a)
      if (kBasisTable<LAT>.m[a][I] != 0.0 && (PAR < 0 || row_parity<LAT>(a) == PAR)) ++n;
    return n;
  }
  // the row of the first term of part<I, PAR>
  template <int I, int PAR>
  static constexpr int first_row() {
    constexpr int Q = Lattice<LAT>::Q;
    for (int a = 1; a < Q; ++a)
      if (kBasisTable<LAT>.m[a][I] != 0.0 && (PAR < 0 || row_parity<LAT>(a) == PAR)) return a;
    return 0;
  }
  template <int I, int PAR, typename V>
  __host__ __device__ static __forceinline__ V part(const V (&z)[Lattice<LAT>::Q - 1]) {
    constexpr int Q = Lattice<LAT>::Q;
    V acc = splat<V>(0);
    bool first = true;
    static_for<Q - 1>([&](auto A) {
      constexpr int a = decltype(A)::value + 1;
      constexpr double c = kBasis<LAT, a, I> * Lattice<LAT>::w(I);
      if constexpr (c != 0.0 && (PAR < 0 || row_parity<LAT>(a) == PAR)) {
        if (first) {
          acc = mul_rn(cst<V>(c), z[a - 1]);
          first = false;
        } else {
          acc = fma_rn(cst<V>(c), z[a - 1], acc);
        }
      }
    });
    return acc;
  }
  template <typename V>
  __host__ __device__ static __forceinline__ void apply(const V (&z)[Lattice<LAT>::Q - 1], V (&wT)[Lattice<LAT>::Q]) {
    constexpr int Q = Lattice<LAT>::Q;
    static_for<Q>([&](auto I) {
      constexpr int i = decltype(I)::value;
      constexpr int ip = partner<LAT>(i);
      if constexpr (ip == i) {
        wT[i] = part<i, -1>(z);
      } else if constexpr (i < ip) {
        const V E = part<i, 0>(z);
        if constexpr (terms<i, 1>() == 1) {
          constexpr int a = first_row<i, 1>();
          constexpr double c = kBasis<LAT, a, i> * Lattice<LAT>::w(i);
          wT[i] = fma_rn(cst<V>(c), z[a - 1], E);
          wT[ip] = fma_rn(cst<V>(-c), z[a - 1], E);
        } else {
          const V O = part<i, 1>(z);
          wT[i] = add_rn(E, O);
          wT[ip] = sub_rn(E, O);
        }
      }
    });
  }
};

// D2Q9: the basis factorises as mu^p(v_x) mu^q(v_y), so the transform is a
// 3x3 pass over q followed by a 3x3 pass over p (24 multiply-adds).
template <typename R>
struct NoiseTransform<kD2Q9, R> {
  static constexpr bool kWeighted = false;  // returns T_i; the caller applies w_i
  template <typename V>
  __host__ __device__ static __forceinline__ void apply(const V (&z)[8], V (&T)[9]) {
    // zeta[p][q] = z^{3p+q}, zeta[0][0] = 0: the q = 0 terms of p = 0 drop out
    V G[3][3];  // G[p][c]: c = 0 (v_y = 0), 1 (v_y = +1), 2 (v_y = -1)
    G[0][0] = mul_rn(cst<V>(-kInvSqrt2), z[1]);
    {
      const V even = mul_rn(cst<V>(kSqrt2), z[1]);
      G[0][1] = fma_rn(cst<V>(kSqrt3), z[0], even);
      G[0][2] = fma_rn(cst<V>(-kSqrt3), z[0], even);
    }
#pragma unroll
    for (int p = 1; p < 3; ++p) {
      const V z0 = z[3 * p - 1], z1 = z[3 * p], z2 = z[3 * p + 1];
      G[p][0] = fma_rn(cst<V>(-kInvSqrt2), z2, z0);
      const V even = fma_rn(cst<V>(kSqrt2), z2, z0);
      G[p][1] = fma_rn(cst<V>(kSqrt3), z1, even);
      G[p][2] = fma_rn(cst<V>(-kSqrt3), z1, even);
    }
    V H[3][3];  // H[cx][cy]
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      H[0][c] = fma_rn(cst<V>(-kInvSqrt2), G[2][c], G[0][c]);
      const V even = fma_rn(cst<V>(kSqrt2), G[2][c], G[0][c]);
      H[1][c] = fma_rn(cst<V>(kSqrt3), G[1][c], even);
      H[2][c] = fma_rn(cst<V>(-kSqrt3), G[1][c], even);
    }
    // velocity -> (cx, cy): 0 -> 0, +1 -> 1, -1 -> 2
    T[0] = H[0][0];
    T[1] = H[1][0];
    T[2] = H[0][1];
    T[3] = H[2][0];
    T[4] = H[0][2];
    T[5] = H[1][1];
    T[6] = H[2][1];
    T[7] = H[2][2];
    T[8] = H[1][2];
  }
};

// D1Q3: T(0) = -z^2/sqrt2, T(+-1) = +-sqrt3 z^1 + sqrt2 z^2.
template <typename R>
struct NoiseTransform<kD1Q3, R> {
  static constexpr bool kWeighted = false;
  template <typename V>
  __host__ __device__ static __forceinline__ void apply(const V (&z)[2], V (&T)[3]) {
    T[0] = mul_rn(cst<V>(-kInvSqrt2), z[1]);
    const V even = mul_rn(cst<V>(kSqrt2), z[1]);
    T[1] = fma_rn(cst<V>(kSqrt3), z[0], even);
    T[2] = fma_rn(cst<V>(-kSqrt3), z[0], even);
  }
};

// Full moment matrix of the D2Q9 product basis, for export and checks.
__host__ __device__ constexpr double d1q3_mu(int p, int v) {
  return p == 0 ? 1.0 : (p == 1 ? kSqrt3 * v : (v == 0 ? -kInvSqrt2 : kSqrt2));
}

}  // namespace lbfd
