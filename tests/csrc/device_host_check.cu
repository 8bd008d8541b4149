// Host build of the device header's arithmetic, for CPU unit tests: the
// noise variates and the noise back-transform the step kernel uses,
// evaluated by the same source on the host.
#include <stdint.h>
#include <string.h>

#include "device.cuh"

using namespace lbfd;

// Returns 1 when the transform folds the weights in (T_i = w_i sum_a ...).
template <int LAT, typename R>
static int transform_t(const double *z, double *T) {
  constexpr int Q = Lattice<LAT>::Q;
  R zz[Q - 1], TT[Q];
  for (int a = 0; a < Q - 1; ++a) zz[a] = static_cast<R>(z[a]);
  NoiseTransform<LAT, R>::apply(zz, TT);
  for (int i = 0; i < Q; ++i) T[i] = static_cast<double>(TT[i]);
  return NoiseTransform<LAT, R>::kWeighted ? 1 : 0;
}

// The transform on two sites' variates at once (value type float2) and on
// each alone (float): lane l of T2 against T of z lane l, as bit patterns.
// Returns the number of values that differ.
template <int LAT>
static int transform_pair_t(const double *z2, double *T2) {
  constexpr int Q = Lattice<LAT>::Q;
  float2 zz[Q - 1], TT[Q];
  float za[Q - 1], zb[Q - 1], Ta[Q], Tb[Q];
  for (int a = 0; a < Q - 1; ++a) {
    za[a] = static_cast<float>(z2[a]);
    zb[a] = static_cast<float>(z2[Q - 1 + a]);
    zz[a] = make_float2(za[a], zb[a]);
  }
  NoiseTransform<LAT, float>::apply(zz, TT);
  NoiseTransform<LAT, float>::apply(za, Ta);
  NoiseTransform<LAT, float>::apply(zb, Tb);
  int bad = 0;
  for (int i = 0; i < Q; ++i) {
    T2[i] = static_cast<double>(TT[i].x);
    T2[Q + i] = static_cast<double>(TT[i].y);
    bad += memcmp(&TT[i].x, &Ta[i], sizeof(float)) != 0;
    bad += memcmp(&TT[i].y, &Tb[i], sizeof(float)) != 0;
  }
  return bad;
}

template <typename R, int NMOM>
static void variates_t(int dist, uint64_t seed, uint32_t lid, uint32_t site, uint64_t t, double *z) {
  R zz[NMOM];
  const PhiloxStep P = make_philox_step(seed, lid, t);
  draw_variates<R, NMOM>(zz, site, P, dist);
  for (int a = 0; a < NMOM; ++a) z[a] = static_cast<double>(zz[a]);
}

extern "C" {

int dhc_transform(int lattice, int f64, const double *z, double *T) {
  switch (lattice) {
    case kD1Q3: return f64 ? transform_t<kD1Q3, double>(z, T) : transform_t<kD1Q3, float>(z, T);
    case kD2Q9: return f64 ? transform_t<kD2Q9, double>(z, T) : transform_t<kD2Q9, float>(z, T);
    case kD3Q19: return f64 ? transform_t<kD3Q19, double>(z, T) : transform_t<kD3Q19, float>(z, T);
  }
  return -1;
}

int dhc_transform_pair(int lattice, const double *z2, double *T2) {
  switch (lattice) {
    case kD1Q3: return transform_pair_t<kD1Q3>(z2, T2);
    case kD2Q9: return transform_pair_t<kD2Q9>(z2, T2);
    case kD3Q19: return transform_pair_t<kD3Q19>(z2, T2);
  }
  return -1;
}

// flat_variate of two words at once (float2) against each alone (float):
// the number of the n pairs whose lanes differ as bit patterns.
int dhc_flat_pair_mismatches(const uint32_t *words, int64_t n) {
  int bad = 0;
  for (int64_t k = 0; k + 1 < 2 * n; k += 2) {
    const float a = static_cast<float>(words[k] >> 8), b = static_cast<float>(words[k + 1] >> 8);
    const float2 v = flat_variate<float2>(make_float2(a, b));
    const float va = flat_variate<float>(a), vb = flat_variate<float>(b);
    bad += memcmp(&v.x, &va, sizeof(float)) != 0 || memcmp(&v.y, &vb, sizeof(float)) != 0;
  }
  return bad;
}

int dhc_variates(int f64, int nmom, int dist, uint64_t seed, uint32_t lid, uint32_t site, uint64_t t, double *z) {
  if (nmom == 2) { f64 ? variates_t<double, 2>(dist, seed, lid, site, t, z) : variates_t<float, 2>(dist, seed, lid, site, t, z); return 0; }
  if (nmom == 8) { f64 ? variates_t<double, 8>(dist, seed, lid, site, t, z) : variates_t<float, 8>(dist, seed, lid, site, t, z); return 0; }
  if (nmom == 18) { f64 ? variates_t<double, 18>(dist, seed, lid, site, t, z) : variates_t<float, 18>(dist, seed, lid, site, t, z); return 0; }
  return -1;
}

// The step kernel's per-site Philox (host-precomputed uniform parts).
int dhc_philox_site(uint64_t seed, uint32_t lid, uint64_t t, uint32_t site, int j, uint32_t *out) {
  const PhiloxStep P = make_philox_step(seed, lid, t);
  const uint64_t sp = uint64_t(site) * Philox::M0;
  uint4 r = philox_site(uint32_t(sp >> 32), uint32_t(sp), P, j);
  out[0] = r.x; out[1] = r.y; out[2] = r.z; out[3] = r.w;
  return 0;
}

int dhc_philox(const uint32_t *ctr, const uint32_t *key, uint32_t *out) {
  uint4 r = philox4x32_10(make_uint4(ctr[0], ctr[1], ctr[2], ctr[3]), key[0], key[1]);
  out[0] = r.x; out[1] = r.y; out[2] = r.z; out[3] = r.w;
  return 0;
}
}

// Multiply-shift division of the batched kernel's index split, against the
// hardware division: every (d, n) pair given; returns the number of mismatches.
#include "fastdiv.cuh"

extern "C" int64_t dhc_fastdiv_mismatches(const uint32_t *d, int64_t nd, const uint32_t *n, int64_t nn) {
  int64_t bad = 0;
  for (int64_t i = 0; i < nd; ++i) {
    const FastDiv f = make_fastdiv(d[i]);
    for (int64_t k = 0; k < nn; ++k) bad += fastdiv(n[k], f) != n[k] / d[i];
  }
  return bad;
}
