// Multiple-relaxation-time steps (mrt_kernels.cuh) for every lattice, FP32
// and FP64, and the run-time tables of D2Q5.
#include <cmath>

#include "mrt_kernels.cuh"

namespace lbfd {

cudaError_t launch_step_mrt(int lattice, int precision, const void *src, void *dst, const StepArgs &a, const double *m,
                            const double *w, const double *tau, cudaStream_t stream) {
  if (precision != kStoreF32 && precision != kStoreF64) return cudaErrorInvalidValue;
  return dispatch_lattice(lattice, [&](auto lat) -> cudaError_t {
    constexpr int LAT = decltype(lat)::value;
    if (precision == kStoreF64) return step_mrt_t<LAT, double>(src, dst, a, m, w, tau, stream);
    return step_mrt_t<LAT, float>(src, dst, a, m, w, tau, stream);
  });
}

// D2Q5 with second moment theta (Sec. II): weights w_0 = 1 - 2 theta,
// w_1..4 = theta / 2, and the basis by weighted Gram-Schmidt of the paper's
// list 1, v_x, v_y, v_x^2 - v_y^2, v_x^2 + v_y^2 (Sec. II).
void d2q5_tables(double theta, double *w, double *m) {
  using L = Lattice<kD2Q5>;
  for (int i = 0; i < 5; ++i) w[i] = i == 0 ? 1.0 - 2.0 * theta : 0.5 * theta;
  for (int a = 0; a < 5; ++a) {
    double u[5];
    for (int i = 0; i < 5; ++i) {
      const double vx = L::v(i, 0), vy = L::v(i, 1);
      const double seed[5] = {1.0, vx, vy, vx * vx - vy * vy, vx * vx + vy * vy};
      u[i] = seed[a];
    }
    for (int b = 0; b < a; ++b) {
      double proj = 0.0;
      for (int i = 0; i < 5; ++i) proj += u[i] * w[i] * m[b * 5 + i];
      for (int i = 0; i < 5; ++i) u[i] -= proj * m[b * 5 + i];
    }
    double n2 = 0.0;
    for (int i = 0; i < 5; ++i) n2 += u[i] * w[i] * u[i];
    const double inv = 1.0 / std::sqrt(n2);
    for (int i = 0; i < 5; ++i) m[a * 5 + i] = u[i] * inv;
  }
}

}  // namespace lbfd
