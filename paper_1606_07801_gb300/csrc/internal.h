// Host-side declarations shared by the library's translation units.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <cstdlib>
#include <string>

#include <nvtx3/nvToolsExt.h>

#include "device.cuh"
#include "step_shape.h"

#define LBFD_MAX_MODES_DEV 16
#define LBFD_MAX_Q_DEV 19

namespace lbfd {

// A named NVTX range for the scope (seen by nsys / ncu timelines; a no-op
// when no tool is attached).
struct NvtxRange {
  explicit NvtxRange(const char *name) { nvtxRangePushA(name); }
  ~NvtxRange() { nvtxRangePop(); }
  NvtxRange(const NvtxRange &) = delete;
  NvtxRange &operator=(const NvtxRange &) = delete;
};

// Per-launch arguments of the step kernel (passed by value).
struct StepArgs {
  int32_t Lx, Ly, Lz;
  int32_t sweep;       // one-launch-per-step kernels: 0 = work blocks in grid order, 1 = reversed
  int64_t N;           // sites
  double omega;        // 1 - 1/tau (what is left of the non-equilibrium part)
  double inv_tau;      // 1/tau
  double noise_var;    // (2 tau - 1)/tau^2: noise variance per unit density
  double rho_eq;       // density of the global-noise variant
  // the same four in FP32, so FP32 kernels never convert from FP64 on the
  // device (GB300's FP64 unit is narrow)
  float omega_f, inv_tau_f, noise_var_f, rho_eq_f;
  int32_t noise_mode;  // kNoiseLocal / kNoiseGlobal / kNoiseOff
  int32_t noise_dist;  // kGaussian / kUniform
  PhiloxStep ph;       // Philox key and counter words of this step (seed, lattice id, t)
};

// Relaxation and noise parameters of a step from tau and rho_mean (FP64 and
// their FP32 copies).  Every path that steps a lattice uses this one
// function, so a lattice gets bit-identical parameters alone or in an
// ensemble.
__host__ __device__ inline void fill_step_params(StepArgs &a, double tau, double rho_mean) {
  a.omega = 1.0 - 1.0 / tau;
  a.inv_tau = 1.0 / tau;
  a.noise_var = (2.0 * tau - 1.0) / (tau * tau);
  a.rho_eq = rho_mean;
  a.omega_f = static_cast<float>(a.omega);
  a.inv_tau_f = static_cast<float>(a.inv_tau);
  a.noise_var_f = static_cast<float>(a.noise_var);
  a.rho_eq_f = static_cast<float>(a.rho_eq);
}

// Calls f(std::integral_constant<int, LAT>, Tag<S>) for a lattice id and a
// storage id (0 FP32, 1 FP64, 2 FP16 deviations, 3 BF16 deviations).
template <class F>
inline cudaError_t dispatch_storage(int precision, F &&f) {
  switch (precision) {
    case kStoreF32: return f(Tag<float>{});
    case kStoreF64: return f(Tag<double>{});
    case kStoreF16: return f(Tag<__half>{});
    case kStoreBF16: return f(Tag<__nv_bfloat16>{});
  }
  return cudaErrorInvalidValue;
}
template <class F>
inline cudaError_t dispatch_lattice(int lattice, F &&f) {
  switch (lattice) {
    case kD1Q3: return f(std::integral_constant<int, kD1Q3>{});
    case kD2Q9: return f(std::integral_constant<int, kD2Q9>{});
    case kD3Q19: return f(std::integral_constant<int, kD3Q19>{});
    case kD2Q5: return f(std::integral_constant<int, kD2Q5>{});
  }
  return cudaErrorInvalidValue;
}
template <class F>
inline cudaError_t dispatch_lattice_storage(int lattice, int precision, F &&f) {
  return dispatch_lattice(lattice, [&](auto lat) {
    return dispatch_storage(precision, [&](auto tag) { return f(lat, tag); });
  });
}

// Bytes of one stored value for a storage id.
inline int storage_bytes(int precision) { return precision == kStoreF64 ? 8 : (precision == kStoreF32 ? 4 : 2); }

// The step parameter in the kernel's precision.
template <typename R>
__host__ __device__ __forceinline__ R step_param(double d, float f);
template <>
__host__ __device__ __forceinline__ double step_param<double>(double d, float) { return d; }
template <>
__host__ __device__ __forceinline__ float step_param<float>(double, float f) { return f; }

// CTAs of the many-steps-per-launch path for a small lattice: 1 = one block
// (k_step_small), 2..8 = a thread-block cluster (k_step_cluster), 0 = the
// lattice does not fit it (or its lattice type has no such path).
int small_path_ctas(int lattice, int precision, int64_t N);

// Per-lattice step launchers (one translation unit each).  vec_width: 2
// runs k_step_vec (Lx even), 1 runs k_step.
cudaError_t launch_step_d1q3(int precision, const void *src, void *dst, const StepArgs &a, cudaStream_t stream,
                             int vec_width);
cudaError_t launch_step_d2q9(int precision, const void *src, void *dst, const StepArgs &a, cudaStream_t stream,
                             int vec_width);
cudaError_t launch_step_d3q19(int precision, const void *src, void *dst, const StepArgs &a, cudaStream_t stream,
                              int vec_width);

// Rows a staged launch updates, and the key offset of their sites (see
// staged_kernels.cuh).
struct StagedRows {
  uint32_t row_begin, nrows, row_key;
};

// The same step by the shared-memory staged kernel (staged_kernels.cuh).
// Needs Lx * (bytes per stored value) to be a multiple of 16, both buffers
// 16-byte aligned and fewer than 2^31 sites (staged_fits); a bounded wait
// that gives up sets *status (device-visible memory) to a non-zero code.
cudaError_t launch_step_staged_d1q3(int precision, const void *src, void *dst, const StepArgs &a, 
                                   const StagedRows &rows, int *status, uint32_t wait_test_bytes, cudaStream_t stream);
cudaError_t launch_step_staged_d2q9(int precision, const void *src, void *dst, const StepArgs &a, 
                                   const StagedRows &rows, int *status, uint32_t wait_test_bytes, cudaStream_t stream);
cudaError_t launch_step_staged_d3q19(int precision, const void *src, void *dst, const StepArgs &a, 
                                    const StagedRows &rows, int *status, uint32_t wait_test_bytes, cudaStream_t stream);
inline bool staged_fits(int lattice, int precision, int64_t Lx, int64_t N, const void *f0, const void *f1) {
  if (lattice != kD1Q3 && lattice != kD2Q9 && lattice != kD3Q19) return false;
  const int64_t elem = storage_bytes(precision);
  return (Lx * elem) % 16 == 0 && N < (int64_t(1) << 31) && reinterpret_cast<uintptr_t>(f0) % 16 == 0 &&
         reinterpret_cast<uintptr_t>(f1) % 16 == 0;
}
// wait_test_bytes > 0 only in tests of the bounded wait: the first tile of
// every CTA waits for that many bytes more than its copies deliver.
inline cudaError_t launch_step_staged(int lattice, int precision, const void *src, void *dst, const StepArgs &a,
                                      const StagedRows &rows, int *status, uint32_t wait_test_bytes,
                                      cudaStream_t stream) {
  switch (lattice) {
    case kD1Q3: return launch_step_staged_d1q3(precision, src, dst, a, rows, status, wait_test_bytes, stream);
    case kD2Q9: return launch_step_staged_d2q9(precision, src, dst, a, rows, status, wait_test_bytes, stream);
    case kD3Q19: return launch_step_staged_d3q19(precision, src, dst, a, rows, status, wait_test_bytes, stream);
  }
  return cudaErrorInvalidValue;
}

// One step of eq. LB from src to dst (pull streaming, two buffers); by
// default with the library's choice of sites per thread.
cudaError_t launch_step(int lattice, int precision, const void *src, void *dst, const StepArgs &a,
                        cudaStream_t stream, int vec_width = 0);

// Streaming shift between the stored post-collision state g and the
// paper's f: dir = +1 gives f_i(x) = g_i(x - v_i), dir = -1 the inverse.
cudaError_t launch_shift(int lattice, int value_bytes, const void *src, void *dst, int32_t Lx, int32_t Ly, int32_t Lz,
                         int dir, cudaStream_t stream);

// f_i = w_i rho(x), rho = rho_mean (+ amp sin(2 pi k.x / L)); w (Q values)
// overrides the lattice's compiled weights (D2Q5 with theta != 1/3).  The
// sine's coordinates are (c + phase_off) mod phase_len per axis (default:
// the stored lattice itself), so a slab takes its part of the global mode.
cudaError_t launch_init(int lattice, int precision, void *f, int32_t Lx, int32_t Ly, int32_t Lz, double rho_mean,
                        double amp, const int32_t *k, cudaStream_t stream, const double *w = nullptr,
                        const int32_t *phase_off = nullptr, const int32_t *phase_len = nullptr);

// Multiple-relaxation-time step (mrt_kernels.cuh), FP32 or FP64 storage:
// m (Q*Q, [a][i]) and w (Q) the basis and weights (run-time for D2Q5), tau
// the relaxation time of each moment (entry 0 unused).
cudaError_t launch_step_mrt(int lattice, int precision, const void *src, void *dst, const StepArgs &a, const double *m,
                            const double *w, const double *tau, cudaStream_t stream);

// Many steps of a small lattice in one launch (step_small.cu), in one
// block's shared memory or in a thread-block cluster's distributed shared
// memory (up to 8 x kSmallMaxBytes): src holds the stored state at step t0,
// dst receives it after nsteps steps (dst may equal src).
constexpr size_t kSmallMaxBytes = 200 * 1024;
bool small_path_fits(int lattice, int precision, int64_t N);
cudaError_t launch_step_small(int lattice, int precision, const void *src, void *dst, const StepArgs &a, uint64_t seed,
                              uint32_t lattice_id, uint64_t t0, int nsteps, cudaStream_t stream);

// D2Q5 weights and moment basis (m[a*5 + i]) for second moment theta.
void d2q5_tables(double theta, double *w, double *m);

// rho(x) of the paper's f(x, t) straight from the stored post-collision state
// g (populations pulled, FP64 sum in velocity order): the same values as a
// streaming shift followed by launch_moments, without the shift.
cudaError_t launch_density_of_state(int lattice, int precision, const void *g, int32_t Lx, int32_t Ly, int32_t Lz,
                                    double rho_mean, double *rho, cudaStream_t stream);
// rho(x) = sum_i f_i, j_a(x) = sum_i f_i v_ia (FP64 outputs; j may be null).
// rho_mean decodes the 16-bit deviation formats.
cudaError_t launch_moments(int lattice, int precision, const void *f, int32_t Lx, int32_t Ly, int32_t Lz,
                           double rho_mean, double *rho, double *j, cudaStream_t stream);

// Noise variates of sites [site0, site0 + nsites) at step t into z[site][moment] (FP64).
cudaError_t launch_noise_draw(int precision, int dist, const PhiloxStep &ph, int64_t site0, int64_t nsites, int nmom,
                              double *z, cudaStream_t stream);

// Box-Muller pairs of given Philox words: words[2k], words[2k+1] -> z[2k], z[2k+1].
cudaError_t launch_box_muller_probe(int precision, const uint32_t *words, int64_t npairs, double *z,
                                    cudaStream_t stream);

// The collision's arithmetic on given operands, once per value and once on
// two values per packed instruction: out[(2 op + form) n + k] for the
// operations op = add, sub, mul, fma, mul then add, mul then sub of
// (a[k], b[k], c[k]), form 0 one value at a time, form 1 packed with the
// neighbour k ^ 1 (n even).
cudaError_t launch_lane_ops_probe(const float *a, const float *b, const float *c, int64_t n, float *out,
                                  cudaStream_t stream);

// Deterministic FP64 reductions.
//   Stage 1 writes per-block partials of `nq` quantities to partials[block][nq];
//   stage 2 sums them in block order and adds the totals into acc[nq] (or
//   stores them when accumulate == 0).
constexpr int kReduceBlocks = 304;   // 2 x 152 SMs
constexpr int kReduceThreads = 256;
constexpr int kObsBlocks = 608;      // 4 x 152 SMs: the FP32 observable pass (partials sized for it)

// Number of FP64 quantities the observable pass produces for a lattice and mode count.
int obs_quantities(int Q, int n_modes);

// FP64 sum_i sum_s f_i(s) over N sites whose population i starts at f + i
// stride (stride 0: N, a whole lattice).
cudaError_t launch_mass(int lattice, int precision, const void *f, int64_t N, double rho_mean, double *partials,
                        double *out, cudaStream_t stream, int64_t stride = 0);

cudaError_t launch_observables(int lattice, int precision, const void *f, int32_t Lx, int32_t Ly, int32_t Lz,
                               double rho_mean, int n_modes, const int32_t *modes /*device, n_modes*3*/,
                               double *partials, double *acc, cudaStream_t stream);

// The same observables for FP32 arithmetic (FP32, FP16, BF16 storage; not
// FP64) from the stored post-collision state g, pulled per population (no
// streamed copy); N < 2^31.  Per-tile FP32 sums of deviations, FP64 beyond.
// phase (optional): the per-axis factors of the structure-factor modes,
// obs_phase_values() float pairs filled by obs_phase_fill(); without it the
// kernel evaluates each phase with sincospif.
// fin: stage-2 scratch of obs_quantities(Q, LBFD_MAX_MODES_DEV) + 1 doubles,
// its last word zero before the first call (the kernels leave it zero).
cudaError_t launch_observables_pull(int lattice, int precision, const void *g, int32_t Lx, int32_t Ly, int32_t Lz,
                                    double rho_mean, int n_modes, const int32_t *modes, const void *phase,
                                    double *partials, double *fin, double *acc, cudaStream_t stream);
// Stage 1 alone over the sites s0 .. s0 + count - 1 of the stored lattice
// (a slab's owned planes): per-block partials, *nblocks of them, in the
// layout above, for the caller to sum.
cudaError_t launch_observables_pull_partials(int lattice, int precision, const void *g, int32_t Lx, int32_t Ly,
                                             int32_t Lz, int64_t s0, int64_t count, double rho_mean, int n_modes,
                                             const int32_t *modes, const void *phase, double *partials, int *nblocks,
                                             cudaStream_t stream);
size_t obs_phase_values(int n_modes, int32_t Lx, int32_t Ly, int32_t Lz);
// period, offset (optional, per axis): coordinate u of the table is the
// global coordinate (offset + u) mod period (a slab's stored planes).
void obs_phase_fill(int n_modes, const int32_t *modes, int32_t Lx, int32_t Ly, int32_t Lz, float *out,
                    const int64_t *period = nullptr, const int64_t *offset = nullptr);

// c_i = w_i rho_mean in FP32, the constants the FP32-arithmetic observables
// take their deviations e_i = f_i - c_i from (rounded so that every kernel
// forms the same value).
template <int LAT>
__host__ __device__ __forceinline__ float obs_offset(int i, float rho_f) {
  return mul_rn(static_cast<float>(Lattice<LAT>::w(i)), rho_f);
}

// Entry k of the observable accumulators ([sum rho, sum rho^2, sum f_i (Q),
// sum f_i f_j (Q x Q), |rho(k_m)|^2 (K)]) from the totals tt of a sample's
// deviation sums in the layout of the FP32 observable pass ([sum delta,
// sum delta^2, sum e_i (Q), (re, im) of the K modes, pairs i <= j
// row-major]), with cs[i] = c_i, C = sum_i c_i and Nd sites: rho = C +
// delta and f_i = c_i + e_i expanded, in FP64.
template <int Q>
__host__ __device__ __forceinline__ double obs_restore(int k, const double *tt, const double *cs, double C, double Nd,
                                                       int K) {
  const int nq1 = 2 + Q + 2 * K;
  if (k == 0) return tt[0] + Nd * C;
  if (k == 1) return tt[1] + 2.0 * C * tt[0] + Nd * C * C;
  if (k < 2 + Q) return tt[k] + Nd * cs[k - 2];
  if (k < 2 + Q + Q * Q) {
    const int r = k - 2 - Q, a = r / Q, b = r - a * Q;
    const int i = a < b ? a : b, j = a < b ? b : a;
    const int p = i * Q - i * (i - 1) / 2 + (j - i);
    return tt[nq1 + p] + cs[j] * tt[2 + i] + cs[i] * tt[2 + j] + Nd * cs[i] * cs[j];
  }
  const int m = k - 2 - Q - Q * Q;
  const double re = tt[2 + Q + 2 * m], im = tt[3 + Q + 2 * m];
  return re * re + im * im;
}

// Stage 2 for partials in the layout of the FP32-arithmetic observable pass
// (nblocks <= kObsBlocks): sums them in block order, restores the sums of rho,
// f and f f from the deviation sums, and adds them into acc.
cudaError_t launch_obs_pull_finalize(int lattice, const double *partials, int nblocks, int n_modes, int64_t N,
                                     double rho_mean, double *fin, double *acc, cudaStream_t stream);

// A step fused with the sampled observables of the state it reads (the
// FP32-arithmetic formats; sample_kernels.cuh): f(x, t) is advanced one step
// from src to dst exactly as launch_step does, its observables go into
// per-block partials (*nblocks sets, at most kObsBlocks, in the layout of
// the FP32 observable pass) for launch_obs_pull_finalize.  phase: the
// per-axis structure-factor tables (obs_phase_fill); n_modes <=
// kFusedModes.
constexpr int kFusedModes = 4;
// Whether a lattice can take the fused step-and-sample kernel: FP32
// arithmetic, fewer than 2^31 sites, at most kFusedModes modes with their
// phase tables, and a work block of 256 threads with whole warps along x
// (the one-launch-per-step kernel's shape).
inline bool sample_fusable(int lattice, int precision, int32_t Lx, int32_t Ly, int32_t Lz, int n_modes,
                           const void *phase) {
  if (lattice != kD1Q3 && lattice != kD2Q9 && lattice != kD3Q19) return false;
  if (precision == kStoreF64 || n_modes > kFusedModes || (n_modes > 0 && !phase)) return false;
  if (int64_t(Lx) * Ly * Lz >= (int64_t(1) << 31)) return false;
  dim3 grid, block;
  step_shape(Lx, Ly, Lz, grid, block, step_vec_width(lattice, precision, Lx) >= 2 ? 2 : 1);
  return block.x * block.y == 256 && block.x % 32 == 0;
}
cudaError_t launch_step_sample_d1q3(int precision, const void *src, void *dst, const StepArgs &a, int n_modes,
                                    const void *phase, double *partials, int *nblocks, bool staged_ok,
                                    int *status, cudaStream_t stream);
cudaError_t launch_step_sample_d2q9(int precision, const void *src, void *dst, const StepArgs &a, int n_modes,
                                    const void *phase, double *partials, int *nblocks, bool staged_ok,
                                    int *status, cudaStream_t stream);
cudaError_t launch_step_sample_d3q19(int precision, const void *src, void *dst, const StepArgs &a, int n_modes,
                                     const void *phase, double *partials, int *nblocks, bool staged_ok,
                                     int *status, cudaStream_t stream);
// staged_ok: the lattice and buffers meet the staged kernel's requirements
// (staged_fits); status: its bounded waits' status word.
inline cudaError_t launch_step_sample(int lattice, int precision, const void *src, void *dst, const StepArgs &a,
                                      int n_modes, const void *phase, double *partials, int *nblocks, bool staged_ok,
                                      int *status, cudaStream_t stream) {
  switch (lattice) {
    case kD1Q3:
      return launch_step_sample_d1q3(precision, src, dst, a, n_modes, phase, partials, nblocks, staged_ok, status,
                                     stream);
    case kD2Q9:
      return launch_step_sample_d2q9(precision, src, dst, a, n_modes, phase, partials, nblocks, staged_ok, status,
                                     stream);
    case kD3Q19:
      return launch_step_sample_d3q19(precision, src, dst, a, n_modes, phase, partials, nblocks, staged_ok, status,
                                      stream);
  }
  return cudaErrorInvalidValue;
}

// The observables of a state without a step, for the register-sampler
// lattices (D1Q3, D2Q9; FP32 arithmetic; the shape sample_fusable accepts):
// the sampler of the fused step as the separate sampling pass, in the
// partials layout of k_obs_pull (then launch_obs_pull_finalize).
// cudaErrorInvalidValue for other lattices.
cudaError_t launch_obs_sample_d1q3(int precision, const void *src, const StepArgs &a, int n_modes,
                                   const void *phase, double *partials, int *nblocks, cudaStream_t stream);
cudaError_t launch_obs_sample_d2q9(int precision, const void *src, const StepArgs &a, int n_modes,
                                   const void *phase, double *partials, int *nblocks, cudaStream_t stream);
inline cudaError_t launch_obs_sample(int lattice, int precision, const void *src, const StepArgs &a, int n_modes,
                                     const void *phase, double *partials, int *nblocks, cudaStream_t stream) {
  if (lattice == kD1Q3) return launch_obs_sample_d1q3(precision, src, a, n_modes, phase, partials, nblocks, stream);
  if (lattice == kD2Q9) return launch_obs_sample_d2q9(precision, src, a, n_modes, phase, partials, nblocks, stream);
  return cudaErrorInvalidValue;
}

// Records msg as the calling thread's lbfd_last_error() and returns code.
int set_last_error(int code, const std::string &msg);

// Batched step (batch_kernels.cuh): many lattices of one type per launch.
struct BatchMember;
struct BatchStep;
cudaError_t launch_batch_step_d1q3(int precision, void *base, const BatchStep *steps, const int64_t *tile_start,
                                   int nmembers, int64_t ntiles, int passes, int occ, int walk, int vx_max,
                                   int noise_mode, int noise_dist, int grid, cudaStream_t stream);
cudaError_t launch_batch_step_d2q9(int precision, void *base, const BatchStep *steps, const int64_t *tile_start,
                                   int nmembers, int64_t ntiles, int passes, int occ, int walk, int vx_max,
                                   int noise_mode, int noise_dist, int grid, cudaStream_t stream);
cudaError_t launch_batch_step_d3q19(int precision, void *base, const BatchStep *steps, const int64_t *tile_start,
                                    int nmembers, int64_t ntiles, int passes, int occ, int walk, int vx_max,
                                    int noise_mode, int noise_dist, int grid, cudaStream_t stream);
struct BatchParams;
cudaError_t launch_batch_param_d1q3(int precision, void *base, const BatchParams *groups, int ngroups,
                                    const BatchStep *steps, int passes, int occ, int vx_max, int noise_mode,
                                    int noise_dist, cudaStream_t stream);
cudaError_t launch_batch_param_d2q9(int precision, void *base, const BatchParams *groups, int ngroups,
                                    const BatchStep *steps, int passes, int occ, int vx_max, int noise_mode,
                                    int noise_dist, cudaStream_t stream);
cudaError_t launch_batch_param_d3q19(int precision, void *base, const BatchParams *groups, int ngroups,
                                     const BatchStep *steps, int passes, int occ, int vx_max, int noise_mode,
                                     int noise_dist, cudaStream_t stream);
int batch_blocks_per_sm_d1q3(int precision, int occ, int vx_max, int walk, int noise_mode, int noise_dist);
int batch_blocks_per_sm_d2q9(int precision, int occ, int vx_max, int walk, int noise_mode, int noise_dist);
int batch_blocks_per_sm_d3q19(int precision, int occ, int vx_max, int walk, int noise_mode, int noise_dist);

// batch.cu: lattice dispatch of the above, the per-launch argument kernel
// and the tile assignment.  walk: 0 = a block of the persistent grid takes
// every grid-th tile, 1 = one run of consecutive tiles, 2 = one block per
// tile (grid ignored); vx_max: the largest sites
// per item of any member (1 selects a kernel without the two-site path).
cudaError_t launch_batch_step(int lattice, int precision, void *base, const BatchStep *steps, const int64_t *tile_start,
                              int nmembers, int64_t ntiles, int passes, int occ, int walk, int vx_max, int noise_mode,
                              int noise_dist, int grid, cudaStream_t stream);
// One launch per group of at most kParamMembers members, their arguments in
// the kernel parameters (tile order 3); steps holds k_batch_prep's output.
cudaError_t launch_batch_param(int lattice, int precision, void *base, const BatchParams *groups, int ngroups,
                               const BatchStep *steps, int passes, int occ, int vx_max, int noise_mode, int noise_dist,
                               cudaStream_t stream);
int batch_blocks_per_sm(int lattice, int precision, int occ, int vx_max, int walk, int noise_mode, int noise_dist);
// Step arguments of members[0..n) for the clock *clock_dev (clock when null).
cudaError_t launch_batch_prep(const BatchMember *members, int n, const uint64_t *clock_dev, uint64_t clock,
                              int noise_mode, int noise_dist, BatchStep *out, cudaStream_t stream);
// clock += 1 on the device (between the launches of a captured graph).
cudaError_t launch_clock_advance(uint64_t *clock_dev, cudaStream_t stream);

// Records n launches of this library's kernels (lbfd_kernel_launches).
void count_launches(int64_t n);

// Host copy of the moment matrix the kernels use, m[a*Q + i].
int basis_table(int lattice, double *m);
int lattice_table(int lattice, int *Q, int *D, int *v, double *w);

}  // namespace lbfd
