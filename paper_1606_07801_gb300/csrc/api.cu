// C ABI of the library (declared in include/lbfd.h): argument checks, device
// memory, the step loop and the reductions.  No torch types cross it.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "internal.h"
#include "lbfd.h"

using namespace lbfd;

namespace {

thread_local std::string g_err;
std::atomic<int64_t> g_launches{0};

int fail(int code, const std::string &msg) {
  g_err = msg;
  return code;
}

int cuda_fail(const char *what, cudaError_t e) {
  // the runtime keeps a failed call's error as the thread's last error;
  // clear it so that the next launch check does not report it again
  (void)cudaGetLastError();
  return fail(e == cudaErrorMemoryAllocation ? LBFD_ENOMEM : LBFD_ECUDA,
              std::string(what) + ": " + cudaGetErrorName(e) + " (" + cudaGetErrorString(e) + ")");
}

#define LBFD_CU(call)                                 \
  do {                                                \
    cudaError_t e_ = (call);                          \
    if (e_ != cudaSuccess) return cuda_fail(#call, e_); \
  } while (0)

// Makes a device current for the scope of an entry point, then restores.
struct DeviceGuard {
  int prev = -1;
  bool ok = true;
  explicit DeviceGuard(int dev) {
    if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
    if (dev >= 0 && dev != prev) ok = cudaSetDevice(dev) == cudaSuccess;
  }
  ~DeviceGuard() {
    int cur = -1;
    if (prev >= 0 && cudaGetDevice(&cur) == cudaSuccess && cur != prev) cudaSetDevice(prev);
  }
};

int lattice_dims(int lattice) { return lattice == LBFD_D1Q3 ? 1 : (lattice == LBFD_D3Q19 ? 3 : 2); }
int lattice_q(int lattice) {
  return lattice == LBFD_D1Q3 ? 3 : (lattice == LBFD_D2Q9 ? 9 : (lattice == LBFD_D2Q5 ? 5 : 19));
}

}  // namespace

int lbfd::set_last_error(int code, const std::string &msg) { return fail(code, msg); }

void lbfd::count_launches(int64_t n) { g_launches.fetch_add(n, std::memory_order_relaxed); }

struct lbfd_sim {
  lbfd_options opt{};
  int Q = 0, D = 0, elem = 0;
  int64_t N = 0;
  void *f[2] = {nullptr, nullptr};
  bool owns_f = false;
  int cur = 0;
  int64_t t = 0;
  cudaStream_t stream = nullptr;
  int device = 0;
  double *partials = nullptr;  // reduction scratch, kReduceBlocks x obs_quantities
  double *acc = nullptr;       // observable accumulators
  int acc_n = 0;
  double *d_mass = nullptr;
  double *fin = nullptr;  // stage-2 scratch of the FP32 observables (totals and a ticket word)
  // stage 2 of a sampled step runs on a side stream, overlapping the next
  // steps; ev_obs marks its end, and obs_pending says that the handle's own
  // stream has not waited for it yet (obs_join)
  cudaStream_t obs_stream = nullptr;
  cudaEvent_t ev_sampled = nullptr, ev_obs = nullptr;
  bool obs_pending = false;
  double *mom = nullptr;  // rho and j for lbfd_moments, allocated on first use
  int64_t n_samples = 0;
  int32_t modes_host[LBFD_MAX_MODES][3] = {};
  void *phase = nullptr;  // per-axis structure-factor factors (FP32 sampling), or null
  // moment-space (multiple-relaxation-time) kernel: taken for D2Q5 and when
  // any tau^a differs from tau; tables of the lattice at its theta
  bool mrt = false;
  double w[LBFD_MAX_Q] = {}, m[LBFD_MAX_Q * LBFD_MAX_Q] = {}, tau_m[LBFD_MAX_Q] = {};
  // status word of the staged kernel's bounded waits: pinned host memory
  // mapped into the device, so the host reads it after a sync without a copy
  int *status_host = nullptr;
  int *status_dev = nullptr;
  bool staged_ok = false;  // the lattice and buffers meet the staged kernel's requirements
  bool alt_sweep = true;  // one-launch-per-step kernels sweep every other step in reverse (sweep_default)
  // the stored lattice: dims itself, or for a slab its n owned planes plus
  // a halo plane on each side along the slowest axis
  int32_t sd[3] = {1, 1, 1};
  int64_t NS = 0;     // stored sites (N for a whole lattice)
  bool slab = false;
  int64_t plane = 0;  // sites of one plane along the slowest axis (slabs)
};

static int slow_axis_of(int lattice) { return lattice == LBFD_D3Q19 ? 2 : (lattice == LBFD_D2Q9 ? 1 : 0); }

// LBFD_ETIMEOUT if a staged step kernel recorded a wait that gave up (call
// after a stream synchronisation); clears the word.
static int check_status(lbfd_sim *h) {
  if (!h->status_host) return LBFD_OK;
  volatile int *st = h->status_host;
  const int v = *st;
  if (v == 0) return LBFD_OK;
  *st = 0;
  return fail(LBFD_ETIMEOUT, "a bounded wait of the staged step kernel gave up (status " + std::to_string(v) +
                                 "); the state is not valid");
}

// The handle stores the post-collision populations g of the last step (the
// pull kernel's natural state).  The paper's f(x, t) is g streamed once.
// These helpers convert through the spare buffer, which the next step
// overwrites anyway.
static cudaError_t materialize_f(lbfd_sim *h) {
  const lbfd_options &o = h->opt;
  return launch_shift(o.lattice, h->elem, h->f[h->cur], h->f[h->cur ^ 1], h->sd[0], h->sd[1], h->sd[2], +1,
                      h->stream);
}

static cudaError_t store_f_from_spare(lbfd_sim *h) {
  const lbfd_options &o = h->opt;
  return launch_shift(o.lattice, h->elem, h->f[h->cur ^ 1], h->f[h->cur], h->sd[0], h->sd[1], h->sd[2], -1,
                      h->stream);
}

// Host conversion between FP64 populations and the storage format (16-bit
// formats hold f_i - w_i rho_mean).
template <typename S>
static void decode_host(const S *raw, double *f, int lattice, int64_t N, double rho_mean) {
  int Q = 0, D = 0, v[LBFD_MAX_Q * 3];
  double w[LBFD_MAX_Q];
  lattice_table(lattice, &Q, &D, v, w);
  for (int i = 0; i < Q; ++i)
    for (int64_t s = 0; s < N; ++s) f[i * N + s] = Store<S>::getd(raw[i * N + s], w[i] * rho_mean);
}
template <typename S>
static void encode_host(const double *f, S *raw, int lattice, int64_t N, double rho_mean) {
  int Q = 0, D = 0, v[LBFD_MAX_Q * 3];
  double w[LBFD_MAX_Q];
  lattice_table(lattice, &Q, &D, v, w);
  for (int i = 0; i < Q; ++i)
    for (int64_t s = 0; s < N; ++s) raw[i * N + s] = Store<S>::putd(f[i * N + s], w[i] * rho_mean);
}

extern "C" {

int lbfd_options_init(lbfd_options *o) {
  if (!o) return fail(LBFD_EINVAL, "lbfd_options_init: null options");
  std::memset(o, 0, sizeof(*o));
  o->lattice = LBFD_D2Q9;
  o->precision = LBFD_F32;
  o->noise_mode = LBFD_NOISE_LOCAL;
  o->noise_dist = LBFD_GAUSSIAN;
  o->init = LBFD_INIT_UNIFORM;
  o->device = -1;
  o->dims[0] = o->dims[1] = o->dims[2] = 1;
  o->tau = 1.0;
  o->rho_mean = 1.0;
  o->seed = 1;
  return LBFD_OK;
}

static int validate(const lbfd_options *o) {
  if (o->lattice < LBFD_D1Q3 || o->lattice > LBFD_D2Q5) return fail(LBFD_EINVAL, "unknown lattice");
  if (o->precision < LBFD_F32 || o->precision > LBFD_F32_BF16) return fail(LBFD_EINVAL, "unknown precision");
  if (o->noise_mode < LBFD_NOISE_LOCAL || o->noise_mode > LBFD_NOISE_OFF)
    return fail(LBFD_EINVAL, "unknown noise mode");
  if (o->noise_dist != LBFD_GAUSSIAN && o->noise_dist != LBFD_UNIFORM)
    return fail(LBFD_EINVAL, "unknown noise distribution");
  if (o->init < LBFD_INIT_UNIFORM || o->init > LBFD_INIT_NONE) return fail(LBFD_EINVAL, "unknown init");
  const int D = lattice_dims(o->lattice);
  for (int a = 0; a < 3; ++a) {
    if (o->dims[a] < 1) return fail(LBFD_EINVAL, "every dimension must be >= 1");
    if (a >= D && o->dims[a] != 1) return fail(LBFD_EINVAL, "dimensions beyond the lattice's D must be 1");
  }
  if (o->dims[0] > 0x7fffffffLL) return fail(LBFD_EINVAL, "Lx too large");
  if (o->dims[1] > 65535 || o->dims[2] > 65535) return fail(LBFD_EINVAL, "Ly and Lz must be <= 65535");
  const double n = double(o->dims[0]) * double(o->dims[1]) * double(o->dims[2]);
  if (n >= 2147483648.0) return fail(LBFD_EINVAL, "lattice has 2^31 sites or more");
  if (!(o->tau > 0.5) || !std::isfinite(o->tau)) return fail(LBFD_EINVAL, "tau must be a finite number > 1/2");
  if (!(o->rho_mean >= 0.0) || !std::isfinite(o->rho_mean))
    return fail(LBFD_EINVAL, "rho_mean must be finite and >= 0");
  if (!std::isfinite(o->sine_amp)) return fail(LBFD_EINVAL, "sine_amp must be finite");
  if (o->n_modes < 0 || o->n_modes > LBFD_MAX_MODES) return fail(LBFD_EINVAL, "n_modes out of range");
  if ((o->f_dev[0] == nullptr) != (o->f_dev[1] == nullptr))
    return fail(LBFD_EINVAL, "give both f_dev buffers or neither");
  if (o->lattice == LBFD_D2Q5) {
    if (!(o->theta == 0.0 || (o->theta > 0.0 && o->theta < 0.5)))
      return fail(LBFD_EINVAL, "theta of D2Q5 must be in (0, 1/2) (or 0 for 1/3)");
  } else if (!(o->theta == 0.0 || std::fabs(o->theta - 1.0 / 3.0) < 1e-15)) {
    return fail(LBFD_EINVAL, "theta is 1/3 for D1Q3, D2Q9 and D3Q19");
  }
  bool mrt = o->lattice == LBFD_D2Q5;
  for (int a = 1; a < lattice_q(o->lattice); ++a) {
    const double ta = o->tau_moments[a];
    if (ta == 0.0 || ta == o->tau) continue;
    if (!(ta > 0.5) || !std::isfinite(ta)) return fail(LBFD_EINVAL, "tau_moments entries must be 0 or finite > 1/2");
    mrt = true;
  }
  if (mrt && o->precision != LBFD_F32 && o->precision != LBFD_F64)
    return fail(LBFD_ENOTSUP, "D2Q5 and multiple relaxation times need FP32 or FP64 storage");
  if (mrt && double(lattice_q(o->lattice)) * n > 4294967295.0)
    return fail(LBFD_ENOTSUP, "D2Q5 and multiple relaxation times need Q * sites < 2^32");
  if (o->f_dev[0] && o->f_dev[0] == o->f_dev[1]) return fail(LBFD_EINVAL, "the two f_dev buffers must differ");
  if (o->step_kernel != LBFD_KERNEL_AUTO && o->step_kernel != LBFD_KERNEL_VEC &&
      o->step_kernel != LBFD_KERNEL_SCALAR && o->step_kernel != LBFD_KERNEL_STAGED)
    return fail(LBFD_EINVAL,
                "step_kernel must be LBFD_KERNEL_AUTO, LBFD_KERNEL_VEC, LBFD_KERNEL_SCALAR or LBFD_KERNEL_STAGED");
  if (o->step_kernel != LBFD_KERNEL_AUTO && mrt)
    return fail(LBFD_EINVAL, "D2Q5 and multiple relaxation times run the moment-space kernel only");
  if (o->wait_test_bytes < 0 || o->wait_test_bytes >= (1 << 20))
    return fail(LBFD_EINVAL, "wait_test_bytes must be in [0, 2^20)");
  if (o->wait_test_bytes != 0 && o->step_kernel != LBFD_KERNEL_STAGED)
    return fail(LBFD_EINVAL, "wait_test_bytes needs step_kernel = LBFD_KERNEL_STAGED");
  if (o->slab_global != 0) {
    if (o->lattice != LBFD_D2Q9 && o->lattice != LBFD_D3Q19)
      return fail(LBFD_EINVAL, "slabs are cut along y (D2Q9) or z (D3Q19)");
    const int ax = slow_axis_of(o->lattice);
    if (o->slab_global < 1 || o->slab_first < 0 || o->slab_first + o->dims[ax] > o->slab_global)
      return fail(LBFD_EINVAL, "slab planes must lie within [0, slab_global)");
    if (o->dims[ax] + 2 > 65535) return fail(LBFD_EINVAL, "a slab stores its planes plus two: at most 65535");
    if (mrt) return fail(LBFD_EINVAL, "slabs run single relaxation on D2Q9 / D3Q19");
    if (o->step_kernel != LBFD_KERNEL_AUTO && o->step_kernel != LBFD_KERNEL_STAGED)
      return fail(LBFD_EINVAL, "slabs run the staged kernel");
  } else if (o->slab_first != 0) {
    return fail(LBFD_EINVAL, "slab_first needs slab_global > 0");
  }
  if (o->sample_every < 0) return fail(LBFD_EINVAL, "sample_every must be >= 0");
  if (o->sample_every > 0 && o->slab_global > 0) return fail(LBFD_EINVAL, "slab handles do not sample");
  for (int k = 0; k < 3; ++k)
    if (o->reserved[k] != 0) return fail(LBFD_EINVAL, "reserved option fields must be 0");
  return LBFD_OK;
}

// Whether the library's own choice takes the staged kernel where it can run.
// On GB300 the register-pull kernel is faster for every lattice (both run
// about the same instructions per site, and the staged kernel's producer
// warp and copies cost a few per cent), so the default is off;
// LBFD_STEP_STAGED = 1 turns it on (a tuning knob; results do not depend on
// the kernel).
static bool staged_default() {
  static const bool v = [] {
    const char *e = getenv("LBFD_STEP_STAGED");
    return e && atoi(e) == 1;
  }();
  return v;
}

// The kernel lbfd_step(h, n) runs.  The small-lattice paths hold many steps
// per launch, so they need n >= 2; otherwise one launch per step.
static int step_path(const lbfd_sim *h, int64_t n) {
  const lbfd_options &o = h->opt;
  if (h->mrt) return LBFD_KERNEL_MRT;
  if (h->slab) return LBFD_KERNEL_STAGED;
  if (n >= 2) {
    const int ctas = small_path_ctas(o.lattice, o.precision, h->N);
    if (ctas == 1) return LBFD_KERNEL_SMALL;
    if (ctas > 1) return LBFD_KERNEL_CLUSTER;
  }
  if (o.step_kernel != LBFD_KERNEL_AUTO) return o.step_kernel;
  if (h->staged_ok && staged_default()) return LBFD_KERNEL_STAGED;
  return step_vec_width(o.lattice, o.precision, int32_t(o.dims[0])) >= 2 ? LBFD_KERNEL_VEC : LBFD_KERNEL_SCALAR;
}

static void free_sim(lbfd_sim *h) {
  if (!h) return;
  if (h->owns_f) {
    cudaFree(h->f[0]);
    cudaFree(h->f[1]);
  }
  cudaFree(h->partials);
  cudaFree(h->phase);
  cudaFree(h->acc);
  cudaFree(h->d_mass);
  cudaFree(h->fin);
  cudaFree(h->mom);
  if (h->status_host) cudaFreeHost(h->status_host);
  if (h->ev_sampled) cudaEventDestroy(h->ev_sampled);
  if (h->ev_obs) cudaEventDestroy(h->ev_obs);
  if (h->obs_stream) cudaStreamDestroy(h->obs_stream);
  delete h;
}

// Whether the one-launch-per-step kernels sweep every other step in reverse
// (StepArgs::sweep): a step that starts where the previous one ended reads
// from L2 the part of the state that is still there.  Measured on GB300:
// D2Q9 2048^2 FP32 (151 MB per buffer against 126 MB of L2) 83.7 -> 86.0
// GLUPS; D3Q19 256^3 (1.27 GB) and its FP16 form unchanged within 0.2%.  On
// by default; LBFD_STEP_SWEEP = 0 turns it off (a tuning knob: results do not
// depend on it).
static bool sweep_default() {
  const char *e = getenv("LBFD_STEP_SWEEP");
  return !(e && atoi(e) == 0);
}

// The handle's stream waits for the last sampled step's stage 2 (before
// anything that reads or rewrites the observable scratch or accumulators).
static cudaError_t obs_join(lbfd_sim *h) {
  if (!h->obs_pending) return cudaSuccess;
  h->obs_pending = false;
  return cudaStreamWaitEvent(h->stream, h->ev_obs, 0);
}

int lbfd_create_ex(lbfd_t *out, const lbfd_options *opt) {
  if (!out || !opt) return fail(LBFD_EINVAL, "lbfd_create_ex: null argument");
  *out = nullptr;
  int rc = validate(opt);
  if (rc) return rc;
  int dev = opt->device;
  if (dev < 0) LBFD_CU(cudaGetDevice(&dev));
  DeviceGuard g(dev);
  if (!g.ok) return fail(LBFD_ECUDA, "cannot make device current");
  lbfd_sim *h = new (std::nothrow) lbfd_sim();
  if (!h) return fail(LBFD_ENOMEM, "host allocation failed");
  h->opt = *opt;
  h->device = dev;
  h->Q = lattice_q(opt->lattice);
  h->D = lattice_dims(opt->lattice);
  h->N = opt->dims[0] * opt->dims[1] * opt->dims[2];
  for (int a = 0; a < 3; ++a) h->sd[a] = int32_t(opt->dims[a]);
  h->slab = opt->slab_global > 0;
  if (h->slab) {
    const int ax = slow_axis_of(opt->lattice);
    h->sd[ax] += 2;
    h->plane = ax == 1 ? opt->dims[0] : opt->dims[0] * opt->dims[1];
  }
  h->NS = int64_t(h->sd[0]) * h->sd[1] * h->sd[2];
  h->elem = storage_bytes(opt->precision);
  h->stream = static_cast<cudaStream_t>(opt->stream);
  for (int m = 0; m < opt->n_modes; ++m)
    for (int k = 0; k < 3; ++k) h->modes_host[m][k] = opt->modes[m][k];
  // tables of the lattice at its theta, and the relaxation time of each moment
  if (opt->lattice == LBFD_D2Q5) {
    d2q5_tables(opt->theta == 0.0 ? 1.0 / 3.0 : opt->theta, h->w, h->m);
  } else {
    int q = 0, d = 0, v[LBFD_MAX_Q * 3];
    lattice_table(opt->lattice, &q, &d, v, h->w);
    basis_table(opt->lattice, h->m);
  }
  h->mrt = opt->lattice == LBFD_D2Q5;
  for (int a = 0; a < h->Q; ++a) {
    const double ta = opt->tau_moments[a];
    h->tau_m[a] = (a == 0 || ta == 0.0) ? opt->tau : ta;
    if (a > 0 && h->tau_m[a] != opt->tau) h->mrt = true;
  }
  const size_t fbytes = size_t(h->Q) * size_t(h->NS) * size_t(h->elem);
  cudaError_t e = cudaSuccess;
  if (opt->f_dev[0]) {
    h->f[0] = opt->f_dev[0];
    h->f[1] = opt->f_dev[1];
    h->owns_f = false;
  } else {
    h->owns_f = true;
    e = cudaMalloc(&h->f[0], fbytes);
    if (e == cudaSuccess) e = cudaMalloc(&h->f[1], fbytes);
  }
  if (e == cudaSuccess) e = cudaHostAlloc(reinterpret_cast<void **>(&h->status_host), sizeof(int), cudaHostAllocMapped);
  if (e == cudaSuccess) {
    *h->status_host = 0;
    e = cudaHostGetDevicePointer(reinterpret_cast<void **>(&h->status_dev), h->status_host, 0);
  }
  h->alt_sweep = sweep_default();
  if (e == cudaSuccess) {
    h->staged_ok = !h->mrt && staged_fits(opt->lattice, opt->precision, opt->dims[0], h->NS, h->f[0], h->f[1]);
    if (h->slab && !h->staged_ok) {
      free_sim(h);
      return fail(LBFD_ENOTSUP, "slab handles run the staged kernel: Lx * (bytes per value) must be a multiple "
                                "of 16 and the buffers 16-byte aligned");
    }
    if (opt->step_kernel == LBFD_KERNEL_STAGED && !h->staged_ok) {
      free_sim(h);
      return fail(LBFD_EINVAL, "LBFD_KERNEL_STAGED needs Lx * (bytes per value) to be a multiple of 16 and "
                               "16-byte aligned buffers");
    }
    if (opt->step_kernel == LBFD_KERNEL_VEC && opt->dims[0] % 2 != 0) {
      free_sim(h);
      return fail(LBFD_EINVAL, "LBFD_KERNEL_VEC needs an even Lx");
    }
  }
  h->acc_n = 2 + h->Q + h->Q * h->Q + LBFD_MAX_MODES;
  if (e == cudaSuccess)
    e = cudaMalloc(&h->partials, sizeof(double) * size_t(std::max(kReduceBlocks, kObsBlocks)) *
                                     obs_quantities(h->Q, LBFD_MAX_MODES));
  if (e == cudaSuccess) e = cudaMalloc(&h->acc, sizeof(double) * h->acc_n);
  if (e == cudaSuccess) e = cudaMalloc(&h->d_mass, sizeof(double));
  const size_t fin_n = size_t(obs_quantities(h->Q, LBFD_MAX_MODES)) + 1;
  if (e == cudaSuccess) e = cudaMalloc(&h->fin, sizeof(double) * fin_n);
  if (e == cudaSuccess) e = cudaMemsetAsync(h->fin, 0, sizeof(double) * fin_n, h->stream);
  // the structure-factor phases of FP32 sampling as per-axis tables (when
  // small), over the stored lattice; a slab's stored plane c is global plane
  // slab_first - 1 + c of slab_global
  const size_t nphase = obs_phase_values(opt->n_modes, h->sd[0], h->sd[1], h->sd[2]);
  if (e == cudaSuccess && opt->precision != LBFD_F64 && nphase > 0 && nphase <= (size_t(1) << 22)) {
    std::vector<float> tab(2 * nphase);
    int64_t period[3] = {h->sd[0], h->sd[1], h->sd[2]}, offset[3] = {0, 0, 0};
    if (h->slab) {
      const int ax = slow_axis_of(opt->lattice);
      period[ax] = opt->slab_global;
      offset[ax] = opt->slab_first - 1;
    }
    obs_phase_fill(opt->n_modes, &h->modes_host[0][0], h->sd[0], h->sd[1], h->sd[2], tab.data(), period, offset);
    e = cudaMalloc(&h->phase, sizeof(float) * tab.size());
    if (e == cudaSuccess) e = cudaMemcpy(h->phase, tab.data(), sizeof(float) * tab.size(), cudaMemcpyHostToDevice);
  }
  if (e == cudaSuccess) e = cudaMemsetAsync(h->acc, 0, sizeof(double) * h->acc_n, h->stream);
  if (e == cudaSuccess && opt->init != LBFD_INIT_NONE) {
    // f(x, 0) into the spare buffer, then stored as g = f shifted back
    const double amp = opt->init == LBFD_INIT_SINE ? opt->sine_amp : 0.0;
    // a slab's stored plane c is global plane slab_first - 1 + c (the halo
    // planes take their neighbours' values, so the owned planes un-stream
    // correctly)
    int32_t off[3] = {0, 0, 0}, len[3] = {int32_t(opt->dims[0]), int32_t(opt->dims[1]), int32_t(opt->dims[2])};
    if (h->slab) {
      const int ax = slow_axis_of(opt->lattice);
      off[ax] = opt->slab_first - 1;
      len[ax] = opt->slab_global;
    }
    e = launch_init(opt->lattice, opt->precision, h->f[1], h->sd[0], h->sd[1], h->sd[2], opt->rho_mean, amp,
                    opt->sine_k, h->stream, h->w, off, len);
    if (e == cudaSuccess) e = store_f_from_spare(h);
  }
  if (e != cudaSuccess) {
    rc = cuda_fail("lbfd_create_ex", e);
    free_sim(h);
    return rc;
  }
  *out = h;
  return LBFD_OK;
}

int lbfd_create(lbfd_t *out, int32_t lattice, const int64_t *dims, double tau, double rho_mean, uint64_t seed) {
  if (!out || !dims) return fail(LBFD_EINVAL, "lbfd_create: null argument");
  if (lattice < LBFD_D1Q3 || lattice > LBFD_D2Q5) return fail(LBFD_EINVAL, "unknown lattice");
  lbfd_options o;
  lbfd_options_init(&o);
  o.lattice = lattice;
  const int D = lattice_dims(lattice);
  for (int a = 0; a < D; ++a) o.dims[a] = dims[a];
  o.tau = tau;
  o.rho_mean = rho_mean;
  o.seed = seed;
  return lbfd_create_ex(out, &o);
}

int lbfd_destroy(lbfd_t h) {
  if (!h) return LBFD_OK;
  DeviceGuard g(h->device);
  cudaError_t e = obs_join(h);
  const cudaError_t e2 = cudaStreamSynchronize(h->stream);
  if (e == cudaSuccess) e = e2;
  free_sim(h);
  if (e != cudaSuccess) return cuda_fail("lbfd_destroy: stream sync", e);
  return LBFD_OK;
}

// The observables of the current state into the accumulators (the body of
// lbfd_sample; a separate pass over the state).
static int sample_now(lbfd_sim *h) {
  const lbfd_options &o = h->opt;
  LBFD_CU(obs_join(h));
  if ((o.lattice == LBFD_D1Q3 || o.lattice == LBFD_D2Q9) && !h->slab &&
      sample_fusable(o.lattice, o.precision, int32_t(o.dims[0]), int32_t(o.dims[1]), int32_t(o.dims[2]), o.n_modes,
                     h->phase)) {
    // FP32 arithmetic, register sampler: the fused step's sampler as a pass
    // of its own over the lattice's register-pull blocks, then stage 2
    StepArgs a{};
    a.Lx = h->sd[0];
    a.Ly = h->sd[1];
    a.Lz = h->sd[2];
    a.N = h->NS;
    fill_step_params(a, o.tau, o.rho_mean);
    int nblocks = 0;
    LBFD_CU(launch_obs_sample(o.lattice, o.precision, h->f[h->cur], a, o.n_modes, h->phase, h->partials, &nblocks,
                              h->stream));
    LBFD_CU(launch_obs_pull_finalize(o.lattice, h->partials, nblocks, o.n_modes, h->N, o.rho_mean, h->fin, h->acc,
                                     h->stream));
    g_launches.fetch_add(2, std::memory_order_relaxed);
  } else if (o.precision != LBFD_F64 && h->N < (int64_t(1) << 31)) {
    // FP32 arithmetic: pulled straight from the stored state
    LBFD_CU(launch_observables_pull(o.lattice, o.precision, h->f[h->cur], int32_t(o.dims[0]), int32_t(o.dims[1]),
                                    int32_t(o.dims[2]), o.rho_mean, o.n_modes, &h->modes_host[0][0], h->phase,
                                    h->partials, h->fin, h->acc, h->stream));
    g_launches.fetch_add(2, std::memory_order_relaxed);
  } else {
    // FP64 storage: FP64 throughout, on the streamed copy of the state
    LBFD_CU(materialize_f(h));
    LBFD_CU(launch_observables(o.lattice, o.precision, h->f[h->cur ^ 1], int32_t(o.dims[0]), int32_t(o.dims[1]),
                               int32_t(o.dims[2]), o.rho_mean, o.n_modes, &h->modes_host[0][0], h->partials, h->acc,
                               h->stream));
    g_launches.fetch_add(3, std::memory_order_relaxed);
  }
  h->n_samples += 1;
  return LBFD_OK;
}

// Steps until the next sampled step counter (t itself if it is sampled).
static int64_t steps_to_sample(const lbfd_sim *h, int64_t t) {
  const int64_t s = h->opt.sample_every;
  return s > 0 ? (s - t % s) % s : INT64_MAX;
}

int lbfd_step(lbfd_t h, int64_t n) {
  NvtxRange nvtx_("lbfd_step");
  if (!h) return fail(LBFD_EINVAL, "lbfd_step: null handle");
  if (n < 0) return fail(LBFD_EINVAL, "lbfd_step: n must be >= 0");
  if (n == 0) return LBFD_OK;
  if (h->slab && n > 1)
    return fail(LBFD_EINVAL, "lbfd_step: a slab takes one step per call (its halo planes are filled between steps)");
  DeviceGuard g(h->device);
  const lbfd_options &o = h->opt;
  StepArgs a{};
  a.Lx = h->sd[0];
  a.Ly = h->sd[1];
  a.Lz = h->sd[2];
  a.N = h->NS;
  // rows updated and their keys: a slab skips its halo planes and keys its
  // rows by their global position
  StagedRows rows{0, uint32_t(h->sd[1]) * uint32_t(h->sd[2]), 0};
  if (h->slab) {
    const uint32_t rpp = uint32_t(h->plane / h->sd[0]);  // rows per plane
    const int ax = slow_axis_of(o.lattice);
    rows.row_begin = rpp;
    rows.nrows = rpp * uint32_t(o.dims[ax]);
    rows.row_key = rpp * uint32_t(o.slab_first) - rpp;
  }
  fill_step_params(a, o.tau, o.rho_mean);
  a.noise_mode = o.noise_mode;
  a.noise_dist = o.noise_dist;
  const int path = step_path(h, n);
  if (path == LBFD_KERNEL_SMALL || path == LBFD_KERNEL_CLUSTER) {
    // a small lattice: many steps per launch in shared memory (bit-identical);
    // chunks end at the sampled steps, which sample by the separate pass
    constexpr int64_t kChunk = 4096;
    int64_t launches = 0, done = 0;
    bool placed = true;
    while (done < n) {
      if (steps_to_sample(h, h->t) == 0) {
        int rc = sample_now(h);
        if (rc) return rc;
      }
      int64_t until = steps_to_sample(h, h->t);
      if (until == 0) until = h->opt.sample_every;
      const int chunk = int(std::min<int64_t>(std::min<int64_t>(kChunk, n - done), until));
      const int to = h->cur ^ (chunk & 1);
      a.ph = make_philox_step(o.seed, o.lattice_id, uint64_t(h->t));
      cudaError_t e = launch_step_small(o.lattice, o.precision, h->f[h->cur], h->f[to], a, o.seed, o.lattice_id,
                                        uint64_t(h->t), chunk, h->stream);
      if (e == cudaErrorNotSupported) {
        // the cluster cannot be placed on this GPU: one launch per step instead
        (void)cudaGetLastError();
        placed = false;
        break;
      }
      if (e != cudaSuccess) return cuda_fail("lbfd_step: launch", e);
      h->cur = to;
      h->t += chunk;
      done += chunk;
      launches += 1;
    }
    g_launches.fetch_add(launches, std::memory_order_relaxed);
    if (placed) return LBFD_OK;
    n -= done;
  }
  const int kernel = step_path(h, 1);
  int vec_width = 1;
  if (kernel == LBFD_KERNEL_VEC) {
    vec_width = step_vec_width(o.lattice, o.precision, a.Lx);
    if (vec_width == 1) vec_width = 2;  // asked for by step_kernel: Lx is even
  }
  const bool fusable = o.sample_every > 0 && !h->mrt &&
                       sample_fusable(o.lattice, o.precision, a.Lx, a.Ly, a.Lz, o.n_modes, h->phase);
  int64_t extra = 0;  // launches besides one step kernel per step
  for (int64_t k = 0; k < n; ++k) {
    a.ph = make_philox_step(o.seed, o.lattice_id, uint64_t(h->t));
    a.sweep = h->alt_sweep ? static_cast<int32_t>(h->t & 1) : 0;
    const void *src = h->f[h->cur];
    void *dst = h->f[h->cur ^ 1];
    if (steps_to_sample(h, h->t) == 0) {
      if (fusable) {
        // the step and the observables of the state it reads in one pass,
        // then stage 2 of the observables on the side stream
        cudaError_t e = obs_join(h);
        int nblocks = 0;
        if (e == cudaSuccess)
          e = launch_step_sample(o.lattice, o.precision, src, dst, a, o.n_modes, h->phase, h->partials, &nblocks,
                                 h->staged_ok, h->status_dev, h->stream);
        if (e == cudaSuccess && !h->obs_stream) {
          e = cudaStreamCreateWithFlags(&h->obs_stream, cudaStreamNonBlocking);
          if (e == cudaSuccess) e = cudaEventCreateWithFlags(&h->ev_sampled, cudaEventDisableTiming);
          if (e == cudaSuccess) e = cudaEventCreateWithFlags(&h->ev_obs, cudaEventDisableTiming);
        }
        if (e == cudaSuccess) e = cudaEventRecord(h->ev_sampled, h->stream);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(h->obs_stream, h->ev_sampled, 0);
        if (e == cudaSuccess)
          e = launch_obs_pull_finalize(o.lattice, h->partials, nblocks, o.n_modes, h->N, o.rho_mean, h->fin, h->acc,
                                       h->obs_stream);
        if (e == cudaSuccess) e = cudaEventRecord(h->ev_obs, h->obs_stream);
        if (e != cudaSuccess) return cuda_fail("lbfd_step: sampled step", e);
        h->obs_pending = true;
        h->n_samples += 1;
        h->cur ^= 1;
        h->t += 1;
        extra += 1;
        continue;
      }
      int rc = sample_now(h);
      if (rc) return rc;
    }
    cudaError_t e =
        kernel == LBFD_KERNEL_MRT ? launch_step_mrt(o.lattice, o.precision, src, dst, a, h->m, h->w, h->tau_m, h->stream)
        : kernel == LBFD_KERNEL_STAGED ? launch_step_staged(o.lattice, o.precision, src, dst, a, rows, h->status_dev,
                                                            uint32_t(o.wait_test_bytes), h->stream)
                                       : launch_step(o.lattice, o.precision, src, dst, a, h->stream, vec_width);
    if (e != cudaSuccess) return cuda_fail("lbfd_step: launch", e);
    h->cur ^= 1;
    h->t += 1;
  }
  g_launches.fetch_add(n + extra, std::memory_order_relaxed);
  return LBFD_OK;
}

int lbfd_set_sample_every(lbfd_t h, int32_t every) {
  if (!h || every < 0) return fail(LBFD_EINVAL, "lbfd_set_sample_every: null handle or every < 0");
  if (h->slab && every > 0) return fail(LBFD_EINVAL, "lbfd_set_sample_every: slab handles do not sample");
  h->opt.sample_every = every;
  return LBFD_OK;
}

int lbfd_step_kernel(lbfd_t h, int64_t n, int32_t *kernel) {
  if (!h || !kernel || n < 0) return fail(LBFD_EINVAL, "lbfd_step_kernel: bad argument");
  *kernel = step_path(h, n);
  return LBFD_OK;
}

int lbfd_sync(lbfd_t h) {
  if (!h) return fail(LBFD_EINVAL, "lbfd_sync: null handle");
  DeviceGuard g(h->device);
  LBFD_CU(obs_join(h));
  LBFD_CU(cudaStreamSynchronize(h->stream));
  return check_status(h);
}

int lbfd_get_t(lbfd_t h, int64_t *t) {
  if (!h || !t) return fail(LBFD_EINVAL, "lbfd_get_t: null argument");
  *t = h->t;
  return LBFD_OK;
}

int lbfd_set_t(lbfd_t h, int64_t t) {
  if (!h || t < 0) return fail(LBFD_EINVAL, "lbfd_set_t: null handle or negative t");
  h->t = t;
  return LBFD_OK;
}

int lbfd_get_f_raw(lbfd_t h, void *f_host) {
  if (!h || !f_host) return fail(LBFD_EINVAL, "lbfd_get_f_raw: null argument");
  DeviceGuard g(h->device);
  LBFD_CU(materialize_f(h));
  if (h->slab) {
    // the owned planes of each population (the stored rows between the halo planes)
    const size_t row = size_t(h->N) * h->elem, pitch = size_t(h->NS) * h->elem;
    const char *from = static_cast<const char *>(h->f[h->cur ^ 1]) + size_t(h->plane) * h->elem;
    LBFD_CU(cudaMemcpy2DAsync(f_host, row, from, pitch, row, size_t(h->Q), cudaMemcpyDeviceToHost, h->stream));
  } else {
    LBFD_CU(cudaMemcpyAsync(f_host, h->f[h->cur ^ 1], size_t(h->Q) * h->N * h->elem, cudaMemcpyDeviceToHost,
                            h->stream));
  }
  LBFD_CU(cudaStreamSynchronize(h->stream));
  return check_status(h);
}

int lbfd_set_f_raw(lbfd_t h, const void *f_host) {
  if (!h || !f_host) return fail(LBFD_EINVAL, "lbfd_set_f_raw: null argument");
  DeviceGuard g(h->device);
  // a slab takes its stored planes: the owned ones and both halo planes
  LBFD_CU(cudaMemcpyAsync(h->f[h->cur ^ 1], f_host, size_t(h->Q) * h->NS * h->elem, cudaMemcpyHostToDevice, h->stream));
  LBFD_CU(store_f_from_spare(h));
  LBFD_CU(cudaStreamSynchronize(h->stream));
  return LBFD_OK;
}

int lbfd_get_f(lbfd_t h, double *f_host) {
  if (!h || !f_host) return fail(LBFD_EINVAL, "lbfd_get_f: null argument");
  if (h->opt.precision == LBFD_F64) return lbfd_get_f_raw(h, f_host);
  std::vector<uint8_t> tmp;
  try {
    tmp.resize(size_t(h->Q) * h->N * h->elem);
  } catch (...) {
    return fail(LBFD_ENOMEM, "lbfd_get_f: host staging allocation failed");
  }
  int rc = lbfd_get_f_raw(h, tmp.data());
  if (rc) return rc;
  const lbfd_options &o = h->opt;
  dispatch_storage(o.precision, [&](auto tag) {
    using S = typename decltype(tag)::type;
    decode_host<S>(reinterpret_cast<const S *>(tmp.data()), f_host, o.lattice, h->N, o.rho_mean);
    return cudaSuccess;
  });
  return LBFD_OK;
}

int lbfd_set_f(lbfd_t h, const double *f_host) {
  if (!h || !f_host) return fail(LBFD_EINVAL, "lbfd_set_f: null argument");
  if (h->opt.precision == LBFD_F64) return lbfd_set_f_raw(h, f_host);
  std::vector<uint8_t> tmp;
  try {
    tmp.resize(size_t(h->Q) * h->NS * h->elem);
  } catch (...) {
    return fail(LBFD_ENOMEM, "lbfd_set_f: host staging allocation failed");
  }
  const lbfd_options &o = h->opt;
  dispatch_storage(o.precision, [&](auto tag) {
    using S = typename decltype(tag)::type;
    encode_host<S>(f_host, reinterpret_cast<S *>(tmp.data()), o.lattice, h->NS, o.rho_mean);
    return cudaSuccess;
  });
  return lbfd_set_f_raw(h, tmp.data());
}

// A slab's density and flux: computed over its stored planes into h->mom,
// then the owned planes copied to rho_dev / j_dev (D2D or D2H by kind).
static int slab_moments(lbfd_sim *h, double *rho_out, double *j_out, cudaMemcpyKind kind) {
  const lbfd_options &o = h->opt;
  if (!h->mom) LBFD_CU(cudaMalloc(&h->mom, sizeof(double) * size_t(h->NS) * (1 + h->D)));
  if (!j_out) {
    LBFD_CU(launch_density_of_state(o.lattice, o.precision, h->f[h->cur], h->sd[0], h->sd[1], h->sd[2], o.rho_mean,
                                    h->mom, h->stream));
  } else {
    LBFD_CU(materialize_f(h));
    LBFD_CU(launch_moments(o.lattice, o.precision, h->f[h->cur ^ 1], h->sd[0], h->sd[1], h->sd[2], o.rho_mean, h->mom,
                           h->mom + h->NS, h->stream));
  }
  LBFD_CU(cudaMemcpyAsync(rho_out, h->mom + h->plane, sizeof(double) * h->N, kind, h->stream));
  if (j_out)
    for (int a = 0; a < h->D; ++a)
      LBFD_CU(cudaMemcpyAsync(j_out + a * h->N, h->mom + (1 + a) * h->NS + h->plane, sizeof(double) * h->N, kind,
                              h->stream));
  return LBFD_OK;
}

int lbfd_moments_device(lbfd_t h, double *rho_dev, double *j_dev) {
  if (!h || !rho_dev) return fail(LBFD_EINVAL, "lbfd_moments_device: null argument");
  DeviceGuard g(h->device);
  const lbfd_options &o = h->opt;
  if (h->slab) return slab_moments(h, rho_dev, j_dev, cudaMemcpyDeviceToDevice);
  if (!j_dev) {
    // density only: pulled from the stored state, no streamed copy
    LBFD_CU(launch_density_of_state(o.lattice, o.precision, h->f[h->cur], int32_t(o.dims[0]), int32_t(o.dims[1]),
                                    int32_t(o.dims[2]), o.rho_mean, rho_dev, h->stream));
    return LBFD_OK;
  }
  LBFD_CU(materialize_f(h));
  LBFD_CU(launch_moments(o.lattice, o.precision, h->f[h->cur ^ 1], int32_t(o.dims[0]), int32_t(o.dims[1]),
                         int32_t(o.dims[2]), o.rho_mean, rho_dev, j_dev, h->stream));
  return LBFD_OK;
}

int lbfd_moments(lbfd_t h, double *rho_host, double *j_host) {
  if (!h || !rho_host) return fail(LBFD_EINVAL, "lbfd_moments: null argument");
  DeviceGuard g(h->device);
  if (h->slab) {
    int rc = slab_moments(h, rho_host, j_host, cudaMemcpyDeviceToHost);
    if (rc) return rc;
    LBFD_CU(cudaStreamSynchronize(h->stream));
    return check_status(h);
  }
  if (!h->mom) LBFD_CU(cudaMalloc(&h->mom, sizeof(double) * size_t(h->N) * (1 + h->D)));
  int rc = lbfd_moments_device(h, h->mom, j_host ? h->mom + h->N : nullptr);
  if (rc) return rc;
  LBFD_CU(cudaMemcpyAsync(rho_host, h->mom, sizeof(double) * h->N, cudaMemcpyDeviceToHost, h->stream));
  if (j_host)
    LBFD_CU(cudaMemcpyAsync(j_host, h->mom + h->N, sizeof(double) * h->N * h->D, cudaMemcpyDeviceToHost, h->stream));
  LBFD_CU(cudaStreamSynchronize(h->stream));
  return check_status(h);
}

int lbfd_mass(lbfd_t h, double *mass) {
  if (!h || !mass) return fail(LBFD_EINVAL, "lbfd_mass: null argument");
  DeviceGuard g(h->device);
  const lbfd_options &o = h->opt;
  LBFD_CU(obs_join(h));
  if (h->slab) {
    // the owned planes of the stored state (a permutation of the lattice's
    // values, so the slabs' masses sum to the lattice's)
    const char *f = static_cast<const char *>(h->f[h->cur]) + h->plane * h->elem;
    LBFD_CU(launch_mass(o.lattice, o.precision, f, h->N, o.rho_mean, h->partials, h->d_mass, h->stream, h->NS));
  } else {
    LBFD_CU(launch_mass(o.lattice, o.precision, h->f[h->cur], h->N, o.rho_mean, h->partials, h->d_mass, h->stream));
  }
  LBFD_CU(cudaMemcpyAsync(mass, h->d_mass, sizeof(double), cudaMemcpyDeviceToHost, h->stream));
  LBFD_CU(cudaStreamSynchronize(h->stream));
  return check_status(h);
}

int lbfd_sample(lbfd_t h) {
  if (!h) return fail(LBFD_EINVAL, "lbfd_sample: null handle");
  if (h->slab) return fail(LBFD_ENOTSUP, "lbfd_sample: not offered for slab handles");
  DeviceGuard g(h->device);
  return sample_now(h);
}

int lbfd_reset_obs(lbfd_t h) {
  if (!h) return fail(LBFD_EINVAL, "lbfd_reset_obs: null handle");
  DeviceGuard g(h->device);
  LBFD_CU(obs_join(h));
  LBFD_CU(cudaMemsetAsync(h->acc, 0, sizeof(double) * h->acc_n, h->stream));
  h->n_samples = 0;
  return LBFD_OK;
}

int lbfd_sample_totals(lbfd_t h, double *totals) {
  if (!h || !totals) return fail(LBFD_EINVAL, "lbfd_sample_totals: null argument");
  const lbfd_options &o = h->opt;
  if (o.precision == LBFD_F64) return fail(LBFD_ENOTSUP, "lbfd_sample_totals: FP32-arithmetic formats only");
  if (h->NS >= (int64_t(1) << 31)) return fail(LBFD_ENOTSUP, "lbfd_sample_totals: 2^31 stored sites or more");
  if (h->slab && o.n_modes > 0 && !h->phase)
    return fail(LBFD_ENOTSUP, "lbfd_sample_totals: the slab's phase tables are too large");
  DeviceGuard g(h->device);
  LBFD_CU(obs_join(h));
  // the owned sites: planes 1 .. n of a slab's stored lattice, or all of it
  const int64_t s0 = h->slab ? h->plane : 0;
  int nblocks = 0;
  LBFD_CU(launch_observables_pull_partials(o.lattice, o.precision, h->f[h->cur], h->sd[0], h->sd[1], h->sd[2], s0, h->N,
                                           o.rho_mean, o.n_modes, &h->modes_host[0][0], h->phase, h->partials,
                                           &nblocks, h->stream));
  g_launches.fetch_add(1, std::memory_order_relaxed);
  const int nq = obs_quantities(h->Q, o.n_modes);
  std::vector<double> part(size_t(nblocks) * nq);
  LBFD_CU(cudaMemcpyAsync(part.data(), h->partials, sizeof(double) * part.size(), cudaMemcpyDeviceToHost, h->stream));
  LBFD_CU(cudaStreamSynchronize(h->stream));
  if (int rc = check_status(h)) return rc;
  for (int q = 0; q < nq; ++q) {
    double t = 0.0;
    for (int b = 0; b < nblocks; ++b) t += part[size_t(b) * nq + q];  // block order
    totals[q] = t;
  }
  return LBFD_OK;
}

int lbfd_obs_restore(int32_t lattice, int32_t n_modes, double rho_mean, int64_t n_sites, const double *totals,
                     double *acc_out) {
  if (!totals || !acc_out) return fail(LBFD_EINVAL, "lbfd_obs_restore: null argument");
  if (lattice < LBFD_D1Q3 || lattice > LBFD_D3Q19) return fail(LBFD_EINVAL, "lbfd_obs_restore: D1Q3, D2Q9 or D3Q19");
  if (n_modes < 0 || n_modes > LBFD_MAX_MODES || n_sites < 0 || !(rho_mean >= 0.0))
    return fail(LBFD_EINVAL, "lbfd_obs_restore: bad argument");
  const float rho_f = static_cast<float>(rho_mean);
  return dispatch_lattice(lattice, [&](auto lat) -> cudaError_t {
           constexpr int LAT = decltype(lat)::value;
           constexpr int Q = Lattice<LAT>::Q;
           double cs[Q];
           double C = 0.0;
           for (int i = 0; i < Q; ++i) {
             cs[i] = static_cast<double>(obs_offset<LAT>(i, rho_f));
             C += cs[i];
           }
           const int nacc = 2 + Q + Q * Q + n_modes;
           for (int k = 0; k < nacc; ++k) acc_out[k] = obs_restore<Q>(k, totals, cs, C, double(n_sites), n_modes);
           return cudaSuccess;
         }) == cudaSuccess
             ? LBFD_OK
             : fail(LBFD_EINVAL, "lbfd_obs_restore: unknown lattice");
}

int lbfd_obs_add(lbfd_t h, const double *acc_sample) {
  if (!h || !acc_sample) return fail(LBFD_EINVAL, "lbfd_obs_add: null argument");
  DeviceGuard g(h->device);
  std::vector<double> acc(h->acc_n);
  LBFD_CU(obs_join(h));
  LBFD_CU(cudaMemcpyAsync(acc.data(), h->acc, sizeof(double) * h->acc_n, cudaMemcpyDeviceToHost, h->stream));
  LBFD_CU(cudaStreamSynchronize(h->stream));
  const int nacc = 2 + h->Q + h->Q * h->Q + h->opt.n_modes;
  for (int k = 0; k < nacc; ++k) acc[k] += acc_sample[k];
  LBFD_CU(cudaMemcpyAsync(h->acc, acc.data(), sizeof(double) * h->acc_n, cudaMemcpyHostToDevice, h->stream));
  LBFD_CU(cudaStreamSynchronize(h->stream));
  h->n_samples += 1;
  return check_status(h);
}

int lbfd_observables(lbfd_t h, lbfd_obs *obs) {
  if (!h || !obs) return fail(LBFD_EINVAL, "lbfd_observables: null argument");
  DeviceGuard g(h->device);
  std::vector<double> acc(h->acc_n);
  LBFD_CU(obs_join(h));
  LBFD_CU(cudaMemcpyAsync(acc.data(), h->acc, sizeof(double) * h->acc_n, cudaMemcpyDeviceToHost, h->stream));
  LBFD_CU(cudaStreamSynchronize(h->stream));
  if (int rc = check_status(h)) return rc;
  std::memset(obs, 0, sizeof(*obs));
  obs->t = h->t;
  obs->n_samples = h->n_samples;
  obs->Q = h->Q;
  obs->n_modes = h->opt.n_modes;
  const int Q = h->Q;
  obs->sum_rho = acc[0];
  obs->sum_rho2 = acc[1];
  for (int i = 0; i < Q; ++i) obs->sum_f[i] = acc[2 + i];
  for (int i = 0; i < Q * Q; ++i) obs->sum_ff[i] = acc[2 + Q + i];
  for (int m = 0; m < h->opt.n_modes; ++m) obs->sum_sk[m] = acc[2 + Q + Q * Q + m];
  return LBFD_OK;
}

int lbfd_query(lbfd_t h, int32_t *Q, int32_t *D, int64_t *N, int32_t *value_bytes) {
  if (!h) return fail(LBFD_EINVAL, "lbfd_query: null handle");
  if (Q) *Q = h->Q;
  if (D) *D = h->D;
  if (N) *N = h->N;
  if (value_bytes) *value_bytes = h->elem;
  return LBFD_OK;
}

int lbfd_state_device(lbfd_t h, void **f_dev, void **stream) {
  if (!h) return fail(LBFD_EINVAL, "lbfd_state_device: null handle");
  if (h->obs_pending) {
    DeviceGuard g(h->device);
    LBFD_CU(obs_join(h));  // so that the stream handed out covers all of the handle's work
  }
  if (f_dev) *f_dev = h->f[h->cur];
  if (stream) *stream = static_cast<void *>(h->stream);
  return LBFD_OK;
}

int lbfd_lattice_tables_ex(int32_t lattice, double theta, int32_t *Q, int32_t *v, double *w, double *m) {
  if (lattice < LBFD_D1Q3 || lattice > LBFD_D2Q5) return fail(LBFD_EINVAL, "unknown lattice");
  if (theta == 0.0) theta = 1.0 / 3.0;
  if (lattice == LBFD_D2Q5 ? !(theta > 0.0 && theta < 0.5) : std::fabs(theta - 1.0 / 3.0) > 1e-15)
    return fail(LBFD_EINVAL, "theta out of range for the lattice");
  int q = 0, d = 0;
  int vv[LBFD_MAX_Q * 3];
  double ww[LBFD_MAX_Q], mm[LBFD_MAX_Q * LBFD_MAX_Q];
  lattice_table(lattice, &q, &d, vv, ww);
  if (lattice == LBFD_D2Q5)
    d2q5_tables(theta, ww, mm);
  else
    basis_table(lattice, mm);
  if (Q) *Q = q;
  if (v)
    for (int k = 0; k < 3 * q; ++k) v[k] = vv[k];
  if (w)
    for (int k = 0; k < q; ++k) w[k] = ww[k];
  if (m)
    for (int k = 0; k < q * q; ++k) m[k] = mm[k];
  return LBFD_OK;
}

int lbfd_lattice_tables(int32_t lattice, int32_t *Q, int32_t *v, double *w, double *m) {
  return lbfd_lattice_tables_ex(lattice, 1.0 / 3.0, Q, v, w, m);
}

int lbfd_noise_draw(int32_t precision, int32_t dist, uint64_t seed, uint32_t lattice_id, uint64_t t, int64_t site0,
                    int64_t nsites, int32_t nmom, double *z_host) {
  if (!z_host || nsites < 0 || site0 < 0) return fail(LBFD_EINVAL, "lbfd_noise_draw: bad argument");
  if (precision != LBFD_F32 && precision != LBFD_F64) return fail(LBFD_EINVAL, "unknown precision");
  if (dist != LBFD_GAUSSIAN && dist != LBFD_UNIFORM) return fail(LBFD_EINVAL, "unknown noise distribution");
  if (nmom != 2 && nmom != 4 && nmom != 8 && nmom != 18) return fail(LBFD_EINVAL, "nmom must be 2, 4, 8 or 18");
  if (site0 + nsites > 0xffffffffLL) return fail(LBFD_EINVAL, "site index beyond 32 bits");
  if (nsites == 0) return LBFD_OK;
  double *d = nullptr;
  const size_t bytes = sizeof(double) * size_t(nsites) * nmom;
  LBFD_CU(cudaMalloc(&d, bytes));
  cudaError_t e = launch_noise_draw(precision, dist, make_philox_step(seed, lattice_id, t), site0, nsites, nmom, d,
                                    nullptr);
  if (e == cudaSuccess) e = cudaMemcpy(z_host, d, bytes, cudaMemcpyDeviceToHost);
  cudaFree(d);
  if (e != cudaSuccess) return cuda_fail("lbfd_noise_draw", e);
  return LBFD_OK;
}

int lbfd_box_muller_probe(int32_t precision, const uint32_t *words_host, int64_t npairs, double *z_host) {
  if (!words_host || !z_host || npairs < 0) return fail(LBFD_EINVAL, "lbfd_box_muller_probe: bad argument");
  if (precision != LBFD_F32 && precision != LBFD_F64) return fail(LBFD_EINVAL, "unknown precision");
  if (npairs == 0) return LBFD_OK;
  uint32_t *dw = nullptr;
  double *dz = nullptr;
  cudaError_t e = cudaMalloc(&dw, sizeof(uint32_t) * 2 * size_t(npairs));
  if (e == cudaSuccess) e = cudaMalloc(&dz, sizeof(double) * 2 * size_t(npairs));
  if (e == cudaSuccess) e = cudaMemcpy(dw, words_host, sizeof(uint32_t) * 2 * size_t(npairs), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = launch_box_muller_probe(precision, dw, npairs, dz, nullptr);
  if (e == cudaSuccess) e = cudaMemcpy(z_host, dz, sizeof(double) * 2 * size_t(npairs), cudaMemcpyDeviceToHost);
  cudaFree(dw);
  cudaFree(dz);
  if (e != cudaSuccess) return cuda_fail("lbfd_box_muller_probe", e);
  return LBFD_OK;
}

int lbfd_lane_ops_probe(const float *a_host, const float *b_host, const float *c_host, int64_t n, float *out_host) {
  if (!a_host || !b_host || !c_host || !out_host || n < 0 || n % 2)
    return fail(LBFD_EINVAL, "lbfd_lane_ops_probe: bad argument");
  if (n == 0) return LBFD_OK;
  const size_t in_bytes = sizeof(float) * size_t(n), out_bytes = 12 * in_bytes;
  float *d = nullptr;
  cudaError_t e = cudaMalloc(&d, 3 * in_bytes + out_bytes);
  if (e == cudaSuccess) e = cudaMemcpy(d, a_host, in_bytes, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(d + n, b_host, in_bytes, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(d + 2 * n, c_host, in_bytes, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = launch_lane_ops_probe(d, d + n, d + 2 * n, n, d + 3 * n, nullptr);
  if (e == cudaSuccess) e = cudaMemcpy(out_host, d + 3 * n, out_bytes, cudaMemcpyDeviceToHost);
  cudaFree(d);
  if (e != cudaSuccess) return cuda_fail("lbfd_lane_ops_probe", e);
  return LBFD_OK;
}

const char *lbfd_last_error(void) { return g_err.c_str(); }

int64_t lbfd_kernel_launches(void) { return g_launches.load(std::memory_order_relaxed); }

int lbfd_struct_sizes(int64_t *options_bytes, int64_t *obs_bytes, int64_t *member_bytes) {
  if (options_bytes) *options_bytes = int64_t(sizeof(lbfd_options));
  if (obs_bytes) *obs_bytes = int64_t(sizeof(lbfd_obs));
  if (member_bytes) *member_bytes = int64_t(sizeof(lbfd_member));
  return LBFD_OK;
}

}  // extern "C"
