// C ABI of the batched ensemble (declared in include/lbfd.h): many
// independent lattices advanced together, one launch per time step for the
// whole ensemble, with the launches of a chunk of steps captured once into
// a CUDA graph and replayed.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "ensemble_kernels.cuh"
#include "internal.h"
#include "lbfd.h"

using namespace lbfd;

namespace lbfd {
// t += 1 on the device, between the steps of a captured graph.
__global__ void k_ens_advance(uint64_t *t_dev) {
  if (threadIdx.x == 0 && blockIdx.x == 0) *t_dev += 1;
}
}  // namespace lbfd

namespace {

constexpr int kGraphSteps = 16;  // steps per captured graph (even: the buffers end where they started)

int ens_fail(int code, const std::string &msg) { return set_last_error(code, msg); }

int ens_cuda(const char *what, cudaError_t e) {
  return ens_fail(e == cudaErrorMemoryAllocation ? LBFD_ENOMEM : LBFD_ECUDA,
                  std::string(what) + ": " + cudaGetErrorName(e) + " (" + cudaGetErrorString(e) + ")");
}

#define ENS_CU(call)                                   \
  do {                                                 \
    cudaError_t e_ = (call);                           \
    if (e_ != cudaSuccess) return ens_cuda(#call, e_); \
  } while (0)

struct DevGuard {
  int prev = -1;
  explicit DevGuard(int dev) {
    if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
    if (dev >= 0 && dev != prev) cudaSetDevice(dev);
  }
  ~DevGuard() {
    int cur = -1;
    if (prev >= 0 && cudaGetDevice(&cur) == cudaSuccess && cur != prev) cudaSetDevice(prev);
  }
};

int q_of(int lattice) { return lattice == LBFD_D1Q3 ? 3 : (lattice == LBFD_D2Q9 ? 9 : 19); }
int d_of(int lattice) { return lattice == LBFD_D1Q3 ? 1 : (lattice == LBFD_D2Q9 ? 2 : 3); }

}  // namespace

struct lbfd_ens {
  int lattice = 0, precision = 0, noise_mode = 0, noise_dist = 0, elem = 4, Q = 0, device = 0, n = 0;
  int vx = 1, grid = 1, ntiles = 0;
  std::vector<EnsMember> hmem;
  EnsMember *dmem = nullptr;
  EnsTile *dtiles = nullptr;
  void *f[2] = {nullptr, nullptr};
  int cur = 0;
  int64_t total_values = 0, total_sites = 0, t = 0;
  uint64_t *t_dev = nullptr;
  bool t_dev_valid = false;
  cudaStream_t stream = nullptr;
  double *partials = nullptr, *d_mass = nullptr;
  cudaGraphExec_t graph = nullptr;
  int graph_vx = 0;
  bool owns_stream = false;
};

static cudaError_t ens_launch(lbfd_ens *e, const void *src, void *dst) {
  switch (e->lattice) {
    case LBFD_D1Q3:
      return launch_ens_step_d1q3(e->precision, e->vx, src, dst, e->dmem, e->dtiles, e->ntiles, e->t_dev, e->noise_mode,
                                  e->noise_dist, e->grid, e->stream);
    case LBFD_D2Q9:
      return launch_ens_step_d2q9(e->precision, e->vx, src, dst, e->dmem, e->dtiles, e->ntiles, e->t_dev, e->noise_mode,
                                  e->noise_dist, e->grid, e->stream);
    default:
      return launch_ens_step_d3q19(e->precision, e->vx, src, dst, e->dmem, e->dtiles, e->ntiles, e->t_dev,
                                   e->noise_mode, e->noise_dist, e->grid, e->stream);
  }
}

// Tiles and persistent grid for sites-per-item vx.
static int ens_plan(lbfd_ens *e, int vx) {
  std::vector<EnsTile> tiles;
  for (int m = 0; m < e->n; ++m) {
    const EnsMember &mm = e->hmem[m];
    const int64_t items = int64_t(mm.Lx / vx) * mm.Ly * mm.Lz;
    for (int64_t i0 = 0; i0 < items; i0 += kEnsThreads) {
      EnsTile t{};
      t.member = m;
      t.item0 = i0;
      tiles.push_back(t);
    }
  }
  if (tiles.size() > size_t(0x7fffffff)) return ens_fail(LBFD_EINVAL, "ensemble too large");
  if (e->dtiles) cudaFree(e->dtiles);
  e->dtiles = nullptr;
  ENS_CU(cudaMalloc(&e->dtiles, sizeof(EnsTile) * tiles.size()));
  ENS_CU(cudaMemcpy(e->dtiles, tiles.data(), sizeof(EnsTile) * tiles.size(), cudaMemcpyHostToDevice));
  e->ntiles = int(tiles.size());
  e->vx = vx;
  int bps = 1;
  switch (e->lattice) {
    case LBFD_D1Q3: bps = ens_blocks_per_sm_d1q3(e->precision, vx, e->noise_mode, e->noise_dist); break;
    case LBFD_D2Q9: bps = ens_blocks_per_sm_d2q9(e->precision, vx, e->noise_mode, e->noise_dist); break;
    default: bps = ens_blocks_per_sm_d3q19(e->precision, vx, e->noise_mode, e->noise_dist); break;
  }
  int sms = 0;
  ENS_CU(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, e->device));
  e->grid = std::max(1, std::min(e->ntiles, sms * bps));
  if (e->graph) {
    cudaGraphExecDestroy(e->graph);
    e->graph = nullptr;
  }
  return LBFD_OK;
}

static void ens_free(lbfd_ens *e) {
  if (!e) return;
  if (e->graph) cudaGraphExecDestroy(e->graph);
  cudaFree(e->dmem);
  cudaFree(e->dtiles);
  cudaFree(e->f[0]);
  cudaFree(e->f[1]);
  cudaFree(e->t_dev);
  cudaFree(e->partials);
  cudaFree(e->d_mass);
  if (e->owns_stream) cudaStreamDestroy(e->stream);
  delete e;
}

static cudaError_t ens_sync_t(lbfd_ens *e) {
  if (e->t_dev_valid) return cudaSuccess;
  const uint64_t t = uint64_t(e->t);
  cudaError_t err = cudaMemcpyAsync(e->t_dev, &t, sizeof(t), cudaMemcpyHostToDevice, e->stream);
  if (err == cudaSuccess) err = cudaStreamSynchronize(e->stream);
  if (err == cudaSuccess) e->t_dev_valid = true;
  return err;
}

// One step: src -> dst for every member, then t += 1 on the device.
static cudaError_t ens_one_step(lbfd_ens *e, int from) {
  cudaError_t err = ens_launch(e, e->f[from], e->f[from ^ 1]);
  if (err == cudaSuccess) {
    k_ens_advance<<<1, 32, 0, e->stream>>>(e->t_dev);
    err = cudaGetLastError();
  }
  return err;
}

static cudaError_t ens_build_graph(lbfd_ens *e) {
  cudaGraph_t g = nullptr;
  cudaError_t err = cudaStreamBeginCapture(e->stream, cudaStreamCaptureModeThreadLocal);
  if (err != cudaSuccess) return err;
  for (int k = 0; k < kGraphSteps && err == cudaSuccess; ++k) err = ens_one_step(e, k & 1);
  cudaError_t end = cudaStreamEndCapture(e->stream, &g);
  if (err == cudaSuccess) err = end;
  if (err == cudaSuccess) err = cudaGraphInstantiate(&e->graph, g, 0);
  if (g) cudaGraphDestroy(g);
  e->graph_vx = e->vx;
  return err;
}

extern "C" {

int lbfd_ensemble_create(lbfd_ens_t *out, int32_t lattice, int32_t precision, int32_t noise_mode, int32_t noise_dist,
                         const lbfd_member *members, int32_t n, void *stream) {
  if (!out || !members || n < 1) return ens_fail(LBFD_EINVAL, "lbfd_ensemble_create: bad argument");
  *out = nullptr;
  if (lattice < LBFD_D1Q3 || lattice > LBFD_D3Q19) return ens_fail(LBFD_EINVAL, "unknown lattice");
  if (precision < LBFD_F32 || precision > LBFD_F32_BF16) return ens_fail(LBFD_EINVAL, "unknown precision");
  if (noise_mode < LBFD_NOISE_LOCAL || noise_mode > LBFD_NOISE_OFF) return ens_fail(LBFD_EINVAL, "unknown noise mode");
  if (noise_dist != LBFD_GAUSSIAN && noise_dist != LBFD_UNIFORM) return ens_fail(LBFD_EINVAL, "unknown noise distribution");
  const int D = d_of(lattice);
  int dev = 0;
  ENS_CU(cudaGetDevice(&dev));
  lbfd_ens *e = new (std::nothrow) lbfd_ens();
  if (!e) return ens_fail(LBFD_ENOMEM, "host allocation failed");
  e->lattice = lattice;
  e->precision = precision;
  e->noise_mode = noise_mode;
  e->noise_dist = noise_dist;
  e->elem = storage_bytes(precision);
  e->Q = q_of(lattice);
  e->device = dev;
  e->n = n;
  e->stream = static_cast<cudaStream_t>(stream);
  int64_t off = 0;
  bool all_even = true;
  for (int m = 0; m < n; ++m) {
    const lbfd_member &mb = members[m];
    for (int a = 0; a < 3; ++a) {
      if (mb.dims[a] < 1 || (a >= D && mb.dims[a] != 1) || mb.dims[a] > 0x7fffffffLL) {
        delete e;
        return ens_fail(LBFD_EINVAL, "member " + std::to_string(m) + ": bad dimensions");
      }
    }
    const double sites = double(mb.dims[0]) * double(mb.dims[1]) * double(mb.dims[2]);
    if (sites >= 2147483648.0) {
      delete e;
      return ens_fail(LBFD_EINVAL, "member " + std::to_string(m) + ": 2^31 sites or more");
    }
    if (!(mb.tau > 0.5) || !std::isfinite(mb.tau) || !(mb.rho_mean >= 0.0) || !std::isfinite(mb.rho_mean)) {
      delete e;
      return ens_fail(LBFD_EINVAL, "member " + std::to_string(m) + ": tau must be > 1/2 and rho_mean >= 0");
    }
    EnsMember em{};
    em.Lx = int32_t(mb.dims[0]);
    em.Ly = int32_t(mb.dims[1]);
    em.Lz = int32_t(mb.dims[2]);
    em.N = int64_t(sites);
    em.offset = off;
    em.tau = mb.tau;
    em.rho_mean = mb.rho_mean;
    em.seed = mb.seed;
    em.lattice_id = mb.lattice_id;
    off += int64_t(e->Q) * em.N;
    // keep every member's block 16-byte aligned for the vector loads
    const int64_t align = 16 / e->elem;
    off = (off + align - 1) / align * align;
    all_even = all_even && (em.Lx % 2 == 0);
    e->hmem.push_back(em);
    e->total_sites += em.N;
  }
  e->total_values = off;
  DevGuard g(dev);
  cudaError_t err = cudaSuccess;
  if (!e->stream) {
    // graph capture needs a stream other than the legacy default stream
    err = cudaStreamCreateWithFlags(&e->stream, cudaStreamNonBlocking);
    e->owns_stream = err == cudaSuccess;
  }
  if (err == cudaSuccess) err = cudaMalloc(&e->f[0], size_t(off) * e->elem);
  if (err == cudaSuccess) err = cudaMalloc(&e->f[1], size_t(off) * e->elem);
  if (err == cudaSuccess) err = cudaMalloc(&e->dmem, sizeof(EnsMember) * n);
  if (err == cudaSuccess) err = cudaMemcpy(e->dmem, e->hmem.data(), sizeof(EnsMember) * n, cudaMemcpyHostToDevice);
  if (err == cudaSuccess) err = cudaMalloc(&e->t_dev, sizeof(uint64_t));
  if (err == cudaSuccess)
    err = cudaMalloc(&e->partials, sizeof(double) * size_t(kReduceBlocks) * obs_quantities(e->Q, LBFD_MAX_MODES));
  if (err == cudaSuccess) err = cudaMalloc(&e->d_mass, sizeof(double));
  // initial states: f into the spare buffer, stored un-streamed
  for (int m = 0; m < n && err == cudaSuccess; ++m) {
    const lbfd_member &mb = members[m];
    const EnsMember &em = e->hmem[m];
    char *f0 = static_cast<char *>(e->f[0]) + em.offset * e->elem;
    char *f1 = static_cast<char *>(e->f[1]) + em.offset * e->elem;
    const double amp = mb.init == LBFD_INIT_SINE ? mb.sine_amp : 0.0;
    if (mb.init == LBFD_INIT_NONE) continue;
    err = launch_init(lattice, precision, f1, em.Lx, em.Ly, em.Lz, mb.rho_mean, amp, mb.sine_k, e->stream);
    if (err == cudaSuccess) err = launch_shift(lattice, e->elem, f1, f0, em.Lx, em.Ly, em.Lz, -1, e->stream);
  }
  if (err != cudaSuccess) {
    int rc = ens_cuda("lbfd_ensemble_create", err);
    ens_free(e);
    return rc;
  }
  int rc = ens_plan(e, all_even ? 2 : 1);
  if (rc) {
    ens_free(e);
    return rc;
  }
  *out = e;
  return LBFD_OK;
}

int lbfd_ensemble_destroy(lbfd_ens_t e) {
  if (!e) return LBFD_OK;
  DevGuard g(e->device);
  cudaError_t err = cudaStreamSynchronize(e->stream);
  ens_free(e);
  if (err != cudaSuccess) return ens_cuda("lbfd_ensemble_destroy", err);
  return LBFD_OK;
}

int lbfd_ensemble_step(lbfd_ens_t e, int64_t n) {
  if (!e) return ens_fail(LBFD_EINVAL, "lbfd_ensemble_step: null handle");
  if (n < 0) return ens_fail(LBFD_EINVAL, "lbfd_ensemble_step: n must be >= 0");
  if (n == 0) return LBFD_OK;
  DevGuard g(e->device);
  ENS_CU(ens_sync_t(e));
  int64_t done = 0;
  while (done < n) {
    if (e->cur == 0 && n - done >= kGraphSteps) {
      if (!e->graph || e->graph_vx != e->vx) {
        if (e->graph) cudaGraphExecDestroy(e->graph);
        e->graph = nullptr;
        ENS_CU(ens_build_graph(e));
      }
      ENS_CU(cudaGraphLaunch(e->graph, e->stream));
      done += kGraphSteps;
    } else {
      ENS_CU(ens_one_step(e, e->cur));
      e->cur ^= 1;
      done += 1;
    }
  }
  e->t += n;
  return LBFD_OK;
}

int lbfd_ensemble_sync(lbfd_ens_t e) {
  if (!e) return ens_fail(LBFD_EINVAL, "lbfd_ensemble_sync: null handle");
  DevGuard g(e->device);
  ENS_CU(cudaStreamSynchronize(e->stream));
  return LBFD_OK;
}

int lbfd_ensemble_tune(lbfd_ens_t e, int32_t steps, int32_t *vx_chosen) {
  if (!e || steps < 1) return ens_fail(LBFD_EINVAL, "lbfd_ensemble_tune: bad argument");
  DevGuard g(e->device);
  ENS_CU(ens_sync_t(e));
  bool all_even = true;
  for (const EnsMember &m : e->hmem) all_even = all_even && (m.Lx % 2 == 0);
  const int candidates[2] = {1, 2};
  float best_ms = -1.0f;
  int best = e->vx;
  cudaEvent_t a = nullptr, b = nullptr;
  ENS_CU(cudaEventCreate(&a));
  ENS_CU(cudaEventCreate(&b));
  for (int vx : candidates) {
    if (vx == 2 && !all_even) continue;
    int rc = ens_plan(e, vx);
    if (rc) return rc;
    // timing launches read the state and write the spare buffer only
    ENS_CU(ens_launch(e, e->f[e->cur], e->f[e->cur ^ 1]));
    ENS_CU(cudaEventRecord(a, e->stream));
    for (int k = 0; k < steps; ++k) ENS_CU(ens_launch(e, e->f[e->cur], e->f[e->cur ^ 1]));
    ENS_CU(cudaEventRecord(b, e->stream));
    ENS_CU(cudaEventSynchronize(b));
    float ms = 0.0f;
    ENS_CU(cudaEventElapsedTime(&ms, a, b));
    if (best_ms < 0.0f || ms < best_ms) {
      best_ms = ms;
      best = vx;
    }
  }
  cudaEventDestroy(a);
  cudaEventDestroy(b);
  int rc = ens_plan(e, best);
  if (rc) return rc;
  if (vx_chosen) *vx_chosen = best;
  return LBFD_OK;
}

int lbfd_ensemble_query(lbfd_ens_t e, int32_t *n_members, int64_t *total_sites, int64_t *t, int32_t *vx) {
  if (!e) return ens_fail(LBFD_EINVAL, "lbfd_ensemble_query: null handle");
  if (n_members) *n_members = e->n;
  if (total_sites) *total_sites = e->total_sites;
  if (t) *t = e->t;
  if (vx) *vx = e->vx;
  return LBFD_OK;
}

static int ens_member_ok(lbfd_ens_t e, int32_t m) { return e && m >= 0 && m < e->n; }

int lbfd_ensemble_get_f(lbfd_ens_t e, int32_t member, double *f_host) {
  if (!ens_member_ok(e, member) || !f_host) return ens_fail(LBFD_EINVAL, "lbfd_ensemble_get_f: bad argument");
  DevGuard g(e->device);
  const EnsMember &em = e->hmem[member];
  const size_t count = size_t(e->Q) * em.N;
  const char *cur = static_cast<const char *>(e->f[e->cur]) + em.offset * e->elem;
  char *spare = static_cast<char *>(e->f[e->cur ^ 1]) + em.offset * e->elem;
  ENS_CU(launch_shift(e->lattice, e->elem, cur, spare, em.Lx, em.Ly, em.Lz, +1, e->stream));
  std::vector<uint8_t> raw(count * e->elem);
  ENS_CU(cudaMemcpyAsync(raw.data(), spare, raw.size(), cudaMemcpyDeviceToHost, e->stream));
  ENS_CU(cudaStreamSynchronize(e->stream));
  int Q = 0, D = 0, v[LBFD_MAX_Q * 3];
  double w[LBFD_MAX_Q];
  lattice_table(e->lattice, &Q, &D, v, w);
  dispatch_storage(e->precision, [&](auto tag) {
    using S = typename decltype(tag)::type;
    const S *p = reinterpret_cast<const S *>(raw.data());
    for (int i = 0; i < Q; ++i)
      for (int64_t s = 0; s < em.N; ++s) f_host[i * em.N + s] = Store<S>::getd(p[i * em.N + s], w[i] * em.rho_mean);
    return cudaSuccess;
  });
  return LBFD_OK;
}

int lbfd_ensemble_set_f(lbfd_ens_t e, int32_t member, const double *f_host) {
  if (!ens_member_ok(e, member) || !f_host) return ens_fail(LBFD_EINVAL, "lbfd_ensemble_set_f: bad argument");
  DevGuard g(e->device);
  const EnsMember &em = e->hmem[member];
  const size_t count = size_t(e->Q) * em.N;
  std::vector<uint8_t> raw(count * e->elem);
  int Q = 0, D = 0, v[LBFD_MAX_Q * 3];
  double w[LBFD_MAX_Q];
  lattice_table(e->lattice, &Q, &D, v, w);
  dispatch_storage(e->precision, [&](auto tag) {
    using S = typename decltype(tag)::type;
    S *p = reinterpret_cast<S *>(raw.data());
    for (int i = 0; i < Q; ++i)
      for (int64_t s = 0; s < em.N; ++s) p[i * em.N + s] = Store<S>::putd(f_host[i * em.N + s], w[i] * em.rho_mean);
    return cudaSuccess;
  });
  char *cur = static_cast<char *>(e->f[e->cur]) + em.offset * e->elem;
  char *spare = static_cast<char *>(e->f[e->cur ^ 1]) + em.offset * e->elem;
  ENS_CU(cudaMemcpyAsync(spare, raw.data(), raw.size(), cudaMemcpyHostToDevice, e->stream));
  ENS_CU(launch_shift(e->lattice, e->elem, spare, cur, em.Lx, em.Ly, em.Lz, -1, e->stream));
  ENS_CU(cudaStreamSynchronize(e->stream));
  return LBFD_OK;
}

int lbfd_ensemble_mass(lbfd_ens_t e, int32_t member, double *mass) {
  if (!ens_member_ok(e, member) || !mass) return ens_fail(LBFD_EINVAL, "lbfd_ensemble_mass: bad argument");
  DevGuard g(e->device);
  const EnsMember &em = e->hmem[member];
  const char *cur = static_cast<const char *>(e->f[e->cur]) + em.offset * e->elem;
  ENS_CU(launch_mass(e->lattice, e->precision, cur, em.N, em.rho_mean, e->partials, e->d_mass, e->stream));
  ENS_CU(cudaMemcpyAsync(mass, e->d_mass, sizeof(double), cudaMemcpyDeviceToHost, e->stream));
  ENS_CU(cudaStreamSynchronize(e->stream));
  return LBFD_OK;
}

}  // extern "C"
