// C ABI of the batched ensemble (declared in include/lbfd.h): many
// independent lattices advanced together by the batched step kernel
// (batch_kernels.cuh), one launch per time step for the whole ensemble, with
// the launches of a chunk of steps captured once into a CUDA graph and
// replayed.  All members start at t = 0 and share t; the ensemble clock is t.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "batch.h"
#include "lbfd.h"

using namespace lbfd;

namespace {

constexpr int kGraphSteps = 16;  // steps per captured graph

int ens_fail(int code, const std::string &msg) { return set_last_error(code, msg); }

int ens_cuda(const char *what, cudaError_t e) {
  // the runtime keeps a failed call's error as the thread's last error;
  // clear it so that the next launch check does not report it again
  (void)cudaGetLastError();
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
  int vx_max = 2, kvx = 2, passes = 1, occ = 0, walk = 0, grid = 1, bps = 1;  // kvx: largest vx of a member
  int64_t ntiles = 0;
  std::vector<BatchMember> hmem;
  std::vector<int64_t> tile_start;
  std::vector<BatchParams> groups;  // parameter-space launches (tile order 3)
  BatchMember *dmem = nullptr;
  int64_t *dtile_start = nullptr;
  BatchStep *dsteps = nullptr;
  void *buf = nullptr;  // both population blocks of every member
  int64_t total_values = 0, total_sites = 0, t = 0;
  uint64_t *t_dev = nullptr;
  bool t_dev_valid = false;
  cudaStream_t stream = nullptr;
  double *partials = nullptr, *d_mass = nullptr;
  cudaGraphExec_t graph = nullptr;
  bool owns_stream = false;
  // side streams for the parameter-space launches: the groups of a step run
  // concurrently (parallel branches of the captured graph), joined before the
  // clock advances
  static constexpr int kSide = 4;
  cudaStream_t side[kSide] = {};
  cudaEvent_t fork_ev = nullptr, join_ev[kSide] = {};
  // member m's block holding its stored state (which = 0) or the spare one (1)
  char *block(int m, int which) const {
    const int p = static_cast<int>(t & 1) ^ which;
    return static_cast<char *>(buf) + hmem[m].off[p] * elem;
  }
};

// Kernel launches of one step of the batched kernel.
static int ens_step_launches(const lbfd_ens *e) {
  return e->walk == kWalkParam ? static_cast<int>(e->groups.size()) : 1;
}

static cudaError_t ens_launch(lbfd_ens *e) {
  if (e->walk == kWalkParam) {
    // groups k, k + kSide, ... on side stream k, forked from and joined to the ensemble's stream
    const int G = static_cast<int>(e->groups.size());
    const int nside = std::min(G, int(lbfd_ens::kSide));
    if (nside <= 1)
      return launch_batch_param(e->lattice, e->precision, e->buf, e->groups.data(), G, e->dsteps, e->passes, e->occ,
                                e->kvx, e->noise_mode, e->noise_dist, e->stream);
    cudaError_t err = cudaEventRecord(e->fork_ev, e->stream);
    for (int k = 0; k < nside && err == cudaSuccess; ++k) {
      err = cudaStreamWaitEvent(e->side[k], e->fork_ev, 0);
      for (int g = k; g < G && err == cudaSuccess; g += nside)
        err = launch_batch_param(e->lattice, e->precision, e->buf, &e->groups[g], 1, e->dsteps, e->passes, e->occ,
                                 e->kvx, e->noise_mode, e->noise_dist, e->side[k]);
      if (err == cudaSuccess) err = cudaEventRecord(e->join_ev[k], e->side[k]);
      if (err == cudaSuccess) err = cudaStreamWaitEvent(e->stream, e->join_ev[k], 0);
    }
    return err;
  }
  return launch_batch_step(e->lattice, e->precision, e->buf, e->dsteps, e->dtile_start, e->n, e->ntiles, e->passes,
                           e->occ, e->walk, e->kvx, e->noise_mode, e->noise_dist, e->grid, e->stream);
}

// Work decomposition (sites per item, tile passes, occupancy variant, tile
// order), the grid of the persistent orders and the parameter blocks of the
// parameter-bank order.
static int ens_plan(lbfd_ens *e, int vx_max, int passes, int occ, int walk) {
  e->kvx = 1;
  for (BatchMember &m : e->hmem) {
    m.vx = (vx_max >= 2 && m.Lx % 2 == 0) ? 2 : 1;
    e->kvx = std::max(e->kvx, int(m.vx));
  }
  e->tile_start.assign(e->n, 0);
  e->ntiles = batch_assign_tiles(e->hmem.data(), e->n, passes, e->tile_start.data());
  ENS_CU(cudaMemcpy(e->dmem, e->hmem.data(), sizeof(BatchMember) * e->n, cudaMemcpyHostToDevice));
  ENS_CU(cudaMemcpy(e->dtile_start, e->tile_start.data(), sizeof(int64_t) * e->n, cudaMemcpyHostToDevice));
  e->vx_max = vx_max;
  e->passes = passes;
  e->occ = occ;
  e->walk = walk;
  e->groups.clear();
  if (walk == kWalkParam) batch_build_params(e->hmem.data(), e->n, e->ntiles, e->noise_mode, e->noise_dist, e->groups);
  e->bps = batch_blocks_per_sm(e->lattice, e->precision, occ, e->kvx, walk, e->noise_mode, e->noise_dist);
  int sms = 0;
  ENS_CU(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, e->device));
  e->grid = int(std::max<int64_t>(1, std::min<int64_t>(e->ntiles, int64_t(sms) * e->bps)));
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
  cudaFree(e->dtile_start);
  cudaFree(e->dsteps);
  cudaFree(e->buf);
  cudaFree(e->t_dev);
  cudaFree(e->partials);
  cudaFree(e->d_mass);
  for (int k = 0; k < lbfd_ens::kSide; ++k) {
    if (e->side[k]) cudaStreamDestroy(e->side[k]);
    if (e->join_ev[k]) cudaEventDestroy(e->join_ev[k]);
  }
  if (e->fork_ev) cudaEventDestroy(e->fork_ev);
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

// One step of every member (arguments for the current t, the step, t += 1).
static cudaError_t ens_one_step(lbfd_ens *e) {
  cudaError_t err = launch_batch_prep(e->dmem, e->n, e->t_dev, 0, e->noise_mode, e->noise_dist, e->dsteps, e->stream);
  if (err == cudaSuccess) err = ens_launch(e);
  if (err == cudaSuccess) err = launch_clock_advance(e->t_dev, e->stream);
  return err;
}

static cudaError_t ens_build_graph(lbfd_ens *e) {
  cudaGraph_t g = nullptr;
  cudaError_t err = cudaStreamBeginCapture(e->stream, cudaStreamCaptureModeThreadLocal);
  if (err != cudaSuccess) return err;
  for (int k = 0; k < kGraphSteps && err == cudaSuccess; ++k) err = ens_one_step(e);
  cudaError_t end = cudaStreamEndCapture(e->stream, &g);
  if (err == cudaSuccess) err = end;
  if (err == cudaSuccess) err = cudaGraphInstantiate(&e->graph, g, 0);
  if (g) cudaGraphDestroy(g);
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
  if (noise_dist != LBFD_GAUSSIAN && noise_dist != LBFD_UNIFORM)
    return ens_fail(LBFD_EINVAL, "unknown noise distribution");
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
  // pass 1: validate and lay out block 0 of every member (16-byte aligned
  // for the vector loads); block 1 of member m sits at total + offset
  std::vector<int64_t> offs(n);
  int64_t off = 0;
  const int64_t align = 16 / e->elem;
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
    if (double(e->Q) * sites > 4294967295.0) {
      delete e;
      return ens_fail(LBFD_EINVAL, "member " + std::to_string(m) + ": Q * sites must be < 2^32");
    }
    if (mb.dims[1] > 65535 || mb.dims[2] > 65535) {
      delete e;
      return ens_fail(LBFD_EINVAL, "member " + std::to_string(m) + ": Ly and Lz must be <= 65535");
    }
    if (!(mb.tau > 0.5) || !std::isfinite(mb.tau) || !(mb.rho_mean >= 0.0) || !std::isfinite(mb.rho_mean)) {
      delete e;
      return ens_fail(LBFD_EINVAL, "member " + std::to_string(m) + ": tau must be > 1/2 and rho_mean >= 0");
    }
    offs[m] = off;
    off += int64_t(e->Q) * int64_t(sites);
    off = (off + align - 1) / align * align;
  }
  e->total_values = off;
  for (int m = 0; m < n; ++m) {
    const lbfd_member &mb = members[m];
    e->hmem.push_back(
        make_batch_member(mb.dims, mb.tau, mb.rho_mean, mb.seed, mb.lattice_id, offs[m], off + offs[m], 0, 2));
    e->total_sites += e->hmem.back().N;
  }
  DevGuard g(dev);
  cudaError_t err = cudaSuccess;
  if (!e->stream) {
    // graph capture needs a stream other than the legacy default stream
    err = cudaStreamCreateWithFlags(&e->stream, cudaStreamNonBlocking);
    e->owns_stream = err == cudaSuccess;
  }
  for (int k = 0; k < lbfd_ens::kSide && err == cudaSuccess; ++k) {
    err = cudaStreamCreateWithFlags(&e->side[k], cudaStreamNonBlocking);
    if (err == cudaSuccess) err = cudaEventCreateWithFlags(&e->join_ev[k], cudaEventDisableTiming);
  }
  if (err == cudaSuccess) err = cudaEventCreateWithFlags(&e->fork_ev, cudaEventDisableTiming);
  if (err == cudaSuccess) err = cudaMalloc(&e->buf, size_t(2 * off) * e->elem);
  if (err == cudaSuccess) err = cudaMalloc(&e->dmem, sizeof(BatchMember) * n);
  if (err == cudaSuccess) err = cudaMalloc(&e->dtile_start, sizeof(int64_t) * n);
  if (err == cudaSuccess) err = cudaMalloc(&e->dsteps, sizeof(BatchStep) * n);
  if (err == cudaSuccess) err = cudaMalloc(&e->t_dev, sizeof(uint64_t));
  if (err == cudaSuccess)
    err = cudaMalloc(&e->partials, sizeof(double) * size_t(kReduceBlocks) * obs_quantities(e->Q, LBFD_MAX_MODES));
  if (err == cudaSuccess) err = cudaMalloc(&e->d_mass, sizeof(double));
  // initial states: f into the spare block, stored un-streamed (t = 0)
  for (int m = 0; m < n && err == cudaSuccess; ++m) {
    const lbfd_member &mb = members[m];
    const BatchMember &bm = e->hmem[m];
    if (mb.init == LBFD_INIT_NONE) continue;
    const double amp = mb.init == LBFD_INIT_SINE ? mb.sine_amp : 0.0;
    err = launch_init(lattice, precision, e->block(m, 1), bm.Lx, bm.Ly, bm.Lz, mb.rho_mean, amp, mb.sine_k, e->stream);
    if (err == cudaSuccess)
      err = launch_shift(lattice, e->elem, e->block(m, 1), e->block(m, 0), bm.Lx, bm.Ly, bm.Lz, -1, e->stream);
  }
  if (err != cudaSuccess) {
    int rc = ens_cuda("lbfd_ensemble_create", err);
    ens_free(e);
    return rc;
  }
  int rc = ens_plan(e, 2, 4, 0, kWalkPerTile);
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
  NvtxRange nvtx_("lbfd_ensemble_step");
  if (!e) return ens_fail(LBFD_EINVAL, "lbfd_ensemble_step: null handle");
  if (n < 0) return ens_fail(LBFD_EINVAL, "lbfd_ensemble_step: n must be >= 0");
  if (n == 0) return LBFD_OK;
  DevGuard g(e->device);
  ENS_CU(ens_sync_t(e));
  int64_t done = 0;
  while (done < n) {
    // the kernels take the parity of each member's block from t on the
    // device, so a captured chunk can start at any t
    if (n - done >= kGraphSteps) {
      if (!e->graph) ENS_CU(ens_build_graph(e));
      ENS_CU(cudaGraphLaunch(e->graph, e->stream));
      done += kGraphSteps;
    } else {
      ENS_CU(ens_one_step(e));
      done += 1;
    }
  }
  count_launches(n * (2 + ens_step_launches(e)));
  e->t += n;
  return LBFD_OK;
}

int lbfd_ensemble_sync(lbfd_ens_t e) {
  if (!e) return ens_fail(LBFD_EINVAL, "lbfd_ensemble_sync: null handle");
  DevGuard g(e->device);
  ENS_CU(cudaStreamSynchronize(e->stream));
  return LBFD_OK;
}

int lbfd_ensemble_tune(lbfd_ens_t e, int32_t steps, int32_t *vx_chosen, int32_t *passes_chosen,
                       int32_t *blocks_per_sm) {
  NvtxRange nvtx_("lbfd_ensemble_tune");
  if (!e || steps < 1) return ens_fail(LBFD_EINVAL, "lbfd_ensemble_tune: bad argument");
  DevGuard g(e->device);
  ENS_CU(ens_sync_t(e));
  // candidates: sites per item (1, or 2 where Lx is even) x tile passes x
  // occupancy variant of the kernel x tile order
  const int vx_cand[2] = {1, 2};
  const int pass_cand[4] = {1, 2, 4, 8};
  float best_ms = -1.0f;
  int best_vx = e->vx_max, best_passes = e->passes, best_occ = e->occ, best_walk = e->walk;
  // On every early exit: destroy the timing events and put the plan the
  // ensemble had before tuning back (the error of the failed call stays the
  // thread's lbfd_last_error()).
  struct TuneGuard {
    lbfd_ens *e;
    int vx, passes, occ, walk;
    cudaEvent_t a = nullptr, b = nullptr;
    bool finished = false;
    ~TuneGuard() {
      if (a) cudaEventDestroy(a);
      if (b) cudaEventDestroy(b);
      if (!finished) {
        const std::string err = lbfd_last_error();
        (void)ens_plan(e, vx, passes, occ, walk);
        (void)cudaGetLastError();
        set_last_error(LBFD_ECUDA, err);
      }
    }
  } guard{e, e->vx_max, e->passes, e->occ, e->walk};
  ENS_CU(cudaEventCreate(&guard.a));
  ENS_CU(cudaEventCreate(&guard.b));
  cudaEvent_t a = guard.a, b = guard.b;
  // timing launches read the state and write the spare block only (t is not advanced)
  int64_t launched = 0;
  for (int walk = 0; walk < 4; ++walk) {
    for (int occ = 0; occ < 2; ++occ) {
      for (int vx : vx_cand) {
        for (int passes : pass_cand) {
          int rc = ens_plan(e, vx, passes, occ, walk);
          if (rc) return rc;
          ENS_CU(launch_batch_prep(e->dmem, e->n, e->t_dev, 0, e->noise_mode, e->noise_dist, e->dsteps, e->stream));
          ENS_CU(ens_launch(e));
          ENS_CU(cudaEventRecord(a, e->stream));
          for (int k = 0; k < steps; ++k) ENS_CU(ens_launch(e));
          ENS_CU(cudaEventRecord(b, e->stream));
          ENS_CU(cudaEventSynchronize(b));
          launched += 1 + int64_t(1 + steps) * ens_step_launches(e);
          float ms = 0.0f;
          ENS_CU(cudaEventElapsedTime(&ms, a, b));
          if (best_ms < 0.0f || ms < best_ms) {
            best_ms = ms;
            best_vx = vx;
            best_passes = passes;
            best_occ = occ;
            best_walk = walk;
          }
        }
      }
    }
  }
  count_launches(launched);
  int rc = ens_plan(e, best_vx, best_passes, best_occ, best_walk);
  if (rc) return rc;
  guard.finished = true;
  if (vx_chosen) *vx_chosen = best_vx;
  if (passes_chosen) *passes_chosen = best_passes;
  if (blocks_per_sm) *blocks_per_sm = e->bps;
  return LBFD_OK;
}

int lbfd_ensemble_plan(lbfd_ens_t e, int32_t vx_max, int32_t passes, int32_t occupancy, int32_t walk) {
  if (!e || (vx_max != 1 && vx_max != 2) || (passes != 1 && passes != 2 && passes != 4 && passes != 8) ||
      (occupancy != 0 && occupancy != 1) ||
      (walk != LBFD_WALK_STRIDED && walk != LBFD_WALK_CONTIGUOUS && walk != LBFD_WALK_PER_TILE &&
       walk != LBFD_WALK_PARAM))
    return ens_fail(LBFD_EINVAL, "lbfd_ensemble_plan: bad argument");
  DevGuard g(e->device);
  ENS_CU(ens_sync_t(e));
  return ens_plan(e, vx_max, passes, occupancy, walk);
}

int lbfd_ensemble_query(lbfd_ens_t e, int32_t *n_members, int64_t *total_sites, int64_t *t, int32_t *vx,
                        int32_t *passes, int32_t *blocks_per_sm, int32_t *walk) {
  if (!e) return ens_fail(LBFD_EINVAL, "lbfd_ensemble_query: null handle");
  if (n_members) *n_members = e->n;
  if (total_sites) *total_sites = e->total_sites;
  if (t) *t = e->t;
  if (vx) *vx = e->vx_max;
  if (passes) *passes = e->passes;
  if (blocks_per_sm) *blocks_per_sm = e->bps;
  if (walk) *walk = e->walk;
  return LBFD_OK;
}

static int ens_member_ok(lbfd_ens_t e, int32_t m) { return e && m >= 0 && m < e->n; }

int lbfd_ensemble_get_f(lbfd_ens_t e, int32_t member, double *f_host) {
  if (!ens_member_ok(e, member) || !f_host) return ens_fail(LBFD_EINVAL, "lbfd_ensemble_get_f: bad argument");
  DevGuard g(e->device);
  const BatchMember &bm = e->hmem[member];
  const size_t count = size_t(e->Q) * bm.N;
  ENS_CU(launch_shift(e->lattice, e->elem, e->block(member, 0), e->block(member, 1), bm.Lx, bm.Ly, bm.Lz, +1,
                      e->stream));
  std::vector<uint8_t> raw(count * e->elem);
  ENS_CU(cudaMemcpyAsync(raw.data(), e->block(member, 1), raw.size(), cudaMemcpyDeviceToHost, e->stream));
  ENS_CU(cudaStreamSynchronize(e->stream));
  int Q = 0, D = 0, v[LBFD_MAX_Q * 3];
  double w[LBFD_MAX_Q];
  lattice_table(e->lattice, &Q, &D, v, w);
  dispatch_storage(e->precision, [&](auto tag) {
    using S = typename decltype(tag)::type;
    const S *p = reinterpret_cast<const S *>(raw.data());
    for (int i = 0; i < Q; ++i)
      for (int64_t s = 0; s < bm.N; ++s) f_host[i * bm.N + s] = Store<S>::getd(p[i * bm.N + s], w[i] * bm.rho_mean);
    return cudaSuccess;
  });
  return LBFD_OK;
}

int lbfd_ensemble_set_f(lbfd_ens_t e, int32_t member, const double *f_host) {
  if (!ens_member_ok(e, member) || !f_host) return ens_fail(LBFD_EINVAL, "lbfd_ensemble_set_f: bad argument");
  DevGuard g(e->device);
  const BatchMember &bm = e->hmem[member];
  const size_t count = size_t(e->Q) * bm.N;
  std::vector<uint8_t> raw(count * e->elem);
  int Q = 0, D = 0, v[LBFD_MAX_Q * 3];
  double w[LBFD_MAX_Q];
  lattice_table(e->lattice, &Q, &D, v, w);
  dispatch_storage(e->precision, [&](auto tag) {
    using S = typename decltype(tag)::type;
    S *p = reinterpret_cast<S *>(raw.data());
    for (int i = 0; i < Q; ++i)
      for (int64_t s = 0; s < bm.N; ++s) p[i * bm.N + s] = Store<S>::putd(f_host[i * bm.N + s], w[i] * bm.rho_mean);
    return cudaSuccess;
  });
  ENS_CU(cudaMemcpyAsync(e->block(member, 1), raw.data(), raw.size(), cudaMemcpyHostToDevice, e->stream));
  ENS_CU(launch_shift(e->lattice, e->elem, e->block(member, 1), e->block(member, 0), bm.Lx, bm.Ly, bm.Lz, -1,
                      e->stream));
  ENS_CU(cudaStreamSynchronize(e->stream));
  return LBFD_OK;
}

int lbfd_ensemble_mass(lbfd_ens_t e, int32_t member, double *mass) {
  if (!ens_member_ok(e, member) || !mass) return ens_fail(LBFD_EINVAL, "lbfd_ensemble_mass: bad argument");
  DevGuard g(e->device);
  const BatchMember &bm = e->hmem[member];
  ENS_CU(launch_mass(e->lattice, e->precision, e->block(member, 0), bm.N, bm.rho_mean, e->partials, e->d_mass,
                     e->stream));
  ENS_CU(cudaMemcpyAsync(mass, e->d_mass, sizeof(double), cudaMemcpyDeviceToHost, e->stream));
  ENS_CU(cudaStreamSynchronize(e->stream));
  return LBFD_OK;
}

}  // extern "C"
