// The serving loop (include/lbfd.h, "serving"): continuous batching of
// simulation requests on one GPU.
//
// State.  One device arena (the budget) holds every resident simulation: two
// population blocks A and B (the batched kernel's blocks 0 and 1) plus, for
// a density result of a lattice whose block is smaller than N doubles, a
// result area.  Ranges are carved with the host RangePool, so admission and
// retirement never allocate.  A simulation admitted when the server clock is
// c gets t0 = c: its own step counter is t = clock - t0, its state lives in
// block t & 1, and its noise is keyed by (its seed, its lattice id, t), as if
// it ran alone.
//
// One time step (tick) of the server, on the compute stream:
//   [table upload, when the resident set changed]  one copy from pinned staging
//   k_batch_prep                                   step arguments of every member
//   batched step per lattice type                  one launch covers all members of that type
//                                                  (k_batch_tile or k_batch_step, by the walk option)
//   k_step per simulation of >= solo_sites sites   the single-lattice kernel, parameters as
//                                                  kernel arguments
// (forked onto side streams when there is more than one launch, joined after)
// then, for each member that has taken its steps, a result kernel (streaming
// shift or density) into its spare block, and on the copy stream the
// device-to-host copy of that result.  The host sees the copy's event
// complete, stamps the completion time and returns the range to the pool.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstring>
#include <new>
#include <set>
#include <string>
#include <thread>
#include <utility>
#include <vector>

#include "batch.h"
#include "lbfd.h"
#include "pool.h"

using namespace lbfd;


namespace {

constexpr int64_t kAlign = 256;
constexpr int kStageSlots = 4;
constexpr int kMaxSlots = 65536;
constexpr int kAdmitScan = 1024;  // queued requests looked at per admission round

double now_s() {
  return std::chrono::duration<double>(std::chrono::steady_clock::now().time_since_epoch()).count();
}

int srv_fail(int code, const std::string &msg) { return set_last_error(code, msg); }

int srv_cuda(const char *what, cudaError_t e) {
  // the runtime keeps a failed call's error as the thread's last error;
  // clear it so that the next launch check does not report it again
  (void)cudaGetLastError();
  return srv_fail(e == cudaErrorMemoryAllocation ? LBFD_ENOMEM : LBFD_ECUDA,
                  std::string(what) + ": " + cudaGetErrorName(e) + " (" + cudaGetErrorString(e) + ")");
}

#define SRV_CU(call)                                   \
  do {                                                 \
    cudaError_t e_ = (call);                           \
    if (e_ != cudaSuccess) return srv_cuda(#call, e_); \
  } while (0)

#define SRV_RC(call)       \
  do {                     \
    int rc_ = (call);      \
    if (rc_) return rc_;   \
  } while (0)

struct DevScope {
  int prev = -1;
  explicit DevScope(int dev) {
    if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
    if (dev >= 0 && dev != prev) cudaSetDevice(dev);
  }
  ~DevScope() {
    int cur = -1;
    if (prev >= 0 && cudaGetDevice(&cur) == cudaSuccess && cur != prev) cudaSetDevice(prev);
  }
};

int q_of(int lattice) { return lattice == LBFD_D1Q3 ? 3 : (lattice == LBFD_D2Q9 ? 9 : 19); }
int d_of(int lattice) { return lattice == LBFD_D1Q3 ? 1 : (lattice == LBFD_D2Q9 ? 2 : 3); }
int64_t round_up(int64_t v, int64_t a) { return (v + a - 1) / a * a; }

enum ReqState : int { kQueued = LBFD_REQ_QUEUED, kRunning = LBFD_REQ_RUNNING, kDone = LBFD_REQ_DONE, kCopying = 3 };

struct SrvRequest {
  lbfd_request r{};
  int state = kQueued;
  int Q = 0;
  int64_t N = 0;
  int64_t block = 0;          // bytes of one population block (aligned)
  int64_t region_bytes = 0;   // blocks A, B (+ density area)
  int64_t result_bytes = 0;   // bytes copied to the host
  int64_t region = -1;        // arena offset
  int64_t sink = -1;          // sink offset, when the result goes to the trace sink
  uint64_t t0 = 0;
  int64_t work = 0;           // sites x steps
  double t_submit = 0.0, t_done = 0.0;
  cudaEvent_t ev = nullptr;   // result copy finished
};

}  // namespace

struct lbfd_server {
  lbfd_server_options opt{};
  int device = 0, elem = 4, sms = 1;
  int bps[3][2] = {{1, 1}, {1, 1}, {1, 1}};  // per lattice type and largest sites per item (1, 2)
  cudaStream_t cs = nullptr, xs = nullptr;  // compute, copy
  cudaStream_t ls[3] = {nullptr, nullptr, nullptr};  // per lattice type, so the launches of a tick overlap
  cudaEvent_t prep_ev = nullptr, lat_ev[3] = {nullptr, nullptr, nullptr};
  // simulations of at least solo_sites sites take the single-lattice kernel,
  // one launch each per step, spread over these streams
  static constexpr int kSoloStreams = 4;
  cudaStream_t ss[kSoloStreams] = {};
  cudaEvent_t solo_ev[kSoloStreams] = {};
  cudaEvent_t fork_ev = nullptr;
  std::vector<int64_t> solo;
  char *arena = nullptr;
  RangePool *pool = nullptr;
  // result sink of run_trace (caller's pinned buffer)
  char *sink = nullptr;
  RangePool *sink_pool = nullptr;
  // device tables: every member of the resident set, segmented by lattice type
  BatchMember *d_members = nullptr;
  int64_t *d_tile_start = nullptr;
  BatchStep *d_steps = nullptr;
  // pinned staging of the tables, reused round-robin once its copy is done
  char *stage[kStageSlots] = {};
  cudaEvent_t stage_ev[kStageSlots] = {};
  int stage_next = 0;
  std::vector<cudaEvent_t> tick_ev;  // ring of max_ahead: the host waits on the step max_ahead back
  cudaEvent_t ready_ev = nullptr;    // result kernel done (compute -> copy stream)
  std::vector<cudaEvent_t> spare_events;
  std::vector<SrvRequest> reqs;
  std::set<std::pair<int64_t, int64_t>> queue;  // (priority, id)
  std::vector<int64_t> active[3];
  std::vector<int64_t> copying;
  std::vector<int64_t> pending;  // results waiting for room in the trace sink
  bool dirty = true;
  int seg_off[3] = {0, 0, 0}, seg_n[3] = {0, 0, 0}, seg_vx[3] = {1, 1, 1};
  int64_t seg_tiles[3] = {0, 0, 0};
  // parameter-space launches (tile order LBFD_WALK_PARAM): the segment's
  // members in groups of up to kParamMembers, rebuilt with every table upload
  std::vector<BatchParams> groups[3];
  uint64_t clock = 0;
  int64_t n_done = 0, site_updates = 0, resident_bytes = 0, peak_resident_bytes = 0, resident_sites = 0,
          peak_resident_sites = 0, launches = 0;
  int n_active = 0, peak_active = 0;
  int64_t largest_free = 0;
};

namespace {

cudaError_t get_event(lbfd_server *s, cudaEvent_t *ev) {
  if (!s->spare_events.empty()) {
    *ev = s->spare_events.back();
    s->spare_events.pop_back();
    return cudaSuccess;
  }
  return cudaEventCreateWithFlags(ev, cudaEventDisableTiming);
}

void server_free(lbfd_server *s) {
  if (!s) return;
  for (SrvRequest &r : s->reqs)
    if (r.ev) cudaEventDestroy(r.ev);
  for (cudaEvent_t e : s->spare_events) cudaEventDestroy(e);
  for (cudaEvent_t e : s->tick_ev)
    if (e) cudaEventDestroy(e);
  for (int k = 0; k < kStageSlots; ++k) {
    if (s->stage_ev[k]) cudaEventDestroy(s->stage_ev[k]);
    if (s->stage[k]) cudaFreeHost(s->stage[k]);
  }
  if (s->ready_ev) cudaEventDestroy(s->ready_ev);
  if (s->prep_ev) cudaEventDestroy(s->prep_ev);
  if (s->fork_ev) cudaEventDestroy(s->fork_ev);
  for (int k = 0; k < lbfd_server::kSoloStreams; ++k) {
    if (s->solo_ev[k]) cudaEventDestroy(s->solo_ev[k]);
    if (s->ss[k]) cudaStreamDestroy(s->ss[k]);
  }
  for (int L = 0; L < 3; ++L) {
    if (s->lat_ev[L]) cudaEventDestroy(s->lat_ev[L]);
    if (s->ls[L]) cudaStreamDestroy(s->ls[L]);
  }
  cudaFree(s->d_members);
  cudaFree(s->d_tile_start);
  cudaFree(s->d_steps);
  cudaFree(s->arena);
  if (s->cs) cudaStreamDestroy(s->cs);
  if (s->xs) cudaStreamDestroy(s->xs);
  delete s->pool;
  delete s->sink_pool;
  delete s;
}

size_t stage_bytes(const lbfd_server *s) {
  return (sizeof(BatchMember) + sizeof(int64_t)) * static_cast<size_t>(s->opt.max_active);
}

// Validates a request and fills its sizes.  in_trace: results may go to the sink.
int prepare_request(lbfd_server *s, const lbfd_request &r, SrvRequest &q, bool in_trace) {
  if (r.lattice < LBFD_D1Q3 || r.lattice > LBFD_D3Q19) return srv_fail(LBFD_EINVAL, "request: unknown lattice");
  const int D = d_of(r.lattice);
  for (int a = 0; a < 3; ++a)
    if (r.dims[a] < 1 || (a >= D && r.dims[a] != 1) || r.dims[a] > 0x7fffffffLL)
      return srv_fail(LBFD_EINVAL, "request: bad dimensions");
  if (r.dims[1] > 65535 || r.dims[2] > 65535) return srv_fail(LBFD_EINVAL, "request: Ly and Lz must be <= 65535");
  const double sites = double(r.dims[0]) * double(r.dims[1]) * double(r.dims[2]);
  if (sites >= 2147483648.0) return srv_fail(LBFD_EINVAL, "request: 2^31 sites or more");
  if (double(q_of(r.lattice)) * sites > 4294967295.0) return srv_fail(LBFD_EINVAL, "request: Q * sites must be < 2^32");
  if (!(r.tau > 0.5) || !std::isfinite(r.tau)) return srv_fail(LBFD_EINVAL, "request: tau must be > 1/2");
  if (!(r.rho_mean >= 0.0) || !std::isfinite(r.rho_mean))
    return srv_fail(LBFD_EINVAL, "request: rho_mean must be >= 0");
  if (r.steps < 0) return srv_fail(LBFD_EINVAL, "request: steps must be >= 0");
  if (r.init != LBFD_INIT_UNIFORM && r.init != LBFD_INIT_SINE && r.init != LBFD_INIT_HOST)
    return srv_fail(LBFD_EINVAL, "request: init must be LBFD_INIT_UNIFORM, LBFD_INIT_SINE or LBFD_INIT_HOST");
  if (r.init == LBFD_INIT_HOST && !r.in_host) return srv_fail(LBFD_EINVAL, "request: LBFD_INIT_HOST needs in_host");
  if (r.result < LBFD_RESULT_F || r.result > LBFD_RESULT_NONE)
    return srv_fail(LBFD_EINVAL, "request: unknown result kind");
  q.r = r;
  q.Q = q_of(r.lattice);
  q.N = int64_t(sites);
  q.work = q.N * r.steps;
  q.block = round_up(int64_t(q.Q) * q.N * s->elem, kAlign);
  const bool rho_area = r.result == LBFD_RESULT_RHO && int64_t(q.Q) * s->elem < 8;
  q.region_bytes = 2 * q.block + (rho_area ? round_up(8 * q.N, kAlign) : 0);
  q.result_bytes = r.result == LBFD_RESULT_F ? int64_t(q.Q) * q.N * s->elem : (r.result == LBFD_RESULT_RHO ? 8 * q.N : 0);
  if (q.region_bytes > s->pool->capacity())
    return srv_fail(LBFD_EINVAL, "request: its state (" + std::to_string(q.region_bytes) +
                                     " bytes) exceeds the server's device-memory budget");
  if (s->opt.max_active_sites > 0 && q.N > s->opt.max_active_sites)
    return srv_fail(LBFD_EINVAL, "request: more sites than the server's max_active_sites");
  if (q.result_bytes > 0 && !r.out_host) {
    if (!in_trace) return srv_fail(LBFD_EINVAL, "request: out_host is needed for this result kind");
    if (!s->sink_pool || q.result_bytes > s->sink_pool->capacity())
      return srv_fail(LBFD_EINVAL, "request: its result does not fit the trace's sink buffer");
  }
  return LBFD_OK;
}

int64_t submit_request(lbfd_server *s, SrvRequest &&q, double t_submit) {
  const int64_t id = static_cast<int64_t>(s->reqs.size());
  q.t_submit = t_submit;
  q.state = kQueued;
  const int64_t prio = s->opt.policy == LBFD_POLICY_SHORTEST  ? q.work
                       : s->opt.policy == LBFD_POLICY_LONGEST ? -q.work
                                                              : id;
  s->reqs.push_back(std::move(q));
  s->queue.insert({prio, id});
  return id;
}

// Result of request id (its state has taken r.steps steps): result kernel on
// the compute stream, copy on the copy stream, completion event.  A result
// bound for the trace sink waits (state untouched in its blocks) until the
// sink has room.
int schedule_result(lbfd_server *s, int64_t id) {
  SrvRequest &q = s->reqs[id];
  const lbfd_request &r = q.r;
  q.state = kCopying;
  if (q.result_bytes > 0 && !r.out_host && q.sink < 0) {
    q.sink = s->sink_pool ? s->sink_pool->alloc(q.result_bytes) : -1;
    if (q.sink < 0) {
      s->pending.push_back(id);
      return LBFD_OK;
    }
  }
  char *A = s->arena + q.region;
  char *cur = (r.steps & 1) ? A + q.block : A;
  char *spare = (r.steps & 1) ? A : A + q.block;
  const char *src = nullptr;
  if (r.result == LBFD_RESULT_F) {
    SRV_CU(launch_shift(r.lattice, s->elem, cur, spare, int32_t(r.dims[0]), int32_t(r.dims[1]), int32_t(r.dims[2]), +1,
                        s->cs));
    src = spare;
    s->launches += 1;
  } else if (r.result == LBFD_RESULT_RHO) {
    double *rho = reinterpret_cast<double *>(int64_t(q.Q) * s->elem >= 8 ? spare : A + 2 * q.block);
    SRV_CU(launch_density_of_state(r.lattice, s->opt.precision, cur, int32_t(r.dims[0]), int32_t(r.dims[1]),
                                   int32_t(r.dims[2]), r.rho_mean, rho, s->cs));
    src = reinterpret_cast<const char *>(rho);
    s->launches += 1;
  }
  SRV_CU(get_event(s, &q.ev));
  if (src) {
    void *dst = r.out_host ? r.out_host : static_cast<void *>(s->sink + q.sink);
    SRV_CU(cudaEventRecord(s->ready_ev, s->cs));
    SRV_CU(cudaStreamWaitEvent(s->xs, s->ready_ev, 0));
    SRV_CU(cudaMemcpyAsync(dst, src, size_t(q.result_bytes), cudaMemcpyDeviceToHost, s->xs));
    SRV_CU(cudaEventRecord(q.ev, s->xs));
  } else {
    SRV_CU(cudaEventRecord(q.ev, s->cs));
  }
  s->copying.push_back(id);
  return LBFD_OK;
}

// Notes finished result copies: stamps, releases ranges.
int retire(lbfd_server *s) {
  size_t keep = 0;
  for (size_t k = 0; k < s->copying.size(); ++k) {
    const int64_t id = s->copying[k];
    SrvRequest &q = s->reqs[id];
    const cudaError_t e = cudaEventQuery(q.ev);
    if (e == cudaErrorNotReady) {
      s->copying[keep++] = id;
      continue;
    }
    if (e != cudaSuccess) {
      s->copying.resize(keep);  // the rest stay unretired; the server is unusable after a CUDA error
      return srv_cuda("cudaEventQuery(result copy)", e);
    }
    q.t_done = now_s();
    q.state = kDone;
    s->spare_events.push_back(q.ev);
    q.ev = nullptr;
    s->pool->release(q.region);
    if (q.sink >= 0) s->sink_pool->release(q.sink);
    q.region = q.sink = -1;
    s->resident_bytes -= q.region_bytes;
    s->resident_sites -= q.N;
    s->n_done += 1;
    s->site_updates += q.work;
  }
  s->copying.resize(keep);
  s->largest_free = s->pool->largest_free();
  // results that waited for sink space
  if (!s->pending.empty()) {
    std::vector<int64_t> waiting;
    waiting.swap(s->pending);
    for (int64_t id : waiting) SRV_RC(schedule_result(s, id));
  }
  return LBFD_OK;
}

// Initial state of an admitted request into block A (t = 0): f into B, then
// the inverse streaming shift into A.
int start_request(lbfd_server *s, int64_t id) {
  SrvRequest &q = s->reqs[id];
  const lbfd_request &r = q.r;
  char *A = s->arena + q.region, *B = A + q.block;
  const int32_t Lx = int32_t(r.dims[0]), Ly = int32_t(r.dims[1]), Lz = int32_t(r.dims[2]);
  if (r.init == LBFD_INIT_HOST) {
    SRV_CU(cudaMemcpyAsync(B, r.in_host, size_t(q.Q) * q.N * s->elem, cudaMemcpyHostToDevice, s->cs));
  } else {
    const double amp = r.init == LBFD_INIT_SINE ? r.sine_amp : 0.0;
    SRV_CU(launch_init(r.lattice, s->opt.precision, B, Lx, Ly, Lz, r.rho_mean, amp, r.sine_k, s->cs));
    s->launches += 1;
  }
  SRV_CU(launch_shift(r.lattice, s->elem, B, A, Lx, Ly, Lz, -1, s->cs));
  s->launches += 1;
  q.t0 = s->clock;
  q.state = kRunning;
  s->resident_bytes += q.region_bytes;
  s->resident_sites += q.N;
  s->peak_resident_bytes = std::max(s->peak_resident_bytes, s->resident_bytes);
  s->peak_resident_sites = std::max(s->peak_resident_sites, s->resident_sites);
  if (r.steps == 0) return schedule_result(s, id);
  s->active[r.lattice].push_back(id);
  s->n_active += 1;
  s->peak_active = std::max(s->peak_active, s->n_active);
  s->dirty = true;
  return LBFD_OK;
}

// Admits queued requests while slots, memory and the site limit allow.
int admit(lbfd_server *s) {
  int scanned = 0;
  for (auto it = s->queue.begin(); it != s->queue.end() && scanned < kAdmitScan;) {
    if (s->n_active >= s->opt.max_active) break;
    ++scanned;
    const int64_t id = it->second;
    SrvRequest &q = s->reqs[id];
    if (q.region_bytes > s->largest_free ||
        (s->opt.max_active_sites > 0 && s->resident_sites + q.N > s->opt.max_active_sites)) {
      ++it;
      continue;
    }
    const int64_t region = s->pool->alloc(q.region_bytes);
    if (region < 0) {
      ++it;
      continue;
    }
    q.region = region;
    q.sink = -1;
    it = s->queue.erase(it);
    s->largest_free = s->pool->largest_free();
    SRV_RC(start_request(s, id));
  }
  return LBFD_OK;
}

// Uploads the member tables of the resident set (segments D1Q3, D2Q9, D3Q19).
int upload_tables(lbfd_server *s) {
  const int slot = s->stage_next;
  s->stage_next = (s->stage_next + 1) % kStageSlots;
  SRV_CU(cudaEventSynchronize(s->stage_ev[slot]));  // its previous copy has finished
  BatchMember *hm = reinterpret_cast<BatchMember *>(s->stage[slot]);
  int64_t *hts = reinterpret_cast<int64_t *>(s->stage[slot] + sizeof(BatchMember) * size_t(s->opt.max_active));
  int n = 0;
  s->solo.clear();
  for (int L = 0; L < 3; ++L) {
    s->seg_off[L] = n;
    for (int64_t id : s->active[L]) {
      const SrvRequest &q = s->reqs[id];
      if (s->opt.solo_sites > 0 && q.N >= s->opt.solo_sites) {
        s->solo.push_back(id);
        continue;
      }
      hm[n++] = make_batch_member(q.r.dims, q.r.tau, q.r.rho_mean, q.r.seed, q.r.lattice_id, q.region / s->elem,
                                  (q.region + q.block) / s->elem, q.t0, s->opt.vx_max);
    }
    s->seg_n[L] = n - s->seg_off[L];
    s->seg_vx[L] = 1;
    for (int m = s->seg_off[L]; m < n; ++m) s->seg_vx[L] = std::max(s->seg_vx[L], int(hm[m].vx));
    s->seg_tiles[L] = batch_assign_tiles(hm + s->seg_off[L], s->seg_n[L], s->opt.passes, hts + s->seg_off[L]);
    if (s->opt.walk == LBFD_WALK_PARAM)
      batch_build_params(hm + s->seg_off[L], s->seg_n[L], s->seg_tiles[L], s->opt.noise_mode, s->opt.noise_dist,
                         s->groups[L]);
  }
  if (n > 0) {
    SRV_CU(cudaMemcpyAsync(s->d_members, hm, sizeof(BatchMember) * size_t(n), cudaMemcpyHostToDevice, s->cs));
    SRV_CU(cudaMemcpyAsync(s->d_tile_start, hts, sizeof(int64_t) * size_t(n), cudaMemcpyHostToDevice, s->cs));
  }
  SRV_CU(cudaEventRecord(s->stage_ev[slot], s->cs));
  s->dirty = false;
  return LBFD_OK;
}

// One time step of every resident simulation, then results of those done.
int tick(lbfd_server *s) {
  NvtxRange nvtx_("server tick");
  if (s->n_active == 0) return LBFD_OK;
  const int ring = int(s->tick_ev.size());
  const int slot = int(s->clock % uint64_t(ring));
  if (s->clock >= uint64_t(ring)) SRV_CU(cudaEventSynchronize(s->tick_ev[slot]));
  if (s->dirty) SRV_RC(upload_tables(s));
  const int n = s->seg_off[2] + s->seg_n[2];
  int types = 0;
  for (int L = 0; L < 3; ++L) types += s->seg_n[L] > 0;
  const bool fork = types + int64_t(s->solo.size()) > 1;
  if (n > 0) {
    SRV_CU(launch_batch_prep(s->d_members, n, nullptr, s->clock, s->opt.noise_mode, s->opt.noise_dist, s->d_steps,
                             s->cs));
    s->launches += 1;
  }
  // one batched launch per lattice type, and one single-lattice launch per
  // large simulation; with more than one launch they run on their own
  // streams, forked here and joined before anything else uses the state
  if (fork) SRV_CU(cudaEventRecord(s->fork_ev, s->cs));
  for (int L = 0; L < 3; ++L) {
    if (s->seg_n[L] == 0) continue;
    cudaStream_t st = fork ? s->ls[L] : s->cs;
    if (fork) SRV_CU(cudaStreamWaitEvent(st, s->fork_ev, 0));
    const int vx = s->seg_vx[L];
    if (s->opt.walk == LBFD_WALK_PARAM) {
      // one launch per group, the members' arguments in the kernel parameters
      const int G = static_cast<int>(s->groups[L].size());
      SRV_CU(launch_batch_param(L, s->opt.precision, s->arena, s->groups[L].data(), G, s->d_steps + s->seg_off[L],
                                s->opt.passes, s->opt.occupancy, vx, s->opt.noise_mode, s->opt.noise_dist, st));
      s->launches += G;
    } else {
      const int grid =
          int(std::max<int64_t>(1, std::min<int64_t>(s->seg_tiles[L], int64_t(s->sms) * s->bps[L][vx - 1])));
      SRV_CU(launch_batch_step(L, s->opt.precision, s->arena, s->d_steps + s->seg_off[L],
                               s->d_tile_start + s->seg_off[L], s->seg_n[L], s->seg_tiles[L], s->opt.passes,
                               s->opt.occupancy, s->opt.walk, vx, s->opt.noise_mode, s->opt.noise_dist, grid, st));
      s->launches += 1;
    }
    if (fork) {
      SRV_CU(cudaEventRecord(s->lat_ev[L], st));
      SRV_CU(cudaStreamWaitEvent(s->cs, s->lat_ev[L], 0));
    }
  }
  if (!s->solo.empty()) {
    const int nst = std::min<int>(lbfd_server::kSoloStreams, int(s->solo.size()));
    for (int k = 0; k < nst; ++k)
      if (fork) SRV_CU(cudaStreamWaitEvent(s->ss[k], s->fork_ev, 0));
    for (size_t k = 0; k < s->solo.size(); ++k) {
      const SrvRequest &q = s->reqs[s->solo[k]];
      const uint64_t t = s->clock - q.t0;  // the simulation's own step counter
      StepArgs a{};
      a.Lx = int32_t(q.r.dims[0]);
      a.Ly = int32_t(q.r.dims[1]);
      a.Lz = int32_t(q.r.dims[2]);
      a.N = q.N;
      fill_step_params(a, q.r.tau, q.r.rho_mean);
      a.noise_mode = s->opt.noise_mode;
      a.noise_dist = s->opt.noise_dist;
      a.ph = make_philox_step(q.r.seed, q.r.lattice_id, t);
      char *A = s->arena + q.region;
      char *src = (t & 1) ? A + q.block : A;
      char *dst = (t & 1) ? A : A + q.block;
      SRV_CU(launch_step(q.r.lattice, s->opt.precision, src, dst, a, fork ? s->ss[k % nst] : s->cs));
      s->launches += 1;
    }
    for (int k = 0; k < nst && fork; ++k) {
      SRV_CU(cudaEventRecord(s->solo_ev[k], s->ss[k]));
      SRV_CU(cudaStreamWaitEvent(s->cs, s->solo_ev[k], 0));
    }
  }
  SRV_CU(cudaEventRecord(s->tick_ev[slot], s->cs));
  // members whose step counter reaches their step count after this step
  for (int L = 0; L < 3; ++L) {
    std::vector<int64_t> &act = s->active[L];
    size_t keep = 0;
    for (size_t k = 0; k < act.size(); ++k) {
      const int64_t id = act[k];
      const SrvRequest &q = s->reqs[id];
      if (int64_t(s->clock - q.t0) + 1 == q.r.steps) {
        s->n_active -= 1;
        s->dirty = true;
        SRV_RC(schedule_result(s, id));
      } else {
        act[keep++] = id;
      }
    }
    act.resize(keep);
  }
  s->clock += 1;
  return LBFD_OK;
}

int64_t unfinished(const lbfd_server *s) {
  return int64_t(s->queue.size()) + s->n_active + int64_t(s->copying.size()) + int64_t(s->pending.size());
}

int pump(lbfd_server *s, int32_t max_steps) {
  for (int32_t k = 0; k < max_steps; ++k) {
    SRV_RC(retire(s));
    SRV_RC(admit(s));
    if (s->n_active == 0) break;
    SRV_RC(tick(s));
  }
  SRV_RC(retire(s));
  return LBFD_OK;
}

// Blocks until the oldest outstanding result copy has finished.
int wait_oldest_copy(lbfd_server *s) {
  if (s->copying.empty()) return LBFD_OK;
  SRV_CU(cudaEventSynchronize(s->reqs[s->copying.front()].ev));
  return LBFD_OK;
}

}  // namespace

extern "C" {

int lbfd_server_options_init(lbfd_server_options *opt) {
  if (!opt) return srv_fail(LBFD_EINVAL, "lbfd_server_options_init: null");
  std::memset(opt, 0, sizeof(*opt));
  opt->precision = LBFD_F32;
  opt->noise_mode = LBFD_NOISE_LOCAL;
  opt->noise_dist = LBFD_GAUSSIAN;
  opt->device = -1;
  opt->hbm_budget = int64_t(1) << 30;
  opt->max_active_sites = 0;
  opt->max_active = 1024;
  opt->max_ahead = 4;
  opt->passes = 1;
  opt->policy = LBFD_POLICY_FIFO;
  opt->walk = LBFD_WALK_PER_TILE;
  opt->vx_max = 2;
  opt->solo_sites = int64_t(1) << 17;
  return LBFD_OK;
}

int lbfd_server_create(lbfd_server_t *out, const lbfd_server_options *opt) {
  if (!out || !opt) return srv_fail(LBFD_EINVAL, "lbfd_server_create: bad argument");
  *out = nullptr;
  const lbfd_server_options &o = *opt;
  if (o.precision < LBFD_F32 || o.precision > LBFD_F32_BF16) return srv_fail(LBFD_EINVAL, "server: unknown precision");
  if (o.noise_mode < LBFD_NOISE_LOCAL || o.noise_mode > LBFD_NOISE_OFF)
    return srv_fail(LBFD_EINVAL, "server: unknown noise mode");
  if (o.noise_dist != LBFD_GAUSSIAN && o.noise_dist != LBFD_UNIFORM)
    return srv_fail(LBFD_EINVAL, "server: unknown noise distribution");
  if (o.hbm_budget < kAlign) return srv_fail(LBFD_EINVAL, "server: hbm_budget too small");
  if (o.max_active < 1 || o.max_active > kMaxSlots)
    return srv_fail(LBFD_EINVAL, "server: max_active must be in [1, 65536]");
  if (o.max_ahead < 1 || o.max_ahead > 1024) return srv_fail(LBFD_EINVAL, "server: max_ahead must be in [1, 1024]");
  if (o.passes != 1 && o.passes != 2 && o.passes != 4 && o.passes != 8)
    return srv_fail(LBFD_EINVAL, "server: passes must be 1, 2, 4 or 8");
  if (o.policy != LBFD_POLICY_FIFO && o.policy != LBFD_POLICY_SHORTEST && o.policy != LBFD_POLICY_LONGEST)
    return srv_fail(LBFD_EINVAL, "server: unknown policy");
  if (o.occupancy != 0 && o.occupancy != 1) return srv_fail(LBFD_EINVAL, "server: occupancy must be 0 or 1");
  if (o.vx_max != 1 && o.vx_max != 2) return srv_fail(LBFD_EINVAL, "server: vx_max must be 1 or 2");
  if (o.walk != LBFD_WALK_STRIDED && o.walk != LBFD_WALK_CONTIGUOUS && o.walk != LBFD_WALK_PER_TILE &&
      o.walk != LBFD_WALK_PARAM)
    return srv_fail(LBFD_EINVAL, "server: walk must be LBFD_WALK_STRIDED, _CONTIGUOUS, _PER_TILE or _PARAM");
  if (o.max_active_sites < 0) return srv_fail(LBFD_EINVAL, "server: max_active_sites must be >= 0");
  if (o.solo_sites < 0) return srv_fail(LBFD_EINVAL, "server: solo_sites must be >= 0");
  int dev = o.device;
  if (dev < 0) SRV_CU(cudaGetDevice(&dev));
  DevScope scope(dev);
  lbfd_server *s = new (std::nothrow) lbfd_server();
  if (!s) return srv_fail(LBFD_ENOMEM, "server: host allocation failed");
  s->opt = o;
  s->device = dev;
  s->elem = storage_bytes(o.precision);
  s->pool = new (std::nothrow) RangePool(o.hbm_budget, kAlign);
  cudaError_t err = s->pool ? cudaSuccess : cudaErrorMemoryAllocation;
  if (err == cudaSuccess) err = cudaDeviceGetAttribute(&s->sms, cudaDevAttrMultiProcessorCount, dev);
  if (err == cudaSuccess) err = cudaStreamCreateWithFlags(&s->cs, cudaStreamNonBlocking);
  if (err == cudaSuccess) err = cudaStreamCreateWithFlags(&s->xs, cudaStreamNonBlocking);
  if (err == cudaSuccess) err = cudaMalloc(&s->arena, size_t(s->pool->capacity()));
  if (err == cudaSuccess) err = cudaMalloc(&s->d_members, sizeof(BatchMember) * size_t(o.max_active));
  if (err == cudaSuccess) err = cudaMalloc(&s->d_tile_start, sizeof(int64_t) * size_t(o.max_active));
  if (err == cudaSuccess) err = cudaMalloc(&s->d_steps, sizeof(BatchStep) * size_t(o.max_active));
  for (int k = 0; k < kStageSlots && err == cudaSuccess; ++k) {
    err = cudaHostAlloc(reinterpret_cast<void **>(&s->stage[k]), stage_bytes(s), cudaHostAllocDefault);
    if (err == cudaSuccess) err = cudaEventCreateWithFlags(&s->stage_ev[k], cudaEventDisableTiming);
    if (err == cudaSuccess) err = cudaEventRecord(s->stage_ev[k], s->cs);
  }
  if (err == cudaSuccess) err = cudaEventCreateWithFlags(&s->ready_ev, cudaEventDisableTiming);
  if (err == cudaSuccess) err = cudaEventCreateWithFlags(&s->prep_ev, cudaEventDisableTiming);
  if (err == cudaSuccess) err = cudaEventCreateWithFlags(&s->fork_ev, cudaEventDisableTiming);
  for (int k = 0; k < lbfd_server::kSoloStreams && err == cudaSuccess; ++k) {
    err = cudaStreamCreateWithFlags(&s->ss[k], cudaStreamNonBlocking);
    if (err == cudaSuccess) err = cudaEventCreateWithFlags(&s->solo_ev[k], cudaEventDisableTiming);
  }
  for (int L = 0; L < 3 && err == cudaSuccess; ++L) {
    err = cudaStreamCreateWithFlags(&s->ls[L], cudaStreamNonBlocking);
    if (err == cudaSuccess) err = cudaEventCreateWithFlags(&s->lat_ev[L], cudaEventDisableTiming);
  }
  s->tick_ev.assign(size_t(o.max_ahead), nullptr);
  for (int k = 0; k < o.max_ahead && err == cudaSuccess; ++k)
    err = cudaEventCreateWithFlags(&s->tick_ev[k], cudaEventDisableTiming);
  if (err != cudaSuccess) {
    const int rc = srv_cuda("lbfd_server_create", err);
    server_free(s);
    return rc;
  }
  for (int L = 0; L < 3; ++L)
    for (int vx = 1; vx <= 2; ++vx)
      s->bps[L][vx - 1] = batch_blocks_per_sm(L, o.precision, o.occupancy, vx, o.walk, o.noise_mode, o.noise_dist);
  s->largest_free = s->pool->largest_free();
  *out = s;
  return LBFD_OK;
}

int lbfd_server_destroy(lbfd_server_t s) {
  if (!s) return LBFD_OK;
  DevScope scope(s->device);
  cudaError_t e1 = cudaStreamSynchronize(s->cs);
  cudaError_t e2 = cudaStreamSynchronize(s->xs);
  for (int L = 0; L < 3; ++L)
    if (e1 == cudaSuccess) e1 = cudaStreamSynchronize(s->ls[L]);
  for (int k = 0; k < lbfd_server::kSoloStreams; ++k)
    if (e1 == cudaSuccess) e1 = cudaStreamSynchronize(s->ss[k]);
  server_free(s);
  if (e1 != cudaSuccess) return srv_cuda("lbfd_server_destroy", e1);
  if (e2 != cudaSuccess) return srv_cuda("lbfd_server_destroy", e2);
  return LBFD_OK;
}

int lbfd_server_submit(lbfd_server_t s, const lbfd_request *req, int64_t *id) {
  if (!s || !req || !id) return srv_fail(LBFD_EINVAL, "lbfd_server_submit: bad argument");
  SrvRequest q;
  SRV_RC(prepare_request(s, *req, q, false));
  *id = submit_request(s, std::move(q), now_s());
  return LBFD_OK;
}

int lbfd_server_pump(lbfd_server_t s, int32_t max_steps, int64_t *left) {
  NvtxRange nvtx_("lbfd_server_pump");
  if (!s || max_steps < 0) return srv_fail(LBFD_EINVAL, "lbfd_server_pump: bad argument");
  DevScope scope(s->device);
  const int64_t l0 = s->launches;
  const int rc = pump(s, max_steps);
  count_launches(s->launches - l0);
  if (left) *left = unfinished(s);
  return rc;
}

int lbfd_server_drain(lbfd_server_t s) {
  NvtxRange nvtx_("lbfd_server_drain");
  if (!s) return srv_fail(LBFD_EINVAL, "lbfd_server_drain: null server");
  DevScope scope(s->device);
  const int64_t l0 = s->launches;
  int rc = LBFD_OK;
  while (rc == LBFD_OK && unfinished(s) > 0) {
    rc = pump(s, 64);
    if (rc == LBFD_OK && s->n_active == 0 && !s->copying.empty()) rc = wait_oldest_copy(s);
    if (rc == LBFD_OK && s->n_active == 0 && s->copying.empty() && !s->queue.empty()) {
      rc = srv_fail(LBFD_EBUSY, "lbfd_server_drain: queued requests cannot be admitted");
    }
  }
  count_launches(s->launches - l0);
  return rc;
}

int lbfd_server_poll(lbfd_server_t s, int64_t id, int32_t *state, double *latency_s) {
  if (!s || !state) return srv_fail(LBFD_EINVAL, "lbfd_server_poll: bad argument");
  if (id < 0 || id >= int64_t(s->reqs.size())) {
    *state = LBFD_REQ_UNKNOWN;
    return LBFD_OK;
  }
  const SrvRequest &q = s->reqs[id];
  *state = q.state == kCopying ? LBFD_REQ_RUNNING : q.state;
  if (latency_s) *latency_s = q.state == kDone ? q.t_done - q.t_submit : -1.0;
  return LBFD_OK;
}

int lbfd_server_get_stats(lbfd_server_t s, lbfd_server_stats *st) {
  if (!s || !st) return srv_fail(LBFD_EINVAL, "lbfd_server_get_stats: bad argument");
  std::memset(st, 0, sizeof(*st));
  st->submitted = int64_t(s->reqs.size());
  st->queued = int64_t(s->queue.size());
  st->running = s->n_active + int64_t(s->copying.size()) + int64_t(s->pending.size());
  st->done = s->n_done;
  st->clock = int64_t(s->clock);
  st->site_updates = s->site_updates;
  st->resident_bytes = s->resident_bytes;
  st->peak_resident_bytes = s->peak_resident_bytes;
  st->resident_sites = s->resident_sites;
  st->peak_resident_sites = s->peak_resident_sites;
  st->active = s->n_active;
  st->peak_active = s->peak_active;
  st->launches = s->launches;
  return LBFD_OK;
}

int lbfd_server_run_trace(lbfd_server_t s, const lbfd_request *reqs, const double *arrival_s, int32_t n,
                          void *sink_host, int64_t sink_bytes, double *latency_s, double *makespan_s) {
  NvtxRange nvtx_("lbfd_server_run_trace");
  if (!s || n < 0 || (n > 0 && (!reqs || !arrival_s || !latency_s)) || sink_bytes < 0 || (sink_bytes > 0 && !sink_host))
    return srv_fail(LBFD_EINVAL, "lbfd_server_run_trace: bad argument");
  for (int32_t k = 1; k < n; ++k)
    if (!(arrival_s[k] >= arrival_s[k - 1]))
      return srv_fail(LBFD_EINVAL, "lbfd_server_run_trace: arrivals must not decrease");
  if (s->sink_pool) return srv_fail(LBFD_EBUSY, "lbfd_server_run_trace: a trace is already running");
  DevScope scope(s->device);
  s->sink = static_cast<char *>(sink_host);
  s->sink_pool = new (std::nothrow) RangePool(sink_bytes, kAlign);
  if (!s->sink_pool) return srv_fail(LBFD_ENOMEM, "lbfd_server_run_trace: host allocation failed");
  // validate the whole trace before the clock starts
  std::vector<SrvRequest> prepared(static_cast<size_t>(n));
  int rc = LBFD_OK;
  for (int32_t k = 0; k < n && rc == LBFD_OK; ++k) rc = prepare_request(s, reqs[k], prepared[k], true);
  std::vector<int64_t> ids(size_t(n), -1);
  const int64_t l0 = s->launches;
  const double t_start = now_s();
  int32_t next = 0;
  while (rc == LBFD_OK) {
    const double now = now_s() - t_start;
    while (next < n && arrival_s[next] <= now) {
      ids[next] = submit_request(s, std::move(prepared[next]), t_start + arrival_s[next]);
      ++next;
    }
    rc = pump(s, 1);
    if (rc != LBFD_OK) break;
    if (next == n && unfinished(s) == 0) break;
    if (s->n_active == 0 && s->queue.empty() && s->copying.empty() && next < n) {
      // idle until the next arrival
      const double wait = arrival_s[next] - (now_s() - t_start);
      if (wait > 2e-3) std::this_thread::sleep_for(std::chrono::duration<double>(wait - 1e-3));
    }
  }
  double last = t_start;
  for (int32_t k = 0; k < n; ++k) {
    const SrvRequest *q = ids[k] >= 0 ? &s->reqs[ids[k]] : nullptr;
    latency_s[k] = (q && q->state == kDone) ? q->t_done - (t_start + arrival_s[k]) : -1.0;
    if (q && q->state == kDone) last = std::max(last, q->t_done);
  }
  if (makespan_s) *makespan_s = last - t_start;
  if (rc != LBFD_OK) {
    // results still in flight target the sink: wait for them before giving it
    // back, and drop queued trace requests, which have nowhere to write
    cudaStreamSynchronize(s->cs);
    cudaStreamSynchronize(s->xs);
    for (auto it = s->queue.begin(); it != s->queue.end();) {
      const SrvRequest &q = s->reqs[it->second];
      it = (q.result_bytes > 0 && !q.r.out_host) ? s->queue.erase(it) : std::next(it);
    }
  }
  delete s->sink_pool;
  s->sink_pool = nullptr;
  s->sink = nullptr;
  count_launches(s->launches - l0);
  return rc;
}

int lbfd_server_struct_sizes(int64_t *options_bytes, int64_t *request_bytes, int64_t *stats_bytes) {
  if (options_bytes) *options_bytes = int64_t(sizeof(lbfd_server_options));
  if (request_bytes) *request_bytes = int64_t(sizeof(lbfd_request));
  if (stats_bytes) *stats_bytes = int64_t(sizeof(lbfd_server_stats));
  return LBFD_OK;
}

}  // extern "C"
