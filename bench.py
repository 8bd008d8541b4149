"""Benchmark of the fused fluctuating lattice-Boltzmann step on GB300.

One benchmark step is one time step of eq. LB (pull-stream, density, relax,
Philox noise in the non-conserved moments, store) over the whole lattice.
Default workload: D2Q9, FP32, periodic 2048 x 2048, tau = 0.8,
rho_mean = 100, local Gaussian noise, uniform start.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--workload d2q9|d3q19|d1q3] [--impl reference]

Prints one JSON line (rank 0).  Under torchrun each rank runs its own
lattice (seed and Philox lattice id offset by the rank): independent
replicas, weak scaling, no collective on the data path.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import re
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "GLUPS & % of HBM peak vs plain per-sim launch; served p50/p99 latency"
UNIT = "GLUPS"

WORKLOADS = {
    "d2q9": dict(lattice=1, dims=(2048, 2048), tau=0.8, rho=100.0, precision=0,
                 name="D2Q9 FP32 periodic 2048x2048, tau=0.8, rho_mean=100, local Gaussian noise, uniform start"),
    "d3q19": dict(lattice=2, dims=(256, 256, 256), tau=1.0, rho=50.0, precision=0,
                  name="D3Q19 FP32 periodic 256^3, tau=1.0, rho_mean=50, local Gaussian noise, uniform start"),
    "d1q3": dict(lattice=0, dims=(256,), tau=1.0, rho=10.0, precision=1,
                 name="D1Q3 FP64 periodic L=256, tau=1.0, rho_mean=10, local Gaussian noise, sine start"),
    "d3q19_f16": dict(lattice=2, dims=(256, 256, 256), tau=1.0, rho=50.0, precision=2,
                      name="D3Q19 periodic 256^3, tau=1.0, rho_mean=50, FP32 arithmetic, FP16 storage of "
                           "f_i - w_i rho_mean, local Gaussian noise, uniform start"),
    "d3q19_bf16": dict(lattice=2, dims=(256, 256, 256), tau=1.0, rho=50.0, precision=3,
                       name="D3Q19 periodic 256^3, tau=1.0, rho_mean=50, FP32 arithmetic, BF16 storage of "
                            "f_i - w_i rho_mean, local Gaussian noise, uniform start"),
    "d2q9_f16": dict(lattice=1, dims=(2048, 2048), tau=0.8, rho=100.0, precision=2,
                     name="D2Q9 periodic 2048x2048, tau=0.8, rho_mean=100, FP32 arithmetic, FP16 storage of "
                          "f_i - w_i rho_mean, local Gaussian noise, uniform start"),
}
ELEM_BYTES = {0: 4, 1: 8, 2: 2, 3: 2}
DTYPE_NAME = {0: "f32", 1: "f64", 2: "f32 (f16 storage)", 3: "f32 (bf16 storage)"}
Q_OF = {0: 3, 1: 9, 2: 19}
# sources of the step kernel k_step_vec and of the choice of its sites per thread
KERNEL_SOURCES = ["paper_1606_07801_gb300/csrc/step_kernels.cuh", "paper_1606_07801_gb300/csrc/device.cuh",
                  "paper_1606_07801_gb300/csrc/step_shape.h", "paper_1606_07801_gb300/csrc/step_d2q9.cu",
                  "paper_1606_07801_gb300/csrc/step_d3q19.cu"]
# sources of the batched kernel (k_batch_tile / k_batch_step)
BATCH_SOURCES = ["paper_1606_07801_gb300/csrc/step_kernels.cuh", "paper_1606_07801_gb300/csrc/device.cuh",
                 "paper_1606_07801_gb300/csrc/batch_kernels.cuh", "paper_1606_07801_gb300/csrc/fastdiv.cuh",
                 "paper_1606_07801_gb300/csrc/batch_d2q9.cu", "paper_1606_07801_gb300/csrc/batch_d3q19.cu"]


def _code_only(text: str) -> str:
    """Source text without comments and whitespace, so that editing a comment
    or the layout does not invalidate a committed capture of unchanged code."""
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    text = re.sub(r"//[^\n]*", "", text)
    return re.sub(r"\s+", "", text)


def kernel_hash(sources=KERNEL_SOURCES) -> str:
    h = hashlib.sha256()
    for p in sources:
        with open(os.path.join(ROOT, p), encoding="utf-8") as fh:
            h.update(_code_only(fh.read()).encode())
    return h.hexdigest()[:16]


def profiled(workload: str, key: str, name: str = "", sources=KERNEL_SOURCES):
    """A figure of a committed ncu summary (profiles/k_step_<workload>.md, or
    profiles/<name>.md) such as traffic_bytes_per_launch or
    instructions_per_site, or None if there is none or the kernel sources
    changed since it was taken."""
    path = os.path.join(ROOT, "profiles", (name or f"k_step_{workload}") + ".md")
    if not os.path.exists(path):
        return None
    text = open(path).read()
    m_hash = re.search(r"kernel_sources_sha256_16:\s*([0-9a-f]+)", text)
    m_val = re.search(key + r":\s*([0-9.eE+]+)", text)
    if not m_hash or not m_val or m_hash.group(1) != kernel_hash(sources):
        return None
    return float(m_val.group(1))


# Instruction-issue ceiling of GB300: 152 SMs x 4 schedulers x 32 lanes, one
# warp instruction per scheduler and cycle, at the 2070 MHz maximum SM clock.
ISSUE_PEAK = 152 * 4 * 32 * 2.070e9


def replica(rank: int) -> dict:
    """Each rank runs its own lattice: seed 1 + rank and Philox lattice id
    rank, so the replicas draw independent noise (no data-path collective)."""
    return {"seed": 1 + rank, "lattice_id": rank}


def max_over_ranks(x: float, dist=None, device="cpu") -> float:
    """The slowest rank's figure (the timed region ends when every rank has
    finished)."""
    if dist is None:
        return float(x)
    import torch

    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_glups(world: int, sites: int, steps: int, seconds: float) -> float:
    """Whole-job throughput: the site updates of all ranks over the slowest
    rank's time (weak scaling: every rank has the same lattice)."""
    return world * sites * steps / seconds / 1e9


def measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as fh:
            d = json.load(fh)
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons while running."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu: int):
        self.gpu = gpu
        self.proc = None
        self.out = tempfile.NamedTemporaryFile(mode="w+", suffix=".csv", delete=False)

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "100"], stdout=self.out,
                                         stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None
        time.sleep(0.3)
        return self

    def __exit__(self, *exc):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        self.out.flush()
        self.out.seek(0)
        rows = [r.split(",") for r in self.out.read().strip().splitlines() if r.count(",") >= 8]
        os.unlink(self.out.name)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"], "samples": 0}
        sm = [float(r[1]) for r in rows if r[1].strip().replace(".", "").isdigit()]
        smax = max((float(r[2]) for r in rows if r[2].strip().replace(".", "").isdigit()), default=None)
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = [n for k, n in enumerate(names) if any(r[5 + k].strip() == "Active" for r in rows)]
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": smax, "reasons": reasons,
                "samples": len(rows)}


def cpu_baseline(wl: dict, budget_s: float = 12.0):
    """The FP64 oracle as it stands, on all host cores, on a bounded sample of
    the workload (fewer steps or a sub-lattice), in the metric's unit."""
    import oracle

    oracle.build()
    cores = os.cpu_count() or 1
    oracle.set_threads(cores)
    lat, dims = wl["lattice"], wl["dims"]
    Q = Q_OF[lat]
    # probe on a slab to size the sample, then run a bounded number of full-lattice steps
    N = int(np.prod(dims))
    f = oracle.init_equilibrium(lat, np.full(N, wl["rho"]))
    t0 = time.perf_counter()
    f = oracle.run(lat, dims, f, 1, wl["tau"], oracle.NOISE_LOCAL, oracle.GAUSSIAN, rho_eq=wl["rho"], seed=1)
    one = time.perf_counter() - t0
    steps = max(1, min(1000, int(budget_s / max(one, 1e-6))))
    t0 = time.perf_counter()
    oracle.run(lat, dims, f, steps, wl["tau"], oracle.NOISE_LOCAL, oracle.GAUSSIAN, rho_eq=wl["rho"], seed=1, t0=1)
    dt = time.perf_counter() - t0
    glups = N * steps / dt / 1e9
    return {"value": glups, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": f"{steps} full-lattice steps of the workload ({N} sites, Q={Q}) in FP64, {dt:.1f} s"}


def _slab(wl: dict, rows: int):
    """The workload's lattice cut to its first `rows` planes along the slowest
    axis (periodic on its own): the same per-site work on fewer sites."""
    dims = list(wl["dims"])
    dims[-1] = max(1, min(dims[-1], rows))
    return tuple(dims)


def run_reference(args, wl):
    """The FP64 oracle on the host cores.  Each bench step is one LB step of
    the workload on a slab of it, sized so that warm-up plus timed steps take
    about a minute in total."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    import oracle

    oracle.build()
    cores = os.cpu_count() or 1
    oracle.set_threads(cores)
    lat = wl["lattice"]
    # calibrate on a small slab
    probe = _slab(wl, 8 if len(wl["dims"]) > 1 else wl["dims"][0])
    n_probe = int(np.prod(probe))
    f = oracle.init_equilibrium(lat, np.full(n_probe, wl["rho"]))
    f = oracle.run(lat, probe, f, 1, wl["tau"], oracle.NOISE_LOCAL, oracle.GAUSSIAN, rho_eq=wl["rho"], seed=1)
    t0 = time.perf_counter()
    oracle.run(lat, probe, f, 2, wl["tau"], oracle.NOISE_LOCAL, oracle.GAUSSIAN, rho_eq=wl["rho"], seed=1, t0=1)
    per_site = (time.perf_counter() - t0) / (2 * n_probe)
    total_steps = max(1, args.steps + args.warmup)
    plane = n_probe // probe[-1]
    rows = int(60.0 / total_steps / max(per_site, 1e-12) / plane)
    dims = _slab(wl, max(1, rows))
    N = int(np.prod(dims))
    f = oracle.init_equilibrium(lat, np.full(N, wl["rho"]))
    t = 0
    for _ in range(args.warmup):
        f = oracle.run(lat, dims, f, 1, wl["tau"], oracle.NOISE_LOCAL, oracle.GAUSSIAN, rho_eq=wl["rho"], seed=1, t0=t)
        t += 1
    t0 = time.perf_counter()
    for _ in range(args.steps):
        f = oracle.run(lat, dims, f, 1, wl["tau"], oracle.NOISE_LOCAL, oracle.GAUSSIAN, rho_eq=wl["rho"], seed=1, t0=t)
        t += 1
    dt = time.perf_counter() - t0
    value = N * args.steps / dt / 1e9
    sample = (f"each step: one FP64 LB step on a {'x'.join(map(str, dims))} slab of the workload "
              f"({N} of {int(np.prod(wl['dims']))} sites); {args.steps} timed steps")
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": dt / args.steps * 1e3, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": wl["name"], "reference": "FP64 CPU oracle (plain C, OpenMP over sites)"},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sample},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


# tile orders of the batched kernel, in the order of the library's LBFD_WALK_* values
WALKS = ["strided", "contiguous", "per_tile", "param"]
ENS_GRAPH_STEPS = 16  # steps per CUDA graph chunk of lbfd_ensemble_step
ENS_LATTICES = {"d1q3": (0, 1, (256, 65536)), "d2q9": (1, 2, (32, 512)), "d3q19": (2, 3, (32, 128))}


def run_ensemble(args):
    """Config 4: 4096 independent D2Q9 FP32 lattices (sides log-uniform in
    [32, 512], rho_mean U[0.5, 200], tau U[0.6, 1.5], distinct seeds), one
    launch per time step for all of them (graph-captured chunks), against the
    plain way of running them: one launch per simulation per step.
    --ens-lattice d3q19 / d1q3 runs the same kind of ensemble of the other
    lattices (cube sides in [32, 128], lengths in [256, 65536])."""
    import torch

    import paper_1606_07801_gb300 as lb
    from paper_1606_07801_gb300 import synth

    torch.cuda.set_device(0)
    lb.load()
    lat, ndim, (lo, hi) = ENS_LATTICES[args.ens_lattice]
    Q = Q_OF[lat]
    specs = synth.ensemble(args.members, side_lo=lo, side_hi=hi, ndim=ndim)
    for k, sp in enumerate(specs):
        sp["lattice_id"] = k
        sp["init"] = lb.INIT_UNIFORM
    stream = torch.cuda.Stream()
    ens = lb.Ensemble(lat, specs, stream=stream)
    n, sites = ens.query()[:2]
    if args.plan:
        # a fixed decomposition (sites per item, passes, occupancy variant, tile order) instead of the tuner's
        pv, pp, po, pw = args.plan.split(",")
        ens.plan(int(pv), int(pp), int(po), WALKS.index(pw))
    else:
        ens.tune(steps=3)
    _, _, _, vx, passes, bps, walk = ens.query()
    # at least one full graph chunk, so that the chunk's one-time capture
    # (lbfd_ensemble_step captures its first 16-step chunk) is not timed
    ens.step(max(args.warmup, ENS_GRAPH_STEPS))
    torch.cuda.synchronize()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    launches0 = lb.abi.lbfd_kernel_launches()
    with ClockSampler(0) as clk:
        torch.cuda.synchronize()
        ev0.record(stream)
        ens.step(args.steps)
        ev1.record(stream)
        torch.cuda.synchronize()
    ms = ev0.elapsed_time(ev1)
    launches = lb.abi.lbfd_kernel_launches() - launches0
    ens.close()
    glups = sites * args.steps / (ms * 1e-3) / 1e9
    # the same members run the plain way: one handle and one launch per simulation per step
    sub = specs[: args.per_sim_members]
    sims = [lb.Simulation(lat, sp["dims"], sp["tau"], sp["rho_mean"], sp["seed"], lattice_id=sp["lattice_id"],
                          stream=stream) for sp in sub]
    for s_ in sims:
        s_.step(3)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.per_sim_steps):
        for s_ in sims:
            s_.step(1)
    e1.record(stream)
    torch.cuda.synchronize()
    ms_ps = e0.elapsed_time(e1)
    sub_sites = sum(int(np.prod(sp["dims"])) for sp in sub)
    per_sim = sub_sites * args.per_sim_steps / (ms_ps * 1e-3) / 1e9
    for s_ in sims:
        s_.close()
    peak, peak_kind = measured_peaks()
    achieved = 8.0 * Q * sites / (ms / args.steps * 1e-3) / 1e9
    kname = {"per_tile": "k_batch_tile", "param": "k_batch_param"}.get(WALKS[walk], "k_batch_step")
    # DRAM bytes per site of one launch from the committed ncu capture of this kernel (same kernel sources),
    # scaled to this ensemble
    per_site = profiled(args.ens_lattice, f"traffic_bytes_per_site_{args.ens_lattice}", f"{kname}_ensemble",
                        BATCH_SOURCES)
    traffic = None if per_site is None else per_site * sites
    line = {
        "metric": METRIC, "value": glups, "unit": UNIT, "n_gpus": 1, "steps": args.steps,
        "warmup": max(args.warmup, ENS_GRAPH_STEPS), "ms_per_step": ms / args.steps, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32", "data": "synthetic",
        "config": {"workload": f"ensemble of {n} {args.ens_lattice.upper()} FP32 lattices, sides log-uniform in "
                               f"[{lo}, {hi}], rho_mean U[0.5, 200], tau U[0.6, 1.5], distinct seeds, local Gaussian "
                               f"noise",
                   "sites": sites, "sites_per_item_max": vx, "tile_passes": passes, "blocks_per_sm": bps,
                   "tile_walk": WALKS[walk], "decomposition": args.plan or "tuned",
                   "graph_steps": ENS_GRAPH_STEPS,
                   "l2": "inputs larger than L2: %.0f MB per population buffer" % (4.0 * Q * sites / 1e6)},
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                     "traffic": traffic, "algorithmic_bytes_per_launch": 8 * Q * sites, "kernel": kname,
                     "peak_source": f"{peak_kind} hbm_gbs"},
        "per_sim_baseline": {"value": per_sim, "unit": UNIT, "sims": len(sub), "steps": args.per_sim_steps,
                             "how": "one lbfd handle and one k_step launch per simulation per step, same stream"},
        "speedup_vs_per_sim": glups / per_sim,
        "e2e": None, "gpu_launches": launches, "clocks": clk.summary(),
    }
    print(json.dumps(line), flush=True)


def served_rate_search(args, lb, abi, synth, sink, make_server) -> dict:
    """The largest Poisson arrival rate at which the p99 latency of the first
    --rate-requests requests of the served trace stays within --p99-bound
    seconds.  The trace's arrival times scale as 1/rate (same seed), so every
    rate serves the same requests.  Halves the rate from --rate until the
    bound holds, then bisects in log space."""
    n = min(args.rate_requests, args.requests)
    arr500, specs = synth.served_trace(n, rate=500.0)
    reqs = [abi.make_request(sp["lattice"], sp["dims"], sp["tau"], sp["rho_mean"], sp["seed"], sp["steps"],
                             lattice_id=sp["lattice_id"], result=lb.RESULT_RHO) for sp in specs]
    tested = []

    def p99_at(rate):
        srv = make_server()
        try:
            lat, makespan = abi.lbfd_server_run_trace(srv.h, reqs, arr500 * (500.0 / rate), sink.data_ptr(),
                                                      sink.nbytes)
        finally:
            srv.close()
        p = float(np.percentile(lat, 99))
        tested.append({"rate": rate, "p99_s": p, "p50_s": float(np.percentile(lat, 50)), "makespan_s": makespan})
        return p

    hi, lo = args.rate, None
    while lo is None and hi > 1.0:
        if p99_at(hi) <= args.p99_bound:
            lo = hi
        else:
            hi /= 2.0
    if lo is not None and lo < args.rate:
        top = min(args.rate, 2.0 * lo)
        for _ in range(3):
            mid = math.sqrt(lo * top)
            if p99_at(mid) <= args.p99_bound:
                lo = mid
            else:
                top = mid
    return {"p99_bound_s": args.p99_bound, "requests": n, "rate_per_s": lo,
            "note": "largest tested rate meeting the bound (None: not even 1/s)", "tested": tested}


def run_served(args):
    """Config 5: a Poisson stream of mixed D1Q3 / D2Q9 / D3Q19 FP32
    simulation requests served by continuous batching under a device-memory
    budget (lbfd_server_run_trace: admission, one batched launch per lattice
    type per time step, result copies on a second stream), against the plain
    way: the same requests taken one at a time in arrival order, each its own
    handle with one launch per time step."""
    import torch

    import paper_1606_07801_gb300 as lb
    from paper_1606_07801_gb300 import lbfd as abi
    from paper_1606_07801_gb300 import synth

    torch.cuda.set_device(0)
    lb.load()
    arrivals, specs = synth.served_trace(args.requests, rate=args.rate)
    reqs = [abi.make_request(sp["lattice"], sp["dims"], sp["tau"], sp["rho_mean"], sp["seed"], sp["steps"],
                             lattice_id=sp["lattice_id"], result=lb.RESULT_RHO) for sp in specs]
    sites = np.array([int(np.prod(sp["dims"])) for sp in specs], dtype=np.int64)
    steps = np.array([sp["steps"] for sp in specs], dtype=np.int64)
    lups = int(np.sum(sites * steps))
    bytes_alg = int(sum(int(np.prod(sp["dims"])) * sp["steps"] * 2 * 4 * Q_OF[sp["lattice"]] for sp in specs))
    d2h = int(np.sum(sites) * 8)
    sink = torch.empty(args.sink_mb << 20, dtype=torch.uint8).pin_memory()
    policy = {"shortest": lb.POLICY_SHORTEST, "longest": lb.POLICY_LONGEST}.get(args.policy, lb.POLICY_FIFO)

    def make_server():
        return lb.Server(hbm_budget=int(args.budget_gb * (1 << 30)), max_active=4096, max_ahead=4,
                         passes=args.passes, policy=policy, max_active_sites=args.max_active_sites,
                         occupancy=args.occupancy, solo_sites=args.solo_sites, walk=WALKS.index(args.walk),
                         vx_max=args.vx_max)

    srv = make_server()
    # warm-up: a short trace of small requests (module load, first launches)
    warm = [abi.make_request(k % 3, [(512,), (64, 64), (16, 16, 16)][k % 3], 1.0, 10.0, 99 + k, 20,
                             result=lb.RESULT_RHO) for k in range(max(3, args.warmup))]
    abi.lbfd_server_run_trace(srv.h, warm, np.zeros(len(warm)), sink.data_ptr(), sink.nbytes)
    launches0 = lb.abi.lbfd_kernel_launches()
    torch.cuda.synchronize()
    with ClockSampler(0) as clk:
        lat, makespan = abi.lbfd_server_run_trace(srv.h, reqs, arrivals, sink.data_ptr(), sink.nbytes)
    launches = lb.abi.lbfd_kernel_launches() - launches0
    st = srv.stats()
    srv.close()
    glups = lups / makespan / 1e9
    p50, p99 = float(np.percentile(lat, 50)), float(np.percentile(lat, 99))
    # the plain way on (a prefix of) the same stream: one request at a time
    nb = args.requests if args.plain_requests < 0 else min(args.requests, args.plain_requests)
    plain = None
    if nb > 0:
        stream = torch.cuda.Stream()
        t_start = time.perf_counter()
        plain_lat = []
        for k in range(nb):
            sp = specs[k]
            wait = arrivals[k] - (time.perf_counter() - t_start)
            if wait > 0:
                time.sleep(wait)
            with lb.Simulation(sp["lattice"], sp["dims"], sp["tau"], sp["rho_mean"], sp["seed"],
                               lattice_id=sp["lattice_id"], stream=stream) as sim:
                sim.step(sp["steps"])
                sim.moments()
            plain_lat.append(time.perf_counter() - t_start - arrivals[k])
        plain_makespan = time.perf_counter() - t_start
        plain_lups = int(np.sum(sites[:nb] * steps[:nb]))
        plain = {"value": plain_lups / plain_makespan / 1e9, "unit": UNIT, "requests": nb,
                 "p50_latency_s": float(np.percentile(plain_lat, 50)),
                 "p99_latency_s": float(np.percentile(plain_lat, 99)), "makespan_s": plain_makespan,
                 "how": "the same stream's requests taken one at a time in arrival order: one lbfd handle per "
                        "request, one k_step launch per time step, density read back"}
    rate_at_bound = served_rate_search(args, lb, abi, synth, sink, make_server) if args.p99_bound > 0 else None
    peak, peak_kind = measured_peaks()
    achieved = bytes_alg / makespan / 1e9
    line = {
        "metric": METRIC, "value": glups, "unit": UNIT, "n_gpus": 1, "steps": args.requests, "warmup": len(warm),
        "ms_per_step": makespan / args.requests * 1e3, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": f"served stream: {args.requests} requests, Poisson arrivals at {args.rate:g}/s, "
                               "lattice uniform over D1Q3 (L log-uniform 256-65536) / D2Q9 (side log-uniform "
                               "32-1024) / D3Q19 (side log-uniform 32-128), steps log-uniform 100-10^4, tau "
                               "U[0.6, 1.5], rho_mean U[0.5, 200], FP32, local Gaussian noise, density result",
                   "hbm_budget_gb": args.budget_gb, "policy": args.policy, "passes": args.passes,
                   "occupancy": args.occupancy, "walk": args.walk, "vx_max": args.vx_max,
                   "solo_sites": args.solo_sites,
                   "max_active_sites": args.max_active_sites, "site_updates": lups,
                   "step": "one bench step = one served request; value = total site updates / makespan"},
        "latency_s": {"p50": p50, "p99": p99, "mean": float(np.mean(lat)), "max": float(np.max(lat))},
        "makespan_s": makespan,
        "max_rate_at_p99_bound": rate_at_bound,
        "server": {k: st[k] for k in ("clock", "peak_active", "peak_resident_bytes", "peak_resident_sites")},
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                     "traffic": None, "kernel": "batched and solo step kernels (whole-job average over the makespan)",
                     "algorithmic_bytes": bytes_alg, "peak_source": f"{peak_kind} hbm_gbs"},
        "per_sim_baseline": plain,
        "e2e": {"value": glups, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": d2h / args.requests,
                "note": "the served value is itself end to end: host clock from the first arrival to the last "
                        "result copied into pinned host memory"},
        "gpu_launches": launches, "clocks": clk.summary(),
    }
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=40000)
    ap.add_argument("--warmup", type=int, default=200)
    ap.add_argument("--workload", default="d2q9", choices=sorted(WORKLOADS) + ["ensemble", "served"])
    ap.add_argument("--impl", default="native", choices=["native", "reference"])
    ap.add_argument("--e2e-steps", type=int, default=20)
    ap.add_argument("--e2e-run-steps", type=int, default=1000,
                    help="steps of the e2e_run figure (state in once, steps, density out once)")
    ap.add_argument("--sample-every", type=int, default=10,
                    help="step workloads: also time the sampled observables, one sample per this many steps")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--members", type=int, default=4096)
    ap.add_argument("--plan", default="", help="ensemble decomposition vx,passes,occupancy,walk (default: tuned)")
    ap.add_argument("--ens-lattice", default="d2q9", choices=sorted(ENS_LATTICES))
    ap.add_argument("--per-sim-members", type=int, default=256)
    ap.add_argument("--per-sim-steps", type=int, default=20)
    ap.add_argument("--requests", type=int, default=1000)
    ap.add_argument("--rate", type=float, default=500.0)
    ap.add_argument("--budget-gb", type=float, default=120.0)
    ap.add_argument("--policy", default="shortest", choices=["fifo", "shortest", "longest"])
    ap.add_argument("--passes", type=int, default=4)
    ap.add_argument("--occupancy", type=int, default=0)
    ap.add_argument("--walk", default="param", choices=WALKS)
    ap.add_argument("--vx-max", type=int, default=2, choices=[1, 2])
    ap.add_argument("--solo-sites", type=int, default=0)
    ap.add_argument("--max-active-sites", type=int, default=20_000_000)
    ap.add_argument("--sink-mb", type=int, default=2048)
    ap.add_argument("--plain-requests", type=int, default=-1)
    ap.add_argument("--p99-bound", type=float, default=0.0,
                    help="served: also search the largest arrival rate whose p99 latency stays within this many s")
    ap.add_argument("--rate-requests", type=int, default=400)
    args = ap.parse_args()
    if args.warmup < 3:
        raise SystemExit("--warmup must be >= 3")
    if args.workload == "ensemble":
        run_ensemble(args)
        return
    if args.workload == "served":
        run_served(args)
        return
    wl = WORKLOADS[args.workload]
    if args.impl == "reference":
        run_reference(args, wl)
        return

    import torch

    import paper_1606_07801_gb300 as lb

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    dist = None
    if world > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    lb.load()

    lat, dims, tau, rho, prec = wl["lattice"], wl["dims"], wl["tau"], wl["rho"], wl["precision"]
    Q, N = Q_OF[lat], int(np.prod(dims))
    elem = ELEM_BYTES[prec]
    stream = torch.cuda.Stream()
    init = lb.INIT_SINE if args.workload == "d1q3" else lb.INIT_UNIFORM
    rep = replica(rank)
    # four structure-factor modes for the sampled observables (they do not touch the step)
    modes = [(1, 0, 0), (2, 0, 0), (0, 1, 0), (1, 1, 1)][: {1: 2, 2: 3, 3: 4}[len(dims)]]
    if len(dims) < 3:
        modes = [tuple(k if d < len(dims) else 0 for d, k in enumerate(m)) for m in modes]
    sim = lb.Simulation(lat, dims, tau, rho, rep["seed"], precision=prec, lattice_id=rep["lattice_id"], stream=stream,
                        torch_buffers=True, device=local, init=init, sine_amp=1.0, sine_k=(1, 0, 0), modes=modes)

    def barrier():
        torch.cuda.synchronize()
        if dist is not None:
            dist.barrier()

    kname = sim.kernel(args.steps)  # the kernel lbfd_step runs for this lattice
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with ClockSampler(local) as clk:
        # the warm-up runs right before the timed region, after the clock
        # sampler has started (its start-up leaves the GPU idle for 0.3 s)
        sim.step(args.warmup)
        barrier()
        launches0 = lb.abi.lbfd_kernel_launches()
        ev0.record(stream)
        sim.step(args.steps)
        ev1.record(stream)
        barrier()
    launches = lb.abi.lbfd_kernel_launches() - launches0
    ms = max_over_ranks(ev0.elapsed_time(ev1), dist, "cuda")
    clocks = clk.summary()
    ms_per_step = ms / args.steps
    value = job_glups(world, N, args.steps, ms * 1e-3)

    # roofline of the dominant kernel (k_step is the only kernel in the timed region)
    bytes_per_launch = 2 * Q * elem * N
    achieved = bytes_per_launch / (ms_per_step * 1e-3) / 1e9
    peak, peak_kind = measured_peaks()
    traffic = profiled(args.workload, "traffic_bytes_per_launch")
    ipsite = profiled(args.workload, "instructions_per_site")
    alu = None
    if ipsite is not None:
        a_alu = ipsite * N / (ms_per_step * 1e-3)
        alu = {"bound": "alu", "achieved": a_alu, "peak": ISSUE_PEAK, "unit": "thread-instructions/s",
               "frac": a_alu / ISSUE_PEAK, "instructions_per_site": ipsite,
               "peak_source": "152 SMs x 4 schedulers x 32 lanes x 2.07 GHz"}

    # the sampled FP64 observables (mass, density variance, S(k), <f_i>, <f_i f_j>):
    # time per sample, and the throughput when a sample follows every
    # --sample-every steps (the fluctuation statistics of a long run)
    obs = None
    if args.sample_every > 0:
        # lbfd_step with a sample every k steps (inside the step kernel where
        # the format allows), timed over the same number of steps as the
        # main region, and the separate sampling pass for comparison
        k = args.sample_every
        lb.abi.lbfd_set_sample_every(sim.h, k)
        sim.step(2 * k)
        torch.cuda.synchronize()
        s_steps = max(k, (args.steps // k) * k)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        sim.step(s_steps)
        lb.abi.lbfd_state_device(sim.h)  # the last sample's stage 2 (side stream) before e1
        e1.record(stream)
        torch.cuda.synchronize()
        ms_sampled = e0.elapsed_time(e1)
        lb.abi.lbfd_set_sample_every(sim.h, 0)
        n_samp = 5
        sim.sample()
        torch.cuda.synchronize()
        e0.record(stream)
        for _ in range(n_samp):
            sim.sample()
        e1.record(stream)
        torch.cuda.synchronize()
        ms_sample = e0.elapsed_time(e1) / n_samp
        fused = bool(kname in ("k_step_vec", "k_step", "k_step_staged") and prec != 1)
        obs = {"sample_every": k, "modes": len(modes), "steps": s_steps,
               "value_with_sampling": job_glups(world, N, s_steps, ms_sampled * 1e-3),
               "fused": fused,
               "ms_per_sampled_step_extra": (ms_sampled / s_steps - ms_per_step) * k,
               "separate_pass": {"ms_per_sample": ms_sample,
                                 "value_with_sampling": job_glups(world, N, k, (k * ms_per_step + ms_sample) * 1e-3),
                                 "algorithmic_bytes_per_sample": Q * elem * N,
                                 "achieved_gbs": Q * elem * N / (ms_sample * 1e-3) / 1e9}}

    # end to end through the C ABI with host buffers: per step, the state goes
    # host -> device (pinned), one step runs, the density comes back
    h_f = torch.empty(Q * N * elem, dtype=torch.uint8).pin_memory()
    h_rho = torch.empty(N, dtype=torch.float64).pin_memory()
    lb.abi.lbfd_get_f_raw(sim.h, h_f.data_ptr())
    barrier()
    e_steps = max(1, args.e2e_steps)
    t0 = time.perf_counter()
    for _ in range(e_steps):
        lb.abi.lbfd_set_f_raw(sim.h, h_f.data_ptr())
        sim.step(1)
        lb.abi.load().lbfd_moments(sim.h, h_rho.data_ptr(), None)
    torch.cuda.synchronize()
    e2e_s = max_over_ranks(time.perf_counter() - t0, dist, "cuda")
    e2e = {"value": job_glups(world, N, e_steps, e2e_s), "unit": UNIT, "h2d_bytes_per_step": Q * N * elem,
           "d2h_bytes_per_step": N * 8,
           "how": "every step: the whole state host -> device (lbfd_set_f_raw, pinned), one lbfd_step, the "
                  "density device -> host (lbfd_moments)"}
    # what a caller running a simulation sees: the state goes in once, a run
    # of steps stays on the device, the density comes back once
    r_steps = max(1, args.e2e_run_steps)
    lb.abi.lbfd_set_f_raw(sim.h, h_f.data_ptr())
    barrier()
    t0 = time.perf_counter()
    lb.abi.lbfd_set_f_raw(sim.h, h_f.data_ptr())
    sim.step(r_steps)
    lb.abi.load().lbfd_moments(sim.h, h_rho.data_ptr(), None)
    torch.cuda.synchronize()
    run_s = max_over_ranks(time.perf_counter() - t0, dist, "cuda")
    e2e_run = {"value": job_glups(world, N, r_steps, run_s), "unit": UNIT,
               "h2d_bytes_per_step": Q * N * elem / r_steps, "d2h_bytes_per_step": N * 8 / r_steps,
               "steps": r_steps,
               "how": f"state host -> device once (pinned), {r_steps} lbfd_step steps, density device -> host once"}
    sim.close()

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": DTYPE_NAME[prec], "data": "synthetic",
            "config": {"workload": wl["name"], "sites": N, "parallelism": f"replicas x{world}",
                       "l2": "inputs larger than L2: %.0f MB per population buffer vs 129 MB L2" % (Q * N * elem / 1e6),
                       "per_sim": "one lattice per GPU, one lbfd_step call for all timed steps",
                       "kernel": kname},
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                         "frac": achieved / peak, "traffic": traffic,
                         "algorithmic_bytes_per_launch": bytes_per_launch, "kernel": kname,
                         "peak_source": f"{peak_kind} hbm_gbs"},
            "roofline_alu": alu,
            "e2e": e2e, "e2e_run": e2e_run, "observables": obs,
            "gpu_launches": launches,
            "clocks": clocks,
        }
        if prec in (2, 3) and alu is not None:
            # 16-bit storage halves the bytes but not the arithmetic: the
            # issue ceiling binds, so it is the primary roofline here
            line["roofline_hbm"], line["roofline"] = line["roofline"], alu
            del line["roofline_alu"]
        if not args.no_cpu_baseline and world == 1:
            line["cpu_baseline"] = cpu_baseline(wl)
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
