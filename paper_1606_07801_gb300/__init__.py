"""GB300-native fluctuating lattice-Boltzmann diffusion (Wagner & Strand, arXiv:1606.07801).

The compute path is the CUDA library ``liblbfd.so`` (sources in ``csrc/``,
C ABI in ``include/lbfd.h``).  This package holds its ctypes binding
(``lbfd``), the build step (``build``), seeded synthetic workloads
(``synth``) and a small convenience wrapper, :class:`Simulation`.  PyTorch,
when used, only provides device memory and streams.
"""
from __future__ import annotations

import ctypes

import numpy as np

from . import build as _build_mod
from .lbfd import (D1Q3, D2Q5, D2Q9, D3Q19, D_OF, EBUSY, ECUDA, EINVAL, ENOMEM, ENOTSUP, ETIMEOUT, F32, F32_BF16, F32_F16,
                   F64, GAUSSIAN, INIT_HOST, INIT_NONE, INIT_SINE, INIT_UNIFORM, KERNEL_AUTO, KERNEL_CLUSTER,
                   KERNEL_MRT, KERNEL_SCALAR, KERNEL_SMALL, KERNEL_STAGED, KERNEL_VEC, MAX_MODES, MAX_Q, NOISE_GLOBAL,
                   NOISE_LOCAL, NOISE_OFF, OK, POLICY_FIFO, POLICY_LONGEST, POLICY_SHORTEST, Q_OF, REQ_DONE,
                   REQ_QUEUED, REQ_RUNNING, REQ_UNKNOWN, RESULT_F, RESULT_NONE, RESULT_RHO, UNIFORM, WALK_CONTIGUOUS, WALK_PARAM, WALK_PER_TILE,
                   WALK_STRIDED, LbfdError, Options, load)
from . import lbfd as abi

__all__ = ["Simulation", "Ensemble", "Server", "STORAGE_DTYPE", "abi", "build", "load", "LbfdError", "Options",
           "D1Q3", "D2Q9", "D3Q19", "D2Q5", "F32", "F64", "F32_F16", "F32_BF16",
           "NOISE_LOCAL", "NOISE_GLOBAL", "NOISE_OFF", "GAUSSIAN", "UNIFORM", "INIT_UNIFORM", "INIT_SINE",
           "INIT_NONE", "INIT_HOST", "RESULT_F", "RESULT_RHO", "RESULT_NONE", "POLICY_FIFO", "POLICY_SHORTEST",
           "POLICY_LONGEST",
           "WALK_STRIDED", "WALK_CONTIGUOUS", "WALK_PER_TILE", "WALK_PARAM", "REQ_QUEUED", "REQ_RUNNING", "REQ_DONE",
           "REQ_UNKNOWN", "Q_OF", "D_OF", "KERNEL_AUTO", "KERNEL_VEC", "KERNEL_SCALAR", "KERNEL_SMALL",
           "KERNEL_CLUSTER", "KERNEL_MRT", "KERNEL_STAGED"]

# numpy type of one stored value per precision (bfloat16 as its raw 16 bits)
STORAGE_DTYPE = {F32: np.float32, F64: np.float64, F32_F16: np.float16, F32_BF16: np.uint16}


def build(force: bool = False) -> str:
    """Compile ``liblbfd.so`` for sm_103a (in-tree) and return its path."""
    return _build_mod.build(force=force)


class Simulation:
    """One lattice on one GPU, owned through an ``lbfd_t`` handle.

    With ``torch_buffers=True`` the two population buffers are torch tensors
    (caller-owned device memory handed to ``lbfd_create_ex``); ``stream`` may
    be a ``torch.cuda.Stream`` or a raw ``cudaStream_t`` integer.
    """

    def __init__(self, lattice: int, dims, tau: float, rho_mean: float, seed: int = 1, *, precision: int = F32,
                 noise_mode: int = NOISE_LOCAL, noise_dist: int = GAUSSIAN, init: int = INIT_UNIFORM,
                 sine_amp: float = 0.0, sine_k=(1, 0, 0), lattice_id: int = 0, modes=(), stream=None,
                 torch_buffers: bool = False, device: int = -1, theta: float = 0.0, tau_moments=None,
                 step_kernel: int = 0, wait_test_bytes: int = 0, slab_global: int = 0, slab_first: int = 0,
                 sample_every: int = 0):
        o = abi.lbfd_options_init()
        o.sample_every = int(sample_every)
        o.step_kernel = int(step_kernel)
        o.wait_test_bytes = int(wait_test_bytes)
        o.slab_global, o.slab_first = int(slab_global), int(slab_first)
        o.lattice, o.precision, o.noise_mode, o.noise_dist, o.init = lattice, precision, noise_mode, noise_dist, init
        d = [int(x) for x in dims] + [1] * (3 - len(dims))
        for a in range(3):
            o.dims[a] = d[a]
        o.tau, o.rho_mean, o.seed, o.lattice_id, o.device = float(tau), float(rho_mean), int(seed), int(lattice_id), device
        o.sine_amp = float(sine_amp)
        o.theta = float(theta)
        if tau_moments is not None:
            tm = [float(x) for x in tau_moments]
            if len(tm) > MAX_Q:
                raise ValueError(f"at most {MAX_Q} relaxation times")
            for a, x in enumerate(tm):
                o.tau_moments[a] = x
        for a in range(3):
            o.sine_k[a] = int(sine_k[a]) if a < len(sine_k) else 0
        modes = list(modes)
        if len(modes) > MAX_MODES:
            raise ValueError(f"at most {MAX_MODES} structure-factor modes")
        o.n_modes = len(modes)
        for m, k in enumerate(modes):
            for a in range(3):
                o.modes[m][a] = int(k[a]) if a < len(k) else 0
        self._keep = []
        if stream is not None:
            o.stream = int(getattr(stream, "cuda_stream", stream))
            self._keep.append(stream)
        self.buffers = None
        if torch_buffers:
            import torch

            q, n = Q_OF[lattice], int(np.prod(d))
            if slab_global:  # a slab stores a halo plane on each side of its slowest axis
                ax = {D2Q9: 1, D3Q19: 2}.get(lattice, 0)
                n = n // d[ax] * (d[ax] + 2)
            dt = {F64: torch.float64, F32: torch.float32, F32_F16: torch.float16, F32_BF16: torch.bfloat16}[precision]
            dev = torch.device("cuda", device if device >= 0 else torch.cuda.current_device())
            bufs = [torch.empty(q * n, dtype=dt, device=dev) for _ in range(2)]
            o.f_dev[0], o.f_dev[1] = bufs[0].data_ptr(), bufs[1].data_ptr()
            self._keep.extend(bufs)
            self.buffers = bufs
        self.lattice, self.dims, self.precision = lattice, tuple(d), precision
        self.Q, self.D, self.N = Q_OF[lattice], D_OF[lattice], int(np.prod(d))
        # sites set_f takes: a slab also takes its two halo planes
        ax = {D2Q9: 1, D3Q19: 2}.get(lattice, 0)
        self.stored_sites = self.N // d[ax] * (d[ax] + 2) if slab_global else self.N
        self.h = abi.lbfd_create_ex(o)

    # -- lifecycle -------------------------------------------------------------
    def close(self) -> None:
        if getattr(self, "h", None):
            h, self.h = self.h, None
            abi.lbfd_destroy(h)

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # -- dynamics ----------------------------------------------------------------
    def step(self, n: int = 1) -> None:
        abi.lbfd_step(self.h, n)

    def sync(self) -> None:
        abi.lbfd_sync(self.h)

    def kernel(self, n: int = 1) -> str:
        """Name of the kernel that step(n) runs."""
        return abi.KERNEL_NAMES[abi.lbfd_step_kernel(self.h, n)]

    @property
    def t(self) -> int:
        return abi.lbfd_get_t(self.h)

    @t.setter
    def t(self, value: int) -> None:
        abi.lbfd_set_t(self.h, value)

    # -- state -------------------------------------------------------------------
    def get_f(self) -> np.ndarray:
        return abi.lbfd_get_f(self.h)

    def set_f(self, f) -> None:
        """f(x, t), [Q, N] (a slab: [Q, owned plus both halo planes])."""
        abi.lbfd_set_f(self.h, np.asarray(f, dtype=np.float64), self.stored_sites)

    def moments(self, with_flux: bool = False):
        return abi.lbfd_moments(self.h, with_flux)

    def mass(self) -> float:
        return abi.lbfd_mass(self.h)

    def sample(self) -> None:
        abi.lbfd_sample(self.h)

    def reset_obs(self) -> None:
        abi.lbfd_reset_obs(self.h)

    def observables(self) -> dict:
        return abi.lbfd_observables(self.h)

    def state_device(self):
        return abi.lbfd_state_device(self.h)


class Ensemble:
    """Many independent lattices of one type advanced together (one launch
    per step for all members, graph-captured).  ``specs`` is a list of dicts
    with dims, tau, rho_mean, seed and optionally lattice_id, init,
    sine_amp, sine_k."""

    def __init__(self, lattice: int, specs, *, precision: int = F32, noise_mode: int = NOISE_LOCAL,
                 noise_dist: int = GAUSSIAN, stream=None):
        self.lattice, self.specs = lattice, list(specs)
        self.Q = Q_OF[lattice]
        self._stream = stream
        s = None if stream is None else int(getattr(stream, "cuda_stream", stream))
        self.h = abi.lbfd_ensemble_create(lattice, precision, noise_mode, noise_dist, self.specs, s)

    def sites(self, member: int) -> int:
        return int(np.prod(self.specs[member]["dims"]))

    def close(self) -> None:
        if getattr(self, "h", None):
            h, self.h = self.h, None
            abi.lbfd_ensemble_destroy(h)

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def step(self, n: int = 1) -> None:
        abi.lbfd_ensemble_step(self.h, n)

    def sync(self) -> None:
        abi.lbfd_ensemble_sync(self.h)

    def tune(self, steps: int = 3):
        """Picks the fastest work decomposition; returns (vx, passes, blocks per SM)."""
        return abi.lbfd_ensemble_tune(self.h, steps)

    def plan(self, vx_max: int, passes: int, occupancy: int = 0, walk: int = WALK_PER_TILE) -> None:
        """Sets the work decomposition without timing (results do not depend on it)."""
        abi.lbfd_ensemble_plan(self.h, vx_max, passes, occupancy, walk)

    def query(self):
        """(members, total sites, t, sites per item at most, tile passes, blocks per SM, tile order)."""
        return abi.lbfd_ensemble_query(self.h)

    def get_f(self, member: int) -> np.ndarray:
        return abi.lbfd_ensemble_get_f(self.h, member, self.Q, self.sites(member))

    def set_f(self, member: int, f) -> None:
        abi.lbfd_ensemble_set_f(self.h, member, f)

    def mass(self, member: int) -> float:
        return abi.lbfd_ensemble_mass(self.h, member)


class Server:
    """Continuous-batching server of simulation requests on one GPU (see
    ``lbfd_server_*`` in include/lbfd.h).  Results land in numpy arrays this
    object allocates (or the caller passes) and keeps alive until read."""

    def __init__(self, *, precision: int = F32, noise_mode: int = NOISE_LOCAL, noise_dist: int = GAUSSIAN,
                 hbm_budget: int = 1 << 30, max_active: int = 1024, max_ahead: int = 4, passes: int = 1,
                 policy: int = POLICY_FIFO, max_active_sites: int = 0, occupancy: int = 0,
                 solo_sites: int = 1 << 17, walk: int = WALK_PER_TILE, vx_max: int = 2, device: int = -1):
        o = abi.lbfd_server_options_init()
        o.precision, o.noise_mode, o.noise_dist, o.device = precision, noise_mode, noise_dist, device
        o.hbm_budget, o.max_active, o.max_ahead, o.passes = int(hbm_budget), max_active, max_ahead, passes
        o.policy, o.max_active_sites, o.occupancy = policy, int(max_active_sites), occupancy
        o.solo_sites, o.walk, o.vx_max = int(solo_sites), walk, vx_max
        self.precision = precision
        self._bufs = {}
        self.h = abi.lbfd_server_create(o)

    def close(self) -> None:
        if getattr(self, "h", None):
            h, self.h = self.h, None
            abi.lbfd_server_destroy(h)

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def submit(self, lattice: int, dims, tau: float, rho_mean: float, seed: int, steps: int, *, lattice_id: int = 0,
               init: int = INIT_UNIFORM, sine_amp: float = 0.0, sine_k=(1, 0, 0), f0=None,
               result: int = RESULT_F, out=None) -> int:
        """Queues a simulation; f0 (storage format, [Q, N]) is its initial f
        when given.  Returns the request id."""
        q, n = Q_OF[lattice], int(np.prod(dims))
        keep = []
        in_ptr = None
        if f0 is not None:
            f0 = np.ascontiguousarray(f0, dtype=STORAGE_DTYPE[self.precision])
            assert f0.size == q * n
            init, in_ptr = INIT_HOST, f0.ctypes.data
            keep.append(f0)
        if result != RESULT_NONE and out is None:
            out = (np.empty((q, n), dtype=STORAGE_DTYPE[self.precision]) if result == RESULT_F
                   else np.empty(n, dtype=np.float64))
        out_ptr = None if out is None else out.ctypes.data
        req = abi.make_request(lattice, dims, tau, rho_mean, seed, steps, lattice_id=lattice_id, init=init,
                               sine_amp=sine_amp, sine_k=sine_k, result=result, in_host=in_ptr, out_host=out_ptr)
        rid = abi.lbfd_server_submit(self.h, req)
        self._bufs[rid] = (out, keep)
        return rid

    def pump(self, max_steps: int = 1) -> int:
        return abi.lbfd_server_pump(self.h, max_steps)

    def drain(self) -> None:
        abi.lbfd_server_drain(self.h)

    def poll(self, rid: int):
        """(state, latency in seconds or -1)."""
        return abi.lbfd_server_poll(self.h, rid)

    def result(self, rid: int):
        """The result array of a finished request (raw storage format for
        RESULT_F, FP64 density for RESULT_RHO)."""
        state, _ = self.poll(rid)
        if state != REQ_DONE:
            raise RuntimeError(f"request {rid} is not done (state {state})")
        return self._bufs[rid][0]

    def stats(self) -> dict:
        return abi.lbfd_server_get_stats(self.h)
