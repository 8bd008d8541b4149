"""ctypes binding of the C ABI in ``include/lbfd.h``.

Argument marshalling only: every step of the method runs in the CUDA
library ``liblbfd.so``.  Loading fails loudly when the library has not been
built; there is no other code path.
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

from . import build as _build

c_int32, c_int64, c_uint32, c_uint64, c_double, c_void_p = (ctypes.c_int32, ctypes.c_int64, ctypes.c_uint32,
                                                            ctypes.c_uint64, ctypes.c_double, ctypes.c_void_p)
P = ctypes.POINTER

OK, EINVAL, ENOMEM, ECUDA, ETIMEOUT, EBUSY, ENOTSUP = 0, -1, -2, -3, -4, -5, -6
D1Q3, D2Q9, D3Q19, D2Q5 = 0, 1, 2, 3
F32, F64, F32_F16, F32_BF16 = 0, 1, 2, 3
NOISE_LOCAL, NOISE_GLOBAL, NOISE_OFF = 0, 1, 2
GAUSSIAN, UNIFORM = 0, 1
INIT_UNIFORM, INIT_SINE, INIT_NONE, INIT_HOST = 0, 1, 2, 3
RESULT_F, RESULT_RHO, RESULT_NONE = 0, 1, 2
POLICY_FIFO, POLICY_SHORTEST, POLICY_LONGEST = 0, 1, 2
WALK_STRIDED, WALK_CONTIGUOUS, WALK_PER_TILE, WALK_PARAM = 0, 1, 2, 3
REQ_UNKNOWN, REQ_QUEUED, REQ_RUNNING, REQ_DONE = -1, 0, 1, 2
MAX_Q, MAX_MODES = 19, 16
KERNEL_AUTO, KERNEL_VEC, KERNEL_SCALAR, KERNEL_SMALL, KERNEL_CLUSTER, KERNEL_MRT, KERNEL_STAGED = 0, 1, 2, 3, 4, 5, 6
KERNEL_NAMES = {KERNEL_VEC: "k_step_vec", KERNEL_SCALAR: "k_step", KERNEL_SMALL: "k_step_small",
                KERNEL_CLUSTER: "k_step_cluster", KERNEL_MRT: "k_step_mrt", KERNEL_STAGED: "k_step_staged"}

Q_OF = {D1Q3: 3, D2Q9: 9, D3Q19: 19, D2Q5: 5}
D_OF = {D1Q3: 1, D2Q9: 2, D3Q19: 3, D2Q5: 2}


class Options(ctypes.Structure):
    """Mirror of ``lbfd_options``."""
    _fields_ = [
        ("lattice", c_int32), ("precision", c_int32), ("noise_mode", c_int32), ("noise_dist", c_int32),
        ("init", c_int32), ("device", c_int32), ("dims", c_int64 * 3), ("tau", c_double),
        ("rho_mean", c_double), ("sine_amp", c_double), ("sine_k", c_int32 * 3), ("lattice_id", c_uint32),
        ("seed", c_uint64), ("stream", c_void_p), ("f_dev", c_void_p * 2), ("n_modes", c_int32),
        ("modes", (c_int32 * 3) * MAX_MODES), ("step_kernel", c_int32), ("wait_test_bytes", c_int32),
        ("slab_global", c_int32), ("slab_first", c_int32), ("sample_every", c_int32),
        ("reserved", c_int32 * 3),
        ("theta", c_double),
        ("tau_moments", c_double * MAX_Q),
    ]


class Obs(ctypes.Structure):
    """Mirror of ``lbfd_obs``."""
    _fields_ = [
        ("t", c_int64), ("n_samples", c_int64), ("Q", c_int32), ("n_modes", c_int32), ("sum_rho", c_double),
        ("sum_rho2", c_double), ("sum_f", c_double * MAX_Q), ("sum_ff", c_double * (MAX_Q * MAX_Q)),
        ("sum_sk", c_double * MAX_MODES),
    ]


class Member(ctypes.Structure):
    """Mirror of ``lbfd_member``."""
    _fields_ = [
        ("dims", c_int64 * 3), ("tau", c_double), ("rho_mean", c_double), ("seed", c_uint64),
        ("lattice_id", c_uint32), ("init", c_int32), ("sine_amp", c_double), ("sine_k", c_int32 * 3),
        ("reserved", c_int32),
    ]


class ServerOptions(ctypes.Structure):
    """Mirror of ``lbfd_server_options``."""
    _fields_ = [
        ("precision", c_int32), ("noise_mode", c_int32), ("noise_dist", c_int32), ("device", c_int32),
        ("hbm_budget", c_int64), ("max_active_sites", c_int64), ("max_active", c_int32), ("max_ahead", c_int32),
        ("passes", c_int32), ("policy", c_int32), ("occupancy", c_int32), ("walk", c_int32),
        ("vx_max", c_int32), ("reserved", c_int32 * 5),
        ("solo_sites", c_int64),
    ]


class Request(ctypes.Structure):
    """Mirror of ``lbfd_request``."""
    _fields_ = [
        ("lattice", c_int32), ("init", c_int32), ("dims", c_int64 * 3), ("tau", c_double), ("rho_mean", c_double),
        ("seed", c_uint64), ("lattice_id", c_uint32), ("result", c_int32), ("steps", c_int64),
        ("sine_amp", c_double), ("sine_k", c_int32 * 3), ("reserved", c_int32), ("in_host", c_void_p),
        ("out_host", c_void_p),
    ]


class ServerStats(ctypes.Structure):
    """Mirror of ``lbfd_server_stats``."""
    _fields_ = [
        ("submitted", c_int64), ("queued", c_int64), ("running", c_int64), ("done", c_int64), ("clock", c_int64),
        ("site_updates", c_int64), ("resident_bytes", c_int64), ("peak_resident_bytes", c_int64),
        ("resident_sites", c_int64), ("peak_resident_sites", c_int64), ("active", c_int32),
        ("peak_active", c_int32), ("launches", c_int64),
    ]


class LbfdError(RuntimeError):
    def __init__(self, code: int, where: str, msg: str):
        super().__init__(f"{where} failed with status {code}: {msg}")
        self.code = code


# name -> (restype, argtypes); every function declared in include/lbfd.h
SIGNATURES = {
    "lbfd_options_init": (c_int32, [P(Options)]),
    "lbfd_create": (c_int32, [P(c_void_p), c_int32, P(c_int64), c_double, c_double, c_uint64]),
    "lbfd_create_ex": (c_int32, [P(c_void_p), P(Options)]),
    "lbfd_destroy": (c_int32, [c_void_p]),
    "lbfd_step": (c_int32, [c_void_p, c_int64]),
    "lbfd_step_kernel": (c_int32, [c_void_p, c_int64, P(c_int32)]),
    "lbfd_set_sample_every": (c_int32, [c_void_p, c_int32]),
    "lbfd_sync": (c_int32, [c_void_p]),
    "lbfd_slab_bounds": (c_int32, [c_int64, c_int32, c_int32, P(c_int64), P(c_int64)]),
    "lbfd_slab_cross": (c_int32, [c_int32, c_int32, c_void_p, P(c_int32)]),
    "lbfd_slab_halo": (c_int32, [c_int32, P(c_int64), c_int32, c_void_p, c_void_p, P(c_int32), P(c_int64)]),
    "lbfd_get_t": (c_int32, [c_void_p, P(c_int64)]),
    "lbfd_set_t": (c_int32, [c_void_p, c_int64]),
    "lbfd_get_f": (c_int32, [c_void_p, c_void_p]),
    "lbfd_set_f": (c_int32, [c_void_p, c_void_p]),
    "lbfd_get_f_raw": (c_int32, [c_void_p, c_void_p]),
    "lbfd_set_f_raw": (c_int32, [c_void_p, c_void_p]),
    "lbfd_moments": (c_int32, [c_void_p, c_void_p, c_void_p]),
    "lbfd_moments_device": (c_int32, [c_void_p, c_void_p, c_void_p]),
    "lbfd_mass": (c_int32, [c_void_p, P(c_double)]),
    "lbfd_sample": (c_int32, [c_void_p]),
    "lbfd_sample_totals": (c_int32, [c_void_p, c_void_p]),
    "lbfd_obs_restore": (c_int32, [c_int32, c_int32, c_double, c_int64, c_void_p, c_void_p]),
    "lbfd_obs_add": (c_int32, [c_void_p, c_void_p]),
    "lbfd_reset_obs": (c_int32, [c_void_p]),
    "lbfd_observables": (c_int32, [c_void_p, P(Obs)]),
    "lbfd_query": (c_int32, [c_void_p, P(c_int32), P(c_int32), P(c_int64), P(c_int32)]),
    "lbfd_state_device": (c_int32, [c_void_p, P(c_void_p), P(c_void_p)]),
    "lbfd_lattice_tables": (c_int32, [c_int32, P(c_int32), c_void_p, c_void_p, c_void_p]),
    "lbfd_lattice_tables_ex": (c_int32, [c_int32, c_double, P(c_int32), c_void_p, c_void_p, c_void_p]),
    "lbfd_noise_draw": (c_int32, [c_int32, c_int32, c_uint64, c_uint32, c_uint64, c_int64, c_int64, c_int32,
                                  c_void_p]),
    "lbfd_box_muller_probe": (c_int32, [c_int32, c_void_p, c_int64, c_void_p]),
    "lbfd_lane_ops_probe": (c_int32, [c_void_p, c_void_p, c_void_p, c_int64, c_void_p]),
    "lbfd_mass_noalloc": (c_int32, [c_int32, c_int32, c_void_p, c_int64, c_void_p, c_void_p]),
    "lbfd_ensemble_create": (c_int32, [P(c_void_p), c_int32, c_int32, c_int32, c_int32, P(Member), c_int32, c_void_p]),
    "lbfd_ensemble_destroy": (c_int32, [c_void_p]),
    "lbfd_ensemble_step": (c_int32, [c_void_p, c_int64]),
    "lbfd_ensemble_sync": (c_int32, [c_void_p]),
    "lbfd_ensemble_tune": (c_int32, [c_void_p, c_int32, P(c_int32), P(c_int32), P(c_int32)]),
    "lbfd_ensemble_plan": (c_int32, [c_void_p, c_int32, c_int32, c_int32, c_int32]),
    "lbfd_ensemble_query": (c_int32, [c_void_p, P(c_int32), P(c_int64), P(c_int64), P(c_int32), P(c_int32),
                                       P(c_int32), P(c_int32)]),
    "lbfd_ensemble_get_f": (c_int32, [c_void_p, c_int32, c_void_p]),
    "lbfd_ensemble_set_f": (c_int32, [c_void_p, c_int32, c_void_p]),
    "lbfd_ensemble_mass": (c_int32, [c_void_p, c_int32, P(c_double)]),
    "lbfd_server_options_init": (c_int32, [P(ServerOptions)]),
    "lbfd_server_create": (c_int32, [P(c_void_p), P(ServerOptions)]),
    "lbfd_server_destroy": (c_int32, [c_void_p]),
    "lbfd_server_submit": (c_int32, [c_void_p, P(Request), P(c_int64)]),
    "lbfd_server_pump": (c_int32, [c_void_p, c_int32, P(c_int64)]),
    "lbfd_server_drain": (c_int32, [c_void_p]),
    "lbfd_server_poll": (c_int32, [c_void_p, c_int64, P(c_int32), P(c_double)]),
    "lbfd_server_get_stats": (c_int32, [c_void_p, P(ServerStats)]),
    "lbfd_server_run_trace": (c_int32, [c_void_p, P(Request), c_void_p, c_int32, c_void_p, c_int64, c_void_p,
                                        P(c_double)]),
    "lbfd_server_struct_sizes": (c_int32, [P(c_int64), P(c_int64), P(c_int64)]),
    "lbfd_pool_create": (c_int32, [P(c_void_p), c_int64, c_int64]),
    "lbfd_pool_destroy": (c_int32, [c_void_p]),
    "lbfd_pool_alloc": (c_int32, [c_void_p, c_int64, P(c_int64)]),
    "lbfd_pool_free": (c_int32, [c_void_p, c_int64]),
    "lbfd_pool_stats": (c_int32, [c_void_p, P(c_int64), P(c_int64), P(c_int32)]),
    "lbfd_last_error": (ctypes.c_char_p, []),
    "lbfd_kernel_launches": (c_int64, []),
    "lbfd_struct_sizes": (c_int32, [P(c_int64), P(c_int64), P(c_int64)]),
}

_lib = None
_lock = threading.Lock()


def library_path() -> str:
    return _build.LIB


def load(build_if_missing: bool = True) -> ctypes.CDLL:
    """Load ``liblbfd.so`` (building it first if asked and needed)."""
    global _lib
    with _lock:
        if _lib is None:
            if build_if_missing and not _build.up_to_date():
                _build.build()
            if not os.path.exists(_build.LIB):
                raise RuntimeError(f"the CUDA library {_build.LIB} is missing: run build() first")
            lib = ctypes.CDLL(_build.LIB)
            for name, (res, args) in SIGNATURES.items():
                fn = getattr(lib, name)
                fn.restype = res
                fn.argtypes = args
            _lib = lib
    return _lib


def last_error() -> str:
    return load().lbfd_last_error().decode()


def _check(rc: int, where: str) -> None:
    if rc != OK:
        raise LbfdError(rc, where, last_error())


def _ptr(a: np.ndarray) -> int:
    return a.ctypes.data


# ---- thin wrappers with the C names ------------------------------------------

def lbfd_options_init() -> Options:
    o = Options()
    _check(load().lbfd_options_init(ctypes.byref(o)), "lbfd_options_init")
    return o


def lbfd_create(lattice: int, dims, tau: float, rho_mean: float, seed: int) -> int:
    h = c_void_p()
    d = (c_int64 * 3)(*[int(x) for x in dims] + [1] * (3 - len(dims)))
    _check(load().lbfd_create(ctypes.byref(h), lattice, d, tau, rho_mean, seed), "lbfd_create")
    return h.value


def lbfd_create_ex(opt: Options) -> int:
    h = c_void_p()
    _check(load().lbfd_create_ex(ctypes.byref(h), ctypes.byref(opt)), "lbfd_create_ex")
    return h.value


def lbfd_destroy(h: int) -> None:
    _check(load().lbfd_destroy(h), "lbfd_destroy")


def lbfd_step(h: int, n: int) -> None:
    _check(load().lbfd_step(h, n), "lbfd_step")


def lbfd_set_sample_every(h: int, every: int) -> None:
    _check(load().lbfd_set_sample_every(h, every), "lbfd_set_sample_every")


def lbfd_step_kernel(h: int, n: int) -> int:
    k = c_int32()
    _check(load().lbfd_step_kernel(h, n, ctypes.byref(k)), "lbfd_step_kernel")
    return k.value


def lbfd_slab_bounds(global_planes: int, nranks: int, rank: int):
    """(first plane, plane count) of rank's slab."""
    first, count = c_int64(), c_int64()
    _check(load().lbfd_slab_bounds(global_planes, nranks, rank, ctypes.byref(first), ctypes.byref(count)),
           "lbfd_slab_bounds")
    return first.value, count.value


def lbfd_slab_cross(lattice: int, direction: int) -> list:
    """Populations with velocity component `direction` along the slowest axis."""
    pops = np.zeros(MAX_Q, dtype=np.int32)
    n = c_int32()
    _check(load().lbfd_slab_cross(lattice, direction, _ptr(pops), ctypes.byref(n)), "lbfd_slab_cross")
    return [int(x) for x in pops[: n.value]]


def lbfd_slab_halo(lattice: int, dims, face: int):
    """(send offsets, receive offsets, values per plane) of one face of a slab
    with owned dims `dims`; offsets are values into its stored state."""
    d = (c_int64 * 3)(*[int(x) for x in dims] + [1] * (3 - len(dims)))
    send = np.zeros(MAX_Q, dtype=np.int64)
    recv = np.zeros(MAX_Q, dtype=np.int64)
    n, plane = c_int32(), c_int64()
    _check(load().lbfd_slab_halo(lattice, d, face, _ptr(send), _ptr(recv), ctypes.byref(n), ctypes.byref(plane)),
           "lbfd_slab_halo")
    return send[: n.value].copy(), recv[: n.value].copy(), plane.value


def lbfd_sync(h: int) -> None:
    _check(load().lbfd_sync(h), "lbfd_sync")


def lbfd_get_t(h: int) -> int:
    t = c_int64()
    _check(load().lbfd_get_t(h, ctypes.byref(t)), "lbfd_get_t")
    return t.value


def lbfd_set_t(h: int, t: int) -> None:
    _check(load().lbfd_set_t(h, t), "lbfd_set_t")


def lbfd_query(h: int):
    Q, D, N, vb = c_int32(), c_int32(), c_int64(), c_int32()
    _check(load().lbfd_query(h, ctypes.byref(Q), ctypes.byref(D), ctypes.byref(N), ctypes.byref(vb)), "lbfd_query")
    return Q.value, D.value, N.value, vb.value


def lbfd_get_f(h: int, out: np.ndarray | None = None) -> np.ndarray:
    Q, D, N, _ = lbfd_query(h)
    if out is None:
        out = np.empty((Q, N), dtype=np.float64)
    assert out.dtype == np.float64 and out.flags.c_contiguous and out.size == Q * N
    _check(load().lbfd_get_f(h, _ptr(out)), "lbfd_get_f")
    return out


def lbfd_set_f(h: int, f: np.ndarray, stored_sites: int | None = None) -> None:
    """stored_sites: for a slab handle, its owned planes plus both halo
    planes (what lbfd_set_f takes); default the handle's N."""
    Q, D, N, _ = lbfd_query(h)
    n = N if stored_sites is None else int(stored_sites)
    f = np.ascontiguousarray(f, dtype=np.float64)
    if f.size != Q * n:
        raise ValueError(f"f must hold Q*N = {Q * n} values")
    _check(load().lbfd_set_f(h, _ptr(f)), "lbfd_set_f")


def lbfd_get_f_raw(h: int, host_ptr: int) -> None:
    _check(load().lbfd_get_f_raw(h, host_ptr), "lbfd_get_f_raw")


def lbfd_set_f_raw(h: int, host_ptr: int) -> None:
    _check(load().lbfd_set_f_raw(h, host_ptr), "lbfd_set_f_raw")


def lbfd_moments(h: int, with_flux: bool = False):
    Q, D, N, _ = lbfd_query(h)
    rho = np.empty(N, dtype=np.float64)
    j = np.empty((D, N), dtype=np.float64) if with_flux else None
    _check(load().lbfd_moments(h, _ptr(rho), _ptr(j) if j is not None else None), "lbfd_moments")
    return (rho, j) if with_flux else rho


def lbfd_moments_device(h: int, rho_dev_ptr: int, j_dev_ptr: int | None = None) -> None:
    _check(load().lbfd_moments_device(h, rho_dev_ptr, j_dev_ptr), "lbfd_moments_device")


def lbfd_mass(h: int) -> float:
    m = c_double()
    _check(load().lbfd_mass(h, ctypes.byref(m)), "lbfd_mass")
    return m.value


def lbfd_sample(h: int) -> None:
    _check(load().lbfd_sample(h), "lbfd_sample")


def lbfd_reset_obs(h: int) -> None:
    _check(load().lbfd_reset_obs(h), "lbfd_reset_obs")


def obs_totals_count(Q: int, n_modes: int) -> int:
    """Entries of one sample's totals (lbfd_sample_totals)."""
    return 2 + Q + 2 * n_modes + Q * (Q + 1) // 2


def lbfd_sample_totals(h: int, Q: int, n_modes: int) -> np.ndarray:
    """One sample's FP64 sums over the handle's own sites (see include/lbfd.h)."""
    out = np.zeros(obs_totals_count(Q, n_modes))
    _check(load().lbfd_sample_totals(h, _ptr(out)), "lbfd_sample_totals")
    return out


def lbfd_obs_restore(lattice: int, n_modes: int, rho_mean: float, n_sites: int, totals) -> np.ndarray:
    """Accumulator entries of one sample from its combined totals (host arithmetic)."""
    Q = Q_OF[lattice]
    t = np.ascontiguousarray(totals, dtype=np.float64)
    if t.size != obs_totals_count(Q, n_modes):
        raise ValueError("totals: wrong length")
    out = np.zeros(2 + Q + Q * Q + n_modes)
    _check(load().lbfd_obs_restore(lattice, n_modes, rho_mean, n_sites, _ptr(t), _ptr(out)), "lbfd_obs_restore")
    return out


def lbfd_obs_add(h: int, acc) -> None:
    a = np.ascontiguousarray(acc, dtype=np.float64)
    _check(load().lbfd_obs_add(h, _ptr(a)), "lbfd_obs_add")


def lbfd_observables(h: int) -> dict:
    o = Obs()
    _check(load().lbfd_observables(h, ctypes.byref(o)), "lbfd_observables")
    Q, K = o.Q, o.n_modes
    return {
        "t": o.t, "n_samples": o.n_samples, "Q": Q, "n_modes": K, "sum_rho": o.sum_rho, "sum_rho2": o.sum_rho2,
        "sum_f": np.array(o.sum_f[:Q]), "sum_ff": np.array(o.sum_ff[:Q * Q]).reshape(Q, Q),
        "sum_sk": np.array(o.sum_sk[:K]),
    }


def lbfd_state_device(h: int):
    f, s = c_void_p(), c_void_p()
    _check(load().lbfd_state_device(h, ctypes.byref(f), ctypes.byref(s)), "lbfd_state_device")
    return f.value, s.value


def lbfd_lattice_tables(lattice: int, theta: float = 0.0):
    """(v[Q,3], w[Q], m[Q,Q]) the kernels use (theta: D2Q5's second moment, 0 = 1/3)."""
    Q = c_int32()
    v = np.zeros(3 * MAX_Q, dtype=np.int32)
    w = np.zeros(MAX_Q)
    m = np.zeros(MAX_Q * MAX_Q)
    _check(load().lbfd_lattice_tables_ex(lattice, theta, ctypes.byref(Q), _ptr(v), _ptr(w), _ptr(m)),
           "lbfd_lattice_tables_ex")
    q = Q.value
    return v[:3 * q].reshape(q, 3).astype(np.int64), w[:q].copy(), m[:q * q].reshape(q, q).copy()


def lbfd_noise_draw(precision: int, dist: int, seed: int, lattice_id: int, t: int, site0: int, nsites: int,
                    nmom: int) -> np.ndarray:
    z = np.empty((nsites, nmom), dtype=np.float64)
    _check(load().lbfd_noise_draw(precision, dist, seed, lattice_id, t, site0, nsites, nmom, _ptr(z)),
           "lbfd_noise_draw")
    return z


def lbfd_box_muller_probe(precision: int, words: np.ndarray) -> np.ndarray:
    w = np.ascontiguousarray(words, dtype=np.uint32).ravel()
    if w.size % 2:
        raise ValueError("words must come in pairs")
    z = np.empty(w.size, dtype=np.float64)
    _check(load().lbfd_box_muller_probe(precision, _ptr(w), w.size // 2, _ptr(z)), "lbfd_box_muller_probe")
    return z


def lbfd_lane_ops_probe(a: np.ndarray, b: np.ndarray, c: np.ndarray) -> np.ndarray:
    """[6, 2, n] float32: the collision's six lane operations on (a, b, c),
    form 0 one value at a time, form 1 two values per packed instruction."""
    a = np.ascontiguousarray(a, dtype=np.float32)
    b = np.ascontiguousarray(b, dtype=np.float32)
    c = np.ascontiguousarray(c, dtype=np.float32)
    if not (a.shape == b.shape == c.shape) or a.ndim != 1:
        raise ValueError("a, b and c must be 1-D arrays of one length")
    out = np.empty(12 * a.size, dtype=np.float32)
    _check(load().lbfd_lane_ops_probe(_ptr(a), _ptr(b), _ptr(c), a.size, _ptr(out)), "lbfd_lane_ops_probe")
    return out.reshape(6, 2, a.size)


def lbfd_mass_noalloc(lattice: int, precision: int, f_dev_ptr: int, n_sites: int, mass_dev_ptr: int,
                      stream: int | None = None) -> None:
    """Mass of a caller-owned device array into a caller-owned device double,
    with no device allocation (fixed internal scratch; see include/lbfd.h)."""
    _check(load().lbfd_mass_noalloc(lattice, precision, f_dev_ptr, n_sites, mass_dev_ptr, stream),
           "lbfd_mass_noalloc")


def make_members(specs) -> ctypes.Array:
    """specs: dicts with dims, tau, rho_mean, seed and optionally lattice_id,
    init, sine_amp, sine_k."""
    arr = (Member * len(specs))()
    for k, sp in enumerate(specs):
        d = [int(x) for x in sp["dims"]] + [1] * (3 - len(sp["dims"]))
        m = arr[k]
        for a in range(3):
            m.dims[a] = d[a]
        m.tau, m.rho_mean, m.seed = float(sp["tau"]), float(sp["rho_mean"]), int(sp["seed"])
        m.lattice_id = int(sp.get("lattice_id", 0))
        m.init = int(sp.get("init", INIT_UNIFORM))
        m.sine_amp = float(sp.get("sine_amp", 0.0))
        sk = list(sp.get("sine_k", (1, 0, 0))) + [0, 0, 0]
        for a in range(3):
            m.sine_k[a] = int(sk[a])
    return arr


def lbfd_ensemble_create(lattice: int, precision: int, noise_mode: int, noise_dist: int, specs, stream=None) -> int:
    h = c_void_p()
    arr = make_members(specs)
    _check(load().lbfd_ensemble_create(ctypes.byref(h), lattice, precision, noise_mode, noise_dist, arr, len(specs),
                                       stream), "lbfd_ensemble_create")
    return h.value


def lbfd_ensemble_destroy(e: int) -> None:
    _check(load().lbfd_ensemble_destroy(e), "lbfd_ensemble_destroy")


def lbfd_ensemble_step(e: int, n: int) -> None:
    _check(load().lbfd_ensemble_step(e, n), "lbfd_ensemble_step")


def lbfd_ensemble_sync(e: int) -> None:
    _check(load().lbfd_ensemble_sync(e), "lbfd_ensemble_sync")


def lbfd_ensemble_tune(e: int, steps: int = 3):
    """Returns the chosen (sites per item at most, tile passes, blocks per SM)."""
    v, p, b = c_int32(), c_int32(), c_int32()
    _check(load().lbfd_ensemble_tune(e, steps, ctypes.byref(v), ctypes.byref(p), ctypes.byref(b)),
           "lbfd_ensemble_tune")
    return v.value, p.value, b.value


def lbfd_ensemble_plan(e: int, vx_max: int, passes: int, occupancy: int, walk: int) -> None:
    _check(load().lbfd_ensemble_plan(e, vx_max, passes, occupancy, walk), "lbfd_ensemble_plan")


def lbfd_ensemble_query(e: int):
    """Returns (members, total sites, t, sites per item at most, tile passes, blocks per SM, tile order)."""
    n, sites, t, vx, passes, bps, walk = c_int32(), c_int64(), c_int64(), c_int32(), c_int32(), c_int32(), c_int32()
    _check(load().lbfd_ensemble_query(e, ctypes.byref(n), ctypes.byref(sites), ctypes.byref(t), ctypes.byref(vx),
                                      ctypes.byref(passes), ctypes.byref(bps), ctypes.byref(walk)),
           "lbfd_ensemble_query")
    return n.value, sites.value, t.value, vx.value, passes.value, bps.value, walk.value


def lbfd_ensemble_get_f(e: int, member: int, Q: int, N: int) -> np.ndarray:
    out = np.empty((Q, N), dtype=np.float64)
    _check(load().lbfd_ensemble_get_f(e, member, _ptr(out)), "lbfd_ensemble_get_f")
    return out


def lbfd_ensemble_set_f(e: int, member: int, f: np.ndarray) -> None:
    f = np.ascontiguousarray(f, dtype=np.float64)
    _check(load().lbfd_ensemble_set_f(e, member, _ptr(f)), "lbfd_ensemble_set_f")


def lbfd_ensemble_mass(e: int, member: int) -> float:
    m = c_double()
    _check(load().lbfd_ensemble_mass(e, member, ctypes.byref(m)), "lbfd_ensemble_mass")
    return m.value


# ---- serving -----------------------------------------------------------------

def lbfd_server_options_init() -> ServerOptions:
    o = ServerOptions()
    _check(load().lbfd_server_options_init(ctypes.byref(o)), "lbfd_server_options_init")
    return o


def lbfd_server_create(opt: ServerOptions) -> int:
    h = c_void_p()
    _check(load().lbfd_server_create(ctypes.byref(h), ctypes.byref(opt)), "lbfd_server_create")
    return h.value


def lbfd_server_destroy(s: int) -> None:
    _check(load().lbfd_server_destroy(s), "lbfd_server_destroy")


def make_request(lattice: int, dims, tau: float, rho_mean: float, seed: int, steps: int, *, lattice_id: int = 0,
                 init: int = INIT_UNIFORM, sine_amp: float = 0.0, sine_k=(1, 0, 0), result: int = RESULT_F,
                 in_host: int | None = None, out_host: int | None = None) -> Request:
    r = Request()
    d = [int(x) for x in dims] + [1] * (3 - len(dims))
    r.lattice, r.init, r.tau, r.rho_mean, r.seed = lattice, init, float(tau), float(rho_mean), int(seed)
    for a in range(3):
        r.dims[a] = d[a]
    sk = list(sine_k) + [0, 0, 0]
    for a in range(3):
        r.sine_k[a] = int(sk[a])
    r.lattice_id, r.result, r.steps, r.sine_amp = int(lattice_id), int(result), int(steps), float(sine_amp)
    r.in_host, r.out_host = in_host, out_host
    return r


def lbfd_server_submit(s: int, req: Request) -> int:
    i = c_int64()
    _check(load().lbfd_server_submit(s, ctypes.byref(req), ctypes.byref(i)), "lbfd_server_submit")
    return i.value


def lbfd_server_pump(s: int, max_steps: int = 1) -> int:
    left = c_int64()
    _check(load().lbfd_server_pump(s, max_steps, ctypes.byref(left)), "lbfd_server_pump")
    return left.value


def lbfd_server_drain(s: int) -> None:
    _check(load().lbfd_server_drain(s), "lbfd_server_drain")


def lbfd_server_poll(s: int, rid: int):
    st, lat = c_int32(), c_double()
    _check(load().lbfd_server_poll(s, rid, ctypes.byref(st), ctypes.byref(lat)), "lbfd_server_poll")
    return st.value, lat.value


def lbfd_server_get_stats(s: int) -> dict:
    st = ServerStats()
    _check(load().lbfd_server_get_stats(s, ctypes.byref(st)), "lbfd_server_get_stats")
    return {name: getattr(st, name) for name, _ in ServerStats._fields_}


def lbfd_server_run_trace(s: int, reqs, arrival_s, sink_ptr: int | None, sink_bytes: int):
    """Runs a fixed trace (see include/lbfd.h); returns (latencies [s], makespan [s])."""
    n = len(reqs)
    arr = (Request * n)(*reqs)
    arrival = np.ascontiguousarray(arrival_s, dtype=np.float64)
    lat = np.empty(n, dtype=np.float64)
    mk = c_double()
    _check(load().lbfd_server_run_trace(s, arr, _ptr(arrival), n, sink_ptr, int(sink_bytes), _ptr(lat),
                                        ctypes.byref(mk)), "lbfd_server_run_trace")
    return lat, mk.value


def lbfd_server_struct_sizes():
    a, b, c = c_int64(), c_int64(), c_int64()
    _check(load().lbfd_server_struct_sizes(ctypes.byref(a), ctypes.byref(b), ctypes.byref(c)),
           "lbfd_server_struct_sizes")
    return a.value, b.value, c.value


# ---- host range allocator ---------------------------------------------------------

def lbfd_pool_create(capacity: int, align: int) -> int:
    h = c_void_p()
    _check(load().lbfd_pool_create(ctypes.byref(h), capacity, align), "lbfd_pool_create")
    return h.value


def lbfd_pool_destroy(p: int) -> None:
    _check(load().lbfd_pool_destroy(p), "lbfd_pool_destroy")


def lbfd_pool_alloc(p: int, size: int) -> int:
    """Offset of a free range, or -1 when none fits."""
    off = c_int64()
    rc = load().lbfd_pool_alloc(p, size, ctypes.byref(off))
    if rc == EBUSY:
        return -1
    _check(rc, "lbfd_pool_alloc")
    return off.value


def lbfd_pool_free(p: int, offset: int) -> None:
    _check(load().lbfd_pool_free(p, offset), "lbfd_pool_free")


def lbfd_pool_stats(p: int):
    used, largest, nfree = c_int64(), c_int64(), c_int32()
    _check(load().lbfd_pool_stats(p, ctypes.byref(used), ctypes.byref(largest), ctypes.byref(nfree)),
           "lbfd_pool_stats")
    return used.value, largest.value, nfree.value


def lbfd_kernel_launches() -> int:
    return int(load().lbfd_kernel_launches())


def lbfd_struct_sizes():
    a, b, c = c_int64(), c_int64(), c_int64()
    _check(load().lbfd_struct_sizes(ctypes.byref(a), ctypes.byref(b), ctypes.byref(c)), "lbfd_struct_sizes")
    return a.value, b.value, c.value
