"""ORACLE for the fluctuating lattice-Boltzmann diffusion step (arXiv:1606.07801).

Test infrastructure only: the test suite, the smoke check and the CPU-baseline
leg of the benchmark may import this package; the product path never does.
It is a thin ctypes binding over ``lbfd_oracle.c``, a plain FP64 C
restatement of the method (Sec. II eqs. LB, collision, coll, xiglobal,
xilocal; Sec. IV noise distribution and zero-density clamp).  It shares no
code with the CUDA library.

Every function here is pinned by ``tests/test_oracle_*.py`` against what the
paper and the mathematics fix (closed forms, printed values, invariants,
brute force on tiny lattices).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

D1Q3, D2Q9, D3Q19, D2Q5 = 0, 1, 2, 3
NOISE_LOCAL, NOISE_GLOBAL, NOISE_OFF = 0, 1, 2
GAUSSIAN, UNIFORM = 0, 1
QMAX = 19

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "lbfd_oracle.c")
_LIB = os.path.join(_HERE, "liblbfd_oracle.so")
_lock = threading.Lock()
_lib = None

_QOF = {D1Q3: 3, D2Q9: 9, D3Q19: 19, D2Q5: 5}


def build(force: bool = False) -> str:
    """Compile the oracle with gcc into ``oracle/liblbfd_oracle.so``."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fopenmp", _SRC, "-o", tmp, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is None:
            build()
            lib = ctypes.CDLL(_LIB)
            P = ctypes.POINTER
            lib.orc_lattice.argtypes = [ctypes.c_int, ctypes.c_double, P(ctypes.c_int), P(ctypes.c_int),
                                        P(ctypes.c_int), P(ctypes.c_double)]
            lib.orc_basis.argtypes = [ctypes.c_int, ctypes.c_double, P(ctypes.c_double)]
            lib.orc_philox4x32_10.argtypes = [P(ctypes.c_uint32), P(ctypes.c_uint32), P(ctypes.c_uint32)]
            lib.orc_philox4x32_10.restype = None
            lib.orc_site_noise.argtypes = [ctypes.c_uint64, ctypes.c_uint32, ctypes.c_uint64, ctypes.c_uint64,
                                           ctypes.c_int, ctypes.c_int, P(ctypes.c_double)]
            lib.orc_site_noise.restype = None
            lib.orc_collide.argtypes = [ctypes.c_int, ctypes.c_double, P(ctypes.c_double), ctypes.c_int,
                                        ctypes.c_double, P(ctypes.c_double), P(ctypes.c_double),
                                        P(ctypes.c_double)]
            lib.orc_run.argtypes = [ctypes.c_int, ctypes.c_double, P(ctypes.c_int64), P(ctypes.c_double),
                                    ctypes.c_int, ctypes.c_int, ctypes.c_double, ctypes.c_uint64,
                                    ctypes.c_uint32, ctypes.c_uint64, ctypes.c_int64, P(ctypes.c_double)]
            lib.orc_init_equilibrium.argtypes = [ctypes.c_int, ctypes.c_double, ctypes.c_int64,
                                                 P(ctypes.c_double), P(ctypes.c_double)]
            _lib = lib
    return _lib


def _dp(a: np.ndarray):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _check(rc: int, what: str):
    if rc < 0:
        raise ValueError(f"oracle {what} failed (rc={rc})")


def lattice(lat: int, theta: float = 1.0 / 3.0):
    """(D, Q, v[Q,3], w[Q]) of a lattice (Sec. II; D2Q5 uses ``theta``)."""
    lib = _load()
    D, Q = ctypes.c_int(), ctypes.c_int()
    v = (ctypes.c_int * (QMAX * 3))()
    w = np.zeros(QMAX)
    _check(lib.orc_lattice(lat, theta, ctypes.byref(D), ctypes.byref(Q), v, _dp(w)), "lattice")
    q = Q.value
    return D.value, q, np.array(v[: 3 * q], dtype=np.int64).reshape(q, 3), w[:q].copy()


def basis(lat: int, theta: float = 1.0 / 3.0) -> np.ndarray:
    """Moment matrix m[a, i] = m_i^a by weighted Gram-Schmidt (Sec. II)."""
    lib = _load()
    m = np.zeros(QMAX * QMAX)
    q = lib.orc_basis(lat, theta, _dp(m))
    _check(q, "basis")
    return m[: q * q].reshape(q, q).copy()


def philox4x32_10(ctr, key) -> np.ndarray:
    """One Philox4x32-10 block (Salmon et al., SC'11)."""
    lib = _load()
    c = (ctypes.c_uint32 * 4)(*[int(x) & 0xFFFFFFFF for x in ctr])
    k = (ctypes.c_uint32 * 2)(*[int(x) & 0xFFFFFFFF for x in key])
    o = (ctypes.c_uint32 * 4)()
    lib.orc_philox4x32_10(c, k, o)
    return np.array(list(o), dtype=np.uint32)


def site_noise(seed: int, lattice_id: int, site: int, t: int, nmom: int, dist: int = GAUSSIAN) -> np.ndarray:
    """Unit variates z^1..z^nmom the oracle draws at (site, step)."""
    lib = _load()
    z = np.zeros(max(nmom, 1) + 4)
    lib.orc_site_noise(seed, lattice_id, site, t, nmom, dist, _dp(z))
    return z[:nmom].copy()


def _taus(lat: int, tau) -> np.ndarray:
    q = _QOF[lat]
    t = np.broadcast_to(np.asarray(tau, dtype=np.float64), (q,)).copy()
    return t


def collide(lat: int, fin, z, tau, noise_mode: int = NOISE_LOCAL, rho_eq: float = 0.0,
            theta: float = 1.0 / 3.0) -> np.ndarray:
    """Post-collision populations of one site for given unit variates z."""
    lib = _load()
    q = _QOF[lat]
    fin = np.ascontiguousarray(fin, dtype=np.float64)
    zz = np.zeros(QMAX)
    zz[: q - 1] = np.asarray(z, dtype=np.float64)[: q - 1]
    out = np.zeros(q)
    taus = _taus(lat, tau)
    _check(lib.orc_collide(lat, theta, _dp(taus), noise_mode, rho_eq, _dp(fin), _dp(zz), _dp(out)), "collide")
    return out


def init_equilibrium(lat: int, rho, theta: float = 1.0 / 3.0) -> np.ndarray:
    """f_i(x, 0) = w_i rho(x, 0), layout [i, site] (eq. f0def)."""
    lib = _load()
    rho = np.ascontiguousarray(np.ravel(rho), dtype=np.float64)
    q = _QOF[lat]
    f = np.zeros((q, rho.size))
    _check(lib.orc_init_equilibrium(lat, theta, rho.size, _dp(rho), _dp(f)), "init")
    return f


def run(lat: int, dims, f, nsteps: int, tau, noise_mode: int = NOISE_LOCAL, dist: int = GAUSSIAN,
        rho_eq: float | None = None, seed: int = 1, lattice_id: int = 0, t0: int = 0,
        theta: float = 1.0 / 3.0) -> np.ndarray:
    """Evolve f ([Q, N] FP64, site = x + Lx (y + Ly z)) by ``nsteps`` LB steps.

    ``rho_eq`` defaults to the mean density of ``f`` (global noise uses the
    initial mass per site, which the dynamics conserve).
    """
    lib = _load()
    d = [int(x) for x in dims] + [1] * (3 - len(dims))
    dd = np.array(d, dtype=np.int64)
    f = np.array(f, dtype=np.float64, order="C", copy=True)
    q = _QOF[lat]
    n = int(np.prod(d))
    if f.shape != (q, n):
        f = f.reshape(q, n)
    if rho_eq is None:
        rho_eq = float(f.sum() / n)
    taus = _taus(lat, tau)
    rc = lib.orc_run(lat, theta, dd.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)), _dp(taus), noise_mode, dist,
                     float(rho_eq), int(seed) & (2**64 - 1), int(lattice_id), int(t0), int(nsteps), _dp(f))
    _check(rc, "run")
    return f


def set_threads(n: int) -> None:
    """Number of OpenMP threads the oracle's site loop may use."""
    try:
        omp = ctypes.CDLL("libgomp.so.1")
        omp.omp_set_num_threads(int(n))
    except OSError:
        pass


def q_of(lat: int) -> int:
    return _QOF[lat]
