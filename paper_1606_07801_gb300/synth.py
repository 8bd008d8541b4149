"""Seeded synthetic inputs for tests and the benchmark.

Nothing here computes any part of the method: these are random arrays,
density fields and workload descriptions with the shapes and value ranges of
the paper's experiments (periodic lattices at a given mean density, single
Fourier modes, ensembles of lattices of mixed size).  Both the CUDA path and
the oracle consume them.
"""
from __future__ import annotations

import math

import numpy as np


def rng(seed: int) -> np.random.Generator:
    return np.random.default_rng(np.random.SeedSequence(int(seed)))


def random_populations(Q: int, N: int, rho_mean: float, spread: float, seed: int,
                       dtype=np.float64) -> np.ndarray:
    """[Q, N] values rho_mean/Q * (1 + spread * U(-1, 1)): a positive,
    non-equilibrium state with mean density about rho_mean."""
    g = rng(seed)
    if dtype == np.float64:
        return (rho_mean / Q) * (1.0 + spread * g.uniform(-1.0, 1.0, size=(Q, N)))
    out = g.random(size=(Q, N), dtype=np.float32)
    out *= np.float32(2.0 * spread)
    out += np.float32(1.0 - spread)
    out *= np.float32(rho_mean / Q)
    return out


def density_sine(dims, k, amp: float, rho_mean: float) -> np.ndarray:
    """rho(x) = rho_mean + amp * sin(2 pi (kx x/Lx + ky y/Ly + kz z/Lz)), site order x fastest."""
    d = [int(v) for v in dims] + [1] * (3 - len(dims))
    kk = [int(v) for v in k] + [0] * (3 - len(k))
    z, y, x = np.meshgrid(np.arange(d[2]), np.arange(d[1]), np.arange(d[0]), indexing="ij")
    frac = (kk[0] * x % d[0]) / d[0] + (kk[1] * y % d[1]) / d[1] + (kk[2] * z % d[2]) / d[2]
    return (rho_mean + amp * np.sin(2 * np.pi * frac)).ravel()


def density_noise(N: int, rho_mean: float, sd: float, seed: int) -> np.ndarray:
    """Gaussian density field around rho_mean."""
    return rho_mean + sd * rng(seed).normal(size=N)


def ensemble(n: int, side_lo: int = 32, side_hi: int = 512, rho_lo: float = 0.5, rho_hi: float = 200.0,
             tau_lo: float = 0.6, tau_hi: float = 1.5, seed: int = 12345, ndim: int = 2):
    """n lattices of ndim dimensions: sides drawn independently log-uniform in
    [side_lo, side_hi] (rounded), mean density and tau uniform in their
    ranges, distinct seeds."""
    g = rng(seed)
    sides = [np.rint(np.exp(g.uniform(math.log(side_lo), math.log(side_hi), n))).astype(np.int64)
             for _ in range(ndim)]
    rho = g.uniform(rho_lo, rho_hi, n)
    tau = g.uniform(tau_lo, tau_hi, n)
    seeds = (int(seed) * 1000003 + np.arange(n)).astype(np.uint64)
    return [dict(dims=tuple(int(sd[i]) for sd in sides), rho_mean=float(rho[i]), tau=float(tau[i]),
                 seed=int(seeds[i])) for i in range(n)]


def served_trace(n: int, rate: float = 500.0, seed: int = 777, d1_range=(256, 65536), d2_side=(32, 1024),
                 d3_side=(32, 128), steps_range=(100, 10000), rho_lo: float = 0.5, rho_hi: float = 200.0,
                 tau_lo: float = 0.6, tau_hi: float = 1.5):
    """A stream of n simulation requests with Poisson arrivals at `rate` per
    second.  The lattice type is uniform over D1Q3 / D2Q9 / D3Q19; D1Q3
    lengths, D2Q9 square sides and D3Q19 cube sides are log-uniform in their
    ranges (rounded), step counts log-uniform in steps_range, mean density
    and tau uniform, seeds distinct.  Returns (arrival times [s], specs)."""
    g = rng(seed)
    arrivals = np.cumsum(g.exponential(1.0 / rate, n))
    arrivals -= arrivals[0]
    kinds = g.integers(0, 3, n)
    u = g.uniform(0.0, 1.0, n)
    steps = np.rint(np.exp(g.uniform(math.log(steps_range[0]), math.log(steps_range[1]), n))).astype(np.int64)
    rho = g.uniform(rho_lo, rho_hi, n)
    tau = g.uniform(tau_lo, tau_hi, n)

    def logu(lo, hi, x):
        return int(round(math.exp(math.log(lo) + x * (math.log(hi) - math.log(lo)))))

    specs = []
    for i in range(n):
        k = int(kinds[i])
        if k == 0:
            dims = (logu(*d1_range, u[i]),)
        elif k == 1:
            s = logu(*d2_side, u[i])
            dims = (s, s)
        else:
            s = logu(*d3_side, u[i])
            dims = (s, s, s)
        specs.append(dict(lattice=k, dims=dims, steps=int(steps[i]), rho_mean=float(rho[i]), tau=float(tau[i]),
                          seed=int(seed) * 1000003 + i, lattice_id=i))
    return arrivals, specs
