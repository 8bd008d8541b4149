"""Pins of the oracle's whole-lattice evolution (eq. LB, collide then stream).

- Noise off, the evolution is linear: it must equal a dense operator built
  here in f-space from the lattice tables (BGK form of eq. collision plus a
  periodic shift by v_i), including lattices with sides of 1 and 2 where the
  wrap aliases neighbours.
- Single Fourier modes decay by the transfer matrix A(k) = diag(e^{-i k.v})
  [(1 - 1/tau) I + (1/tau) w 1^T]; at tau = 1 on D1Q3 the density mode decays
  by lambda^t with lambda = 2/3 + cos(k)/3 (the density recursion of the
  equilibrium-dynamics passage, Sec. IV).
- With noise, the exact stationary covariance of the linear-Gaussian system
  (brute-force Lyapunov sum on 4-8 sites) equals the paper's Poisson
  second moment (eq. ffluct) corrected for global mass conservation:
  rho (w_i delta_ij delta_xx' - w_i w_j / N).
- Mass is conserved to rounding, and a run split in two equals one run.
"""
import math

import numpy as np
import pytest


def _shift_operator(v, dims, Q):
    """P[(i, x+v_i), (i, x)] = 1 on the periodic lattice, layout i*N + site."""
    Lx, Ly, Lz = dims
    N = Lx * Ly * Lz
    P = np.zeros((Q * N, Q * N))
    for i in range(Q):
        for z in range(Lz):
            for y in range(Ly):
                for x in range(Lx):
                    s = x + Lx * (y + Ly * z)
                    d = ((x + v[i, 0]) % Lx) + Lx * (((y + v[i, 1]) % Ly) + Ly * ((z + v[i, 2]) % Lz))
                    P[i * N + d, i * N + s] += 1.0
    return P


def _bgk_operator(w, tau, N):
    """Block collision K: f*_i = f_i + (w_i rho - f_i)/tau at every site."""
    Q = w.size
    Ks = (1 - 1.0 / tau) * np.eye(Q) + np.outer(w, np.ones(Q)) / tau
    return np.kron(Ks, np.eye(N))  # acts on layout i*N + s


def _oracle_operator(orc, lat, dims, tau, theta=1.0 / 3.0):
    Q = orc.q_of(lat)
    N = int(np.prod(dims))
    A = np.zeros((Q * N, Q * N))
    for k in range(Q * N):
        e = np.zeros((Q, N))
        e.flat[k] = 1.0
        A[:, k] = orc.run(lat, dims, e, 1, tau, orc.NOISE_OFF, theta=theta, rho_eq=0.0).ravel()
    return A


CASES = [
    ("D1Q3", (5, 1, 1), 0.8),
    ("D1Q3", (1, 1, 1), 0.7),
    ("D1Q3", (2, 1, 1), 1.3),
    ("D2Q9", (3, 4, 1), 0.8),
    ("D2Q9", (2, 1, 1), 0.6),
    ("D2Q9", (1, 3, 1), 1.0),
    ("D3Q19", (2, 3, 2), 1.0),
    ("D3Q19", (3, 1, 2), 0.55),
    ("D2Q5", (3, 3, 1), 1.0),
]


@pytest.mark.parametrize("name,dims,tau", CASES)
def test_noise_off_equals_dense_operator(orc, name, dims, tau):
    lat = getattr(orc, name)
    D, Q, v, w = orc.lattice(lat)
    N = int(np.prod(dims))
    A_test = _shift_operator(v, dims, Q) @ _bgk_operator(w, tau, N)
    A_orc = _oracle_operator(orc, lat, dims, tau)
    assert np.max(np.abs(A_orc - A_test)) < 1e-15


@pytest.mark.parametrize("t,expect", [(1000, 0.9044766338315362), (10000, 0.3664152311782258)])
def test_d1q3_sine_decay_closed_form(orc, t, expect):
    """D1Q3, tau = 1, L = 256, rho = 10 + sin(2 pi x / 256), noise off:
    the sine amplitude after t steps is lambda^t, lambda = 2/3 + cos(2 pi/256)/3."""
    L = 256
    lam = 2.0 / 3.0 + math.cos(2 * math.pi / L) / 3.0
    assert abs(lam**t - expect) < 1e-13
    x = np.arange(L)
    rho0 = 10.0 + np.sin(2 * np.pi * x / L)
    f = orc.init_equilibrium(orc.D1Q3, rho0)
    f = orc.run(orc.D1Q3, (L,), f, t, 1.0, orc.NOISE_OFF)
    rho = f.sum(0)
    amp = 2.0 / L * ((rho - 10.0) * np.sin(2 * np.pi * x / L)).sum()
    assert abs(amp - lam**t) < 1e-13 + 1e-15 * t
    # pointwise: FP64 rounding accumulates over t steps on values near 10
    assert np.max(np.abs(rho - (10.0 + lam**t * np.sin(2 * np.pi * x / L)))) < 1e-15 * 10.0 * t


@pytest.mark.parametrize("name,dims,k,tau,t", [
    ("D2Q9", (64, 32, 1), (3, 1, 0), 0.8, 150),
    ("D3Q19", (16, 8, 8), (1, 2, 1), 0.6, 60),
    ("D2Q5", (40, 30, 1), (2, 5, 0), 1.4, 80),
])
def test_fourier_mode_transfer_matrix(orc, name, dims, k, tau, t):
    """f(k, t) = A(k)^t f(k, 0) for a single-mode start, any tau."""
    lat = getattr(orc, name)
    D, Q, v, w = orc.lattice(lat)
    Lx, Ly, Lz = dims
    kv = 2 * np.pi * np.array(k) / np.array(dims)
    zz, yy, xx = np.meshgrid(np.arange(Lz), np.arange(Ly), np.arange(Lx), indexing="ij")
    phase = kv[0] * xx + kv[1] * yy + kv[2] * zz  # shape (Lz, Ly, Lx) -> ravel = site order
    rho0 = 5.0 + np.cos(phase).ravel()
    f = orc.init_equilibrium(lat, rho0)
    f = orc.run(lat, dims, f, t, tau, orc.NOISE_OFF)
    K = (1 - 1.0 / tau) * np.eye(Q) + np.outer(w, np.ones(Q)) / tau
    A = np.diag(np.exp(-1j * (v @ kv))) @ K
    fk = np.linalg.matrix_power(A, t) @ (0.5 * w.astype(complex))
    pred = 5.0 * w[:, None] + 2.0 * np.real(fk[:, None] * np.exp(1j * phase.ravel())[None, :])
    assert np.max(np.abs(f - pred)) < 1e-12


def _streamed_noise_cov(v, dims, Q, sigma_f):
    """Covariance of the streamed noise: xi_i(x) lands on (i, x + v_i)."""
    N = int(np.prod(dims))
    P = _shift_operator(v, dims, Q)
    S0 = np.kron(sigma_f, np.eye(N))
    return P @ S0 @ P.T


def _lyapunov_sum(A, S, w_full, doublings=22):
    """sum_k A^k S A^kT by doubling.  The mass mode (right eigenvector w_full,
    left eigenvector 1, eigenvalue 1) carries no noise; it is projected out of
    A so that rounding in that direction cannot grow."""
    n = w_full.size
    N_sites = w_full.sum()
    Pi = np.eye(n) - np.outer(w_full, np.ones(n)) / N_sites
    C, Ak = S.copy(), A @ Pi
    for _ in range(doublings):
        C = C + Ak @ C @ Ak.T
        Ak = Ak @ Ak
    return C


@pytest.mark.parametrize("name,dims,tau", [
    ("D1Q3", (4, 1, 1), 1.0),
    ("D1Q3", (5, 1, 1), 0.6),
    ("D1Q3", (8, 1, 1), 1.5),
    ("D2Q9", (2, 2, 1), 0.8),
    ("D2Q9", (2, 4, 1), 1.2),
    ("D3Q19", (2, 2, 2), 1.0),
    ("D2Q5", (3, 3, 1), 1.0),
])
def test_exact_stationary_covariance(orc, name, dims, tau):
    """Brute force: the stationary covariance of the oracle's dynamics (its
    noise-off operator and its per-site noise map, global noise) equals
    rho (w_i delta_ij delta_xx' - w_i w_j / N): the Poisson second moment of
    eq. ffluct with the total mass held fixed (Sec. IV, Table I discussion)."""
    lat = getattr(orc, name)
    D, Q, v, w = orc.lattice(lat)
    N = int(np.prod(dims))
    rho = 7.0
    A = _oracle_operator(orc, lat, dims, tau)
    # per-site noise map of the oracle's collision
    base = orc.collide(lat, rho * w, np.zeros(Q - 1), tau, orc.NOISE_GLOBAL, rho)
    B = np.zeros((Q, Q - 1))
    for a in range(Q - 1):
        z = np.zeros(Q - 1)
        z[a] = 1.0
        B[:, a] = orc.collide(lat, rho * w, z, tau, orc.NOISE_GLOBAL, rho) - base
    S = _streamed_noise_cov(v, dims, Q, B @ B.T)
    wf = np.repeat(w, N)
    C = _lyapunov_sum(A, S, wf)
    expect = rho * (np.diag(wf) - np.outer(wf, wf) / N)
    assert np.max(np.abs(C - expect)) < 1e-11 * rho


def test_mass_conserved_with_noise(orc):
    lat = orc.D2Q9
    dims = (32, 24, 1)
    N = 32 * 24
    rng = np.random.default_rng(1)
    rho0 = 100.0 + rng.normal(0, 3, N)
    f = orc.init_equilibrium(lat, rho0)
    m0 = f.sum()
    t = 300
    f = orc.run(lat, dims, f, t, 0.8, orc.NOISE_LOCAL, seed=9)
    eps = 2.0**-53
    # Mass is exact in real arithmetic (Sec. IV: the total density is
    # conserved).  In FP64 each stored population carries a rounding of
    # relative size ~eps, and sum_i w_i = 1 holds only to rounding, which
    # makes the drift systematic: bound it by Q eps rho t N.
    assert abs(f.sum() - m0) <= 9 * eps * 100.0 * t * N
    # and the noise did act
    assert np.std(f.sum(0)) > 3.5


def test_noise_is_streamed_with_populations(orc):
    """One step from a uniform state: the noise each site emits sums to zero
    over the populations it sends out (noise lives in non-conserved moments,
    then streams)."""
    lat = orc.D2Q9
    D, Q, v, w = orc.lattice(lat)
    dims = (6, 5, 1)
    N = 30
    f0 = orc.init_equilibrium(lat, np.full(N, 20.0))
    noisy = orc.run(lat, dims, f0, 1, 0.9, orc.NOISE_LOCAL, seed=4, t0=17)
    quiet = orc.run(lat, dims, f0, 1, 0.9, orc.NOISE_OFF)
    d = (noisy - quiet).reshape(Q, 5, 6)
    for y in range(5):
        for x in range(6):
            tot = sum(d[i, (y + v[i, 1]) % 5, (x + v[i, 0]) % 6] for i in range(Q))
            assert abs(tot) < 1e-13
    assert np.max(np.abs(d)) > 0.1


@pytest.mark.parametrize("mode", ["NOISE_LOCAL", "NOISE_GLOBAL"])
def test_split_run_is_bit_identical(orc, mode):
    lat = orc.D3Q19
    dims = (5, 4, 3)
    rng = np.random.default_rng(2)
    f0 = orc.init_equilibrium(lat, 30 + rng.normal(0, 1, 60))
    nm = getattr(orc, mode)
    whole = orc.run(lat, dims, f0, 7, 0.7, nm, seed=99, rho_eq=30.0)
    part = orc.run(lat, dims, f0, 3, 0.7, nm, seed=99, rho_eq=30.0)
    part = orc.run(lat, dims, part, 4, 0.7, nm, seed=99, rho_eq=30.0, t0=3)
    assert np.array_equal(whole, part)
