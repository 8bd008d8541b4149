"""Time correlators of the density (Sec. IV, "Equilibrium dynamics", eq.
TimeCorrEqn): in equilibrium the normalised correlation
<rho_k(s + t) rho_k(s)*> / <|rho_k|^2> of a Fourier mode k != 0 follows the
density row of the lattice's transfer matrix,
    C_k(t) = 1^T A(k)^t w,   A(k) = diag(e^{-i k.v_i}) [(1 - 1/tau) I + (1/tau) w 1^T],
because the equal-time covariance of f(k) is N rho diag(w) (the flat
structure factor) and the noise has zero mean given the present state.  At
tau = 1 this is lambda(k)^t, lambda(k) = sum_i w_i cos(k.v_i); the paper's
exponential with gamma(k) is its continuum form.  The oracle's noisy runs
must reproduce it within their statistical error (batch means, 5 sigma)."""
import math

import numpy as np
import pytest


def transfer_correlation(v, w, k, tau, t):
    """Re 1^T A(k)^t w for wave vector k (radians per lattice unit)."""
    Q = len(w)
    omega = (1.0 - 1.0 / tau) * np.eye(Q) + np.outer(w, np.ones(Q)) / tau
    A = np.diag(np.exp(-1j * (v[:, :2] @ k))) @ omega
    return np.real(np.ones(Q) @ np.linalg.matrix_power(A, t) @ w)


def correlations(series, lags, nb=20):
    """Normalised autocorrelation of a complex series at the given lags, with
    batch-mean standard errors."""
    T = series.shape[0] - max(lags)
    T -= T % nb
    out, err = [], []
    for L in lags:
        prod = np.real(series[L:L + T] * np.conj(series[:T])) / np.mean(np.abs(series[:T]) ** 2)
        b = prod.reshape(nb, -1).mean(1)
        out.append(b.mean())
        err.append(b.std(ddof=1) / math.sqrt(nb))
    return np.array(out), np.array(err)


@pytest.mark.parametrize("tau", [0.8, 1.0, 1.4])
def test_density_time_correlation_follows_transfer_matrix(orc, tau):
    lat, (Lx, Ly), rho = orc.D2Q9, (12, 10), 50.0
    D, Q, v, w = orc.lattice(lat)
    N = Lx * Ly
    f = orc.init_equilibrium(lat, np.full(N, rho))
    f = orc.run(lat, (Lx, Ly), f, 300, tau, orc.NOISE_GLOBAL, rho_eq=rho, seed=8)
    T = 12000
    modes = [(1, 0), (0, 1), (2, 1), (3, 2)]
    series = np.empty((T, len(modes)), dtype=complex)
    for t in range(T):
        f = orc.run(lat, (Lx, Ly), f, 1, tau, orc.NOISE_GLOBAL, rho_eq=rho, seed=8, t0=300 + t)
        rk = np.fft.fft2(f.sum(0).reshape(Ly, Lx))
        for m, (kx, ky) in enumerate(modes):
            series[t, m] = rk[ky % Ly, kx % Lx]
    lags = [1, 2, 4, 8]
    for m, (kx, ky) in enumerate(modes):
        k = np.array([2 * np.pi * kx / Lx, 2 * np.pi * ky / Ly])
        want = np.array([transfer_correlation(v, w, k, tau, L) for L in lags])
        got, err = correlations(series[:, m], lags)
        assert np.all(np.abs(got - want) < 5 * err + 0.01), (tau, (kx, ky), got, want, err)


def test_tau_one_is_the_power_of_lambda():
    """At tau = 1 the transfer-matrix correlation is lambda(k)^t exactly."""
    import oracle

    oracle.build()
    D, Q, v, w = oracle.lattice(oracle.D2Q5, 1.0 / 3.0)
    for kx, ky in [(1, 0), (5, 3), (20, 20)]:
        k = np.array([2 * np.pi * kx / 81, 2 * np.pi * ky / 81])
        lam = float(np.sum(w * np.cos(v[:, :2] @ k)))
        for t in (1, 3, 10, 40):
            assert abs(transfer_correlation(v, w, k, 1.0, t) - lam ** t) < 1e-12
