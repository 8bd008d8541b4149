"""Statistical pins of the oracle: long noisy runs on small lattices must
reproduce the equilibrium statistics the paper derives and prints.

- d_ij (eqs. dij, dijexp) on the paper's 3x3 D2Q5 lattice against Table I
  and against the finite-size closed form delta_ij - sqrt(w_i w_j)/N.
- Var(rho_x) = rho (1 - 1/N) and the flat structure factor
  S_ij(k) = N f^eq_i delta_ij for k != 0 (eq. fkfk and the S^th passage).
- Global noise keeps the second moments exact at low density; local noise
  raises them there (Sec. IV, "Limit of low density").

Error bars come from batch means; every bound is 5 sigma.
"""
import math

import numpy as np
import pytest

from tests import golden_io


def _trajectory(orc, lat, dims, rho_bar, tau, T, mode, seed, burn=200, dist=0):
    Q = orc.q_of(lat)
    N = int(np.prod(dims))
    f = orc.init_equilibrium(lat, np.full(N, rho_bar))
    f = orc.run(lat, dims, f, burn, tau, mode, dist=dist, seed=seed, rho_eq=rho_bar)
    out = np.empty((T, Q, N))
    for t in range(T):
        f = orc.run(lat, dims, f, 1, tau, mode, dist=dist, seed=seed, rho_eq=rho_bar, t0=burn + t)
        out[t] = f
    return out


def _batch_mean(x, nb=40):
    """Mean and standard error of a time series by batch means (axis 0)."""
    T = x.shape[0] - x.shape[0] % nb
    b = x[:T].reshape(nb, T // nb, *x.shape[1:]).mean(1)
    return b.mean(0), b.std(0, ddof=1) / math.sqrt(nb)


def _dij_series(f, rho_bar, w):
    """Per-step lattice average of (f_i - rho w_i)(f_j - rho w_j)/(rho sqrt(w_i w_j)).
    Its expectation equals that of eq. dijexp, since <f_i> = rho w_i: the
    linear terms of f_i f_j - (rho w_i)(rho w_j) average to zero."""
    d = f - rho_bar * w[None, :, None]
    prod = np.einsum("tix,tjx->tij", d, d) / d.shape[2]
    return prod / (rho_bar * np.sqrt(np.outer(w, w)))[None]


@pytest.mark.parametrize("mode", ["NOISE_LOCAL", "NOISE_GLOBAL"])
def test_table1_dij_3x3(orc, mode):
    lat = orc.D2Q5
    D, Q, v, w = orc.lattice(lat)
    rho = 120.0
    f = _trajectory(orc, lat, (3, 3, 1), rho, 1.0, 30000, getattr(orc, mode), seed=2024)
    d, err = _batch_mean(_dij_series(f, rho, w))
    closed = np.eye(Q) - np.sqrt(np.outer(w, w)) / 9.0
    assert np.all(np.abs(d - closed) < 5 * err + 1e-4)
    printed = golden_io.table1()[3]
    # the paper's own estimate carries ~1e-3 statistical error
    assert np.all(np.abs(d - printed) < 5 * err + 1.5e-3)
    # and the finite-size correction is resolved: d_00 is clearly below 1
    assert 1.0 - d[0, 0] > 10 * err[0, 0]


def test_table1_closed_form_matches_printed_values():
    """The finite-size closed form reproduces every printed Table I entry
    within the paper's statistical error (about 1e-3 at 3x3)."""
    theta = 1.0 / 3.0
    w = np.array([1 - 2 * theta] + [theta / 2] * 4)
    for L, tab in golden_io.table1().items():
        closed = np.eye(5) - np.sqrt(np.outer(w, w)) / (L * L)
        tol = 1.5e-3 if L == 3 else 2.5e-4
        assert np.max(np.abs(closed - tab)) < tol


def test_density_variance_and_structure_factor(orc):
    lat = orc.D2Q9
    D, Q, v, w = orc.lattice(lat)
    Lx, Ly = 8, 6
    N = Lx * Ly
    rho = 50.0
    f = _trajectory(orc, lat, (Lx, Ly, 1), rho, 0.8, 12000, orc.NOISE_LOCAL, seed=77)
    r = f.sum(1)  # (T, N)
    var, err = _batch_mean(((r - rho) ** 2).mean(1) / rho)
    assert abs(var - (1 - 1 / N)) < 5 * err
    # structure factor S_ij(k) = <f_i(k) f_j(-k)>, k != 0: N rho w_i delta_ij
    T = f.shape[0]
    nb = 40
    Tb = T // nb
    fk = np.fft.fft2(f[: nb * Tb].reshape(nb * Tb, Q, Ly, Lx), axes=(2, 3)).reshape(nb, Tb, Q, Ly * Lx)
    A = np.ascontiguousarray(fk.transpose(3, 0, 2, 1))  # (k, batch, i, t)
    Sb = (A @ np.conj(A.transpose(0, 1, 3, 2))).real / (Tb * N * rho)  # (k, batch, i, j)
    Sm, Se = Sb.mean(1), Sb.std(1, ddof=1) / math.sqrt(nb)
    expect = np.diag(w)[None, :, :]
    dev = np.abs(Sm - expect)[1:]  # drop k = 0 (flat index 0)
    assert np.all(dev < 5 * Se[1:] + 1e-4)
    # k = 0: mass is fixed, so the density mode does not fluctuate
    assert np.max(np.abs(r.sum(1) - N * rho)) < 1e-9 * N * rho
    # S_rho(k)/(N rho) = 1 for all k != 0 (flat)
    Sr = (np.abs(np.fft.fft2(r.reshape(-1, Ly, Lx))) ** 2).reshape(T, -1) / (N * rho)
    m, e = _batch_mean(Sr)
    assert np.all(np.abs(m[1:] - 1.0) < 5 * e[1:])


def test_low_density_global_exact_local_inflated(orc):
    """rho = 0.5: global noise leaves the dynamics linear with additive noise,
    so the second moments stay exact; the zero-density clamp of local noise
    makes them larger (Sec. IV, limit of low density)."""
    lat = orc.D2Q5
    D, Q, v, w = orc.lattice(lat)
    rho = 0.5
    fg = _trajectory(orc, lat, (3, 3, 1), rho, 1.0, 20000, orc.NOISE_GLOBAL, seed=5)
    dg, eg = _batch_mean(_dij_series(fg, rho, w))
    closed = np.eye(Q) - np.sqrt(np.outer(w, w)) / 9.0
    assert np.all(np.abs(dg - closed) < 5 * eg + 1e-4)
    fl = _trajectory(orc, lat, (3, 3, 1), rho, 1.0, 20000, orc.NOISE_LOCAL, seed=5)
    dl, el = _batch_mean(_dij_series(fl, rho, w))
    assert dl[0, 0] - closed[0, 0] > 5 * el[0, 0]
    # some sites do go negative at this density
    assert (fl.sum(1) < 0).mean() > 0.01
