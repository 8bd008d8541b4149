"""The non-equilibrium workload of the paper (Sec. IV, "Non-equilibrium
dynamics"): a block of density rho_1 on [L/4, 3L/4) in material of density
rho_2, periodic in x.  Without noise the lattice-Boltzmann density must
follow the periodic erf series of the diffusion equation with
D = theta (tau^j - 1/2), the hydrodynamic result of Sec. III, up to the
lattice's discretisation error, which falls with time.  With several
relaxation times only the flux time tau^j may set D (the moment-space
collision matrix diag(tau^rho, tau^j, tau^j, tau^n, tau^s)): a D taken from
another moment's time misses by far more than the tolerance."""
import math

import numpy as np
import pytest
from scipy.special import erf

L, R1, R2 = 100, 120.0, 20.0


def front_theory(D, t):
    """rho^th(x, t) of the paper's front (sum over periodic images); the
    block's edges sit half-way between sites 24|25 and 74|75."""
    x = np.arange(L, dtype=float)
    rho = np.full(L, R2)
    s = 2.0 * math.sqrt(D * t)
    for i in range(-3, 4):
        rho += (R1 - R2) / 2 * (erf((x - (i * L + 24.5)) / s) - erf((x - (i * L + 74.5)) / s))
    return rho


def front_start():
    x = np.arange(L)
    return np.where((x >= 25) & (x < 75), R1, R2).astype(float)


@pytest.mark.parametrize("theta,tau", [(1.0 / 3.0, 1.0), (0.2, 0.8), (0.45, 1.3)])
def test_srt_front_follows_erf_series(orc, theta, tau):
    f0 = orc.init_equilibrium(orc.D2Q5, front_start(), theta=theta)
    D = theta * (tau - 0.5)
    for t, tol in [(100, 2e-3), (400, 5e-4), (1600, 1.5e-4)]:
        rho = orc.run(orc.D2Q5, (L, 1), f0, t, tau, orc.NOISE_OFF, theta=theta).sum(0)
        err = np.max(np.abs(rho - front_theory(D, t))) / (R1 - R2)
        assert err < tol, (theta, tau, t, err)
        assert abs(rho.sum() - front_start().sum()) < 1e-9 * rho.sum()


@pytest.mark.parametrize("theta,taus", [(1.0 / 3.0, [1.0, 0.8, 0.8, 1.4, 0.6]), (0.25, [1.0, 1.2, 1.2, 0.7, 1.6])])
def test_mrt_front_is_set_by_the_flux_time(orc, theta, taus):
    f0 = orc.init_equilibrium(orc.D2Q5, front_start(), theta=theta)
    rho = orc.run(orc.D2Q5, (L, 1), f0, 400, taus, orc.NOISE_OFF, theta=theta).sum(0)
    good = np.max(np.abs(rho - front_theory(theta * (taus[1] - 0.5), 400))) / (R1 - R2)
    wrong = np.max(np.abs(rho - front_theory(theta * (taus[3] - 0.5), 400))) / (R1 - R2)
    assert good < 5e-4 and wrong > 0.05
