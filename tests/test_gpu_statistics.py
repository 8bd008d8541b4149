"""Equilibrium statistics the paper derives, measured on the GPU with the
library's own FP64 accumulators (lbfd_sample / lbfd_observables):

- the density variance Var(rho_x) = rho (1 - 1/N) and the flat structure
  factor S(k) = N rho for k != 0 (the fluctuation-dissipation result the
  paper's S^th passage and eq. fkfk state), for D2Q9 and D3Q19 in FP32;
- the per-population covariance <f_i f_j> - <f_i><f_j> = rho (w_i delta_ij -
  w_i w_j / N) (eq. ffluct with the mass fixed);
- at low density (rho = 0.5, Sec. IV) global noise keeps the variance
  exact while the zero-density clamp of local noise raises it.

Samples are taken every few steps after a burn-in; error bars come from
batch means over independent blocks of samples, and every bound is 5
sigma."""
import math

import numpy as np
import pytest

import paper_1606_07801_gb300 as lb
from paper_1606_07801_gb300 import abi

pytestmark = pytest.mark.gpu


def _blocks(sim, nblocks, per_block, every):
    """Per block: mean over samples of (sum_x rho^2, sum_x f_i f_j, sum_x f_i,
    |rho(k)|^2 for the configured modes)."""
    out = []
    for _ in range(nblocks):
        sim.reset_obs()
        for _ in range(per_block):
            sim.step(every)
            sim.sample()
        ob = sim.observables()
        n = ob["n_samples"]
        out.append((ob["sum_rho2"] / n, ob["sum_ff"] / n, ob["sum_f"] / n, ob["sum_sk"] / n))
    return out


def _mean_err(x):
    x = np.array(x)
    return x.mean(0), x.std(0, ddof=1) / math.sqrt(len(x))


@pytest.mark.parametrize("lat,dims,tau,rho", [(lb.D2Q9, (24, 16), 0.8, 100.0), (lb.D3Q19, (8, 6, 5), 1.0, 50.0)])
def test_variance_structure_factor_and_covariance(lat, dims, tau, rho):
    N = int(np.prod(dims))
    modes = [(1, 0, 0), (0, 1, 0), (3, 2, 0), (dims[0] // 2, 0, 0)] + ([(1, 1, 1), (2, 0, 3)] if lat == lb.D3Q19 else [])
    _, w, _ = abi.lbfd_lattice_tables(lat)
    with lb.Simulation(lat, dims, tau, rho, 21, modes=modes) as s:
        s.step(500)
        blocks = _blocks(s, 20, 150, 4)
    r2, e_r2 = _mean_err([b[0] / N for b in blocks])
    # mass is fixed, so <rho_x> = rho exactly and Var = <rho^2> - rho^2
    assert abs((r2 - rho * rho) / rho - (1.0 - 1.0 / N)) < 5 * e_r2 / rho + 2e-3
    sk, e_sk = _mean_err([b[3] / (N * rho) for b in blocks])
    assert np.all(np.abs(sk - 1.0) < 5 * e_sk + 2e-3), (sk, e_sk)
    cov = [(b[1] - np.outer(b[2], b[2]) / N) / N for b in blocks]
    c, e_c = _mean_err(cov)
    want = rho * (np.diag(w) - np.outer(w, w) / N)
    assert np.all(np.abs(c - want) < 5 * e_c + 2e-3 * rho)


def test_low_density_global_exact_local_inflated():
    """rho = 0.5 on a 16 x 16 D2Q9 lattice: with global noise the density
    variance is rho (1 - 1/N) at any density; with local noise the clamp at
    rho = 0 raises it."""
    dims, rho = (16, 16), 0.5
    N = 256
    res = {}
    for mode in (lb.NOISE_GLOBAL, lb.NOISE_LOCAL):
        with lb.Simulation(lb.D2Q9, dims, 1.0, rho, 33, noise_mode=mode, precision=lb.F64) as s:
            s.step(300)
            blocks = _blocks(s, 20, 200, 3)
        res[mode] = _mean_err([(b[0] / N - rho * rho) / rho for b in blocks])
    g, eg = res[lb.NOISE_GLOBAL]
    loc, el = res[lb.NOISE_LOCAL]
    assert abs(g - (1.0 - 1.0 / N)) < 5 * eg + 2e-3
    assert loc - g > 5 * math.hypot(el, eg)
