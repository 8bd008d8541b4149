"""16-bit storage (FP16 or BF16 deviations f_i - w_i rho_mean, FP32
arithmetic) against the FP64 oracle.

The stored deviation is rounded to nearest even each step, so paths drift
from the oracle's like a random walk of that rounding: about 2^-11 |d| per
value and step for FP16, 2^-8 |d| for BF16, |d| being a few units at the
densities below.  After 100 steps the bounds are 1e-3 rho_mean (FP16) and
1e-2 rho_mean (BF16); the measured errors are printed.  Equilibrium
statistics must still hold after longer runs."""
import numpy as np
import pytest

import paper_1606_07801_gb300 as lb
from paper_1606_07801_gb300 import abi, synth

pytestmark = pytest.mark.gpu

FORMATS = [(lb.F32_F16, 1e-3, 2.0**-11), (lb.F32_BF16, 1e-2, 2.0**-8)]


@pytest.mark.parametrize("precision,tol,ulp", FORMATS)
def test_storage_round_trip(precision, tol, ulp):
    Q, dims, rho = 19, (12, 10, 8), 50.0
    N = int(np.prod(dims))
    _, w, _ = abi.lbfd_lattice_tables(lb.D3Q19)
    f0 = synth.random_populations(Q, N, rho, 0.3, seed=3)
    with lb.Simulation(lb.D3Q19, dims, 1.0, rho, 1, precision=precision, init=lb.INIT_NONE) as s:
        s.set_f(f0)
        back = s.get_f()
    dev = np.abs(f0 - rho * w[:, None])
    assert np.all(np.abs(back - f0) <= ulp * dev + 1e-12)


@pytest.mark.parametrize("precision,tol,ulp", FORMATS)
@pytest.mark.parametrize("lat,dims,tau,rho", [(lb.D2Q9, (64, 48), 0.8, 100.0), (lb.D3Q19, (16, 12, 10), 1.0, 50.0)])
def test_parity_against_fp64_oracle(orc, lat, dims, tau, rho, precision, tol, ulp):
    Q, N = lb.Q_OF[lat], int(np.prod(dims))
    f0 = synth.random_populations(Q, N, rho, 0.2, seed=17)
    # start from the exactly representable state the GPU holds
    with lb.Simulation(lat, dims, tau, rho, 2, precision=precision, init=lb.INIT_NONE) as s:
        s.set_f(f0)
        start = s.get_f()
        s.step(100)
        g = s.get_f()
        mass = s.mass()
    o = orc.run(lat, dims, start, 100, tau, orc.NOISE_LOCAL, orc.GAUSSIAN, rho_eq=rho, seed=2)
    err = np.max(np.abs(g - o))
    print(f"precision {precision}, lattice {lat}: max |f - f_oracle| after 100 steps = {err:.3e} = {err / rho:.2e} rho")
    assert err <= tol * rho
    assert abs(mass - o.sum()) <= 1e-4 * o.sum()


@pytest.mark.parametrize("precision", [lb.F32_F16, lb.F32_BF16])
def test_equilibrium_statistics_hold(precision):
    """D3Q19 40^3, rho 50, 300 steps from a uniform start: the density variance
    approaches rho (1 - 1/N) and the mean populations stay at w_i rho."""
    dims, rho = (40, 40, 40), 50.0
    N = 40 ** 3
    with lb.Simulation(lb.D3Q19, dims, 1.0, rho, 5, precision=precision) as s:
        m0 = s.mass()
        s.step(300)
        m1 = s.mass()
        s.sample()
        ob = s.observables()
        _, w, _ = abi.lbfd_lattice_tables(lb.D3Q19)
    var = ob["sum_rho2"] / N - (ob["sum_rho"] / N) ** 2
    assert abs(var / rho - 1.0) < 0.03
    assert np.max(np.abs(ob["sum_f"] / N - w * rho)) < 2e-3 * rho
    assert abs(m1 - m0) < 1e-4 * m0
