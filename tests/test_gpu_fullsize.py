"""Parity at the benchmark's full sizes, in the launch configuration the
benchmark times: one step from a random state, checked site by site against
the oracle's collision of the source sites (f_i(x, t+1) is the collision
output of site x - v_i), plus properties that hold at any size."""
import numpy as np
import pytest

import paper_1606_07801_gb300 as lb
from paper_1606_07801_gb300 import synth

pytestmark = pytest.mark.gpu


def _coords(s, dims):
    Lx, Ly, Lz = dims
    return s % Lx, (s // Lx) % Ly, s // (Lx * Ly)


def _site(x, y, z, dims):
    Lx, Ly, Lz = dims
    return (x % Lx) + Lx * ((y % Ly) + Ly * (z % Lz))


def _expected_at(orc, lat, dims, f0, sites, tau, mode, rho_eq, seed, t):
    D, Q, v, w = orc.lattice(lat)
    out = np.empty((len(sites), Q))
    for k, s in enumerate(sites):
        x, y, z = _coords(int(s), dims)
        for i in range(Q):
            src = _site(x - v[i, 0], y - v[i, 1], z - v[i, 2], dims)
            zz = orc.site_noise(seed, 0, src, t, Q - 1, lb.GAUSSIAN)
            out[k, i] = orc.collide(lat, f0[:, src].astype(np.float64), zz, tau, mode, rho_eq)[i]
    return out


def _sample_sites(dims, n, seed):
    N = int(np.prod(dims))
    g = np.random.default_rng(seed)
    Lx, Ly, Lz = dims
    corners = [_site(x, y, z, dims) for x in (0, Lx - 1) for y in (0, Ly - 1) for z in (0, Lz - 1)]
    return np.unique(np.concatenate([g.integers(0, N, n), corners]))


@pytest.mark.parametrize("lat,dims,tau,rho", [
    (lb.D2Q9, (2048, 2048, 1), 0.8, 100.0),
    (lb.D3Q19, (256, 256, 256), 1.0, 50.0),
])
def test_full_size_one_step_sampled(orc, lat, dims, tau, rho):
    Q, N = lb.Q_OF[lat], int(np.prod(dims))
    f0 = synth.random_populations(Q, N, rho, 0.3, seed=123, dtype=np.float32)
    t = 4321
    with lb.Simulation(lat, dims[: lb.D_OF[lat]], tau, rho, 1, precision=lb.F32, init=lb.INIT_NONE) as s:
        lb.abi.lbfd_set_f_raw(s.h, f0.ctypes.data)
        s.t = t
        m0 = s.mass()
        s.step(1)
        f1 = np.empty_like(f0)
        lb.abi.lbfd_get_f_raw(s.h, f1.ctypes.data)
        m1 = s.mass()
    sites = _sample_sites(dims, 1500 if lat == lb.D2Q9 else 600, seed=7)
    exp = _expected_at(orc, lat, dims, f0, sites, tau, lb.NOISE_LOCAL, rho, 1, t)
    got = f1[:, sites].T.astype(np.float64)
    assert np.max(np.abs(got - exp)) <= 2e-5 * rho
    assert abs(m1 - m0) <= 1e-6 * abs(m0)


def test_full_size_many_steps_properties():
    """D2Q9 2048^2 FP32, 200 steps from a uniform start: mass conserved,
    mean populations stay at w_i rho, and the density variance grows toward
    its equilibrium value rho (1 - 1/N)."""
    dims, rho = (2048, 2048), 100.0
    with lb.Simulation(lb.D2Q9, dims, 0.8, rho, 1, precision=lb.F32) as s:
        m0 = s.mass()
        s.step(200)
        m1 = s.mass()
        s.sample()
        ob = s.observables()
        v, w, m = lb.abi.lbfd_lattice_tables(lb.D2Q9)
    N = dims[0] * dims[1]
    assert abs(m1 - m0) <= 1e-5 * m0
    assert np.max(np.abs(ob["sum_f"] / N - w * rho)) < 1e-3 * rho
    var = ob["sum_rho2"] / N - (ob["sum_rho"] / N) ** 2
    assert 0.5 * rho < var < 1.05 * rho
