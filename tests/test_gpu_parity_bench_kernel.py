"""Parity over 1000 steps of the kernel the benchmark times, and of the D1Q3
FP64 workload in full, against the FP64 oracle (element by element, same
seeded inputs, same Philox noise stream).

The benchmark's lattices (D2Q9 2048^2, D3Q19 256^3) take one launch of the
one-launch-per-step kernel per step.  A lattice whose two buffers fit the
many-steps-per-launch paths (one block's or one cluster's shared memory)
takes those paths instead, so the cases here are sized above that limit and
each test first checks that lbfd_step picks the same kernel for its lattice
as for the benchmark's.

Tolerances (spec bar, paper Sec. II eq. LB iterated 1000 times):
max |f_gpu - f_oracle| <= 1e-12 rho_mean (FP64), <= 2e-5 rho_mean (FP32).
"""
import os
import sys

import numpy as np
import pytest

import paper_1606_07801_gb300 as lb
from paper_1606_07801_gb300 import synth

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)
import bench  # noqa: E402  (the benchmark's workload table)

from .slope_bound import oracle_run_with_slope  # noqa: E402

pytestmark = pytest.mark.gpu

TOL = {lb.F64: 1e-12, lb.F32: 2e-5}


@pytest.fixture(scope="module")
def orc_mt(orc):
    """The oracle on every host core (its result does not depend on the
    thread count: each site's update is computed on its own)."""
    orc.set_threads(os.cpu_count() or 1)
    yield orc
    orc.set_threads(1)


def _bench_kernel(workload: str, n: int) -> str:
    wl = bench.WORKLOADS[workload]
    with lb.Simulation(wl["lattice"], wl["dims"], wl["tau"], wl["rho"], 1, precision=wl["precision"],
                       init=lb.INIT_NONE) as s:
        return s.kernel(n)


@pytest.mark.parametrize("workload,lat,dims,tau,rho", [
    ("d2q9", lb.D2Q9, (256, 200), 0.8, 100.0),
    ("d3q19", lb.D3Q19, (48, 40, 36), 1.0, 50.0),
])
def test_bench_kernel_1000_steps(orc_mt, workload, lat, dims, tau, rho):
    Q, N = lb.Q_OF[lat], int(np.prod(dims))
    f0 = synth.random_populations(Q, N, rho, 0.3, seed=101 + lat)
    want = orc_mt.run(lat, dims, f0, 1000, tau, orc_mt.NOISE_LOCAL, orc_mt.GAUSSIAN, rho_eq=rho, seed=1)
    assert np.max(np.abs(want - f0)) > 0.1 * rho / Q  # the run moved far from its start
    for precision in (lb.F32, lb.F64):
        expect = _bench_kernel(workload, 1000) if precision == bench.WORKLOADS[workload]["precision"] else None
        with lb.Simulation(lat, dims, tau, rho, 1, precision=precision, init=lb.INIT_NONE) as s:
            if expect is not None:
                assert s.kernel(1000) == expect, (s.kernel(1000), expect)
            s.set_f(f0)
            s.step(1000)
            got = s.get_f()
        err = float(np.max(np.abs(got - want)))
        print(f"{workload} {dims} precision {precision}: max |f_gpu - f_oracle| = {err:.3e} "
              f"({err / rho:.2e} rho_mean)")
        assert err <= TOL[precision] * rho, err


def test_d1q3_fp64_workload_in_full(orc_mt):
    """The D1Q3 workload itself: FP64, L = 256, tau = 1, rho_mean = 10,
    f_i = w_i (10 + sin(2 pi x / 256)) at t = 0, local Gaussian noise, seed 1,
    10^4 steps, through the same lbfd_step call the benchmark makes.  At
    rho_mean = 10 the equilibrium density has variance rho_mean, so over
    2.56e6 site updates some sites pass close to zero density; the FP64 bar is
    scaled by the slope of the clamped noise amplitude there
    (tests/slope_bound.py)."""
    wl = bench.WORKLOADS["d1q3"]
    lat, dims, tau, rho = wl["lattice"], wl["dims"], wl["tau"], wl["rho"]
    with lb.Simulation(lat, dims, tau, rho, 1, precision=wl["precision"], init=lb.INIT_SINE, sine_amp=1.0,
                       sine_k=(1, 0, 0)) as s:
        assert s.kernel(10_000) == _bench_kernel("d1q3", 10_000)
        s.step(10_000)
        got = s.get_f()
    f0 = orc_mt.init_equilibrium(lat, synth.density_sine(dims, (1,), 1.0, rho))
    want, amp = oracle_run_with_slope(orc_mt, lat, dims, f0, 10_000, tau, rho, 1)
    err = float(np.max(np.abs(got - want)))
    print(f"D1Q3 FP64 L=256, 10^4 steps: max |f_gpu - f_oracle| = {err:.3e} against the run's bound "
          f"{1e-12 * rho * amp:.3e} (slope factor {amp:.3g})")
    assert err <= 1e-12 * rho * amp, err


@pytest.mark.parametrize("t,expect", [(1000, 0.9044766338315362), (10_000, 0.3664152311782258)])
def test_d1q3_fp64_workload_noise_off_closed_form(t, expect):
    """The D1Q3 workload with the noise off, on the benchmark's path: at tau = 1
    the sine mode of rho decays by lambda^t, lambda = 2/3 + cos(2 pi/256)/3
    (the density-mode row of the lattice transfer matrix; paper Sec. IV, the
    equilibrium-dynamics passage, read without its misprints)."""
    wl = bench.WORKLOADS["d1q3"]
    lat, dims, tau, rho = wl["lattice"], wl["dims"], wl["tau"], wl["rho"]
    L = dims[0]
    with lb.Simulation(lat, dims, tau, rho, 1, precision=wl["precision"], init=lb.INIT_SINE, sine_amp=1.0,
                       sine_k=(1, 0, 0), noise_mode=lb.NOISE_OFF) as s:
        assert s.kernel(t) == _bench_kernel("d1q3", t)
        s.step(t)
        r = s.moments()
    x = np.arange(L)
    amp = 2.0 / L * ((r - rho) * np.sin(2 * np.pi * x / L)).sum()
    assert abs(amp - expect) < 1e-13 + 1e-15 * t
    assert np.max(np.abs(r - (rho + expect * np.sin(2 * np.pi * x / L)))) < 1e-15 * rho * t
