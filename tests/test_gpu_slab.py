"""Slab handles on the GPU: one lattice cut into slabs along its slowest axis,
all held by this process and exchanging their halo planes by device copies
(paper_1606_07801_gb300.slab.step_local), must evolve bit for bit as the
unsplit lattice (paper Sec. II, eq. LB reads nearest neighbours only; the
noise is keyed by the global site index).  The same slab handles serve one
GPU per process with NCCL messages in place of the copies."""
import numpy as np
import pytest

import paper_1606_07801_gb300 as lb
from paper_1606_07801_gb300 import abi, slab, synth

pytestmark = pytest.mark.gpu


def _stored_planes(f, gdims, plan):
    """Global f [Q, N] cut to the slab's stored planes (owned plus one halo
    plane on each side, periodic), [Q, stored sites]."""
    Q = f.shape[0]
    L = gdims[plan.axis]
    planes = [(plan.first - 1 + c) % L for c in range(plan.count + 2)]
    f3 = f.reshape(Q, gdims[2], gdims[1], gdims[0])
    return (f3[:, :, planes, :] if plan.axis == 1 else f3[:, planes, :, :]).reshape(Q, -1)


@pytest.mark.parametrize("lat,gdims,precision,nranks,mode", [
    (lb.D2Q9, (264, 40, 1), lb.F32, 2, lb.NOISE_LOCAL),
    (lb.D2Q9, (256, 9, 1), lb.F64, 3, lb.NOISE_LOCAL),
    (lb.D2Q9, (520, 7, 1), lb.F32_F16, 2, lb.NOISE_GLOBAL),
    (lb.D3Q19, (24, 10, 12), lb.F32, 2, lb.NOISE_LOCAL),
    (lb.D3Q19, (32, 6, 5), lb.F32_BF16, 3, lb.NOISE_LOCAL),
    (lb.D3Q19, (16, 4, 8), lb.F64, 4, lb.NOISE_OFF),
])
def test_slabs_bit_identical_to_whole(lat, gdims, precision, nranks, mode):
    Q, N = lb.Q_OF[lat], int(np.prod(gdims))
    dims = gdims[:2] if lat == lb.D2Q9 else gdims
    rho, tau, seed, steps = 25.0, 0.9, 11, 9
    f0 = synth.random_populations(Q, N, rho, 0.3, seed=N)
    with lb.Simulation(lat, dims, tau, rho, seed, precision=precision, noise_mode=mode, init=lb.INIT_NONE,
                       lattice_id=4) as whole:
        whole.set_f(f0)
        whole.step(steps)
        want = whole.get_f()
    slabs = [slab.SlabSimulation(lat, dims, tau, rho, seed, nranks=nranks, rank=r, local=True, precision=precision,
                                 noise_mode=mode, init=lb.INIT_NONE, lattice_id=4) for r in range(nranks)]
    try:
        for sl in slabs:
            assert sl.sim.kernel(1) == "k_step_staged"
            sl.sim.set_f(_stored_planes(f0, gdims, sl.plan))
        slab.step_local(slabs)
        slab.step_local(slabs, steps)
        got = np.concatenate([sl.get_f() for sl in slabs], axis=1)
        rho_slabs = np.concatenate([sl.sim.moments() for sl in slabs])
    finally:
        for sl in slabs:
            sl.close()
    assert np.array_equal(got, want)
    assert np.array_equal(rho_slabs, want.sum(0)) or np.max(np.abs(rho_slabs - want.sum(0))) < 1e-12 * rho


def test_slabs_sine_start_match_whole():
    """The initial state of a slab takes its part of the global sine mode."""
    lat, dims, rho = lb.D3Q19, (16, 8, 10), 40.0
    kw = dict(init=lb.INIT_SINE, sine_amp=2.0, sine_k=(1, 2, 3))
    with lb.Simulation(lat, dims, 1.1, rho, 5, **kw) as whole:
        whole.step(4)
        want = whole.get_f()
    slabs = [slab.SlabSimulation(lat, dims, 1.1, rho, 5, nranks=3, rank=r, local=True, **kw) for r in range(3)]
    try:
        slab.step_local(slabs)
        slab.step_local(slabs, 4)
        got = np.concatenate([sl.get_f() for sl in slabs], axis=1)
    finally:
        for sl in slabs:
            sl.close()
    assert np.array_equal(got, want)


def test_slab_handle_limits():
    with slab.SlabSimulation(lb.D2Q9, (64, 16), 0.8, 10.0, 1, nranks=2, rank=1, local=True) as sl:
        with pytest.raises(abi.LbfdError) as e:
            sl.sim.step(2)
        assert e.value.code == abi.EINVAL
        with pytest.raises(abi.LbfdError) as e:  # its sampling goes through lbfd_sample_totals
            sl.sim.sample()
        assert e.value.code == abi.ENOTSUP
    with pytest.raises(abi.LbfdError) as e:  # rows not on 16-byte boundaries: no staged kernel, no slab
        lb.Simulation(lb.D2Q9, (66, 8), 0.8, 10.0, 1, slab_global=16, slab_first=8)
    assert e.value.code == abi.ENOTSUP
    with pytest.raises(abi.LbfdError):
        lb.Simulation(lb.D2Q9, (64, 8), 0.8, 10.0, 1, slab_global=12, slab_first=8)


@pytest.mark.parametrize("lat,gdims,prec,nranks,modes", [
    (lb.D2Q9, (264, 40, 1), lb.F32, 2, [(1, 0, 0), (2, 3, 0)]),
    (lb.D2Q9, (520, 7, 1), lb.F32_BF16, 3, [(0, 1, 0)]),
    (lb.D3Q19, (24, 10, 12), lb.F32, 3, [(1, 0, 0), (0, 1, 2), (1, 1, 1)]),
    (lb.D3Q19, (32, 6, 8), lb.F32_F16, 2, [(0, 0, 1)]),
])
def test_slab_mass_and_observables_sum_to_the_whole(lat, gdims, prec, nranks, modes):
    """The slabs' FP64 masses (owned planes of the stored state) add up to the
    lattice's mass, and their observable totals (lbfd_sample_totals, modes at
    global coordinates), summed and combined by lbfd_obs_restore, give the
    whole lattice's sampled sums (paper Sec. IV) to FP32-tile accuracy; the
    slab path runs the same FP32 pass over other tiles, so the sums agree to
    the rounding of 256-term FP32 tiles, not bit for bit."""
    Q, N = lb.Q_OF[lat], int(np.prod(gdims))
    dims = gdims[:2] if lat == lb.D2Q9 else gdims
    rho, tau, seed = 25.0, 0.9, 11
    f0 = synth.random_populations(Q, N, rho, 0.3, seed=N + 1)
    kw = dict(precision=prec, init=lb.INIT_NONE, lattice_id=4, modes=modes)
    with lb.Simulation(lat, dims, tau, rho, seed, **kw) as whole:
        whole.set_f(f0)
        masses, obs_whole = [], None
        for _ in range(3):
            whole.step(2)
            whole.sample()
            masses.append(whole.mass())
        obs_whole = whole.observables()
    slabs = [slab.SlabSimulation(lat, dims, tau, rho, seed, nranks=nranks, rank=r, local=True, **kw)
             for r in range(nranks)]
    try:
        for sl in slabs:
            sl.sim.set_f(_stored_planes(f0, gdims, sl.plan))
        slab.step_local(slabs)
        for k in range(3):
            slab.step_local(slabs, 2)
            slab.sample_local(slabs)
            assert slab.mass_local(slabs) == pytest.approx(masses[k], rel=1e-13)
        obs = [sl.observables() for sl in slabs]
    finally:
        for sl in slabs:
            sl.close()
    n = 3 * N
    var = obs_whole["sum_rho2"] / n - (obs_whole["sum_rho"] / n) ** 2
    cov = np.asarray(obs_whole["sum_ff"]) / n - np.outer(obs_whole["sum_f"], obs_whole["sum_f"]) / n ** 2
    for ob in obs:
        # the bounds of the FP32 sampling tests, doubled (both sides carry FP32 tile sums)
        assert ob["n_samples"] == 3
        assert abs(ob["sum_rho"] - obs_whole["sum_rho"]) <= 1e-6 * obs_whole["sum_rho"]
        assert abs(ob["sum_rho2"] - obs_whole["sum_rho2"]) / n <= 2e-4 * var
        assert np.max(np.abs(ob["sum_f"] - obs_whole["sum_f"])) <= 1e-6 * np.max(obs_whole["sum_f"])
        assert np.max(np.abs(np.asarray(ob["sum_ff"]) - obs_whole["sum_ff"])) / n <= 2e-4 * np.max(np.abs(cov))
        assert np.all(np.abs(ob["sum_sk"] - obs_whole["sum_sk"]) <= 2e-4 * obs_whole["sum_sk"] + 2e-3 * n * var)
    assert all(np.array_equal(obs[0]["sum_ff"], o["sum_ff"]) for o in obs)


def test_sample_totals_of_a_whole_handle_match_lbfd_sample():
    """For a whole lattice, lbfd_sample_totals + lbfd_obs_restore gives the
    observables of lbfd_sample's separate pass with the stage-2 sum taken on
    the host.  (For D2Q9 the separate pass runs the step's register sampler,
    and lbfd_sample_totals the site-range pass: the same FP32 values summed
    in another order, hence FP32-level tolerances.)"""
    lat, dims, modes = lb.D2Q9, (96, 70), [(1, 2, 0), (3, 0, 0)]
    rho, N = 40.0, 96 * 70
    with lb.Simulation(lat, dims, 0.8, rho, 2, modes=modes) as s:
        s.step(5)
        s.sample()
        want = s.observables()
        t = abi.lbfd_sample_totals(s.h, 9, len(modes))
        got = abi.lbfd_obs_restore(lat, len(modes), rho, N, t)
    flat = np.concatenate([[want["sum_rho"], want["sum_rho2"]], want["sum_f"], np.ravel(want["sum_ff"])])
    nk = len(modes)
    assert np.allclose(got[:-nk], flat, rtol=2e-6, atol=0.0)
    sk = np.asarray(want["sum_sk"])
    assert np.all(np.abs(got[-nk:] - sk) <= 1e-4 * sk + 1e-3 * N * rho)
