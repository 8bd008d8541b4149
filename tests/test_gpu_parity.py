"""Parity of the CUDA path with the FP64 oracle, element by element, on the
same seeded inputs and the same Philox noise stream.

Tolerances (max |f_gpu - f_oracle| after the stated number of steps):
  FP64 arithmetic: 1e-12 * rho_mean
  FP32 arithmetic: 2e-5  * rho_mean, where the local density stays away
                   from zero.  Local noise has amplitude sqrt(max(rho, 0)),
                   whose slope is unbounded at rho = 0: a site that comes
                   within FP32 rounding of zero density draws visibly
                   different noise in FP32 and FP64, and the difference
                   then diffuses.  Runs that reach rho ~ 0 are compared
                   pathwise in FP64 and statistically in FP32.
Lattices span several thread blocks and end in ragged tails in x and y.
"""
import numpy as np
import pytest

import paper_1606_07801_gb300 as lb
from paper_1606_07801_gb300 import abi, synth

from .slope_bound import oracle_run_with_slope

pytestmark = pytest.mark.gpu

TOL = {lb.F64: 1e-12, lb.F32: 2e-5}


def _gpu_run(lat, dims, f0, nsteps, tau, precision, mode=lb.NOISE_LOCAL, dist=lb.GAUSSIAN, rho_mean=1.0, seed=1,
             lattice_id=0, t0=0, **kw):
    with lb.Simulation(lat, dims, tau, rho_mean, seed, precision=precision, noise_mode=mode, noise_dist=dist,
                       init=lb.INIT_NONE, lattice_id=lattice_id, **kw) as s:
        s.set_f(f0)
        s.t = t0
        s.step(nsteps)
        return s.get_f()


def _oracle_run(orc, lat, dims, f0, nsteps, tau, mode=lb.NOISE_LOCAL, dist=lb.GAUSSIAN, rho_mean=1.0, seed=1,
                lattice_id=0, t0=0):
    return orc.run(lat, dims, f0, nsteps, tau, mode, dist, rho_eq=rho_mean, seed=seed, lattice_id=lattice_id, t0=t0)


CASES = [
    # lattice, dims, tau, rho_mean, precision
    (lb.D1Q3, (1000,), 1.0, 10.0, lb.F64),   # the D1Q3 workload's density; reaches rho ~ 0 at times
    (lb.D1Q3, (1000,), 1.0, 100.0, lb.F32),
    (lb.D2Q9, (67, 45), 0.8, 100.0, lb.F64),
    (lb.D2Q9, (67, 45), 0.8, 100.0, lb.F32),
    (lb.D3Q19, (19, 13, 11), 1.0, 50.0, lb.F64),
    (lb.D3Q19, (19, 13, 11), 1.0, 50.0, lb.F32),
]


@pytest.mark.parametrize("lat,dims,tau,rho,precision", CASES)
def test_parity_1000_steps_local_gaussian(orc, lat, dims, tau, rho, precision):
    Q, N = lb.Q_OF[lat], int(np.prod(dims))
    f0 = synth.random_populations(Q, N, rho, 0.3, seed=11 + lat)
    g = _gpu_run(lat, dims, f0, 1000, tau, precision, rho_mean=rho, seed=1)
    o = _oracle_run(orc, lat, dims, f0, 1000, tau, rho_mean=rho, seed=1)
    err = np.max(np.abs(g - o))
    assert err <= TOL[precision] * rho, err
    # the run did move far from its start
    assert np.max(np.abs(o - f0)) > 0.1 * rho / Q


@pytest.mark.parametrize("precision", [lb.F64, lb.F32])
@pytest.mark.parametrize("mode,dist", [(lb.NOISE_GLOBAL, lb.GAUSSIAN), (lb.NOISE_OFF, lb.GAUSSIAN),
                                       (lb.NOISE_LOCAL, lb.UNIFORM), (lb.NOISE_GLOBAL, lb.UNIFORM)])
@pytest.mark.parametrize("lat,dims,tau,rho", [(lb.D2Q9, (40, 33), 0.6, 20.0), (lb.D3Q19, (9, 10, 7), 1.4, 30.0),
                                              (lb.D1Q3, (300,), 0.75, 60.0)])
def test_parity_noise_variants(orc, lat, dims, tau, rho, mode, dist, precision):
    Q, N = lb.Q_OF[lat], int(np.prod(dims))
    f0 = synth.random_populations(Q, N, rho, 0.2, seed=5)
    g = _gpu_run(lat, dims, f0, 300, tau, precision, mode, dist, rho_mean=rho, seed=77, lattice_id=3)
    o = _oracle_run(orc, lat, dims, f0, 300, tau, mode, dist, rho_mean=rho, seed=77, lattice_id=3)
    assert np.max(np.abs(g - o)) <= TOL[precision] * rho


@pytest.mark.parametrize("lat,dims", [
    (lb.D1Q3, (1,)), (lb.D1Q3, (2,)), (lb.D2Q9, (1, 1)), (lb.D2Q9, (2, 1)), (lb.D2Q9, (1, 2)), (lb.D2Q9, (2, 2)),
    (lb.D2Q9, (3, 300)), (lb.D2Q9, (513, 2)), (lb.D3Q19, (1, 1, 1)), (lb.D3Q19, (2, 2, 2)), (lb.D3Q19, (1, 5, 2)),
    (lb.D3Q19, (33, 1, 3)),
])
def test_degenerate_sizes(orc, lat, dims):
    """Sides of 1 and 2 (the periodic wrap aliases a site's neighbours) and
    thin lattices."""
    Q, N = lb.Q_OF[lat], int(np.prod(dims))
    f0 = synth.random_populations(Q, N, 8.0, 0.5, seed=N)
    g = _gpu_run(lat, dims, f0, 50, 0.9, lb.F64, rho_mean=8.0, seed=3)
    o = _oracle_run(orc, lat, dims, f0, 50, 0.9, rho_mean=8.0, seed=3)
    assert np.max(np.abs(g - o)) <= 1e-12 * 8.0


@pytest.mark.parametrize("precision", [lb.F64, lb.F32])
def test_zero_density_stays_zero(precision):
    with lb.Simulation(lb.D2Q9, (17, 9), 0.8, 0.0, 5, precision=precision) as s:
        s.step(20)
        assert np.all(s.get_f() == 0.0)


def test_low_density_local_noise(orc):
    """rho = 0.5 with the zero-density clamp: FP64 follows the oracle pathwise;
    FP32 is judged statistically (mass, density variance, share of
    negative-density sites, mean populations), and the share of sites beyond
    the pathwise tolerance is reported."""
    lat, dims, rho = lb.D2Q9, (128, 96), 0.5
    Q, N = 9, 128 * 96
    f0 = synth.random_populations(Q, N, rho, 0.3, seed=99)
    # FP64 bar scaled by the slope of the clamped noise amplitude at the
    # run's closest approach to zero density (tests/slope_bound.py)
    o, amp = oracle_run_with_slope(orc, lat, dims, f0, 200, 0.8, rho, 21)
    assert (o.sum(0) < 0).mean() > 0.01  # the clamp is exercised
    g64 = _gpu_run(lat, dims, f0, 200, 0.8, lb.F64, rho_mean=rho, seed=21)
    err64 = np.abs(g64 - o)
    bound = 1e-12 * rho * amp
    print(f"FP64 at rho = 0.5: max error {err64.max():.2e} against the run's bound {bound:.2e} "
          f"(slope factor {amp:.3g}); {100 * np.any(err64 > 1e-12 * rho, axis=0).mean():.2f}% of sites beyond "
          f"1e-12 rho")
    assert err64.max() <= bound
    g32 = _gpu_run(lat, dims, f0, 200, 0.8, lb.F32, rho_mean=rho, seed=21)
    bad = np.any(np.abs(g32 - o) > 2e-5 * rho, axis=0).mean()
    print(f"FP32 at rho = 0.5: {100 * bad:.1f}% of sites beyond 2e-5 rho after 200 steps")
    assert abs(g32.sum() - o.sum()) < 1e-5 * N * rho
    rg, ro = g32.sum(0), o.sum(0)
    # the two fields are two samples of the same law; with shared noise they
    # are strongly correlated, so their statistics agree well within the
    # sampling error of one field
    se_var = ro.var() * np.sqrt(2.0 / N)
    assert abs(rg.var() - ro.var()) < 3 * se_var
    assert abs((rg < 0).mean() - (ro < 0).mean()) < 3 * np.sqrt((ro < 0).mean() / N)
    assert np.max(np.abs(g32.mean(1) - o.mean(1))) < 5 * o.std(1).max() / np.sqrt(N)


@pytest.mark.parametrize("precision,tol", [(lb.F64, 1e-14), (lb.F32, 3e-6)])
@pytest.mark.parametrize("dist", [lb.GAUSSIAN, lb.UNIFORM])
@pytest.mark.parametrize("nmom", [2, 8, 18])
def test_noise_variates_match_oracle(orc, precision, tol, dist, nmom):
    seed, lid, t = 0x123456789ABCDEF, 7, (5 << 32) + 99
    z = abi.lbfd_noise_draw(precision, dist, seed, lid, t, 1000, 300, nmom)
    zo = np.array([orc.site_noise(seed, lid, s, t, nmom, dist) for s in range(1000, 1300)])
    assert np.max(np.abs(z - zo)) <= tol * max(1.0, np.max(np.abs(zo)))


@pytest.mark.parametrize("precision", [lb.F64, lb.F32])
def test_split_run_bit_identical(precision):
    f0 = synth.random_populations(19, 12 * 7 * 5, 40.0, 0.2, seed=8)
    whole = _gpu_run(lb.D3Q19, (12, 7, 5), f0, 9, 0.7, precision, rho_mean=40.0, seed=5)
    with lb.Simulation(lb.D3Q19, (12, 7, 5), 0.7, 40.0, 5, precision=precision, init=lb.INIT_NONE) as s:
        s.set_f(f0)
        s.step(4)
        mid = s.get_f()
    with lb.Simulation(lb.D3Q19, (12, 7, 5), 0.7, 40.0, 5, precision=precision, init=lb.INIT_NONE) as s:
        s.set_f(mid)
        s.t = 4
        s.step(5)
        assert np.array_equal(s.get_f(), whole)


def test_seed_and_lattice_id_select_streams():
    f0 = synth.random_populations(9, 30 * 20, 10.0, 0.1, seed=1)
    a = _gpu_run(lb.D2Q9, (30, 20), f0, 5, 0.8, lb.F64, rho_mean=10.0, seed=1, lattice_id=0)
    b = _gpu_run(lb.D2Q9, (30, 20), f0, 5, 0.8, lb.F64, rho_mean=10.0, seed=2, lattice_id=0)
    c = _gpu_run(lb.D2Q9, (30, 20), f0, 5, 0.8, lb.F64, rho_mean=10.0, seed=1, lattice_id=1)
    assert not np.allclose(a, b) and not np.allclose(a, c) and not np.allclose(b, c)


@pytest.mark.parametrize("precision", [lb.F64, lb.F32])
def test_init_matches_equilibrium(orc, precision):
    dims, k = (96, 40), (2, 1)
    rho = synth.density_sine(dims, k, 3.0, 20.0)
    with lb.Simulation(lb.D2Q9, dims, 0.8, 20.0, 1, precision=precision, init=lb.INIT_SINE, sine_amp=3.0,
                       sine_k=k) as s:
        g = s.get_f()
    o = orc.init_equilibrium(lb.D2Q9, rho)
    assert np.max(np.abs(g - o)) <= (1e-14 if precision == lb.F64 else 1e-6) * 23.0
    with lb.Simulation(lb.D3Q19, (5, 6, 7), 0.8, 20.0, 1, precision=precision) as s:
        g = s.get_f()
    o = orc.init_equilibrium(lb.D3Q19, np.full(210, 20.0))
    assert np.max(np.abs(g - o)) <= 1e-6 * 20.0


@pytest.mark.parametrize("lat,dims", [(lb.D1Q3, (77,)), (lb.D2Q9, (31, 17)), (lb.D3Q19, (7, 6, 5))])
def test_moments_mass_and_observables(lat, dims):
    Q, N = lb.Q_OF[lat], int(np.prod(dims))
    modes = [(1, 0, 0), (2, 1, 0), (0, 1, 1), (3, 2, 1)][: 2 + (lat != lb.D1Q3)]
    with lb.Simulation(lat, dims, 0.8, 30.0, 4, precision=lb.F64, modes=modes) as s:
        s.step(13)
        f = s.get_f()
        rho, j = s.moments(with_flux=True)
        v, w, m = abi.lbfd_lattice_tables(lat)
        assert np.max(np.abs(rho - f.sum(0))) < 1e-12
        assert np.max(np.abs(j - v[:, : lb.D_OF[lat]].T @ f)) < 1e-12
        assert abs(s.mass() - f.sum()) < 1e-12 * f.sum()
        s.sample()
        s.step(3)
        f2 = s.get_f()
        s.sample()
        ob = s.observables()
    r1, r2 = f.sum(0), f2.sum(0)
    assert ob["n_samples"] == 2 and ob["t"] == 16
    assert abs(ob["sum_rho"] - (r1.sum() + r2.sum())) < 1e-12 * N * 60
    assert abs(ob["sum_rho2"] - ((r1 ** 2).sum() + (r2 ** 2).sum())) < 1e-12 * ob["sum_rho2"]
    assert np.max(np.abs(ob["sum_f"] - (f.sum(1) + f2.sum(1)))) < 1e-10
    ff = f @ f.T + f2 @ f2.T
    assert np.max(np.abs(ob["sum_ff"] - ff)) < 1e-12 * np.max(ff)
    d3 = list(dims) + [1] * (3 - len(dims))
    for mi, k in enumerate(modes):
        sk = 0.0
        for r in (r1, r2):
            field = (r - 30.0).reshape(d3[2], d3[1], d3[0])
            ft = np.fft.fftn(field)
            sk += abs(ft[k[2] % d3[2], k[1] % d3[1], k[0] % d3[0]]) ** 2
        assert abs(ob["sum_sk"][mi] - sk) < 1e-5 * max(sk, 1.0)


@pytest.mark.parametrize("lat,dims,prec", [(lb.D1Q3, (77,), lb.F32), (lb.D2Q9, (31, 17), lb.F32),
                                           (lb.D3Q19, (7, 6, 5), lb.F32), (lb.D2Q9, (300, 261), lb.F32),
                                           (lb.D3Q19, (40, 33, 21), lb.F32_F16), (lb.D2Q9, (64, 48), lb.F32_BF16),
                                           (lb.D1Q3, (50001,), lb.F32), (lb.D2Q5, (45, 38), lb.F32),
                                           (lb.D1Q3, (2200001,), lb.F32)])
def test_fp32_observables_match_fp64_sums(lat, dims, prec):
    """FP32-arithmetic formats sample from the stored state directly (no
    streamed copy), in FP32 per 256-site tile on deviations from w_i rho_mean
    and FP64 beyond.  The restored sums must match FP64 sums over get_f()
    (the same stored values) to what FP32 tiles allow; the central moments
    (density variance, covariance of the f_i) and S(k) are checked directly.
    The structure-factor phases come from per-axis tables, except on the
    2200001-site line (tables too large), which evaluates them directly with
    64-bit products (k x may pass 2^31)."""
    Q, N = lb.Q_OF[lat], int(np.prod(dims))
    modes = [(1, 0, 0), (2, 1, 0), (0, 1, 1), (3, 2, 1)][: 2 + (lat == lb.D3Q19)]
    if len(dims) == 1:
        modes = [(1, 0, 0), (7, 0, 0)]
    rho_mean = 30.0
    kw = dict(theta=0.3) if lat == lb.D2Q5 else {}
    with lb.Simulation(lat, dims, 0.8, rho_mean, 4, precision=prec, modes=modes, **kw) as s:
        s.step(13)
        f1 = s.get_f()
        s.sample()
        s.step(3)
        f2 = s.get_f()
        s.sample()
        ob = s.observables()
    fs = (f1, f2)
    n = 2 * N
    rho_sum = sum(f.sum() for f in fs)
    rho2_sum = sum((f.sum(0) ** 2).sum() for f in fs)
    f_sum = sum(f.sum(1) for f in fs)
    ff_sum = sum(f @ f.T for f in fs)
    assert ob["n_samples"] == 2
    assert abs(ob["sum_rho"] - rho_sum) <= 5e-7 * rho_sum
    var_ref = rho2_sum / n - (rho_sum / n) ** 2
    var_gpu = ob["sum_rho2"] / n - (ob["sum_rho"] / n) ** 2
    assert abs(var_gpu - var_ref) <= 1e-4 * var_ref
    assert np.max(np.abs(ob["sum_f"] - f_sum)) <= 5e-7 * np.max(f_sum)
    cov_ref = ff_sum / n - np.outer(f_sum, f_sum) / n ** 2
    cov_gpu = np.asarray(ob["sum_ff"]) / n - np.outer(ob["sum_f"], ob["sum_f"]) / n ** 2
    assert np.max(np.abs(cov_gpu - cov_ref)) <= 1e-4 * np.max(np.abs(cov_ref))
    d3 = list(dims) + [1] * (3 - len(dims))
    for mi, k in enumerate(modes):
        sk = 0.0
        for f in fs:
            field = (f.sum(0) - rho_mean).reshape(d3[2], d3[1], d3[0])
            ft = np.fft.fftn(field)
            sk += abs(ft[k[2] % d3[2], k[1] % d3[1], k[0] % d3[0]]) ** 2
        assert abs(ob["sum_sk"][mi] - sk) <= 1e-4 * sk + 1e-3 * N * var_ref, (mi, k)


def test_torch_buffers_and_stream_give_same_result():
    import torch

    f0 = synth.random_populations(9, 50 * 40, 10.0, 0.2, seed=2)
    ref = _gpu_run(lb.D2Q9, (50, 40), f0, 25, 0.8, lb.F32, rho_mean=10.0, seed=6)
    st = torch.cuda.Stream()
    got = _gpu_run(lb.D2Q9, (50, 40), f0, 25, 0.8, lb.F32, rho_mean=10.0, seed=6, torch_buffers=True, stream=st)
    assert np.array_equal(ref, got)


def test_error_reporting_on_gpu():
    with pytest.raises(abi.LbfdError):
        abi.lbfd_noise_draw(lb.F32, lb.GAUSSIAN, 1, 0, 0, 0, 10, 5)
    with lb.Simulation(lb.D2Q9, (8, 8), 0.8, 1.0, 1) as s:
        with pytest.raises(abi.LbfdError) as e:
            s.step(-3)
        assert e.value.code == abi.EINVAL


@pytest.mark.parametrize("precision,tol", [(lb.F64, 1e-14), (lb.F32, 3e-6)])
def test_box_muller_grid_edges(precision, tol):
    """The uniform grid's edges: u0 and u1 at their smallest and largest cells
    and around 1/2, where FP32 cannot hold u and the kernel forms 1 - u and
    u - 1/2 from the integer word."""
    edge = np.array([0x00000000, 0x000000FF, 0x00000100, 0x7FFFFF00, 0x7FFFFFFF, 0x80000000, 0x80000100,
                     0xFBFFFFFF, 0xFC000000, 0xFFFFFE00, 0xFFFFFEFF, 0xFFFFFF00, 0xFFFFFFFF], dtype=np.uint64)
    g = np.random.default_rng(4)
    r0 = np.concatenate([np.repeat(edge, edge.size), g.integers(0, 2**32, 20000, dtype=np.uint64)])
    r1 = np.concatenate([np.tile(edge, edge.size), g.integers(0, 2**32, 20000, dtype=np.uint64)])
    words = np.stack([r0, r1], 1).astype(np.uint32)
    z = abi.lbfd_box_muller_probe(precision, words).reshape(-1, 2)
    u0 = ((r0 >> 8).astype(np.float64) + 0.5) / 2**24
    u1 = ((r1 >> 8).astype(np.float64) + 0.5) / 2**24
    rad = np.sqrt(-2 * np.log(u0))
    want = np.stack([rad * np.cos(2 * np.pi * u1), rad * np.sin(2 * np.pi * u1)], 1)
    assert np.all(np.isfinite(z))
    assert np.max(np.abs(z - want)) <= tol * 6.0


@pytest.mark.parametrize("lat,dims,precision", [
    # one block
    (lb.D1Q3, (1001,), lb.F32), (lb.D2Q9, (40, 30), lb.F32), (lb.D3Q19, (9, 8, 7), lb.F32),
    (lb.D3Q19, (6, 5, 4), lb.F32_F16), (lb.D2Q9, (1, 1), lb.F32), (lb.D2Q9, (5, 6), lb.F64),
    # thread-block clusters: FP64 spread one CTA per 32 sites, larger states over several CTAs
    (lb.D1Q3, (256,), lb.F64), (lb.D1Q3, (65,), lb.F64), (lb.D2Q9, (13, 7), lb.F64), (lb.D2Q9, (64, 64), lb.F32),
    (lb.D3Q19, (16, 16, 16), lb.F32), (lb.D3Q19, (10, 10, 10), lb.F64), (lb.D2Q9, (100, 100), lb.F32_F16),
    (lb.D3Q19, (20, 20, 21), lb.F32),
])
@pytest.mark.parametrize("mode,dist", [(lb.NOISE_LOCAL, lb.GAUSSIAN), (lb.NOISE_GLOBAL, lb.UNIFORM)])
def test_small_lattice_many_steps_per_launch(lat, dims, precision, mode, dist):
    """A lattice whose two buffers fit one block's shared memory, or the
    distributed shared memory of a cluster of up to 8 CTAs, takes one launch
    for up to 4096 steps; the result equals one launch per step bit for bit,
    across launch boundaries and odd and even step counts."""
    Q, N = lb.Q_OF[lat], int(np.prod(dims))
    f0 = synth.random_populations(Q, N, 30.0, 0.3, seed=N)
    kw = dict(precision=precision, noise_mode=mode, noise_dist=dist, init=lb.INIT_NONE, lattice_id=5)
    with lb.Simulation(lat, dims, 0.9, 30.0, 11, **kw) as a:
        a.set_f(f0)
        n0 = abi.lbfd_kernel_launches()
        a.step(37)
        a.step(4100)   # two launches: 4096 + 4
        assert abi.lbfd_kernel_launches() - n0 == 3
        fa = a.get_f()
    with lb.Simulation(lat, dims, 0.9, 30.0, 11, **kw) as b:
        b.set_f(f0)
        for _ in range(4137):
            b.step(1)
        fb = b.get_f()
    assert np.array_equal(fa, fb)


def test_allocation_failure_is_reported_and_recoverable():
    """Failure detection on the host: a lattice whose two buffers exceed the
    GPU's memory (2 x 19 x 4 B x 2.0e9 sites = 306 GB) and a server whose
    arena does fail with LBFD_ENOMEM, free what they took, and leave the
    library usable."""
    o = abi.lbfd_options_init()
    o.lattice = lb.D3Q19
    o.dims[0], o.dims[1], o.dims[2] = 1200, 1200, 1400
    with pytest.raises(abi.LbfdError) as e:
        abi.lbfd_create_ex(o)
    assert e.value.code == abi.ENOMEM
    with pytest.raises(abi.LbfdError) as e:
        lb.Server(hbm_budget=1 << 40)
    assert e.value.code == abi.ENOMEM
    with lb.Simulation(lb.D2Q9, (16, 8), 0.8, 10.0, 1) as s:
        s.step(3)
        assert abs(s.mass() - 10.0 * 128) < 1e-3
