"""The serving loop on the GPU.  Every served simulation must end
bit-identical to the same lattice run alone through lbfd_create_ex /
lbfd_step (same arithmetic, same Philox keys, its own t), whatever else
shares the GPU with it: requests arrive while others run, in several
waves, with mixed lattices, sizes, step counts, initial states and result
kinds; admission respects the memory budget, the slot count and the site
limit; and the trace loop serves a Poisson stream."""
import numpy as np
import pytest

import paper_1606_07801_gb300 as lb
from paper_1606_07801_gb300 import lbfd as abi
from paper_1606_07801_gb300 import synth

pytestmark = pytest.mark.gpu


def _spec(lat, dims, steps, k, **kw):
    g = np.random.default_rng(1000 + k)
    sp = dict(lattice=lat, dims=dims, steps=steps, tau=float(g.uniform(0.6, 1.5)),
              rho_mean=float(g.uniform(20.0, 200.0)), seed=int(g.integers(0, 2**63)),
              lattice_id=int(g.integers(0, 2**31)), init=lb.INIT_SINE if k % 3 == 1 else lb.INIT_UNIFORM,
              sine_amp=0.4, sine_k=(1, 2, 1), result=lb.RESULT_F if k % 4 != 3 else lb.RESULT_RHO, f0=None)
    sp.update(kw)
    return sp


def _alone(sp, precision, noise_mode=lb.NOISE_LOCAL, noise_dist=lb.GAUSSIAN):
    """The same simulation through lbfd_create_ex, lbfd_step and
    lbfd_get_f_raw / lbfd_moments."""
    lat, dims = sp["lattice"], sp["dims"]
    Q, N = lb.Q_OF[lat], int(np.prod(dims))
    init = lb.INIT_NONE if sp["f0"] is not None else sp["init"]
    with lb.Simulation(lat, dims, sp["tau"], sp["rho_mean"], sp["seed"], precision=precision, noise_mode=noise_mode,
                       noise_dist=noise_dist, init=init, sine_amp=sp["sine_amp"], sine_k=sp["sine_k"],
                       lattice_id=sp["lattice_id"]) as s:
        if sp["f0"] is not None:
            raw = np.ascontiguousarray(sp["f0"], dtype=lb.STORAGE_DTYPE[precision])
            abi.lbfd_set_f_raw(s.h, raw.ctypes.data)
        s.step(sp["steps"])
        if sp["result"] == lb.RESULT_RHO:
            return s.moments()
        out = np.empty((Q, N), dtype=lb.STORAGE_DTYPE[precision])
        abi.lbfd_get_f_raw(s.h, out.ctypes.data)
        return out


def _submit(srv, sp):
    return srv.submit(sp["lattice"], sp["dims"], sp["tau"], sp["rho_mean"], sp["seed"], sp["steps"],
                      lattice_id=sp["lattice_id"], init=sp["init"], sine_amp=sp["sine_amp"], sine_k=sp["sine_k"],
                      f0=sp["f0"], result=sp["result"])


def _mixed_specs(precision):
    specs = []
    shapes = [(lb.D1Q3, (257,)), (lb.D2Q9, (33, 20)), (lb.D3Q19, (10, 7, 5)), (lb.D2Q9, (64, 48)),
              (lb.D1Q3, (1024,)), (lb.D3Q19, (16, 16, 8)), (lb.D2Q9, (1, 17)), (lb.D2Q9, (130, 3)),
              (lb.D3Q19, (2, 3, 4)), (lb.D1Q3, (6,)), (lb.D2Q9, (96, 96)), (lb.D3Q19, (24, 12, 9))]
    steps = [0, 1, 17, 40, 3, 25, 64, 9, 31, 2, 50, 12]
    for k, ((lat, dims), n) in enumerate(zip(shapes, steps)):
        sp = _spec(lat, dims, n, k)
        if k % 5 == 2:  # a host-given non-equilibrium start
            Q, N = lb.Q_OF[lat], int(np.prod(dims))
            f = synth.random_populations(Q, N, sp["rho_mean"], 0.3, seed=k)
            if precision in (lb.F32_F16, lb.F32_BF16):
                # the 16-bit formats store f_i - w_i rho_mean
                _, w, _ = abi.lbfd_lattice_tables(lat)
                dev = f - w[:, None] * sp["rho_mean"]
                if precision == lb.F32_F16:
                    f = dev.astype(np.float16)
                else:
                    f = (dev.astype(np.float32).view(np.uint32) >> 16).astype(np.uint16)
            sp["f0"] = f
        specs.append(sp)
    return specs


@pytest.mark.parametrize("precision,solo,walk,vx_max", [
    (lb.F32, 0, lb.WALK_STRIDED, 2), (lb.F32, 400, lb.WALK_STRIDED, 2), (lb.F64, 400, lb.WALK_CONTIGUOUS, 2),
    (lb.F32_F16, 0, lb.WALK_CONTIGUOUS, 1), (lb.F32_F16, 1000, lb.WALK_STRIDED, 2), (lb.F32, 0, lb.WALK_CONTIGUOUS, 1),
    (lb.F32, 0, lb.WALK_CONTIGUOUS, 2), (lb.F32, 400, lb.WALK_PER_TILE, 2), (lb.F32_BF16, 0, lb.WALK_PER_TILE, 1),
    (lb.F32, 400, lb.WALK_PARAM, 2), (lb.F32_F16, 0, lb.WALK_PARAM, 1)])
def test_served_results_bit_identical_to_alone(precision, solo, walk, vx_max):
    """solo: simulations of at least this many sites take their own
    single-lattice launch each step (0: all batched); walk and vx_max: tile
    order and sites per item of the batched launch."""
    specs = _mixed_specs(precision)
    with lb.Server(precision=precision, hbm_budget=256 << 20, max_ahead=3, solo_sites=solo, walk=walk,
                   vx_max=vx_max) as srv:
        ids = [_submit(srv, sp) for sp in specs[:5]]
        srv.pump(6)                      # the first wave runs ...
        ids += [_submit(srv, sp) for sp in specs[5:9]]   # ... while the second arrives
        srv.pump(4)
        ids += [_submit(srv, sp) for sp in specs[9:]]
        srv.drain()
        got = [srv.result(i) for i in ids]
        st = srv.stats()
        lat = [srv.poll(i)[1] for i in ids]
    assert st["done"] == len(specs) and st["queued"] == 0 and st["running"] == 0
    assert st["site_updates"] == sum(int(np.prod(sp["dims"])) * sp["steps"] for sp in specs)
    assert st["peak_active"] >= 6   # the waves did overlap on the device
    assert all(x >= 0.0 for x in lat)
    for k, sp in enumerate(specs):
        want = _alone(sp, precision)
        assert got[k].dtype == want.dtype
        assert np.array_equal(got[k], want), (k, sp["lattice"], sp["dims"], sp["steps"])


def test_noise_variants_served_bit_identical():
    for mode, dist in [(lb.NOISE_GLOBAL, lb.UNIFORM), (lb.NOISE_OFF, lb.GAUSSIAN)]:
        specs = [_spec(lb.D2Q9, (40, 22), 23, 0), _spec(lb.D3Q19, (9, 8, 6), 11, 1), _spec(lb.D1Q3, (99,), 30, 2)]
        with lb.Server(noise_mode=mode, noise_dist=dist, hbm_budget=64 << 20) as srv:
            ids = [_submit(srv, sp) for sp in specs]
            srv.drain()
            got = [srv.result(i) for i in ids]
        for k, sp in enumerate(specs):
            assert np.array_equal(got[k], _alone(sp, lb.F32, mode, dist)), (mode, k)


def test_budget_slots_and_site_limit_bound_admission():
    # one D2Q9 64x64 FP32 request holds 2 x 9 x 4096 x 4 bytes = 294912 bytes
    specs = [_spec(lb.D2Q9, (64, 64), 10 + 7 * k, k, result=lb.RESULT_F) for k in range(6)]
    budget = 2 * 294912 + 1000
    with lb.Server(hbm_budget=budget) as srv:
        ids = [_submit(srv, sp) for sp in specs]
        srv.drain()
        st = srv.stats()
        got = [srv.result(i) for i in ids]
    assert st["peak_resident_bytes"] <= budget and st["peak_active"] == 2
    for k, sp in enumerate(specs):
        assert np.array_equal(got[k], _alone(sp, lb.F32))
    # slots
    with lb.Server(hbm_budget=64 << 20, max_active=3) as srv:
        ids = [_submit(srv, sp) for sp in specs]
        srv.drain()
        assert srv.stats()["peak_active"] == 3
    # site limit with shortest-first admission
    with lb.Server(hbm_budget=64 << 20, max_active_sites=3 * 4096, policy=lb.POLICY_SHORTEST) as srv:
        ids = [_submit(srv, sp) for sp in reversed(specs)]
        srv.drain()
        st = srv.stats()
        got = [srv.result(i) for i in ids]
    assert st["peak_resident_sites"] <= 3 * 4096 and st["peak_active"] == 3
    for k, sp in enumerate(reversed(specs)):
        assert np.array_equal(got[k], _alone(sp, lb.F32))
    # longest-work-first admission: other order, same results
    with lb.Server(hbm_budget=64 << 20, max_active_sites=3 * 4096, policy=lb.POLICY_LONGEST) as srv:
        ids = [_submit(srv, sp) for sp in specs]
        srv.drain()
        got = [srv.result(i) for i in ids]
    for k, sp in enumerate(specs):
        assert np.array_equal(got[k], _alone(sp, lb.F32))


def test_requests_that_never_fit_are_rejected():
    with lb.Server(hbm_budget=1 << 20) as srv:
        with pytest.raises(abi.LbfdError) as e:
            srv.submit(lb.D2Q9, (256, 256), 0.8, 10.0, 1, 5)
        assert e.value.code == abi.EINVAL and "budget" in str(e.value)
        with pytest.raises(abi.LbfdError):
            srv.submit(lb.D2Q9, (8, 8), 0.4, 10.0, 1, 5)
        req = abi.make_request(lb.D2Q9, (8, 8), 0.8, 10.0, 1, 5, result=lb.RESULT_F, out_host=None)
        with pytest.raises(abi.LbfdError):
            abi.lbfd_server_submit(srv.h, req)
        assert srv.stats()["submitted"] == 0


def test_trace_loop_serves_a_poisson_stream():
    g = np.random.default_rng(5)
    n = 60
    arrivals = np.cumsum(g.exponential(1.0 / 2000.0, n))
    reqs, specs = [], []
    for k in range(n):
        lat = [lb.D1Q3, lb.D2Q9, lb.D3Q19][k % 3]
        dims = [(int(g.integers(64, 4096)),), (int(g.integers(16, 128)), int(g.integers(16, 128))),
                (int(g.integers(8, 32)),) * 3][k % 3]
        steps = int(g.integers(5, 200))
        sp = _spec(lat, dims, steps, k, result=lb.RESULT_RHO if k % 2 else lb.RESULT_F)
        specs.append(sp)
        reqs.append(abi.make_request(lat, dims, sp["tau"], sp["rho_mean"], sp["seed"], steps,
                                     lattice_id=sp["lattice_id"], init=sp["init"], sine_amp=sp["sine_amp"],
                                     sine_k=sp["sine_k"], result=sp["result"]))
    sink = np.empty(64 << 20, dtype=np.uint8)
    with lb.Server(hbm_budget=512 << 20) as srv:
        lat, makespan = abi.lbfd_server_run_trace(srv.h, reqs, arrivals, sink.ctypes.data, sink.nbytes)
        st = srv.stats()
    assert st["done"] == n and st["queued"] == 0 and st["running"] == 0
    assert st["site_updates"] == sum(int(np.prod(sp["dims"])) * sp["steps"] for sp in specs)
    assert np.all(lat > 0.0) and makespan >= arrivals[-1]
    assert np.all(arrivals + lat <= makespan + 1e-6)
