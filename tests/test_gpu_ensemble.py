"""Batched ensembles: every member must evolve bit-identically to the same
lattice stepped alone (same arithmetic, same Philox keys), across graph
chunks, odd and even row lengths, storage formats and the tuner; and FP64
members must match the oracle."""
import numpy as np
import pytest

import paper_1606_07801_gb300 as lb
from paper_1606_07801_gb300 import synth

pytestmark = pytest.mark.gpu


def _specs(lat, n, seed):
    g = np.random.default_rng(seed)
    out = []
    for k in range(n):
        if lat == lb.D1Q3:
            dims = (int(g.integers(5, 900)),)
        elif lat == lb.D2Q9:
            dims = (int(g.integers(3, 140)), int(g.integers(1, 90)))
        else:
            dims = (int(g.integers(2, 24)), int(g.integers(1, 20)), int(g.integers(1, 16)))
        out.append(dict(dims=dims, tau=float(g.uniform(0.6, 1.5)), rho_mean=float(g.uniform(0.5, 200)),
                        seed=int(g.integers(0, 2**63)), lattice_id=int(g.integers(0, 2**31)),
                        init=lb.INIT_SINE if k % 3 == 0 else lb.INIT_UNIFORM, sine_amp=0.3, sine_k=(1, 1, 0)))
    return out


def _alone(lat, sp, precision, steps, mode=lb.NOISE_LOCAL, dist=lb.GAUSSIAN):
    with lb.Simulation(lat, sp["dims"], sp["tau"], sp["rho_mean"], sp["seed"], precision=precision, noise_mode=mode,
                       noise_dist=dist, init=sp["init"], sine_amp=sp["sine_amp"], sine_k=sp["sine_k"],
                       lattice_id=sp["lattice_id"]) as s:
        s.step(steps)
        return s.get_f()


@pytest.mark.parametrize("lat,precision", [(lb.D2Q9, lb.F32), (lb.D3Q19, lb.F32), (lb.D1Q3, lb.F64),
                                           (lb.D2Q9, lb.F32_F16), (lb.D3Q19, lb.F64)])
def test_members_bit_identical_to_single_lattices(lat, precision):
    specs = _specs(lat, 9, seed=lat * 10 + precision)
    with lb.Ensemble(lat, specs, precision=precision) as e:
        e.step(21)   # one graph chunk of 16 and single steps
        e.step(16)   # starts on the odd buffer: single steps, then a chunk
        e.step(1)
        got = [e.get_f(m) for m in range(len(specs))]
        n, sites, t, vx, passes, bps, walk = e.query()
    assert (n, t) == (len(specs), 38)
    assert sites == sum(int(np.prod(s["dims"])) for s in specs)
    for m, sp in enumerate(specs):
        assert np.array_equal(got[m], _alone(lat, sp, precision, 38)), m


@pytest.mark.parametrize("lat", [lb.D2Q9, lb.D3Q19])
@pytest.mark.parametrize("vx,passes,occ,walk", [(1, 1, 0, lb.WALK_CONTIGUOUS), (2, 8, 1, lb.WALK_CONTIGUOUS),
                                                (2, 1, 0, lb.WALK_CONTIGUOUS), (2, 2, 1, lb.WALK_STRIDED),
                                                (1, 4, 0, lb.WALK_STRIDED), (2, 4, 0, lb.WALK_PER_TILE),
                                                (1, 2, 1, lb.WALK_PER_TILE), (2, 4, 0, lb.WALK_PARAM),
                                                (1, 1, 1, lb.WALK_PARAM)])
def test_every_decomposition_bit_identical(lat, vx, passes, occ, walk):
    """Sites per item, tile passes, occupancy variant and tile order change
    only which thread computes a site, never its value.  The members are
    large enough (about 10^6 sites in all) that a block of the persistent
    grid takes several tiles and, in the contiguous order, crosses members."""
    g = np.random.default_rng(lat * 100 + passes * 10 + walk)
    specs = _specs(lat, 7, seed=lat * 3 + passes)
    for k, sp in enumerate(specs):
        if lat == lb.D2Q9:
            sp["dims"] = (int(g.integers(200, 420)), int(g.integers(150, 330)))
        else:
            sp["dims"] = (int(g.integers(40, 66)), int(g.integers(30, 50)), int(g.integers(20, 41)))
    with lb.Ensemble(lat, specs) as e:
        e.plan(vx, passes, occ, walk)
        q = e.query()
        assert (q[3], q[4], q[6]) == (vx, passes, walk) and q[5] >= 1
        e.step(19)
        got = [e.get_f(m) for m in range(len(specs))]
    for m, sp in enumerate(specs):
        assert np.array_equal(got[m], _alone(lat, sp, lb.F32, 19)), m


@pytest.mark.parametrize("lat,precision,walk", [(lb.D1Q3, lb.F64, lb.WALK_PARAM), (lb.D2Q9, lb.F32_F16, lb.WALK_PARAM),
                                                (lb.D3Q19, lb.F32_BF16, lb.WALK_PARAM), (lb.D2Q9, lb.F64, lb.WALK_PER_TILE),
                                                (lb.D1Q3, lb.F32, lb.WALK_CONTIGUOUS)])
def test_tile_orders_bit_identical_in_every_format(lat, precision, walk):
    """The parameter-bank and other tile orders in the FP64 and 16-bit
    formats and on D1Q3: members equal the same lattices stepped alone.  Over
    112 members so that the parameter order takes more than one launch."""
    specs = _specs(lat, 130, seed=lat * 7 + precision)
    with lb.Ensemble(lat, specs, precision=precision) as e:
        e.plan(2, 2, 0, walk)
        e.step(18)
        got = [e.get_f(m) for m in range(0, len(specs), 9)]
    for k, m in enumerate(range(0, len(specs), 9)):
        assert np.array_equal(got[k], _alone(lat, specs[m], precision, 18)), m


def test_plan_rejects_bad_values():
    specs = _specs(lb.D2Q9, 2, seed=1)
    with lb.Ensemble(lb.D2Q9, specs) as e:
        for bad in [(3, 1, 0, 0), (2, 3, 0, 0), (2, 1, 2, 0), (2, 1, 0, 4), (2, 1, 0, -1)]:
            with pytest.raises(lb.LbfdError):
                e.plan(*bad)


@pytest.mark.parametrize("mode,dist", [(lb.NOISE_GLOBAL, lb.UNIFORM), (lb.NOISE_OFF, lb.GAUSSIAN)])
def test_noise_variants_bit_identical(mode, dist):
    specs = _specs(lb.D2Q9, 5, seed=7)
    with lb.Ensemble(lb.D2Q9, specs, noise_mode=mode, noise_dist=dist) as e:
        e.step(17)
        got = [e.get_f(m) for m in range(5)]
    for m, sp in enumerate(specs):
        assert np.array_equal(got[m], _alone(lb.D2Q9, sp, lb.F32, 17, mode, dist))


def test_tuner_keeps_state_and_results():
    specs = [dict(dims=(64, 40), tau=0.8, rho_mean=50.0, seed=3, lattice_id=1, init=lb.INIT_UNIFORM, sine_amp=0.0,
                  sine_k=(1, 0, 0)),
             dict(dims=(96, 30), tau=1.2, rho_mean=20.0, seed=4, lattice_id=2, init=lb.INIT_SINE, sine_amp=1.0,
                  sine_k=(2, 1, 0))]
    with lb.Ensemble(lb.D2Q9, specs) as e:
        e.step(5)
        before = [e.get_f(m) for m in range(2)]
        vx, passes, bps = e.tune(steps=3)
        assert vx in (1, 2) and passes in (1, 2, 4, 8) and bps >= 1
        assert all(np.array_equal(before[m], e.get_f(m)) for m in range(2))
        e.step(20)
        got = [e.get_f(m) for m in range(2)]
    for m in range(2):
        assert np.array_equal(got[m], _alone(lb.D2Q9, specs[m], lb.F32, 25))


def test_fp64_members_match_oracle(orc):
    specs = _specs(lb.D2Q9, 4, seed=11)
    for sp in specs:
        sp["init"] = lb.INIT_NONE
    with lb.Ensemble(lb.D2Q9, specs, precision=lb.F64) as e:
        f0 = []
        for m, sp in enumerate(specs):
            Q, N = 9, int(np.prod(sp["dims"]))
            f0.append(synth.random_populations(Q, N, sp["rho_mean"], 0.2, seed=m))
            e.set_f(m, f0[-1])
        e.step(40)
        got = [e.get_f(m) for m in range(4)]
        masses = [e.mass(m) for m in range(4)]
    for m, sp in enumerate(specs):
        o = orc.run(lb.D2Q9, sp["dims"], f0[m], 40, sp["tau"], orc.NOISE_LOCAL, orc.GAUSSIAN, rho_eq=sp["rho_mean"],
                    seed=sp["seed"], lattice_id=sp["lattice_id"])
        assert np.max(np.abs(got[m] - o)) <= 1e-12 * max(sp["rho_mean"], 1.0)
        assert abs(masses[m] - o.sum()) <= 1e-10 * o.sum()
