"""Multi-rank paths on CPU ranks (gloo, 127.0.0.1).

1. Slab decomposition of one lattice (paper Sec. II, eq. LB: the update
   reads nearest neighbours only).  Each rank holds a slab along the slowest
   axis with a halo plane on each side, laid out as the library stores a
   slab handle.  It steps its owned planes with a host step built from the
   oracle's collision and the oracle's noise of each site's global index
   (the key the GPU kernel uses), and fills its halo planes between steps
   through the library's plan (lbfd_slab_bounds, lbfd_slab_halo) and
   paper_1606_07801_gb300.slab.exchange over gloo.  The gathered result must
   equal oracle.run on the whole lattice bit for bit.
2. The benchmark's replicas: distinct Philox seed and lattice id per rank,
   the slowest rank's time by an all-reduce MAX.
"""
import queue
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _spawn(target, world, args):
    ctx = mp.get_context("spawn")
    out = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=target, args=(r, world, port, out) + tuple(args)) for r in range(world)]
    for p in procs:
        p.start()
    try:
        got = sorted((out.get(timeout=180) for _ in procs), key=lambda x: x[0])
    except queue.Empty:
        pytest.fail("a rank did not report")
    finally:
        for p in procs:
            p.join(timeout=60)
            if p.is_alive():
                p.kill()
    assert [p.exitcode for p in procs] == [0] * world
    return got


def _roll(f, v, dims, sign):
    """sign = +1: out_i(x) = f_i(x - v_i) (streaming); -1: out_i(x) = f_i(x + v_i)."""
    Lx, Ly, Lz = dims
    out = np.empty_like(f)
    for i in range(f.shape[0]):
        a = f[i].reshape(Lz, Ly, Lx)
        out[i] = np.roll(a, shift=(sign * v[i, 2], sign * v[i, 1], sign * v[i, 0]), axis=(0, 1, 2)).ravel()
    return out


def _host_step(orc, plan, v, g, t, tau, rho, seed, lid):
    """One step of the slab's owned planes from its stored state g [Q, stored
    sites]: site x pulls g_i(x - v_i) (the halo planes hold its neighbours'
    values), collides by the oracle with the oracle's noise of its global
    site index, and stores f*_i(x).  The halo planes are left as they were."""
    Lx, Ly, Lz = plan.stored_dims
    Q = g.shape[0]
    out = g.copy()
    for z in range(Lz):
        for y in range(Ly):
            c = (y, z)[plan.axis - 1]
            if c == 0 or c == plan.count + 1:
                continue
            for x in range(Lx):
                s = x + Lx * (y + Ly * z)
                fin = [g[i, (x - v[i, 0]) % Lx + Lx * ((y - v[i, 1]) % Ly + Ly * ((z - v[i, 2]) % Lz))]
                       for i in range(Q)]
                zeta = orc.site_noise(seed, lid, plan.global_site(s), t, Q - 1, orc.GAUSSIAN)
                out[:, s] = orc.collide(plan.lattice, fin, zeta, tau, orc.NOISE_LOCAL, rho)
    return out


def _slab_rank(rank, world, port, out, lat, gdims, steps):
    import os

    import torch
    import torch.distributed as dist

    os.environ["MASTER_ADDR"], os.environ["MASTER_PORT"] = "127.0.0.1", str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import oracle
        from paper_1606_07801_gb300 import slab, synth

        oracle.build()
        _, Q, v, _ = oracle.lattice(lat)
        N = int(np.prod(gdims))
        tau, rho, seed, lid = 0.8, 30.0, 9, 2
        f0 = synth.random_populations(Q, N, rho, 0.3, seed=123)      # the same global start on every rank
        g0 = _roll(f0, v, gdims, -1)                                 # stored form: g_i(x) = f_i(x + v_i)
        plan = slab.SlabPlan(lat, gdims, world, rank)
        # this rank's stored planes: global planes first - 1 .. first + count (periodic)
        L = gdims[plan.axis]
        planes = [(plan.first - 1 + c) % L for c in range(plan.count + 2)]
        g3 = g0.reshape(Q, gdims[2], gdims[1], gdims[0])
        stored = (g3[:, :, planes, :] if plan.axis == 1 else g3[:, planes, :, :]).reshape(Q, -1).copy()
        for c in (0, plan.count + 1):  # halo planes start unknown: the exchange must fill them
            sl = np.s_[:, :, c, :] if plan.axis == 1 else np.s_[:, c, :, :]
            s4 = stored.reshape(Q, plan.stored_dims[2], plan.stored_dims[1], plan.stored_dims[0])
            s4[sl] = np.nan
        state = torch.from_numpy(stored.reshape(-1))
        slab.exchange(plan, state)
        for t in range(steps):
            g = _host_step(oracle, plan, v, state.numpy().reshape(Q, -1), t, tau, rho, seed, lid)
            state.copy_(torch.from_numpy(g.reshape(-1)))
            slab.exchange(plan, state)
        pieces = [None] * world
        dist.all_gather_object(pieces, (plan.first, plan.count, plan.owned(state.numpy().reshape(Q, -1)).copy()))
        out.put((rank, pieces, plan.faces[0][2]))
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("world,lat,gdims,steps", [
    (2, 1, (12, 10, 1), 6),   # D2Q9 cut along y
    (3, 1, (8, 7, 1), 5),     # uneven slabs: 3, 2, 2 rows
    (2, 2, (6, 4, 6), 4),     # D3Q19 cut along z
])
def test_slab_split_bit_identical_to_whole_lattice(orc, world, lat, gdims, steps):
    got = _spawn(_slab_rank, world, (lat, gdims, steps))
    _, Q, v, _ = orc.lattice(lat)
    pieces = got[0][1]
    # assemble the global stored state from the owned planes
    plane = gdims[0] if lat == 1 else gdims[0] * gdims[1]
    N = int(np.prod(gdims))
    g = np.full((Q, N), np.nan)
    covered = 0
    for first, count, owned in pieces:
        g[:, first * plane:(first + count) * plane] = owned
        covered += count
    assert covered == gdims[1 if lat == 1 else 2]
    f = _roll(g, v, gdims, +1)
    from paper_1606_07801_gb300 import synth

    f0 = synth.random_populations(Q, N, 30.0, 0.3, seed=123)
    want = orc.run(lat, gdims[: 2 if lat == 1 else 3], f0, steps, 0.8, orc.NOISE_LOCAL, orc.GAUSSIAN, rho_eq=30.0,
                   seed=9, lattice_id=2)
    assert np.array_equal(f, want)


def _replica_rank(rank, world, port, out):
    import os

    import torch.distributed as dist

    os.environ["MASTER_ADDR"], os.environ["MASTER_PORT"] = "127.0.0.1", str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import bench

        rep = bench.replica(rank)
        reps = [None] * world
        dist.all_gather_object(reps, rep)
        slowest = bench.max_over_ranks(10.0 + 3.0 * rank, dist)   # rank 1 is the slow one
        value = bench.job_glups(world, 4096, 100, slowest)
        dist.barrier()
        out.put((rank, rep, reps, slowest, value))
    finally:
        dist.destroy_process_group()


def test_bench_replicas_and_slowest_rank_timing():
    (r0, rep0, reps0, t0, v0), (r1, rep1, reps1, t1, v1) = _spawn(_replica_rank, 2, ())
    assert reps0 == reps1 == [rep0, rep1]
    assert rep0["seed"] != rep1["seed"] and rep0["lattice_id"] != rep1["lattice_id"]
    assert t0 == t1 == 13.0
    assert v0 == v1 == pytest.approx(2 * 4096 * 100 / 13.0 / 1e9, rel=1e-15)


def test_slab_plan_host_arithmetic():
    """Bounds cover the axis once, balanced; each face sends and receives the
    populations that cross it, the upper slab's low face receiving exactly
    what the lower slab's high face sends."""
    from paper_1606_07801_gb300 import lbfd as abi
    from paper_1606_07801_gb300 import slab

    for L, n in ((10, 2), (7, 3), (65533, 8), (5, 5)):
        b = [abi.lbfd_slab_bounds(L, n, r) for r in range(n)]
        assert b[0][0] == 0 and all(b[k][0] + b[k][1] == b[k + 1][0] for k in range(n - 1))
        assert sum(c for _, c in b) == L and max(c for _, c in b) - min(c for _, c in b) <= 1
    with pytest.raises(abi.LbfdError):
        abi.lbfd_slab_bounds(3, 4, 0)
    v9 = abi.lbfd_lattice_tables(abi.D2Q9)[0]
    v19 = abi.lbfd_lattice_tables(abi.D3Q19)[0]
    assert abi.lbfd_slab_cross(abi.D2Q9, 1) == [i for i in range(9) if v9[i, 1] == 1] and len(
        abi.lbfd_slab_cross(abi.D2Q9, 1)) == 3
    assert abi.lbfd_slab_cross(abi.D3Q19, -1) == [i for i in range(19) if v19[i, 2] == -1] and len(
        abi.lbfd_slab_cross(abi.D3Q19, -1)) == 5
    lo, hi = slab.SlabPlan(abi.D3Q19, (6, 5, 9), 2, 0), slab.SlabPlan(abi.D3Q19, (6, 5, 9), 2, 1)
    NS_lo, NS_hi = lo.stored_sites, hi.stored_sites
    send_hi = [(int(o) // NS_lo, int(o) % NS_lo // lo.plane) for o in lo.faces[1][0]]
    recv_lo = [(int(o) // NS_hi, int(o) % NS_hi // hi.plane) for o in hi.faces[0][1]]
    assert [p for p, _ in send_hi] == [p for p, _ in recv_lo] == abi.lbfd_slab_cross(abi.D3Q19, 1)
    assert {c for _, c in send_hi} == {lo.count} and {c for _, c in recv_lo} == {0}
    assert lo.faces[0][2] == 30


def _slab_totals(lat, f, gdims, first, count, plane, axis, rho_mean, modes):
    """One slab's totals in the layout of lbfd_sample_totals, by their
    definition: sums over the slab's sites of e_i = f_i - c_i (c_i = w_i
    rho_mean rounded to FP32), delta = sum_i e_i, delta^2, e_i e_j, and
    (rho - rho_mean) e^{-2 pi i k.x / L} at the sites' global coordinates."""
    import oracle

    _, Q, v, w = oracle.lattice(lat)
    c = (np.float32(w) * np.float32(rho_mean)).astype(np.float64)
    e = f - c[:, None]
    delta = e.sum(0)
    Lx, Ly, Lz = gdims
    s = np.arange(count * plane)
    x = s % Lx
    y = (s // Lx) % (Ly if axis == 2 else count) + (first if axis == 1 else 0)
    z = s // (Lx * Ly) + first if axis == 2 else np.zeros_like(s)
    d = f.sum(0) - rho_mean
    out = [delta.sum(), (delta ** 2).sum()] + list(e.sum(1))
    for k in modes:
        ph = 2 * np.pi * (k[0] * x / Lx + k[1] * y / Ly + k[2] * z / Lz)
        out += [(d * np.cos(ph)).sum(), -(d * np.sin(ph)).sum()]
    out += [(e[i] * e[j]).sum() for i in range(Q) for j in range(i, Q)]
    return np.array(out)


def _obs_rank(rank, world, port, out, lat, gdims, modes):
    import os

    import torch.distributed as dist

    os.environ["MASTER_ADDR"], os.environ["MASTER_PORT"] = "127.0.0.1", str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import oracle
        from paper_1606_07801_gb300 import slab, synth

        oracle.build()
        _, Q, v, _ = oracle.lattice(lat)
        N = int(np.prod(gdims))
        rho = 30.0
        f0 = synth.random_populations(Q, N, rho, 0.3, seed=77)
        f = oracle.run(lat, gdims[: 2 if lat == 1 else 3], f0, 3, 0.8, oracle.NOISE_LOCAL, oracle.GAUSSIAN,
                       rho_eq=rho, seed=4, lattice_id=1)
        plan = slab.SlabPlan(lat, gdims, world, rank)
        mine = f[:, plan.first * plan.plane:(plan.first + plan.count) * plan.plane]
        totals = _slab_totals(lat, mine, plan.global_dims, plan.first, plan.count, plan.plane, plan.axis, rho, modes)
        total = slab.allreduce_sum(totals)
        entries = slab.sample_entries(plan, rho, len(modes), total)
        mass = slab.allreduce_sum([mine.sum()])[0]
        out.put((rank, entries, mass))
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("world,lat,gdims,modes", [
    (2, 1, (12, 10, 1), [(1, 0, 0), (2, 3, 0)]),
    (3, 2, (6, 4, 7), [(1, 0, 0), (0, 1, 2), (1, 1, 1)]),
])
def test_slab_observables_allreduce_match_whole_lattice(orc, world, lat, gdims, modes):
    """Each rank sums the observables of its own planes; the FP64 all-reduce
    of those totals (paper_1606_07801_gb300.slab.allreduce_sum), combined by
    the library's lbfd_obs_restore, gives the whole lattice's sums of rho,
    rho^2, f_i, f_i f_j and |rho(k)|^2 (paper Sec. IV, eqs. rhoth, dijexp,
    fkfk), the modes squared after the sum; and the slabs' masses add up to
    the lattice's."""
    got = _spawn(_obs_rank, world, (lat, gdims, modes))
    _, Q, v, w = orc.lattice(lat)
    N = int(np.prod(gdims))
    from paper_1606_07801_gb300 import synth

    f0 = synth.random_populations(Q, N, 30.0, 0.3, seed=77)
    f = orc.run(lat, gdims[: 2 if lat == 1 else 3], f0, 3, 0.8, orc.NOISE_LOCAL, orc.GAUSSIAN, rho_eq=30.0,
                seed=4, lattice_id=1)
    rho = f.sum(0)
    Lx, Ly, Lz = gdims
    field = (rho - 30.0).reshape(Lz, Ly, Lx)
    F = np.fft.fftn(field)
    want = np.concatenate([[rho.sum(), (rho ** 2).sum()], f.sum(1), (f @ f.T).ravel(),
                           [abs(F[k[2] % Lz, k[1] % Ly, k[0] % Lx]) ** 2 for k in modes]])
    for rank, entries, mass in got:
        assert np.allclose(entries, want, rtol=1e-11, atol=1e-9 * abs(want).max()), rank
        assert mass == pytest.approx(f.sum(), rel=1e-13)
    assert all(np.array_equal(got[0][1], g[1]) for g in got)
