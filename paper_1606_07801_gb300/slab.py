"""Slab decomposition of one lattice over several processes, one GPU each.

The step of eq. LB (Wagner & Strand, Sec. II) reads nearest neighbours only.
A lattice cut into slabs along its slowest axis (y for D2Q9, z for D3Q19)
therefore evolves exactly as a whole if, before every step, each slab holds
one plane beyond each face with the populations that cross it: 3 for D2Q9
and 5 for D3Q19, one plane each.  The noise of a site is keyed by its global
index, so the split run is bit-identical to the unsplit one.

This module holds the orchestration around the library:
  SlabPlan        a rank's planes, its neighbours and the exchange plan of
                  both faces (from lbfd_slab_bounds / lbfd_slab_halo)
  exchange        fills the halo planes of a stored state through
                  torch.distributed point-to-point messages (NCCL between
                  GPUs, gloo on CPU); one message per face and direction
  exchange_local  the same for several slabs held by one process
  SlabSimulation  a slab handle on this process's GPU, stepped one step at
                  a time with an exchange after each step
  allreduce_sum   the FP64 all-reduce of the slabs' sums: the mass (each
                  slab's owned planes, lbfd_mass) and the sampled
                  observables (lbfd_sample_totals, combined by
                  lbfd_obs_restore after the sum, so |rho(k)|^2 squares the
                  lattice's mode sum, not the slabs')
Arithmetic of the method stays in the CUDA library; here are only index
ranges, copies and the sums over ranks.
"""
from __future__ import annotations

import numpy as np

from . import lbfd as abi

SLOW_AXIS = {abi.D2Q9: 1, abi.D3Q19: 2}


class SlabPlan:
    """The slab of `rank` out of `nranks` of a lattice of global dims."""

    def __init__(self, lattice: int, global_dims, nranks: int, rank: int):
        if lattice not in SLOW_AXIS:
            raise ValueError("slabs are cut along y (D2Q9) or z (D3Q19)")
        self.lattice, self.nranks, self.rank = lattice, int(nranks), int(rank)
        g = [int(x) for x in global_dims] + [1] * (3 - len(global_dims))
        self.global_dims = tuple(g)
        self.axis = ax = SLOW_AXIS[lattice]
        self.first, self.count = abi.lbfd_slab_bounds(g[ax], self.nranks, self.rank)
        d = list(g)
        d[ax] = self.count
        self.dims = tuple(d)  # owned planes
        sd = list(d)
        sd[ax] += 2
        self.stored_dims = tuple(sd)  # with a halo plane on each side
        self.Q = abi.Q_OF[lattice]
        self.plane = g[0] if ax == 1 else g[0] * g[1]
        self.stored_sites = self.plane * (self.count + 2)
        self.below = (self.rank - 1) % self.nranks
        self.above = (self.rank + 1) % self.nranks
        # face 0 = low face (to and from `below`), face 1 = high face
        self.faces = [abi.lbfd_slab_halo(lattice, self.dims, face) for face in (0, 1)]

    def global_site(self, stored_site: int) -> int:
        """Global index x + Lx (y + Ly z) of a stored site (owned planes:
        stored plane c is global plane first - 1 + c)."""
        return int(stored_site) - self.plane + self.first * self.plane

    def owned(self, stored: np.ndarray) -> np.ndarray:
        """The owned planes of a [Q, stored sites] array."""
        return stored[:, self.plane: self.plane * (self.count + 1)]


def _views(plan: SlabPlan, state, face: int, which: int):
    off = plan.faces[face][which]
    p = plan.faces[face][2]
    return [state[int(o): int(o) + p] for o in off]


def _pack(plan, state, face):
    import torch

    return torch.cat(_views(plan, state, face, 0))


def _unpack(plan, state, face, buf):
    p = plan.faces[face][2]
    for k, v in enumerate(_views(plan, state, face, 1)):
        v.copy_(buf[k * p:(k + 1) * p])


def exchange(plan: SlabPlan, state, group=None) -> None:
    """Fill the halo planes of `state` (this rank's stored state, a flat
    tensor) from its neighbours.  The high face's populations go up and
    arrive in the upper slab's low halo plane; the low face's go down into
    the lower slab's high halo plane.  Messages between one pair of ranks are
    posted in the same order on both sides (and tagged by the receiving
    face), so two ranks that are each other's upper and lower neighbour
    match them correctly."""
    import torch
    import torch.distributed as dist

    if plan.nranks == 1:
        up, down = _pack(plan, state, 1), _pack(plan, state, 0)
        _unpack(plan, state, 0, up)
        _unpack(plan, state, 1, down)
        return
    send_up, send_down = _pack(plan, state, 1), _pack(plan, state, 0)
    recv_low, recv_high = torch.empty_like(send_up), torch.empty_like(send_down)
    ops = [dist.P2POp(dist.isend, send_up, plan.above, group, tag=0),
           dist.P2POp(dist.isend, send_down, plan.below, group, tag=1),
           dist.P2POp(dist.irecv, recv_low, plan.below, group, tag=0),
           dist.P2POp(dist.irecv, recv_high, plan.above, group, tag=1)]
    for req in dist.batch_isend_irecv(ops):
        req.wait()
    _unpack(plan, state, 0, recv_low)
    _unpack(plan, state, 1, recv_high)


def exchange_local(plans, states) -> None:
    """exchange() for all slabs of a lattice held by one process."""
    ups = [_pack(p, s, 1) for p, s in zip(plans, states)]
    downs = [_pack(p, s, 0) for p, s in zip(plans, states)]
    for p, s in zip(plans, states):
        _unpack(p, s, 0, ups[p.below])
        _unpack(p, s, 1, downs[p.above])


def allreduce_sum(values, group=None) -> np.ndarray:
    """FP64 sum of `values` over the ranks of `group`; every rank gets it
    (a copy when there is no process group or one rank)."""
    a = np.array(values, dtype=np.float64, copy=True).reshape(-1)
    try:
        import torch
        import torch.distributed as dist
    except ImportError:  # pragma: no cover
        return a
    if not dist.is_available() or not dist.is_initialized() or dist.get_world_size(group) == 1:
        return a
    t = torch.from_numpy(a)
    if dist.get_backend(group) == "nccl":
        t = t.cuda(torch.cuda.current_device())
    dist.all_reduce(t, op=dist.ReduceOp.SUM, group=group)
    return t.cpu().numpy()


def sample_entries(plan: SlabPlan, rho_mean: float, n_modes: int, totals) -> np.ndarray:
    """The accumulator entries of one sample of the whole lattice from the
    totals summed over all its slabs."""
    n_sites = int(np.prod(plan.global_dims))
    return abi.lbfd_obs_restore(plan.lattice, n_modes, rho_mean, n_sites, totals)


class SlabSimulation:
    """This rank's slab of one lattice on its GPU: a slab handle of the
    library whose buffers are torch tensors, on torch's current stream (so
    the library's kernels, the exchange's copies and the messages are
    ordered), stepped one step at a time with a halo exchange after each.
    With local=True the slab exchanges nothing by itself: several slabs held
    by one process are stepped together by step_local()."""

    def __init__(self, lattice: int, global_dims, tau: float, rho_mean: float, seed: int = 1, *, nranks: int,
                 rank: int, group=None, device: int = -1, local: bool = False, **kw):
        import torch

        from . import Simulation

        self.plan = SlabPlan(lattice, global_dims, nranks, rank)
        self.group = group
        self.rho_mean = float(rho_mean)
        self.n_modes = len(kw.get("modes") or ())
        kw.setdefault("stream", torch.cuda.current_stream())
        self.sim = Simulation(lattice, self.plan.dims, tau, rho_mean, seed, torch_buffers=True, device=device,
                              slab_global=self.plan.global_dims[self.plan.axis], slab_first=self.plan.first, **kw)
        self.local = local
        if not local:
            self.exchange()

    def state(self):
        """The current stored state as a flat torch tensor (one of the two buffers)."""
        ptr, _ = self.sim.state_device()
        for b in self.sim.buffers:
            if b.data_ptr() == ptr:
                return b
        raise RuntimeError("the handle's state is not one of its torch buffers")

    def exchange(self) -> None:
        exchange(self.plan, self.state(), self.group)

    def step(self, n: int = 1) -> None:
        if self.local:
            raise RuntimeError("local slabs are stepped together by step_local()")
        for _ in range(int(n)):
            self.sim.step(1)
            self.exchange()

    def get_f(self) -> np.ndarray:
        """f(x, t) on the owned planes, [Q, owned sites]."""
        return self.sim.get_f()

    def mass(self) -> float:
        """The lattice's mass: the slabs' FP64 masses summed over the ranks."""
        return float(allreduce_sum([abi.lbfd_mass(self.sim.h)], self.group)[0])

    def sample(self) -> None:
        """Adds the lattice's observables of the current state to this
        slab's accumulators (every rank's hold the same sums): the slabs'
        totals, summed over the ranks, then combined."""
        totals = abi.lbfd_sample_totals(self.sim.h, self.plan.Q, self.n_modes)
        total = allreduce_sum(totals, self.group)
        abi.lbfd_obs_add(self.sim.h, sample_entries(self.plan, self.rho_mean, self.n_modes, total))

    def observables(self) -> dict:
        return self.sim.observables()

    def close(self) -> None:
        self.sim.close()

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


def mass_local(slabs) -> float:
    """The lattice's mass from all of its slabs held by this process."""
    return float(sum(abi.lbfd_mass(sl.sim.h) for sl in slabs))


def sample_local(slabs) -> None:
    """sample() for all slabs of a lattice held by this process: their
    totals summed in slab order, combined, and added to every slab."""
    total = None
    for sl in slabs:
        t = abi.lbfd_sample_totals(sl.sim.h, sl.plan.Q, sl.n_modes)
        total = t if total is None else total + t
    entries = sample_entries(slabs[0].plan, slabs[0].rho_mean, slabs[0].n_modes, total)
    for sl in slabs:
        abi.lbfd_obs_add(sl.sim.h, entries)


def step_local(slabs, n: int = 0) -> None:
    """Several slabs of one lattice held by this process: the halo exchange
    after creation (n = 0), or n steps of all of them, each followed by the
    exchange among them."""
    plans = [sl.plan for sl in slabs]
    if n == 0:
        exchange_local(plans, [sl.state() for sl in slabs])
    for _ in range(int(n)):
        for sl in slabs:
            sl.sim.step(1)
        exchange_local(plans, [sl.state() for sl in slabs])
