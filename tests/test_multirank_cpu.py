"""The bench's multi-rank path, on CPU ranks (gloo, world size 2, 127.0.0.1).

Under torchrun every rank runs its own replica lattice: distinct Philox seed
and lattice id, no collective on the data path.  The timed region's length
is the slowest rank's, taken with an all-reduce MAX, and the reported value
is the site updates of all ranks over that time.  The GPU runs use NCCL for
the same two collectives (barrier, MAX); these ranks use gloo."""
import queue
import socket

import pytest
import torch.multiprocessing as mp


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
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


def test_replicas_and_slowest_rank_timing():
    ctx = mp.get_context("spawn")
    out = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, out)) for r in range(2)]
    for p in procs:
        p.start()
    try:
        got = sorted((out.get(timeout=120) for _ in procs), key=lambda x: x[0])
    except queue.Empty:
        pytest.fail("a rank did not report")
    finally:
        for p in procs:
            p.join(timeout=60)
            if p.is_alive():
                p.kill()
    assert [p.exitcode for p in procs] == [0, 0]
    (r0, rep0, reps0, t0, v0), (r1, rep1, reps1, t1, v1) = got
    assert reps0 == reps1 == [rep0, rep1]
    assert rep0["seed"] != rep1["seed"] and rep0["lattice_id"] != rep1["lattice_id"]
    assert t0 == t1 == 13.0
    assert v0 == v1 == pytest.approx(2 * 4096 * 100 / 13.0 / 1e9, rel=1e-15)


def test_single_rank_needs_no_collective():
    import bench

    assert bench.max_over_ranks(2.5) == 2.5
    assert bench.replica(0) == {"seed": 1, "lattice_id": 0}
