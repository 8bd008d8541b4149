"""Host logic of the serving loop, no GPU: the first-fit range allocator the
server carves its device arena and result staging with (checked against a
plain model of free and used ranges), the struct layouts of the binding, and
argument checks that fail before any CUDA call."""
import ctypes

import numpy as np
import pytest

import paper_1606_07801_gb300 as lb
from paper_1606_07801_gb300 import lbfd as abi


class Model:
    """Byte-level model: a range is free iff no live allocation covers it."""

    def __init__(self, capacity, align):
        self.cap, self.align = capacity // align * align, align
        self.live = {}

    def first_fit(self, size):
        size = max(1, size)
        size = (size + self.align - 1) // self.align * self.align
        used = sorted(self.live.items())
        pos = 0
        for off, sz in used:
            if off - pos >= size:
                return pos, size
            pos = off + sz
        return (pos, size) if self.cap - pos >= size else (-1, size)

    def largest_free(self):
        used = sorted(self.live.items())
        pos, best = 0, 0
        for off, sz in used:
            best = max(best, off - pos)
            pos = off + sz
        return max(best, self.cap - pos)


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_pool_matches_first_fit_model(seed):
    g = np.random.default_rng(seed)
    cap, align = 1 << 20, 256
    p = abi.lbfd_pool_create(cap, align)
    m = Model(cap, align)
    try:
        for _ in range(3000):
            if m.live and g.random() < 0.45:
                off = int(g.choice(list(m.live)))
                abi.lbfd_pool_free(p, off)
                del m.live[off]
            else:
                size = int(g.integers(1, 1 << 16))
                want, rounded = m.first_fit(size)
                got = abi.lbfd_pool_alloc(p, size)
                assert got == want
                if got >= 0:
                    assert got % align == 0
                    m.live[got] = rounded
            used, largest, nfree = abi.lbfd_pool_stats(p)
            assert used == sum(m.live.values())
            assert largest == m.largest_free()
        # freeing everything coalesces back to one range
        for off in list(m.live):
            abi.lbfd_pool_free(p, off)
        assert abi.lbfd_pool_stats(p) == (0, cap, 1)
    finally:
        abi.lbfd_pool_destroy(p)


def test_pool_rejects_bad_frees_and_sizes():
    p = abi.lbfd_pool_create(4096, 256)
    try:
        a = abi.lbfd_pool_alloc(p, 100)
        assert a == 0
        with pytest.raises(abi.LbfdError) as e:
            abi.lbfd_pool_free(p, 128)  # inside a range, not its start
        assert e.value.code == abi.EINVAL
        abi.lbfd_pool_free(p, a)
        with pytest.raises(abi.LbfdError):
            abi.lbfd_pool_free(p, a)  # double free
        assert abi.lbfd_pool_alloc(p, 4097) == -1
        assert abi.lbfd_pool_alloc(p, 4096) == 0
    finally:
        abi.lbfd_pool_destroy(p)
    h = ctypes.c_void_p()
    assert abi.load().lbfd_pool_create(ctypes.byref(h), 1024, 3) == abi.EINVAL


def test_server_structs_match_binding():
    o, r, s = abi.lbfd_server_struct_sizes()
    assert o == ctypes.sizeof(abi.ServerOptions)
    assert r == ctypes.sizeof(abi.Request)
    assert s == ctypes.sizeof(abi.ServerStats)


def test_server_option_defaults_and_checks():
    o = abi.lbfd_server_options_init()
    assert (o.precision, o.noise_mode, o.noise_dist, o.device) == (lb.F32, lb.NOISE_LOCAL, lb.GAUSSIAN, -1)
    assert (o.hbm_budget, o.max_active, o.max_ahead, o.passes, o.policy) == (1 << 30, 1024, 4, 1, lb.POLICY_FIFO)
    assert o.solo_sites == 1 << 17 and o.occupancy == 0 and o.walk == lb.WALK_PER_TILE and o.vx_max == 2
    lib = abi.load()
    h = ctypes.c_void_p()
    for field, bad in [("passes", 3), ("max_active", 0), ("max_ahead", 0), ("policy", 7), ("precision", 9),
                       ("hbm_budget", 16), ("solo_sites", -1), ("occupancy", 2),
                       ("walk", 4), ("vx_max", 0), ("vx_max", 3)]:
        b = abi.lbfd_server_options_init()
        setattr(b, field, bad)
        assert lib.lbfd_server_create(ctypes.byref(h), ctypes.byref(b)) == abi.EINVAL, field


def test_server_null_handles():
    lib = abi.load()
    st = ctypes.c_int32()
    assert lib.lbfd_server_destroy(None) == abi.OK
    assert lib.lbfd_server_pump(None, 1, None) == abi.EINVAL
    assert lib.lbfd_server_drain(None) == abi.EINVAL
    assert lib.lbfd_server_poll(None, 0, ctypes.byref(st), None) == abi.EINVAL
    req = abi.make_request(lb.D2Q9, (8, 8), 0.8, 1.0, 1, 10)
    i = ctypes.c_int64()
    assert lib.lbfd_server_submit(None, ctypes.byref(req), ctypes.byref(i)) == abi.EINVAL
