"""CPU unit tests of the device header's arithmetic (device.cuh compiled for
the host by nvcc): Philox4x32-10, the noise variates and the noise
back-transform the step kernel uses, against the oracle."""
import ctypes
import os
import shutil
import subprocess

import numpy as np
import pytest

import paper_1606_07801_gb300 as lb
from tests import golden_io

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def dhc(tmp_path_factory):
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(nvcc):
        pytest.skip("nvcc not available")
    out = str(tmp_path_factory.mktemp("dhc") / "libdhc.so")
    src = os.path.join(ROOT, "tests", "csrc", "device_host_check.cu")
    inc = os.path.join(ROOT, "paper_1606_07801_gb300", "csrc")
    subprocess.run([nvcc, "-std=c++17", "-O2", "-Xcompiler", "-fPIC", "-shared", "-I", inc, "-I",
                    os.path.join(ROOT, "include"), src, "-o", out], check=True)
    lib = ctypes.CDLL(out)
    lib.dhc_transform.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p]
    lib.dhc_variates.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_uint64, ctypes.c_uint32,
                                 ctypes.c_uint32, ctypes.c_uint64, ctypes.c_void_p]
    lib.dhc_philox.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]
    lib.dhc_philox_site.argtypes = [ctypes.c_uint64, ctypes.c_uint32, ctypes.c_uint64, ctypes.c_uint32, ctypes.c_int,
                                    ctypes.c_void_p]
    lib.dhc_transform_pair.argtypes = [ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p]
    lib.dhc_flat_pair_mismatches.argtypes = [ctypes.c_void_p, ctypes.c_int64]
    lib.dhc_fastdiv_mismatches.restype = ctypes.c_int64
    lib.dhc_fastdiv_mismatches.argtypes = [ctypes.c_void_p, ctypes.c_int64, ctypes.c_void_p, ctypes.c_int64]
    return lib


def test_step_philox_equals_the_definition(orc, dhc):
    """The kernel's Philox (rounds 0-2 partly precomputed per step) equals
    Philox4x32-10 on the counter (site, lattice id, t_lo, t_hi*8 + j)."""
    g = np.random.default_rng(11)
    for _ in range(400):
        seed = int(g.integers(0, 2**64, dtype=np.uint64))
        lid = int(g.integers(0, 2**32))
        t = int(g.integers(0, 2**40))
        site = int(g.integers(0, 2**32))
        j = int(g.integers(0, 8))
        out = np.zeros(4, dtype=np.uint32)
        dhc.dhc_philox_site(seed, lid, t, site, j, out.ctypes.data)
        ctr = [site, lid, t & 0xFFFFFFFF, (((t >> 32) << 3) | j) & 0xFFFFFFFF]
        key = [seed & 0xFFFFFFFF, seed >> 32]
        assert out.tolist() == orc.philox4x32_10(ctr, key).tolist()


def test_device_philox_known_answers(dhc):
    for ctr, key, out in golden_io.philox_kat():
        c = np.array(ctr, dtype=np.uint32)
        k = np.array(key, dtype=np.uint32)
        o = np.zeros(4, dtype=np.uint32)
        dhc.dhc_philox(c.ctypes.data, k.ctypes.data, o.ctypes.data)
        assert o.tolist() == out


@pytest.mark.parametrize("lat", [lb.D1Q3, lb.D2Q9, lb.D3Q19])
@pytest.mark.parametrize("f64,tol", [(1, 1e-15), (0, 1e-6)])
def test_noise_transform_is_the_basis(orc, dhc, lat, f64, tol):
    """T_i = sum_{a>=1} m_i^a z^a for unit z: the kernel's (factorised, or
    sparse, weighted and parity-split) transform reproduces the oracle's
    Gram-Schmidt basis (times w_i where the transform folds the weights in)."""
    Q = lb.Q_OF[lat]
    m = orc.basis(lat)
    _, _, _, w = orc.lattice(lat)
    for a in range(Q - 1):
        z = np.zeros(Q - 1)
        z[a] = 1.0
        T = np.zeros(Q)
        weighted = dhc.dhc_transform(lat, f64, z.ctypes.data, T.ctypes.data)
        expect = m[a + 1] * w if weighted else m[a + 1]
        assert np.max(np.abs(T - expect)) < tol * 4


@pytest.mark.parametrize("lat", [lb.D1Q3, lb.D2Q9, lb.D3Q19])
def test_two_site_transform_is_lane_by_lane_the_one_site_transform(orc, dhc, lat):
    """The transform instantiated on float2 (two neighbouring sites, as the
    paired collision runs it) gives in each lane the float transform of that
    lane's variates, bit for bit (host build: two scalar operations per
    packed one; the device instructions are checked on the GPU), and both
    lanes are the oracle's transform to FP32 accuracy."""
    Q = lb.Q_OF[lat]
    m = orc.basis(lat)
    _, _, _, w = orc.lattice(lat)
    g = np.random.default_rng(lat + 11)
    for _ in range(20):
        z2 = g.standard_normal(2 * (Q - 1))
        T2 = np.zeros(2 * Q)
        assert dhc.dhc_transform_pair(lat, z2.ctypes.data, T2.ctypes.data) == 0
        T1 = np.zeros(Q)
        weighted = dhc.dhc_transform(lat, 0, z2[: Q - 1].copy().ctypes.data, T1.ctypes.data)
        for lane in range(2):
            zl = z2[lane * (Q - 1):(lane + 1) * (Q - 1)]
            expect = m[1:].T @ zl
            if weighted:
                expect = expect * w
            assert np.max(np.abs(T2[lane * Q:(lane + 1) * Q] - expect)) < 1e-5 * max(1.0, np.max(np.abs(expect)))


def test_two_site_flat_variate_is_lane_by_lane(dhc):
    g = np.random.default_rng(5)
    words = np.concatenate([g.integers(0, 2**32, 4096, dtype=np.uint64),
                            [0, 1, 255, 256, 2**31 - 1, 2**31, 2**32 - 256, 2**32 - 1]]).astype(np.uint32)
    assert dhc.dhc_flat_pair_mismatches(words.ctypes.data, words.size // 2) == 0


@pytest.mark.parametrize("nmom", [2, 8, 18])
@pytest.mark.parametrize("dist", [0, 1])
def test_variates_match_oracle(orc, dhc, nmom, dist):
    for site, t in [(0, 0), (77, 99), (2**31 + 5, 2**33 + 7)]:
        z = np.zeros(nmom)
        dhc.dhc_variates(1, nmom, dist, 0xDEADBEEF12345, 9, site, t, z.ctypes.data)
        zo = orc.site_noise(0xDEADBEEF12345, 9, site, t, nmom, dist)
        assert np.max(np.abs(z - zo)) < 1e-14
        dhc.dhc_variates(0, nmom, dist, 0xDEADBEEF12345, 9, site, t, z.ctypes.data)
        assert np.max(np.abs(z - zo)) < 5e-6 * max(1.0, np.max(np.abs(zo)))


def test_multiply_shift_division_is_exact(dhc):
    """The batched kernel splits work-item indices with multiply-shift
    division; it must equal integer division for every divisor in
    [1, 2^31) and numerator in [0, 2^31): all small divisors, powers of two
    and their neighbours, random large ones, against edge and random
    numerators."""
    g = np.random.default_rng(3)
    d = set(range(1, 4097))
    for e in range(1, 31):
        d |= {2**e - 1, 2**e, 2**e + 1}
    d |= set(int(x) for x in g.integers(1, 2**31, 3000))
    d.add(2**31 - 1)
    d = np.array(sorted(d), dtype=np.uint32)
    n = set(range(0, 70000))
    for e in range(1, 32):
        n |= {2**e - 1, 2**e, 2**e + 1}
    n |= set(int(x) for x in g.integers(0, 2**31, 20000))
    n = np.array(sorted(x for x in n if x < 2**31), dtype=np.uint32)
    # multiples of each divisor and their neighbours, where rounding would show
    for dv in d[::37]:
        k = np.arange(1, 2**31 // int(dv), max(1, (2**31 // int(dv)) // 50), dtype=np.int64) * int(dv)
        extra = np.concatenate([k - 1, k, k + 1])
        extra = extra[(extra >= 0) & (extra < 2**31)].astype(np.uint32)
        assert dhc.dhc_fastdiv_mismatches(np.array([dv]).ctypes.data, 1, extra.ctypes.data, extra.size) == 0
    assert dhc.dhc_fastdiv_mismatches(d.ctypes.data, d.size, n.ctypes.data, n.size) == 0
