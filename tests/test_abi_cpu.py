"""Host-side checks of the C ABI (no GPU needed): the library loads, exports
every function include/lbfd.h declares, its structs match the binding, its
argument checks reject bad input, and the tables compiled into the kernels
agree with the oracle's independent construction."""
import ctypes
import os
import re

import numpy as np
import pytest

import paper_1606_07801_gb300 as lb
from paper_1606_07801_gb300 import lbfd as abi

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    for h in os.listdir(os.path.join(ROOT, "include")):
        if h.endswith(".h"):
            text = open(os.path.join(ROOT, "include", h)).read()
            text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
            names |= set(re.findall(r"\b(lbfd_\w+)\s*\(", text))
    return names


def test_every_declared_symbol_is_exported_and_bound():
    lib = abi.load()
    declared = _declared()
    assert len(declared) >= 20
    for name in declared:
        assert hasattr(lib, name), name
        assert name in abi.SIGNATURES, name


def test_struct_layouts_match_binding():
    o, b, m = abi.lbfd_struct_sizes()
    assert o == ctypes.sizeof(abi.Options)
    assert b == ctypes.sizeof(abi.Obs)
    assert m == ctypes.sizeof(abi.Member)


def test_ensemble_rejects_bad_members_without_gpu():
    lib = abi.load()
    h = ctypes.c_void_p()
    bad = abi.make_members([dict(dims=(8, 8), tau=0.4, rho_mean=1.0, seed=1)])
    assert lib.lbfd_ensemble_create(ctypes.byref(h), lb.D2Q9, lb.F32, 0, 0, bad, 1, None) in (abi.EINVAL, abi.ECUDA)
    assert lib.lbfd_ensemble_create(ctypes.byref(h), lb.D2Q9, 9, 0, 0, bad, 1, None) == abi.EINVAL
    assert lib.lbfd_ensemble_create(ctypes.byref(h), lb.D2Q9, lb.F32, 0, 0, bad, 0, None) == abi.EINVAL
    assert lib.lbfd_ensemble_plan(None, 2, 1, 0, lb.WALK_CONTIGUOUS) == abi.EINVAL
    assert lib.lbfd_ensemble_query(None, None, None, None, None, None, None, None) == abi.EINVAL


def test_options_defaults():
    o = abi.lbfd_options_init()
    assert (o.lattice, o.precision, o.noise_mode, o.noise_dist, o.init, o.device) == (lb.D2Q9, lb.F32, 0, 0, 0, -1)
    assert list(o.dims) == [1, 1, 1] and o.tau == 1.0 and o.rho_mean == 1.0 and o.seed == 1


@pytest.mark.parametrize("kw,msg", [
    (dict(tau=0.5), "tau"),
    (dict(tau=float("nan")), "tau"),
    (dict(rho_mean=-1.0), "rho_mean"),
    (dict(lattice=7), "lattice"),
    (dict(precision=7), "precision"),
    (dict(noise_mode=9), "noise"),
    (dict(noise_dist=5), "distribution"),
    (dict(init=4), "init"),
    (dict(dims=(0, 4, 1)), "dimension"),
    (dict(dims=(4, 4, 2)), "beyond"),
    (dict(dims=(70000, 40000, 1)), "2^31"),
    (dict(dims=(4, 70000, 1)), "65535"),
    (dict(n_modes=17), "n_modes"),
])
def test_create_rejects_bad_options(kw, msg):
    o = abi.lbfd_options_init()
    o.dims[0], o.dims[1] = 8, 8
    for k, v in kw.items():
        if k == "dims":
            for a in range(3):
                o.dims[a] = v[a]
        else:
            setattr(o, k, v)
    with pytest.raises(abi.LbfdError) as e:
        abi.lbfd_create_ex(o)
    assert e.value.code == abi.EINVAL
    assert msg in str(e.value)


def test_null_handles_are_rejected():
    lib = abi.load()
    assert lib.lbfd_step(None, 1) == abi.EINVAL
    assert lib.lbfd_destroy(None) == abi.OK
    assert lib.lbfd_mass(None, None) == abi.EINVAL
    assert "null" in abi.last_error()


@pytest.mark.parametrize("lat", [lb.D1Q3, lb.D2Q9, lb.D3Q19])
def test_kernel_tables_match_oracle(orc, lat):
    """The moment basis compiled into the kernels (constexpr Gram-Schmidt /
    product form) equals the oracle's runtime Gram-Schmidt."""
    v, w, m = abi.lbfd_lattice_tables(lat)
    D, Q, ov, ow = orc.lattice(lat)
    assert np.array_equal(v, ov)
    assert np.max(np.abs(w - ow)) == 0.0
    assert np.max(np.abs(m - orc.basis(lat))) < 1e-14


def test_step_rejects_negative_n_without_gpu():
    lib = abi.load()
    assert lib.lbfd_step(ctypes.c_void_p(1), -1) == abi.EINVAL


@pytest.mark.parametrize("theta", [0.1, 0.2, 1.0 / 3.0, 0.45])
def test_d2q5_tables_match_oracle(orc, theta):
    """D2Q5 at free theta: the run-time weights and Gram-Schmidt basis the
    moment-space kernel receives equal the oracle's."""
    v, w, m = abi.lbfd_lattice_tables(lb.D2Q5, theta)
    D, Q, ov, ow = orc.lattice(orc.D2Q5, theta)
    assert np.array_equal(v, ov)
    assert np.max(np.abs(w - ow)) < 1e-16
    assert np.max(np.abs(m - orc.basis(orc.D2Q5, theta))) < 1e-14


@pytest.mark.parametrize("kw,code,msg", [
    (dict(lattice=3, theta=0.5), abi.EINVAL, "theta"),
    (dict(lattice=3, theta=-0.1), abi.EINVAL, "theta"),
    (dict(lattice=1, theta=0.25), abi.EINVAL, "theta"),
    (dict(lattice=3, precision=2), abi.ENOTSUP, "FP32 or FP64"),
    (dict(lattice=1, precision=3, tau_moments=[0, 0.9]), abi.ENOTSUP, "FP32 or FP64"),
    (dict(lattice=1, tau_moments=[0, 0.4]), abi.EINVAL, "tau_moments"),
])
def test_create_rejects_bad_paper_variants(kw, code, msg):
    o = abi.lbfd_options_init()
    o.dims[0], o.dims[1] = 8, 8
    for k, v in kw.items():
        if k == "tau_moments":
            for a, x in enumerate(v):
                o.tau_moments[a] = x
        else:
            setattr(o, k, v)
    with pytest.raises(abi.LbfdError) as e:
        abi.lbfd_create_ex(o)
    assert e.value.code == code and msg in str(e.value)


def test_lane_ops_probe_rejects_bad_arguments_without_gpu():
    lib = abi.load()
    x = np.zeros(4, np.float32)
    p = x.ctypes.data_as(ctypes.c_void_p)
    out = np.zeros(48, np.float32).ctypes.data_as(ctypes.c_void_p)
    assert lib.lbfd_lane_ops_probe(p, p, p, 3, out) == abi.EINVAL   # odd count
    assert lib.lbfd_lane_ops_probe(p, p, p, -2, out) == abi.EINVAL  # negative count
    assert lib.lbfd_lane_ops_probe(None, p, p, 4, out) == abi.EINVAL
    assert lib.lbfd_lane_ops_probe(p, p, p, 4, None) == abi.EINVAL
    assert lib.lbfd_lane_ops_probe(p, p, p, 0, out) == abi.OK        # nothing to do
