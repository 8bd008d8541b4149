"""Observables sampled inside the step (lbfd_options.sample_every).

With sample_every = s, lbfd_step adds the observables of f(x, t) at every
step t with t mod s == 0 (paper Sec. IV: sums of rho, rho^2, f_i, f_i f_j and
|rho(k)|^2, eqs. rhoth, dijexp, fkfk).  For the FP32-arithmetic formats this
runs in one pass with the step, plus the stage-2 kernel of the sample.  The
state must evolve bit for bit as without sampling; the accumulated sums
must match FP64 sums over the same stored states to what the fused path's
FP32 sums allow, well inside the bounds below (those of the separate
sampling pass's test):
  - D1Q3, D2Q9: each lane adds FP32 products over at most 128 sites, then an
    FP32 butterfly over the warp (5 more additions), then FP64;
  - D3Q19: products of TF32 parts (hi hi + hi lo + lo hi, FP32-accurate)
    added by the tensor cores in FP32 over at most 256 sites, folded in FP32
    over at most 2048, then FP64: about 100 roundings of 2^-24 in all.
The launch count shows that the fused path ran."""
import numpy as np
import pytest

import paper_1606_07801_gb300 as lb

pytestmark = pytest.mark.gpu

EVERY, STEPS = 5, 23  # samples at t = 0, 5, 10, 15, 20


def _modes(lat, dims):
    if len(dims) == 1:
        return [(1, 0, 0), (7, 0, 0)]
    return [(1, 0, 0), (2, 1, 0), (0, 1, 1), (3, 2, 1)][: 3 + (lat == lb.D3Q19)]


def _check_sums(ob, fs, rho_mean, modes, dims):
    N = fs[0].shape[1]
    n = len(fs) * N
    rho_sum = sum(f.sum() for f in fs)
    rho2_sum = sum((f.sum(0) ** 2).sum() for f in fs)
    f_sum = sum(f.sum(1) for f in fs)
    ff_sum = sum(f @ f.T for f in fs)
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
            sk += abs(np.fft.fftn(field)[k[2] % d3[2], k[1] % d3[1], k[0] % d3[0]]) ** 2
        assert abs(ob["sum_sk"][mi] - sk) <= 1e-4 * sk + 1e-3 * N * var_ref, (mi, k)


# every lattice here is above the size of the many-steps-per-launch paths
@pytest.mark.parametrize("lat,dims,prec", [
    (lb.D2Q9, (300, 261), lb.F32),
    (lb.D2Q9, (301, 100), lb.F32),       # odd Lx: one site per thread
    (lb.D2Q9, (256, 200), lb.F32_BF16),
    (lb.D3Q19, (40, 33, 21), lb.F32_F16),
    (lb.D3Q19, (48, 20, 16), lb.F32),
    (lb.D1Q3, (100001,), lb.F32),
])
def test_fused_sampling_matches_fp64_sums_and_keeps_the_state(lat, dims, prec):
    modes = _modes(lat, dims)
    rho_mean = 30.0
    kw = dict(precision=prec, modes=modes)
    # the same run sampled inside the step ...
    with lb.Simulation(lat, dims, 0.8, rho_mean, 4, sample_every=EVERY, **kw) as s:
        l0 = lb.abi.lbfd_kernel_launches()
        s.step(STEPS)
        s.sync()
        launches = lb.abi.lbfd_kernel_launches() - l0
        ob = s.observables()
        fa = s.get_f()
    # ... and stepped one step at a time, reading the state at the sampled steps
    fs = []
    with lb.Simulation(lat, dims, 0.8, rho_mean, 4, **kw) as s:
        for t in range(STEPS):
            if t % EVERY == 0:
                fs.append(s.get_f())
            s.step(1)
        fb = s.get_f()
    assert np.array_equal(fa, fb)
    assert ob["n_samples"] == len(fs) == 5
    # one step kernel per step plus one stage-2 kernel per sample: no separate pass
    assert launches == STEPS + len(fs)
    _check_sums(ob, fs, rho_mean, modes, dims)


@pytest.mark.parametrize("lat,dims,prec", [
    (lb.D1Q3, (256,), lb.F32),     # the many-steps-per-launch path, split at the sampled steps
    (lb.D2Q9, (40, 33), lb.F64),   # FP64 storage samples by its own FP64 pass
    (lb.D2Q9, (30, 4), lb.F32),    # a work block narrower than 256 threads: the separate pass
])
def test_sampling_that_runs_as_a_separate_pass(lat, dims, prec):
    modes = _modes(lat, dims)
    with lb.Simulation(lat, dims, 0.9, 20.0, 6, precision=prec, modes=modes, sample_every=EVERY) as s:
        s.step(STEPS)
        ob = s.observables()
        fa = s.get_f()
    with lb.Simulation(lat, dims, 0.9, 20.0, 6, precision=prec, modes=modes) as s:
        for t in range(STEPS):
            if t % EVERY == 0:
                s.sample()
            s.step(1)
        want = s.observables()
        fb = s.get_f()
    assert np.array_equal(fa, fb)
    assert ob["n_samples"] == want["n_samples"] == 5
    for key in ("sum_rho", "sum_rho2"):
        assert ob[key] == want[key]
    assert np.array_equal(ob["sum_f"], want["sum_f"]) and np.array_equal(ob["sum_ff"], want["sum_ff"])
    assert np.array_equal(ob["sum_sk"], want["sum_sk"])


def test_stage_two_on_the_side_stream_is_joined():
    """Stage 2 of a sampled step runs on the handle's side stream; every
    reader of the accumulators, and the next sampled step, wait for it.
    Reading the observables right after lbfd_step (no sync) and after a sync
    must give the same sums, and resetting between samples must drop only
    the samples before it."""
    dims, prec = (300, 261), lb.F32
    kw = dict(precision=prec, modes=_modes(lb.D2Q9, dims), sample_every=1)
    with lb.Simulation(lb.D2Q9, dims, 0.8, 30.0, 4, **kw) as s:
        s.step(7)
        a = s.observables()             # no sync before: joins the side stream
        s.sync()
        b = s.observables()
        s.reset_obs()                   # after the join, before the next samples
        s.step(3)
        c = s.observables()
    assert a["n_samples"] == b["n_samples"] == 7 and c["n_samples"] == 3
    assert a["sum_rho"] == b["sum_rho"] and np.array_equal(a["sum_ff"], b["sum_ff"])
    with lb.Simulation(lb.D2Q9, dims, 0.8, 30.0, 4, **kw) as s:
        s.step(7)
        s.reset_obs()
        s.step(3)
        d = s.observables()
    assert c["sum_rho"] == d["sum_rho"] and np.array_equal(c["sum_ff"], d["sum_ff"])


STAGED_RUN = """
import sys
sys.path.insert(0, {root!r})
import paper_1606_07801_gb300 as lb
from tests.test_gpu_fused_sampling import test_fused_sampling_matches_fp64_sums_and_keeps_the_state as check
check({lat}, {dims!r}, {prec})
print("staged sampled steps ok")
"""


@pytest.mark.parametrize("lat,dims,prec", [
    (lb.D3Q19, (40, 33, 21), lb.F32_F16),
    (lb.D3Q19, (48, 40, 36), lb.F32_BF16),  # both above the many-steps-per-launch paths
])
def test_staged_sampled_steps_on_request(lat, dims, prec):
    """LBFD_SAMPLE_STAGED = 1 (read once per process, hence a child process)
    samples D3Q19 16-bit lattices in the staged kernel: the same checks as
    the default register-pull path."""
    import os
    import subprocess
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    env = dict(os.environ, LBFD_SAMPLE_STAGED="1")
    r = subprocess.run([sys.executable, "-c", STAGED_RUN.format(root=root, lat=lat, dims=dims, prec=prec)],
                       env=env, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stdout + r.stderr
    assert "staged sampled steps ok" in r.stdout
