"""The shared-memory staged step kernel (bulk copies into shared memory on an
mbarrier, pull from there, bulk stores back).

It runs the same per-site collision as the register-pull kernels, so a
lattice must evolve bit for bit the same under either.  Shapes cover tiles
that end inside a row (Lx not a multiple of the tile width), rows exactly one
16-byte chunk wide (both halo chunks wrap onto the row itself), sides of 1
and 2 in y and z, every storage format and every noise variant; one step per
call keeps the lattices off the many-steps-per-launch paths."""
import numpy as np
import pytest

import paper_1606_07801_gb300 as lb
from paper_1606_07801_gb300 import abi, synth

pytestmark = pytest.mark.gpu


def _run(lat, dims, precision, kernel, f0, steps, rho, tau=0.8, mode=lb.NOISE_LOCAL, dist=lb.GAUSSIAN, seed=3):
    with lb.Simulation(lat, dims, tau, rho, seed, precision=precision, noise_mode=mode, noise_dist=dist,
                       init=lb.INIT_NONE, lattice_id=5, step_kernel=kernel) as s:
        assert s.kernel(1) == abi.KERNEL_NAMES[kernel]
        s.set_f(f0)
        for _ in range(steps):
            s.step(1)
        return s.get_f()


@pytest.mark.parametrize("lat,dims,precision", [
    (lb.D2Q9, (64, 48), lb.F32),        # one tile per row, shorter than the tile width
    (lb.D2Q9, (1040, 37), lb.F32),      # two full tiles and a 16-site tile per row
    (lb.D2Q9, (4, 300), lb.F32),        # a row is one 16-byte chunk
    (lb.D2Q9, (258, 20), lb.F64),       # FP64: a 2-site tile at the end of each row
    (lb.D2Q9, (520, 9), lb.F32_F16),    # 16-bit: an 8-site tile at the end of each row
    (lb.D2Q9, (48, 33), lb.F32_BF16),
    (lb.D2Q9, (512, 2), lb.F32),        # Ly = 2: both y-neighbours are the same row
    (lb.D3Q19, (36, 20, 18), lb.F32),
    (lb.D3Q19, (130, 6, 5), lb.F64),
    (lb.D3Q19, (264, 4, 3), lb.F32_F16),
    (lb.D3Q19, (16, 2, 1), lb.F32_BF16),
    (lb.D3Q19, (8, 1, 2), lb.F32),
    (lb.D1Q3, (100000,), lb.F32),       # 195 full tiles and a 160-site tile
    (lb.D1Q3, (5002,), lb.F64),
])
def test_staged_bit_identical_to_register_pull(lat, dims, precision):
    Q, N = lb.Q_OF[lat], int(np.prod(dims))
    rho = 40.0
    f0 = synth.random_populations(Q, N, rho, 0.3, seed=N + Q)
    ref_kernel = lb.KERNEL_VEC if dims[0] % 2 == 0 else lb.KERNEL_SCALAR
    a = _run(lat, dims, precision, lb.KERNEL_STAGED, f0, 7, rho)
    b = _run(lat, dims, precision, ref_kernel, f0, 7, rho)
    assert np.array_equal(a, b)
    assert not np.array_equal(a, f0)


@pytest.mark.parametrize("mode,dist", [(lb.NOISE_GLOBAL, lb.GAUSSIAN), (lb.NOISE_OFF, lb.GAUSSIAN),
                                       (lb.NOISE_LOCAL, lb.UNIFORM), (lb.NOISE_GLOBAL, lb.UNIFORM)])
@pytest.mark.parametrize("lat,dims", [(lb.D2Q9, (520, 12)), (lb.D3Q19, (24, 10, 7))])
def test_staged_noise_variants_bit_identical(lat, dims, mode, dist):
    Q, N = lb.Q_OF[lat], int(np.prod(dims))
    f0 = synth.random_populations(Q, N, 0.8, 0.5, seed=7)  # low density: the clamp is exercised
    a = _run(lat, dims, lb.F32, lb.KERNEL_STAGED, f0, 5, 0.8, tau=1.3, mode=mode, dist=dist)
    b = _run(lat, dims, lb.F32, lb.KERNEL_VEC, f0, 5, 0.8, tau=1.3, mode=mode, dist=dist)
    assert np.array_equal(a, b)


def test_staged_against_oracle_many_steps(orc):
    """Element-wise parity with the FP64 oracle over 300 steps of one launch
    per step (FP64 and FP32 storage)."""
    lat, dims, tau, rho = lb.D2Q9, (264, 40), 0.8, 60.0
    Q, N = 9, 264 * 40
    f0 = synth.random_populations(Q, N, rho, 0.3, seed=17)
    want = orc.run(lat, dims, f0, 300, tau, orc.NOISE_LOCAL, orc.GAUSSIAN, rho_eq=rho, seed=3, lattice_id=5)
    for precision, tol in ((lb.F64, 1e-12), (lb.F32, 2e-5)):
        got = _run(lat, dims, precision, lb.KERNEL_STAGED, f0, 300, rho)
        assert np.max(np.abs(got - want)) <= tol * rho


@pytest.mark.parametrize("lat,dims,precision", [(lb.D2Q9, (66, 10), lb.F32), (lb.D2Q9, (12, 10), lb.F32_F16),
                                                (lb.D3Q19, (7, 4, 4), lb.F64)])
def test_staged_requirements(lat, dims, precision):
    """Rows that do not start on 16-byte boundaries cannot take the staged
    kernel: asking for it is refused, and the library's own choice falls back
    to a register-pull kernel."""
    with pytest.raises(abi.LbfdError) as e:
        lb.Simulation(lat, dims, 0.8, 10.0, 1, precision=precision, step_kernel=lb.KERNEL_STAGED)
    assert e.value.code == abi.EINVAL
    with lb.Simulation(lat, dims, 0.8, 10.0, 1, precision=precision) as s:
        assert s.kernel(1) in ("k_step_vec", "k_step")


def test_staged_wait_that_runs_out_is_reported():
    """A bounded wait of the staged kernel that runs out (here: the first tile
    of every CTA waits for bytes no copy delivers) stops the kernel after
    about a second and is reported as LBFD_ETIMEOUT by the next synchronous
    call; the device stays usable."""
    dims = (1024, 64)
    with lb.Simulation(lb.D2Q9, dims, 0.8, 10.0, 1, step_kernel=lb.KERNEL_STAGED, wait_test_bytes=16) as s:
        s.step(1)
        with pytest.raises(abi.LbfdError) as e:
            s.sync()
        assert e.value.code == abi.ETIMEOUT
        s.sync()  # reported once
    # a normal simulation runs afterwards on the same device
    f0 = synth.random_populations(9, 1024 * 64, 10.0, 0.2, seed=2)
    a = _run(lb.D2Q9, dims, lb.F32, lb.KERNEL_STAGED, f0, 3, 10.0)
    b = _run(lb.D2Q9, dims, lb.F32, lb.KERNEL_VEC, f0, 3, 10.0)
    assert np.array_equal(a, b)
