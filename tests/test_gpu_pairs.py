"""The paired collision: the vector step kernel updates two neighbouring
sites at once on the packed FP32 instructions (add/mul/fma.rn.f32x2) where
that is faster, and one at a time elsewhere.

Each packed lane rounds as the scalar instruction does and the collision is
one source over both forms, so a lattice must evolve bit for bit the same as
under the one-site-per-thread kernel.  Shapes take the vector kernel at four
sites per thread (Lx a multiple of 4) and at two (Lx = 2 mod 4), for every
lattice, storage format and noise variant, at low density so that the clamp
of the local noise amplitude is exercised too."""
import numpy as np
import pytest

import paper_1606_07801_gb300 as lb
from paper_1606_07801_gb300 import abi, synth

pytestmark = pytest.mark.gpu


def _run(lat, dims, precision, kernel, f0, steps, rho, mode, dist, tau=1.3):
    with lb.Simulation(lat, dims, tau, rho, 11, precision=precision, noise_mode=mode, noise_dist=dist,
                       init=lb.INIT_NONE, lattice_id=2, step_kernel=kernel) as s:
        assert s.kernel(1) == abi.KERNEL_NAMES[kernel]
        s.set_f(f0)
        for _ in range(steps):
            s.step(1)
        return s.get_f()


NOISE = [(lb.NOISE_LOCAL, lb.GAUSSIAN), (lb.NOISE_GLOBAL, lb.GAUSSIAN), (lb.NOISE_LOCAL, lb.UNIFORM),
         (lb.NOISE_OFF, lb.GAUSSIAN)]


@pytest.mark.parametrize("mode,dist", NOISE)
@pytest.mark.parametrize("precision", [lb.F32, lb.F32_F16, lb.F32_BF16, lb.F64])
@pytest.mark.parametrize("lat,dims", [
    (lb.D2Q9, (128, 20)),     # four sites per thread
    (lb.D2Q9, (130, 17)),     # two sites per thread
    (lb.D3Q19, (32, 6, 5)),
    (lb.D3Q19, (34, 5, 4)),
    (lb.D1Q3, (4096,)),
    (lb.D1Q3, (4098,)),
])
def test_vector_kernel_bit_identical_to_one_site_per_thread(lat, dims, precision, mode, dist):
    Q, N = lb.Q_OF[lat], int(np.prod(dims))
    rho = 0.9
    f0 = synth.random_populations(Q, N, rho, 0.5, seed=N + 3 * Q)
    a = _run(lat, dims, precision, lb.KERNEL_VEC, f0, 4, rho, mode, dist)
    b = _run(lat, dims, precision, lb.KERNEL_SCALAR, f0, 4, rho, mode, dist)
    assert np.array_equal(a, b)
    assert not np.array_equal(a, f0)
