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


def _lane_operands(n, seed):
    """Operands that cover what rounding can distinguish: ordinary values at
    several scales, subnormals, signed zeros, infinities, NaN, near-overflow
    and exact cancellation, mixed so that the two lanes of a packed
    instruction see different kinds."""
    g = np.random.default_rng(seed)
    kinds = [
        lambda m: g.standard_normal(m),
        lambda m: g.standard_normal(m) * 1e-30,
        lambda m: g.standard_normal(m) * 1e30,
        lambda m: g.uniform(-1, 1, m) * 1e-38,       # subnormal products and sums
        lambda m: g.choice([1e-45, -1e-45, 1.4e-40, -2.9e-39], m),
        lambda m: g.choice([0.0, -0.0], m),
        lambda m: g.choice([np.inf, -np.inf, np.nan, 3.4e38, -3.4e38], m),
    ]
    cols = []
    for _ in range(3):
        k = g.integers(0, len(kinds), n)
        v = np.empty(n)
        for j, f in enumerate(kinds):
            sel = k == j
            v[sel] = f(int(sel.sum()))
        cols.append(v.astype(np.float32))
    a, b, c = cols
    # exact cancellation: c = -(a b) and b = a at some places
    with np.errstate(all="ignore"):
        c[::7] = -(a[::7] * b[::7])
    b[::5] = a[::5]
    return a, b, c


def _same(x, y):
    both_nan = np.isnan(x) & np.isnan(y)
    return np.all(both_nan | (x.view(np.uint32) == y.view(np.uint32)))


def test_packed_lane_operations_round_as_one_value_at_a_time():
    """add/sub/mul/fma.rn.f32x2 against the scalar operations, bit for bit,
    with subnormals kept (no flush to zero) and a product added to a third
    value rounded twice in both forms (no fusion into an FMA)."""
    n = 1 << 16
    a, b, c = _lane_operands(n, 2024)
    r = abi.lbfd_lane_ops_probe(a, b, c)
    for op in range(6):
        assert _same(r[op, 0], r[op, 1]), f"operation {op}: packed and one-at-a-time forms differ"
    with np.errstate(all="ignore"):
        ref = [a + b, a - b, a * b, None, (a * b) + c, c - (a * b)]
    for op in (0, 1, 2, 4, 5):
        assert _same(r[op, 0], ref[op].astype(np.float32)), f"operation {op} differs from IEEE FP32"
    # a product added to c rounds twice: somewhere it must differ from the fused form
    finite = np.isfinite(r[3, 0]) & np.isfinite(r[4, 0])
    assert np.any(r[3, 0][finite] != r[4, 0][finite])


def test_lane_ops_probe_rejects_bad_sizes():
    with pytest.raises(lb.LbfdError):
        abi.lbfd_lane_ops_probe(np.zeros(3, np.float32), np.zeros(3, np.float32), np.zeros(3, np.float32))
