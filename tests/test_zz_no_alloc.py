"""GPU test of lbfd_mass_noalloc, the mass reduction for callers that cannot
allocate device memory (a framework that owns the GPU's memory, a fixed
budget, a loop that cannot pay for cudaMalloc).  It keeps its partial sums in
a fixed device array inside the library, so here it must agree with the
allocating lbfd_mass on the same state, on consecutive calls that reuse that
array.  This file sorts last so that a run stopping at the first failure has
already run every other test."""
import numpy as np
import pytest
import torch

import paper_1606_07801_gb300 as lb
from paper_1606_07801_gb300 import abi, synth

pytestmark = pytest.mark.gpu

REL = 1e-12  # the FP64 tolerance of the parity tests


@pytest.mark.parametrize("lat,dims,precision", [
    (lb.D2Q9, (300, 200), lb.F32),
    (lb.D3Q19, (24, 20, 18), lb.F64),
    (lb.D1Q3, (5000,), lb.F32),
    (lb.D2Q9, (2048, 2048), lb.F32),
    # exactly the capacity of the fixed scratch: every one of its slots is written and read
    (lb.D1Q3, (16777216,), lb.F32),
])
def test_noalloc_mass_matches_lbfd_mass_on_two_calls(lat, dims, precision):
    Q, N = lb.Q_OF[lat], int(np.prod(dims))
    f0 = synth.random_populations(Q, N, 40.0, 0.3, seed=N)
    out = torch.zeros(2, dtype=torch.float64, device="cuda")
    with lb.Simulation(lat, dims, 0.8, 40.0, 3, precision=precision, init=lb.INIT_NONE) as s:
        s.set_f(f0)
        s.step(3)
        want = []
        for k in range(2):
            want.append(s.mass())  # the allocating entry point
            f_dev, stream = s.state_device()
            abi.lbfd_mass_noalloc(lat, precision, f_dev, N, out.data_ptr() + 8 * k, stream)
            s.sync()
            s.step(2)  # the second call sees a different state
        torch.cuda.synchronize()
        got = out.cpu().numpy()
    assert want[0] != want[1]
    for k in range(2):
        assert abs(got[k] - want[k]) <= REL * abs(want[k]), (k, got[k], want[k])


def test_noalloc_rejects_sizes_beyond_its_scratch():
    out = torch.zeros(1, dtype=torch.float64, device="cuda")
    buf = torch.zeros(16, dtype=torch.float32, device="cuda")
    with pytest.raises(abi.LbfdError) as e:
        abi.lbfd_mass_noalloc(lb.D2Q9, lb.F32, buf.data_ptr(), 16777217, out.data_ptr())
    assert e.value.code == abi.EINVAL and "16777216" in str(e.value)
    with pytest.raises(abi.LbfdError):
        abi.lbfd_mass_noalloc(lb.D2Q9, lb.F32, buf.data_ptr(), 0, out.data_ptr())
