"""Every other step the one-launch-per-step kernels map their CTAs to the
mirror-image work blocks (StepArgs::sweep), so that a step starts on the rows
the previous one wrote last.  Which CTA updates which site must change
nothing: the same run with the alternation switched off (LBFD_STEP_SWEEP=0,
read once per process, hence a child process) gives the same state bit for
bit, on lattices above the many-steps-per-launch paths and over an odd
number of steps."""
import os
import subprocess
import sys

import numpy as np
import pytest

import paper_1606_07801_gb300 as lb
from paper_1606_07801_gb300 import synth

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

RUN = """
import sys
import numpy as np
sys.path.insert(0, {root!r})
import paper_1606_07801_gb300 as lb
from paper_1606_07801_gb300 import synth
lat, dims, prec = {lat}, {dims!r}, {prec}
Q, N = lb.Q_OF[lat], int(np.prod(dims))
f0 = synth.random_populations(Q, N, 40.0, 0.3, seed=5)
with lb.Simulation(lat, dims, 0.9, 40.0, 3, precision=prec, init=lb.INIT_NONE) as s:
    assert s.kernel(7) == {kernel!r}
    s.set_f(f0)
    s.step(7)
    np.save({out!r}, s.get_f())
"""


@pytest.mark.parametrize("lat,dims,prec,kernel", [
    (lb.D2Q9, (320, 200), lb.F32, "k_step_vec"),
    (lb.D2Q9, (301, 97), lb.F32, "k_step"),
    (lb.D3Q19, (48, 40, 36), lb.F32, "k_step_vec"),
    (lb.D3Q19, (32, 30, 28), lb.F32_F16, "k_step_vec"),
])
def test_reverse_sweep_changes_nothing(tmp_path, lat, dims, prec, kernel):
    out = str(tmp_path / "f_off.npy")
    code = RUN.format(root=ROOT, lat=lat, dims=dims, prec=prec, kernel=kernel, out=out)
    subprocess.run([sys.executable, "-c", code], env={**os.environ, "LBFD_STEP_SWEEP": "0"}, check=True,
                   timeout=300)
    f_off = np.load(out)
    Q, N = lb.Q_OF[lat], int(np.prod(dims))
    f0 = synth.random_populations(Q, N, 40.0, 0.3, seed=5)
    with lb.Simulation(lat, dims, 0.9, 40.0, 3, precision=prec, init=lb.INIT_NONE) as s:
        s.set_f(f0)
        s.step(7)
        f_on = s.get_f()
    assert np.array_equal(f_on, f_off)
