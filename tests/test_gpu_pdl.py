"""Programmatic dependent launch changes only when a step's blocks start, not
what they compute.  The launch attribute is read once per process
(LBFD_STEP_PDL), so two child processes run the same lattices with it off and
on, and their results must agree bit for bit.  The lattices are larger than
the small-lattice path takes, so every step is one step-kernel launch; they
cover the two-site kernel (even Lx) and the one-site kernel (odd Lx)."""
import os
import subprocess
import sys

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

SCRIPT = """
import sys
import numpy as np
sys.path.insert(0, {root!r})
import paper_1606_07801_gb300 as lb
out = []
for lat, dims, prec in [(lb.D2Q9, (256, 130), lb.F32), (lb.D3Q19, (64, 40, 33), lb.F32),
                        (lb.D2Q9, (193, 128), lb.F64), (lb.D3Q19, (48, 32, 32), lb.F32_F16)]:
    with lb.Simulation(lat, dims, 0.8, 30.0, 5, precision=prec) as s:
        s.step(25)
        out.append(s.get_f())
np.savez({path!r}, *out)
"""


def _run(pdl: str, path: str) -> list:
    env = dict(os.environ, LBFD_STEP_PDL=pdl)
    subprocess.run([sys.executable, "-c", SCRIPT.format(root=ROOT, path=path)], env=env, check=True, timeout=600)
    with np.load(path) as z:
        return [z[k] for k in sorted(z.files, key=lambda k: int(k.split("_")[1]))]


def test_dependent_launch_is_bit_identical(tmp_path):
    off = _run("0", str(tmp_path / "off.npz"))
    on = _run("1", str(tmp_path / "on.npz"))
    assert len(off) == len(on) == 4
    for a, b in zip(off, on):
        assert a.dtype == b.dtype and np.array_equal(a, b)
