"""Every numeric constant of include/lbfd.h has the same value in the Python
binding, and the bench's names of the tile orders follow LBFD_WALK_* (host
only)."""
import os
import re

import bench
from paper_1606_07801_gb300 import lbfd as abi

HEADER = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include", "lbfd.h")


def _defines():
    out = {}
    for line in open(HEADER):
        m = re.match(r"#define\s+LBFD_(\w+)\s+\(?(-?\d+)\)?", line)
        if m:
            out[m.group(1)] = int(m.group(2))
    return out


def test_binding_constants_match_header():
    d = _defines()
    assert len(d) > 30
    skip = {"ABI_VERSION"}
    missing = []
    for name, value in d.items():
        if name in skip:
            continue
        if not hasattr(abi, name):
            missing.append(name)
            continue
        assert getattr(abi, name) == value, name
    assert not missing, missing


def test_bench_walk_names_follow_header():
    d = _defines()
    walks = {k[len("WALK_"):].lower(): v for k, v in d.items() if k.startswith("WALK_")}
    assert [bench.WALKS.index(n) for n in walks] == list(walks.values())
    assert len(bench.WALKS) == len(walks)
