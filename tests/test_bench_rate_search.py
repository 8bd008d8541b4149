"""The served bench's search for the largest arrival rate that meets a p99
latency bound, run on the host against a fake trace runner whose p99 falls
as the rate falls (no GPU)."""
import types

import numpy as np

import bench
from paper_1606_07801_gb300 import synth


class _FakeAbi:
    """p99 = 200 / rate seconds; records the arrival times it was given."""

    def __init__(self):
        self.calls = []

    @staticmethod
    def make_request(*a, **k):
        return a

    def lbfd_server_run_trace(self, h, reqs, arrivals, sink_ptr, sink_bytes):
        span = float(arrivals[-1])
        rate = (len(arrivals) - 1) / span * 500.0 / self.base_rate
        self.calls.append(rate)
        lat = np.full(len(reqs), 200.0 / rate)
        return lat, span + 1.0


class _Srv:
    h = 1

    def close(self):
        pass


def _search(bound, rate=500.0, n=50):
    arr, _ = synth.served_trace(n, rate=500.0)
    fake = _FakeAbi()
    fake.base_rate = (n - 1) / float(arr[-1])
    args = types.SimpleNamespace(rate=rate, requests=n, rate_requests=n, p99_bound=bound)
    lb = types.SimpleNamespace(RESULT_RHO=1)
    sink = types.SimpleNamespace(data_ptr=lambda: 0, nbytes=0)
    return bench.served_rate_search(args, lb, fake, synth, sink, _Srv), fake


def test_rate_search_brackets_the_bound():
    res, fake = _search(2.0)          # p99 <= 2 s  <=>  rate >= 100 / s  (always true at 500)
    assert res["rate_per_s"] == 500.0 and len(fake.calls) == 1
    res, fake = _search(0.8)          # needs rate >= 250: 500 passes at once
    assert res["rate_per_s"] == 500.0
    res, _ = _search(0.5, rate=300.0)  # needs rate >= 400: 300 fails, 150 fails, ... nothing passes
    assert res["rate_per_s"] is None


def test_rate_search_bisects_between_halvings():
    # a p99 that grows with the rate: bound met only at low rates
    arr, _ = synth.served_trace(40, rate=500.0)

    class Abi(_FakeAbi):
        def lbfd_server_run_trace(self, h, reqs, arrivals, sink_ptr, sink_bytes):
            rate = 500.0 * float(arr[-1]) / float(arrivals[-1])
            self.calls.append(rate)
            return np.full(len(reqs), rate / 100.0), 1.0

    fake = Abi()
    args = types.SimpleNamespace(rate=500.0, requests=40, rate_requests=40, p99_bound=1.5)  # rate <= 150
    res = bench.served_rate_search(args, types.SimpleNamespace(RESULT_RHO=1), fake, synth,
                                   types.SimpleNamespace(data_ptr=lambda: 0, nbytes=0), _Srv)
    # halvings 500, 250 fail, 125 passes; three log-space bisections in (125, 250)
    assert np.allclose(fake.calls[:3], [500.0, 250.0, 125.0])
    assert len(fake.calls) == 6
    assert 125.0 <= res["rate_per_s"] <= 150.0
    assert all(t["p99_s"] <= 1.5 for t in res["tested"] if t["rate"] <= res["rate_per_s"])
