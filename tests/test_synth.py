"""The seeded input generators (shared by the oracle tests, the GPU parity tests and the bench).

They hold none of the method's arithmetic; these checks pin the workload recipes the bench and
DESIGN state: sizes, ranges, validity of every (m, n) pair and determinism under the seed."""
import math

import numpy as np

from paper_1901_00155_gb300 import synth


def test_series_are_deterministic_and_finite():
    for spec in (synth.workload_small(), synth.workloads_medium()[3], synth.SeriesSpec("sine", 5000, 64, 9, ("phase",))):
        a, offs_a = synth.make_series(spec)
        b, offs_b = synth.make_series(spec)
        assert a.dtype == np.float32 and a.size == spec.m
        assert np.array_equal(a, b) and offs_a == offs_b
        assert np.isfinite(a).all()
        # anomalies sit at least n from the ends and 2n from each other
        offs = sorted(offs_a)
        assert all(o >= spec.n and o + spec.n <= spec.m for o in offs)
        assert all(b_ - a_ >= 2 * spec.n for a_, b_ in zip(offs, offs[1:]))


def test_batch_workload_recipe():
    specs = synth.workload_batch(seed=0, count=512)
    assert len(specs) == 512
    assert all(2048 <= s.m <= 65536 for s in specs)
    assert {s.n for s in specs} <= {64, 128, 256}
    assert all(s.m - s.n + 1 >= 2 * s.n for s in specs)  # every series has non-self matches
    assert {s.kind for s in specs} == {"rw", "sine"}
    assert all(len(s.anomalies) == 1 for s in specs)
    # log-uniform: the median length sits near the geometric mean of the range
    med = float(np.median([s.m for s in specs]))
    assert 0.7 * math.sqrt(2048 * 65536) < med < 1.4 * math.sqrt(2048 * 65536)
    assert [s.seed for s in synth.workload_batch(seed=0, count=512)] == [s.seed for s in specs]


def test_serving_trace_recipe():
    trace = synth.serving_requests(seed=0, rate_per_s=200.0, duration_s=5.0)
    t = np.array([x for x, _ in trace])
    assert np.all(np.diff(t) > 0) and t[-1] < 5.0
    # Poisson(200/s) over 5 s: about 1000 arrivals (a 4-sigma band)
    assert abs(len(trace) - 1000) < 4 * math.sqrt(1000)
    specs = [s for _, s in trace]
    assert all(4096 <= s.m <= (1 << 20) for s in specs)
    assert {s.n for s in specs} <= {64, 128, 256, 512, 1024}
    assert all(s.m - s.n + 1 >= 2 * s.n for s in specs)
    assert synth.serving_requests(seed=0, rate_per_s=200.0, duration_s=5.0) == trace
