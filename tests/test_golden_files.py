"""The stored discord goldens (written by oracle/make_goldens.py from the FP64 oracle alone) are
complete, self-consistent and reproducible.

* Every medium (m = 262,144) and large (m = 2^20, n = 256, seeds 0-2) workload has one entry.
* Large entries: O1 (the brute-force definition) on the discord row equals O2's nn^2 bit for bit,
  and no sampled row's O1 value exceeds it.
* Two medium entries (the fastest to recompute) are re-derived with O2 here and must match exactly.
"""
import os

import pytest

import oracle
from paper_1901_00155_gb300 import synth

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def _read(name):
    rows = {}
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            if line.startswith("#") or not line.strip():
                continue
            parts = line.split()
            rows[parts[0]] = parts[1:]
    return rows


def test_medium_goldens_cover_the_workloads():
    rows = _read("discords_medium.txt")
    assert sorted(rows) == sorted(s.name() for s in synth.workloads_medium())
    for spec in synth.workloads_medium():
        m, n, idx, nn2, ev = rows[spec.name()]
        assert (int(m), int(n)) == (spec.m, spec.n)
        assert 0 <= int(idx) < spec.m - spec.n + 1 and float(nn2) > 0 and int(ev) > 0


def test_large_goldens_are_consistent():
    rows = _read("discords_large.txt")
    assert sorted(rows) == sorted(synth.workload_large(s).name() for s in (0, 1, 2))
    for seed in (0, 1, 2):
        spec = synth.workload_large(seed)
        m, n, idx, nn2, ev, o1, ns, smax, sseed = rows[spec.name()]
        assert (int(m), int(n)) == (spec.m, spec.n)
        assert float(o1) == float(nn2)          # O1 on the discord row == O2, bit for bit
        assert float(smax) <= float(nn2)        # no sampled row beats it
        assert int(ns) == 2048 and int(sseed) == 20240 + seed


@pytest.mark.parametrize("name", ["sine_m262144_n128_s0_flat+spike+phase", "sine_m262144_n512_s1_flat+spike+phase"])
def test_medium_golden_recomputes(name):
    spec = next(s for s in synth.workloads_medium() if s.name() == name)
    T, _ = synth.make_series(spec)
    m, n, idx, nn2, ev = _read("discords_medium.txt")[name]
    i, d2, _ = oracle.hotsax(T, spec.n)
    assert i == int(idx) and d2 == float(nn2)
