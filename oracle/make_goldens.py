"""Writes the stored discord goldens under tests/golden/ -- TEST INFRASTRUCTURE.

Every value it writes comes from the FP64 oracle in this directory, run on the
seeded synthetic series of ``paper_1901_00155_gb300.synth`` (the generators
hold none of the method's arithmetic).  Nothing here touches the CUDA library.

Output files (one line per series, whitespace separated):

* ``tests/golden/discords_medium.txt``: the twelve m = 262,144 workloads
  (random walk and sine + noise, n in {128, 256, 512}, seeds 0 and 1, three
  anomalies each).  Columns: name, m, n, index, nn2, evaluated_pairs, where
  (index, nn2) is O2 -- the CPU HOTSAX of Algorithms 2-4 -- and nn2 is the
  squared nearest-neighbour distance on the globally normalised series (Eq. 2).
* ``tests/golden/discords_large.txt``: the m = 2^20, n = 256 random walks
  (five anomalies) for seeds 0, 1, 2.  Columns: name, m, n, index, nn2,
  evaluated_pairs, o1_nn2_of_index, sample_rows, sample_max_nn2,
  sample_seed.  o1_nn2_of_index is O1 (the Section 2.1 definition, brute
  force over every column) on the discord row, and must equal O2's nn2 bit
  for bit; sample_max_nn2 is the largest O1 value over ``sample_rows``
  seeded random rows (numpy default_rng(sample_seed)), which must not exceed
  nn2.  The full O1 profile at this size costs about N^2 n = 2.8e14 FP64
  multiply-adds in dependent chains (half a day on eight cores), so the
  brute-force definition is applied to the discord row and the sample only.

Run: ``python oracle/make_goldens.py [--only medium|large]`` from the
repository root.  Takes about half an hour on eight cores.
"""
from __future__ import annotations

import argparse
import os
import sys
import time

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_ROOT = os.path.dirname(_HERE)
if _ROOT not in sys.path:
    sys.path.insert(0, _ROOT)

import oracle  # noqa: E402
from paper_1901_00155_gb300 import synth  # noqa: E402

GOLDEN = os.path.join(_ROOT, "tests", "golden")
SAMPLE_ROWS = 2048
SAMPLE_SEED = 20240


def _medium(path: str) -> None:
    lines = ["# name m n index nn2 evaluated_pairs  (O2, CPU HOTSAX, FP64; written by oracle/make_goldens.py)"]
    for spec in synth.workloads_medium():
        T, _ = synth.make_series(spec)
        t0 = time.time()
        i, d2, ev = oracle.hotsax(T, spec.n)
        print(f"{spec.name()}: {i} {d2!r} ({time.time() - t0:.1f} s)", flush=True)
        lines.append(f"{spec.name()} {spec.m} {spec.n} {i} {d2!r} {ev}")
    with open(path, "w") as f:
        f.write("\n".join(lines) + "\n")


def _large(path: str) -> None:
    lines = ["# name m n index nn2 evaluated_pairs o1_nn2_of_index sample_rows sample_max_nn2 sample_seed "
             "(O2 + O1 checks, FP64; written by oracle/make_goldens.py)"]
    for seed in (0, 1, 2):
        spec = synth.workload_large(seed)
        T, _ = synth.make_series(spec)
        N = T.size - spec.n + 1
        t0 = time.time()
        i, d2, ev = oracle.hotsax(T, spec.n)
        t1 = time.time()
        o1, _ = oracle.nn_rows(T, spec.n, [i])
        if o1[0] != d2:
            raise SystemExit(f"O1 and O2 disagree on the discord row of {spec.name()}: {o1[0]!r} vs {d2!r}")
        rows = np.random.default_rng(SAMPLE_SEED + seed).integers(0, N, size=SAMPLE_ROWS)
        nns, _ = oracle.nn_rows(T, spec.n, rows)
        smax = float(nns.max())
        if smax > d2:
            raise SystemExit(f"a sampled row beats the O2 discord of {spec.name()}: {smax!r} > {d2!r}")
        print(f"{spec.name()}: {i} {d2!r} O2 {t1 - t0:.1f} s, O1 checks {time.time() - t1:.1f} s", flush=True)
        lines.append(f"{spec.name()} {spec.m} {spec.n} {i} {d2!r} {ev} {float(o1[0])!r} {SAMPLE_ROWS} {smax!r} "
                     f"{SAMPLE_SEED + seed}")
    with open(path, "w") as f:
        f.write("\n".join(lines) + "\n")


def main() -> None:
    ap = argparse.ArgumentParser()
    ap.add_argument("--only", choices=["medium", "large"])
    a = ap.parse_args()
    if a.only in (None, "medium"):
        _medium(os.path.join(GOLDEN, "discords_medium.txt"))
    if a.only in (None, "large"):
        _large(os.path.join(GOLDEN, "discords_large.txt"))


if __name__ == "__main__":
    main()
