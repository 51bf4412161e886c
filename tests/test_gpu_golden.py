"""The discord search on the GPU against stored oracle goldens, for all three arithmetic forms.

The goldens (tests/golden/discords_medium.txt, discords_large.txt) were written by
oracle/make_goldens.py from the FP64 oracle alone: O2 (the CPU HOTSAX of Algorithms 2-4, bitwise
equal to the brute-force definition by construction and by the O1 == O2 pins) on the twelve
m = 262,144 workloads and on the m = 2^20, n = 256 random walks for seeds 0-2, the latter also
checked against O1 (Section 2.1's definition, brute force) on the discord row and on a seeded
sample of rows.

Bars (the required accuracy of each form):
  * FP32 form: the oracle's index, or a row whose oracle nn distance is within 1e-4 relative of
    the oracle's maximum; nn_distance within 1e-4 relative.
  * Tensor-core forms (FP16 / BF16 Gram tiles, FP64 rescoring): the oracle's index (another index
    only where the oracle's own distances tie within 1e-12 relative); nn_distance within 1e-6.
"""
import math
import os

import pytest

import oracle
from paper_1901_00155_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")
FORMS = ["fp32", "tc_fp16", "tc_bf16"]


def _read(name):
    rows = {}
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            if line.startswith("#") or not line.strip():
                continue
            parts = line.split()
            rows[parts[0]] = {"m": int(parts[1]), "n": int(parts[2]), "index": int(parts[3]), "nn2": float(parts[4])}
    return rows


MEDIUM = _read("discords_medium.txt")
LARGE = _read("discords_large.txt")


def _search(T, n, prec):
    import paper_1901_00155_gb300 as dd
    with dd.Plan(T.size, n, prec) as p:
        return p.find_discord(torch.from_numpy(T).cuda())


def _check(T, n, prec, r, ref):
    d_ref = math.sqrt(ref["nn2"])
    if prec == "fp32":
        assert r.nn_distance == pytest.approx(d_ref, rel=1e-4, abs=1e-6), (prec, r, ref)
        if r.index != ref["index"]:
            nn, _ = oracle.nn_rows(T, n, [r.index])
            assert math.sqrt(nn[0]) == pytest.approx(d_ref, rel=1e-4, abs=1e-6), (prec, r, ref)
    else:
        assert r.exact
        assert r.nn_distance == pytest.approx(d_ref, rel=1e-6, abs=1e-9), (prec, r, ref)
        if r.index != ref["index"]:
            nn, _ = oracle.nn_rows(T, n, [r.index])
            assert nn[0] == pytest.approx(ref["nn2"], rel=1e-12, abs=1e-15), (prec, r, ref)
            assert r.index > ref["index"] or nn[0] != ref["nn2"]


def test_goldens_cover_the_workloads():
    assert sorted(MEDIUM) == sorted(s.name() for s in synth.workloads_medium())
    assert sorted(LARGE) == sorted(synth.workload_large(s).name() for s in (0, 1, 2))


@pytest.mark.parametrize("prec", FORMS)
@pytest.mark.parametrize("spec", synth.workloads_medium(), ids=lambda s: s.name())
def test_medium_workloads(spec, prec):
    T, _ = synth.make_series(spec)
    ref = MEDIUM[spec.name()]
    assert (ref["m"], ref["n"]) == (spec.m, spec.n)
    _check(T, spec.n, prec, _search(T, spec.n, prec), ref)


@pytest.mark.parametrize("prec", FORMS)
@pytest.mark.parametrize("seed", [0, 1, 2])
def test_large_workloads(seed, prec):
    """m = 2^20, n = 256: the benchmark's configuration and its two sister seeds."""
    spec = synth.workload_large(seed)
    T, _ = synth.make_series(spec)
    ref = LARGE[spec.name()]
    assert (ref["m"], ref["n"]) == (spec.m, spec.n)
    _check(T, spec.n, prec, _search(T, spec.n, prec), ref)
