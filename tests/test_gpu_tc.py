"""Tensor-core Gram form (tcgen05, FP16 / BF16 operands, FP32 accumulation,
per-row error bound, FP64 rescoring) against the FP64 oracle through the C ABI.

Tolerance: the discord index must equal the oracle's (a different index is
accepted only where the oracle's own distances tie within 1e-12 relative),
and nn_distance must be within 1e-6 relative of the oracle's.
"""
import math

import numpy as np
import pytest

import oracle
from paper_1901_00155_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

RTOL = 1e-6
TIE = 1e-12
PRECS = ["tc_fp16", "tc_bf16"]


def _dd():
    import paper_1901_00155_gb300 as dd
    return dd


def _search(T, n, prec, **opts):
    dd = _dd()
    with dd.Plan(T.size, n, prec, **opts) as p:
        return p.find_discord(torch.from_numpy(np.ascontiguousarray(T)).cuda())


def _check(T, n, r, i_ref, d2_ref):
    d_ref = math.sqrt(d2_ref)
    assert r.exact
    assert r.nn_distance == pytest.approx(d_ref, rel=RTOL, abs=1e-9), (r, i_ref, d_ref)
    if r.index != i_ref:
        nn, _ = oracle.nn_rows(T, n, [r.index])
        assert nn[0] == pytest.approx(d2_ref, rel=TIE, abs=1e-15), (r, i_ref, d_ref)
        assert r.index > i_ref or nn[0] != d2_ref


@pytest.mark.parametrize("prec", PRECS)
def test_small_random_sweep(prec):
    rng = np.random.default_rng(1234)
    for trial in range(40):
        n = int(rng.choice([1, 2, 3, 8, 16, 33, 64, 100, 256]))
        m = int(rng.integers(3 * n - 1, 3 * n + 900))
        T = synth.random_small(rng, m)
        r = _search(T, n, prec)
        i_ref, d2_ref = oracle.discord_brute(T, n)
        _check(T, n, r, i_ref, d2_ref)


@pytest.mark.parametrize("prec", PRECS)
def test_small_workload(prec):
    spec = synth.workload_small()
    T, _ = synth.make_series(spec)
    r = _search(T, spec.n, prec)
    i_ref, d2_ref = oracle.discord_brute(T, spec.n)
    _check(T, spec.n, r, i_ref, d2_ref)


@pytest.mark.parametrize("prec", PRECS)
@pytest.mark.parametrize("n,m", [(16, 3000), (64, 64 * 3 - 1), (128, 128 * 3 + 77), (200, 5000)])
def test_profile_within_bound(prec, n, m):
    """Gram-form profile values stay within a relative error far below the
    fp16 / bf16 unit (their rigorous per-row bound is checked on the device)."""
    dd = _dd()
    rng = np.random.default_rng(n + m)
    T = np.cumsum(rng.standard_normal(m)).astype(np.float32)
    with dd.Plan(m, n, prec) as p:
        prof = p.nn_profile(torch.from_numpy(T).cuda()).cpu().numpy()
    ref = oracle.nn_profile(T, n)
    u = 2.0 ** -11 if prec == "tc_fp16" else 2.0 ** -8
    # |D - d^2| <= ~4 u sqrt(c_i c_j) + ...; c <= S2 of a window of t^
    _, c = oracle.window_stats(T, n)
    tol = 8 * u * c.max() + 1e-6
    assert np.max(np.abs(prof - ref)) <= tol


@pytest.mark.parametrize("prec", PRECS)
def test_tc_matches_fp32_and_exhaustive(prec):
    rng = np.random.default_rng(44)
    T = np.cumsum(rng.standard_normal(12000)).astype(np.float32)
    a = _search(T, 96, prec)
    b = _search(T, 96, prec, early_abandon=False)
    c = _search(T, 96, "fp32")
    assert a.index == b.index == c.index
    assert a.nn_distance == b.nn_distance
    assert c.nn_distance == pytest.approx(a.nn_distance, rel=1e-4)


@pytest.mark.parametrize("prec", PRECS)
def test_edge_cases(prec):
    r = _search(np.full(900, -1.25, np.float32), 10, prec)
    assert r.index == 0 and r.nn_distance == 0.0
    unit = np.array([0, 3, 1, 4, 1, 5, 9, 2], dtype=np.float32)
    T = np.tile(unit, 60)
    T[203] += 1.0
    r = _search(T, 6, prec)
    i_ref, d2_ref = oracle.discord_brute(T, 6)
    _check(T, 6, r, i_ref, d2_ref)


@pytest.mark.parametrize("prec", PRECS)
@pytest.mark.parametrize("n,m", [(700, 2200), (1000, 5000), (1024, 3100)])
def test_long_subsequences(n, m, prec):
    """k = n spans many 64-element operand chunks (and ragged tails)."""
    rng = np.random.default_rng(n)
    T = np.cumsum(rng.standard_normal(m)).astype(np.float32)
    r = _search(T, n, prec)
    i_ref, d2_ref = oracle.discord_brute(T, n)
    _check(T, n, r, i_ref, d2_ref)


def test_expired_wait_reports_timeout_and_plan_stays_usable():
    """Failure handling without a GPU fault: the injected stall leaves the tensor-core kernel's
    operand stages armed but never filled, so its waits (bounded by %globaltimer) expire; the call
    returns DD_ETIMEOUT, and the same plan then searches normally."""
    import paper_1901_00155_gb300 as dd
    spec = synth.workload_small()
    T, _ = synth.make_series(spec)
    Td = torch.from_numpy(T).cuda()
    with dd.Plan(T.size, spec.n, "tc_fp16") as p:
        p.set_graph(False)
        ok = p.find_discord(Td)
        p.inject(1)
        with pytest.raises(dd.DDError) as ei:
            p.find_discord(Td)
        assert ei.value.status == 4  # DD_ETIMEOUT
        again = p.find_discord(Td)
        assert (again.index, again.nn_distance) == (ok.index, ok.nn_distance)
