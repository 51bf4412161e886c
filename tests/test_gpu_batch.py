"""Fused batch (dd_batch_*): many series searched by one launch per step of the
search, through the C ABI.

Each series' result must be the FP64 oracle's discord (index equal unless the
oracle's own distances tie within 1e-12 relative; nn_distance within 1e-6
relative), and equal to the result of a single-series plan on the same series
(index equal, distance within 1e-9 relative: both are exact FP64 rescorings of
the same rows, normalised with statistics summed in different orders; a
different index only where the oracle's distances of the two rows tie within
1e-12).
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
SOLO = 1e-9


def _dd():
    import paper_1901_00155_gb300 as dd
    return dd


def _cuda(T):
    return torch.from_numpy(np.ascontiguousarray(T, dtype=np.float32)).cuda()


def _check_oracle(T, n, r, i_ref, d2_ref):
    assert not isinstance(r, Exception), r
    assert r.exact
    assert r.nn_distance == pytest.approx(math.sqrt(d2_ref), rel=RTOL, abs=1e-9), (r, i_ref, d2_ref)
    if r.index != i_ref:
        nn, _ = oracle.nn_rows(T, n, [r.index])
        assert nn[0] == pytest.approx(d2_ref, rel=TIE, abs=1e-15), (r, i_ref, d2_ref)
        assert r.index > i_ref or nn[0] != d2_ref


def _same_as_solo(T, n, r, s):
    """The fused and the single-series results agree: the same index and distance, or, where the
    two (normalised with FP64 sums in different orders) picked different rows, rows whose oracle
    distances tie within 1e-12."""
    assert not isinstance(r, Exception) and not isinstance(s, Exception), (r, s)
    assert r.nn_distance == pytest.approx(s.nn_distance, rel=SOLO), (r, s)
    if r.index != s.index:
        nn, _ = oracle.nn_rows(T, n, [r.index, s.index])
        assert nn[0] == pytest.approx(nn[1], rel=TIE, abs=1e-15), (r, s, nn)


def _solo(T, n, prec):
    dd = _dd()
    with dd.Plan(T.size, n, prec) as p:
        return p.find_discord(_cuda(T))


def _random_mix(seed, count, m_hi=6000, ns=(1, 3, 8, 33, 64, 100, 128, 256)):
    rng = np.random.default_rng(seed)
    out = []
    for _ in range(count):
        n = int(rng.choice(ns))
        m = int(rng.integers(3 * n - 1, max(3 * n, m_hi)))
        if rng.random() < 0.5:
            T = np.cumsum(rng.standard_normal(m))
        else:
            k = np.arange(m)
            T = np.sin(2 * np.pi * k / rng.uniform(20, 200)) + 0.1 * rng.standard_normal(m)
            a = int(rng.integers(0, m - n + 1))
            T[a:a + n] += rng.standard_normal(n)
        out.append((T.astype(np.float32), n))
    return out


@pytest.mark.parametrize("prec", ["tc_fp16", "tc_bf16"])
def test_batch_matches_oracle_small(prec):
    dd = _dd()
    items = _random_mix(11 if prec == "tc_fp16" else 12, 40)
    with dd.Batch(len(items), sum(T.size for T, _ in items), 256, prec) as b:
        res = b.search([_cuda(T) for T, _ in items], [n for _, n in items])
    for (T, n), r in zip(items, res):
        i_ref, d2_ref = oracle.discord_brute(T, n)
        _check_oracle(T, n, r, i_ref, d2_ref)


def test_batch_workload_equals_solo_and_oracle():
    """The 512-series workload (m log-uniform in [2048, 65536], n in {64, 128, 256}, random walk
    and sine + noise, one anomaly each): every result equals the single-series plan's; a sample
    of the shorter series is checked against the oracle's HOTSAX."""
    dd = _dd()
    specs = synth.workload_batch(0)
    series = [synth.make_series(s)[0] for s in specs]
    ns = [s.n for s in specs]
    dev = [_cuda(T) for T in series]
    with dd.Batch(len(specs), sum(T.size for T in series), 256, "tc_fp16") as b:
        res = b.search(dev, ns)
        again = b.search(dev, ns)
        assert b.graph_replays() == 1
    for r, q in zip(res, again):
        assert (r.index, r.nn_distance) == (q.index, q.nn_distance)
    solo = dd.find_discord_batched(dev, ns, "tc_fp16")
    for k, (r, s) in enumerate(zip(res, solo)):
        _same_as_solo(series[k], ns[k], r, s)
    short = [k for k, s in enumerate(specs) if s.m <= 12000][:10]
    assert len(short) >= 5
    for k in short:
        i_ref, d2_ref = oracle.hotsax(series[k], ns[k])[:2]
        _check_oracle(series[k], ns[k], res[k], i_ref, d2_ref)


def test_batch_replay_with_new_data():
    """The second call with the same shapes replays the captured graph; its series pointers
    and values are new and its results are those of the new data."""
    dd = _dd()
    first = _random_mix(21, 12)
    second = _random_mix(22, 12)
    # the same shapes, other values
    second = [(np.resize(T2, T1.size).astype(np.float32) + np.float32(0.5), n1)
              for (T1, n1), (T2, _) in zip(first, second)]
    with dd.Batch(12, sum(T.size for T, _ in first), 256, "tc_fp16") as b:
        b.search([_cuda(T) for T, _ in first], [n for _, n in first])
        res = b.search([_cuda(T) for T, _ in second], [n for _, n in second])
        assert b.graph_replays() == 1
    for (T, n), r in zip(second, res):
        _same_as_solo(T, n, r, _solo(T, n, "tc_fp16"))


def test_batch_edge_cases():
    """Constant, non-finite, too-short and n > n_max series complete on their own; the others
    are unaffected; the shortest valid series (N = 2n) and a periodic series with an exact tie
    structure match the oracle."""
    dd = _dd()
    rng = np.random.default_rng(5)
    unit = np.array([0, 3, 1, 4, 1, 5, 9, 2], dtype=np.float32)
    tied = np.tile(unit, 60)
    tied[203] += 1.0
    nan = np.cumsum(rng.standard_normal(3000)).astype(np.float32)
    nan[1234] = np.nan
    good = [(np.cumsum(rng.standard_normal(5000)).astype(np.float32), 64),
            (np.cumsum(rng.standard_normal(3 * 50 - 1)).astype(np.float32), 50),
            (tied, 6)]
    items = [good[0], (np.full(900, -1.25, np.float32), 10), good[1], (nan, 32),
             (np.cumsum(rng.standard_normal(100)).astype(np.float32), 40),  # N < 2n
             (np.cumsum(rng.standard_normal(4000)).astype(np.float32), 300),  # n > n_max
             good[2]]
    with dd.Batch(len(items), sum(T.size for T, _ in items), 256, "tc_fp16") as b:
        res = b.search([_cuda(T) for T, _ in items], [n for _, n in items])
        assert b.search([], []) == []
    assert res[1].index == 0 and res[1].nn_distance == 0.0
    assert isinstance(res[3], dd.DDError) and res[3].status == 3   # DD_ENONFINITE
    assert isinstance(res[4], dd.DDError) and res[4].status == 1   # DD_EINVAL
    assert isinstance(res[5], dd.DDError) and res[5].status == 1
    for k in (0, 2, 6):
        T, n = items[k]
        i_ref, d2_ref = oracle.discord_brute(T, n)
        _check_oracle(T, n, res[k], i_ref, d2_ref)


def test_batch_many_lengths_and_capacity():
    """Twelve distinct n (twelve groups in one call); calls beyond the capacity fail whole."""
    dd = _dd()
    rng = np.random.default_rng(9)
    items = []
    for n in (2, 5, 16, 31, 64, 65, 127, 128, 129, 200, 255, 256):
        m = int(rng.integers(3 * n, 3 * n + 2500))
        items.append((np.cumsum(rng.standard_normal(m)).astype(np.float32), n))
    total = sum(T.size for T, _ in items)
    with dd.Batch(len(items), total, 256, "tc_fp16") as b:
        res = b.search([_cuda(T) for T, _ in items], [n for _, n in items])
        for (T, n), r in zip(items, res):
            i_ref, d2_ref = oracle.discord_brute(T, n)
            _check_oracle(T, n, r, i_ref, d2_ref)
        big = np.cumsum(rng.standard_normal(total + 1000)).astype(np.float32)
        with pytest.raises(dd.DDError) as e:
            b.search([_cuda(big)], [64])
        assert e.value.status == 2  # DD_ENOMEM
        with pytest.raises(dd.DDError):
            b.search([_cuda(items[0][0])] * (len(items) + 1), [items[0][1]] * (len(items) + 1))


def test_batch_schedules_change_speed_only():
    """Per-n schedules (columns per work item, settle threshold 0 = every candidate settled in
    FP32 first, or never, FP32 settle tiles of 32, 64 or 128 rows) give the same exact results; a
    new schedule recaptures the graph."""
    dd = _dd()
    items = _random_mix(31, 24, m_hi=9000, ns=(64, 128, 256))
    series = [_cuda(T) for T, _ in items]
    ns = [n for _, n in items]
    with dd.Batch(len(items), sum(T.size for T, _ in items), 256, "tc_fp16") as b:
        ref = b.search(series, ns)
        for sched in ({64: (256, 0, 32), 128: (1024, 0, 64), 256: (512, 0, 128)},
                      {64: (512, 0, 128), 128: (512, 0, 32), 256: (256, 0, 32)},
                      {64: (2048, 10 ** 6, 64), 128: (256, 10 ** 6, 64), 256: (256, 1, 64)}):
            for n, (sc, st, sr) in sched.items():
                b.set_schedule(n, sc, st, sr)
            got = b.search(series, ns)
            for r, q in zip(ref, got):
                assert (r.index, r.nn_distance) == (q.index, q.nn_distance)
        assert b.graph_replays() == 0
        b.set_schedule(64)  # back to the batch's own
        again = b.search(series, ns)
        assert [(r.index, r.nn_distance) for r in again] == [(r.index, r.nn_distance) for r in ref]
