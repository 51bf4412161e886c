"""Per-window z-normalised discords and the diagonal-recurrence profile on the GPU (C ABI)
against the FP64 oracle.

Tolerances:
- per-window discord: exact FP64 rescoring on the GPU, so the index equals the oracle's (or,
  where the oracle's values tie within 1e-9 relative, a row of that value) and the distance
  agrees within 1e-6 relative;
- per-window profile: the exact FP64 distance from each row to the argument the recurrence
  found, so never below the oracle's nearest-neighbour value (1e-6 relative, the float
  rounding of the output); above it only where FP32 rounding of the recurrence picked a
  near-tie (at most 1e-3 relative, and for >= 99% of rows not at all);
- global diagonal profile: the FP32 direct distance to that argument (Eq. 1 squared), so
  within the FP32 form's error (1e-4 relative) of the oracle's distance for that pair, and
  of the nearest-neighbour value up to the same near-tie slack.
"""
import math

import numpy as np
import pytest

import oracle
from paper_1901_00155_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TIE = 1e-9
RTOL = 1e-6


def _dd():
    import paper_1901_00155_gb300 as dd
    return dd


def _cuda(T):
    return torch.from_numpy(np.ascontiguousarray(T, dtype=np.float32)).cuda()


def _check_discord(T, n, r, i_ref, d2_ref):
    assert r.exact
    assert r.nn_distance == pytest.approx(math.sqrt(d2_ref), rel=RTOL, abs=1e-9), (r, i_ref, d2_ref)
    if r.index != i_ref:
        nn, _ = oracle.nn_rows(T, n, [r.index], "window")
        assert nn[0] == pytest.approx(d2_ref, rel=TIE, abs=1e-12), (r, i_ref, d2_ref)


def test_window_discord_small_sweep():
    dd = _dd()
    rng = np.random.default_rng(2024)
    for trial in range(40):
        n = int(rng.choice([1, 2, 3, 8, 16, 33, 64]))
        m = int(rng.integers(3 * n - 1, 3 * n + 600))
        T = synth.random_small(rng, m)
        with dd.Plan(T.size, n, znorm="window") as p:
            r = p.find_discord(_cuda(T))
        i_ref, d2_ref = oracle.discord_brute(T, n, "window")
        _check_discord(T, n, r, i_ref, d2_ref)


def test_window_discord_across_tiles_and_flat_windows():
    """Several diagonal blocks and row blocks of the recurrence kernel, ragged edges, a planted
    flat stretch (constant windows) and a planted shape anomaly."""
    dd = _dd()
    for seed, m, n in [(1, 5000, 32), (2, 4500, 100), (3, 6200, 17)]:
        rng = np.random.default_rng(seed)
        T = np.cumsum(rng.standard_normal(m)).astype(np.float32)
        T[1200:1200 + 2 * n] = T[1200]
        T[3000:3000 + n] += np.sin(np.arange(n) / 3.0).astype(np.float32) * 4
        with dd.Plan(m, n, znorm="window") as p:
            r = p.find_discord(_cuda(T))
            waves = p.waves()
        i_ref, d2_ref = oracle.discord_brute(T, n, "window")
        _check_discord(T, n, r, i_ref, d2_ref)
        N = m - n + 1
        assert [w["kind"] for w in waves] == ["diag"]
        assert waves[0]["pairs"] == (N - n) * (N - n + 1) // 2 == r.computed_pairs
        assert 1 <= r.candidates < N


def test_window_profile_and_arguments():
    dd = _dd()
    rng = np.random.default_rng(5)
    m, n = 5000, 32
    T = (np.cumsum(rng.standard_normal(m)) + 0.3 * rng.standard_normal(m)).astype(np.float32)
    T[2000:2000 + 3 * n] = 1.5
    ref = oracle.nn_profile(T, n, "window")
    with dd.Plan(m, n, znorm="window") as p:
        Tc = _cuda(T)
        prof = p.nn_profile(Tc).cpu().numpy().astype(np.float64)
        prof2, idx = p.nn_profile_diag(Tc, index=True)
    prof2 = prof2.cpu().numpy().astype(np.float64)
    idx = idx.cpu().numpy()
    assert np.array_equal(prof, prof2)
    N = m - n + 1
    assert np.all(np.abs(idx - np.arange(N)) >= n) and idx.min() >= 0 and idx.max() < N
    assert np.all(prof >= ref * (1 - RTOL) - 1e-9)
    assert np.all(prof <= ref * (1 + 1e-3) + 1e-6)
    assert np.mean(np.abs(prof - ref) <= RTOL * ref + 1e-9) >= 0.99
    for i in np.random.default_rng(0).choice(N, 64, replace=False):
        assert prof[i] == pytest.approx(oracle.dist2(T, n, int(i), int(idx[i]), "window"), rel=RTOL, abs=1e-9)


def test_global_diag_profile():
    dd = _dd()
    rng = np.random.default_rng(6)
    m, n = 6000, 64
    T = np.cumsum(rng.standard_normal(m)).astype(np.float32)
    ref = oracle.nn_profile(T, n)
    with dd.Plan(m, n, diag=True) as p:
        prof, idx = p.nn_profile_diag(_cuda(T), index=True)
        waves = p.waves()
    prof = prof.cpu().numpy().astype(np.float64)
    idx = idx.cpu().numpy()
    N = m - n + 1
    assert waves[0]["kind"] == "diag" and waves[0]["pairs"] == (N - n) * (N - n + 1) // 2
    assert np.all(np.abs(idx - np.arange(N)) >= n)
    assert np.all(prof >= ref * (1 - 1e-4) - 1e-5)
    assert np.all(prof <= ref * (1 + 2e-3) + 1e-4)
    for i in np.random.default_rng(1).choice(N, 64, replace=False):
        assert prof[i] == pytest.approx(oracle.dist2(T, n, int(i), int(idx[i])), rel=1e-4, abs=1e-5)


def test_window_rows_exact():
    dd = _dd()
    rng = np.random.default_rng(7)
    m, n = 3000, 40
    T = np.cumsum(rng.standard_normal(m)).astype(np.float32)
    rows = np.array([0, 1, 17, 500, 1501, m - n], dtype=np.int32)
    ref, _ = oracle.nn_rows(T, n, rows.astype(np.int64), "window")
    with dd.Plan(m, n, znorm="window") as p:
        got = p.nn_rows(_cuda(T), torch.from_numpy(rows).cuda()).cpu().numpy()
    assert np.allclose(got, ref, rtol=RTOL, atol=1e-9)


def test_window_topk():
    dd = _dd()
    rng = np.random.default_rng(8)
    m, n = 3000, 24
    T = np.cumsum(rng.standard_normal(m)).astype(np.float32)
    with dd.Plan(m, n, znorm="window") as p:
        got = p.find_discords(_cuda(T), 3)
    ref = oracle.discords_brute(T, n, 3, "window")
    assert [g.index for g in got] == [i for i, _ in ref]
    for g, (_, d2) in zip(got, ref):
        assert g.nn_distance == pytest.approx(math.sqrt(d2), rel=RTOL)


def test_window_graph_eager_async_engine_agree():
    dd = _dd()
    rng = np.random.default_rng(9)
    series = [np.cumsum(rng.standard_normal(m)).astype(np.float32) for m in (2500, 4000, 3100)]
    n = 30
    solo = []
    for T in series:
        with dd.Plan(T.size, n, znorm="window") as p:
            a = p.find_discord(_cuda(T))
            p.set_graph(False)
            b = p.find_discord(_cuda(T))
            assert (a.index, a.nn_distance) == (b.index, b.nn_distance)
            solo.append(a)
    batched = dd.find_discord_batched([_cuda(T) for T in series], [n] * 3, znorm="window")
    for s, b in zip(solo, batched):
        assert (s.index, s.nn_distance) == (b.index, b.nn_distance)


def test_window_errors():
    dd = _dd()
    T = np.cumsum(np.random.default_rng(0).standard_normal(600)).astype(np.float32)
    T[200] = np.inf
    with dd.Plan(T.size, 16, znorm="window") as p:
        with pytest.raises(dd.DDError) as e:
            p.find_discord(_cuda(T))
    assert e.value.status == 3
    with dd.Plan(T.size, 16) as p:
        with pytest.raises(dd.DDError) as e:
            p.nn_profile_diag(_cuda(np.zeros(600, np.float32)))
    assert e.value.status == 7


def test_window_discord_full_size_sampled():
    """m = 2^20, n = 256 (the benchmark's size) per window: the GPU discord's distance is its
    exact nearest-neighbour distance, and no sampled row -- the GPU profile's largest values
    included -- has a larger one."""
    dd = _dd()
    spec = synth.workload_large(0)
    T, _ = synth.make_series(spec)
    n = spec.n
    with dd.Plan(T.size, n, znorm="window") as p:
        Tc = _cuda(T)
        r = p.find_discord(Tc)
        prof = p.nn_profile(Tc).cpu().numpy()
    top = np.argsort(prof)[-6:]
    rows = np.unique(np.concatenate([[r.index], top, np.random.default_rng(3).choice(prof.size, 3)]))
    nn, _ = oracle.nn_rows(T, n, rows.astype(np.int64), "window")
    got = dict(zip(rows.tolist(), nn.tolist()))
    assert r.nn_distance == pytest.approx(math.sqrt(got[r.index]), rel=RTOL)
    assert max(got.values()) <= got[r.index] * (1 + TIE)
