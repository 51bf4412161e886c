"""Discord search on the GPU (C ABI) against the FP64 oracle.

FP32 form (tolerance from the required accuracy of the plain FP32 path):
  * index: identical to the oracle's, or -- where the oracle's distances tie
    within the tolerance -- a row whose oracle nn distance is within RTOL of
    the oracle's maximum;
  * nn_distance within RTOL (relative) of the oracle's.
"""
import math

import numpy as np
import pytest

import oracle
from paper_1901_00155_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

RTOL = 1e-4


def _dd():
    import paper_1901_00155_gb300 as dd
    return dd


def _search(T, n, **opts):
    dd = _dd()
    with dd.Plan(T.size, n, **opts) as p:
        r = p.find_discord(torch.from_numpy(np.ascontiguousarray(T)).cuda())
    return r


def _check_against(T, n, r, i_ref, d2_ref):
    d_ref = math.sqrt(d2_ref)
    assert r.nn_distance == pytest.approx(d_ref, rel=RTOL, abs=1e-6), (r, i_ref, d_ref)
    if r.index != i_ref:
        nn, _ = oracle.nn_rows(T, n, [r.index])
        assert math.sqrt(nn[0]) == pytest.approx(d_ref, rel=RTOL, abs=1e-6), (r, i_ref, d_ref)


def test_small_random_sweep():
    rng = np.random.default_rng(77)
    for trial in range(60):
        n = int(rng.choice([1, 2, 3, 8, 16, 33, 64, 100]))
        m = int(rng.integers(3 * n - 1, 3 * n + 700))
        T = synth.random_small(rng, m)
        r = _search(T, n)
        i_ref, d2_ref = oracle.discord_brute(T, n)
        _check_against(T, n, r, i_ref, d2_ref)


def test_small_workload_exact():
    spec = synth.workload_small()
    T, _ = synth.make_series(spec)
    r = _search(T, spec.n)
    i_ref, d2_ref = oracle.discord_brute(T, spec.n)
    assert r.index == i_ref
    assert r.nn_distance == pytest.approx(math.sqrt(d2_ref), rel=RTOL)


@pytest.mark.parametrize("n,m", [(16, 3000), (64, 64 * 3 - 1), (128, 128 * 3 + 77), (1, 50)])
def test_profile_matches_oracle(n, m):
    dd = _dd()
    rng = np.random.default_rng(n + m)
    T = np.cumsum(rng.standard_normal(m)).astype(np.float32)
    with dd.Plan(m, n) as p:
        prof = p.nn_profile(torch.from_numpy(T).cuda()).cpu().numpy()
    ref = oracle.nn_profile(T, n)
    np.testing.assert_allclose(prof, ref, rtol=RTOL, atol=1e-5 * max(1.0, ref.max()))


def test_nn_rows_matches_oracle():
    dd = _dd()
    rng = np.random.default_rng(5)
    T = np.cumsum(rng.standard_normal(20000)).astype(np.float32)
    n = 96
    rows = np.array([0, 1, 777, 5000, 19904, 12345, 12345], dtype=np.int32)
    with dd.Plan(T.size, n) as p:
        got = p.nn_rows(torch.from_numpy(T).cuda(), torch.from_numpy(rows).cuda()).cpu().numpy()
    ref, _ = oracle.nn_rows(T, n, rows)
    np.testing.assert_allclose(got, ref, rtol=RTOL, atol=1e-6)


def test_exhaustive_equals_abandon():
    rng = np.random.default_rng(9)
    for _ in range(4):
        T = np.cumsum(rng.standard_normal(6000)).astype(np.float32)
        a = _search(T, 50)
        b = _search(T, 50, early_abandon=False)
        assert a.index == b.index
        assert a.nn_distance == b.nn_distance
        assert b.computed_pairs > a.computed_pairs


def test_ordering_options_do_not_change_result():
    rng = np.random.default_rng(10)
    T = np.cumsum(rng.standard_normal(9000)).astype(np.float32)
    base = _search(T, 64)
    for opts in [dict(paa_mode=1), dict(alphabet=3, paa_w=5), dict(refine_k=0), dict(phase1_max=0),
                 dict(phase1_max=1, refine_k=1)]:
        r = _search(T, 64, **opts)
        assert (r.index, r.nn_distance) == (base.index, base.nn_distance), opts


def test_constant_series():
    r = _search(np.full(1000, 3.5, np.float32), 10)
    assert r.index == 0 and r.nn_distance == 0.0


def test_periodic_ties_pick_smallest_index():
    # every window has an exact copy except those holding the spike
    unit = np.array([0, 3, 1, 4, 1, 5, 9, 2], dtype=np.float32)
    T = np.tile(unit, 50)
    T[203] += 1.0
    n = 6
    r = _search(T, n)
    i_ref, d2_ref = oracle.discord_brute(T, n)
    assert i_ref == 203 - n + 1
    assert r.index == i_ref
    assert r.nn_distance == pytest.approx(math.sqrt(d2_ref), rel=RTOL)


def test_errors():
    dd = _dd()
    with pytest.raises(dd.DDError) as e:
        dd.Plan(100, 40)
    assert e.value.status == 1
    T = np.cumsum(np.random.default_rng(0).standard_normal(500)).astype(np.float32)
    T[17] = np.nan
    with dd.Plan(T.size, 8) as p:
        with pytest.raises(dd.DDError) as e:
            p.find_discord(torch.from_numpy(T).cuda())
    assert e.value.status == 3


def test_host_entry_point_and_async():
    dd = _dd()
    spec = synth.workload_small()
    T, _ = synth.make_series(spec)
    with dd.Plan(T.size, spec.n) as p:
        r1 = p.find_discord(torch.from_numpy(T).cuda())
        r2 = p.find_discord_host(T)
        r3 = p.find_discord_host(torch.from_numpy(T).pin_memory())
        buf = torch.zeros(64, dtype=torch.uint8, device="cuda")
        p.find_discord_async(torch.from_numpy(T).cuda(), buf)
        torch.cuda.synchronize()
        r4 = dd.Plan.decode_result(buf)
    for r in (r2, r3, r4):
        assert (r.index, r.nn_distance) == (r1.index, r1.nn_distance)


def test_batched_uneven():
    dd = _dd()
    rng = np.random.default_rng(21)
    series, ns, refs = [], [], []
    for k in range(6):
        n = int(rng.choice([16, 32, 64]))
        m = int(rng.integers(3 * n + 10, 4000))
        T = synth.random_small(rng, m, "rw")
        series.append(torch.from_numpy(T).cuda())
        ns.append(n)
        refs.append((T, n) + oracle.discord_brute(T, n))
    out = dd.find_discord_batched(series, ns)
    for r, (T, n, i_ref, d2_ref) in zip(out, refs):
        _check_against(T, n, r, i_ref, d2_ref)


@pytest.mark.parametrize("precision", ["fp32", "tc_fp16"])
def test_wave_trace(precision):
    """The per-wave trace accounts for every evaluated pair, in the wave order
    of Algorithm 2 (nearest-mean neighbourhood first, then Cand, top, rest)."""
    dd = _dd()
    spec = synth.workloads_medium()[2]
    T, _ = synth.make_series(spec)
    Td = torch.from_numpy(T).cuda()
    with dd.Plan(T.size, spec.n, precision) as p:
        p.set_profiling(True)
        for _ in range(2):  # the second call replays the captured graph
            r = p.find_discord(Td)
            waves = p.waves()
            assert waves, waves
            assert sum(w["pairs"] for w in waves) == r.computed_pairs
            first = "band" if precision != "fp32" else "local"
            assert waves[0]["kind"] == first and waves[0]["rows"] == T.size - spec.n + 1
            kinds = [w["kind"] for w in waves]
            assert "cand" in kinds and "rest" in kinds, kinds
            assert kinds[-1] == ("settle" if precision != "fp32" else "rest"), kinds
            # waves inside conditional graph bodies (run only when many rows survive) are not timed
            timed = [w for w in waves if w["ms"] >= 0.0]
            assert {w["kind"] for w in timed} >= {first, "cand", "rest"}, waves
            assert all(w["items"] >= 0 and w["rows"] >= 0 for w in waves)
            assert p.profile()["dist_launches"] == len(timed)


@pytest.mark.parametrize("precision", ["fp32", "tc_fp16"])
def test_eager_equals_graph(precision):
    """dd_plan_set_graph(0): the same search enqueued directly (its conditional waves gate
    themselves on the device) gives the graph replay's result."""
    dd = _dd()
    for spec in (synth.workloads_medium()[2], synth.SeriesSpec("sine", 60000, 512, 7, ("spike",))):
        T, _ = synth.make_series(spec)
        Td = torch.from_numpy(T).cuda()
        with dd.Plan(T.size, spec.n, precision) as p:
            g = p.find_discord(Td)
            p.set_graph(False)
            e = p.find_discord(Td)
        assert (g.index, g.nn_distance) == (e.index, e.nn_distance), (spec, g, e)


@pytest.mark.parametrize("precision", ["fp32", "tc_fp16"])
def test_top_k_discords(precision):
    """dd_find_discords against the oracle's definition, and the plan searches normally after."""
    dd = _dd()
    for spec, k in ((synth.workload_small(), 4), (synth.SeriesSpec("sine", 30000, 128, 5, ("spike", "burst", "flat")), 3)):
        T, _ = synth.make_series(spec)
        Td = torch.from_numpy(T).cuda()
        ref = oracle.discords_brute(T, spec.n, k)
        with dd.Plan(T.size, spec.n, precision) as p:
            got = p.find_discords(Td, k)
            again = p.find_discord(Td)
        assert len(got) == len(ref)
        for g, (i, d2) in zip(got, ref):
            assert g.nn_distance == pytest.approx(math.sqrt(d2), rel=RTOL if precision == "fp32" else 1e-6)
            if precision != "fp32":
                assert g.index == i
        assert again.index == ref[0][0]


@pytest.mark.parametrize("precision", ["fp32", "tc_fp16", "tc_bf16"])
def test_top_k_hand_examples(precision):
    """dd_find_discords on the hand-worked top-k examples of tests/golden/topk_examples.txt."""
    import os
    dd = _dd()
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "topk_examples.txt")
    cases = []
    with open(path) as f:
        for line in f:
            line = line.strip()
            if line and not line.startswith("#"):
                T, n, k, picks, _ = [x.strip() for x in line.split("|")]
                cases.append((np.array([float(v) for v in T.split(",")], dtype=np.float32), int(n), int(k),
                              [(int(a), float(b)) for a, b in (p.split(":") for p in picks.split(","))]))
    assert len(cases) == 2
    for T, n, k, want in cases:
        with dd.Plan(T.size, n, precision) as p:
            got = p.find_discords(torch.from_numpy(T).cuda(), k)
        assert [g.index for g in got] == [w[0] for w in want], (precision, got, want)
        for g, (_, d) in zip(got, want):
            assert g.nn_distance == pytest.approx(d, rel=RTOL if precision == "fp32" else 1e-6, abs=1e-6)


def test_launch_count_excludes_skipped_conditional_waves():
    """A graph replay that skips the conditional waves launches fewer kernels than the same
    search enqueued eagerly (where every gated kernel is launched and exits on its own)."""
    dd = _dd()
    spec = synth.workload_small()
    T, _ = synth.make_series(spec)
    Td = torch.from_numpy(T).cuda()
    with dd.Plan(T.size, spec.n, "tc_fp16") as p:
        p.find_discord(Td)
        p.find_discord(Td)
        g = p.last_launches()
        p.set_graph(False)
        p.find_discord(Td)
        e = p.last_launches()
    assert 0 < g < e


@pytest.mark.parametrize("form", ["fp32", "tc_fp16", "window"])
def test_nn_rows_out_of_range_entries(form):
    """dd_nn_rows with entries outside [0, N): they give non-finite values, are never used as
    indices, and leave the valid rows' values (against the oracle) untouched."""
    dd = _dd()
    rng = np.random.default_rng(15)
    T = np.cumsum(rng.standard_normal(6000)).astype(np.float32)
    n = 64
    N = T.size - n + 1
    rows = np.array([5, -1, N, 100, -(2 ** 31), N + 777, 4000, 2 ** 31 - 1, N - 1], dtype=np.int32)
    valid = (rows >= 0) & (rows < N)
    kw = {"znorm": "window"} if form == "window" else {}
    prec = "fp32" if form == "window" else form
    with dd.Plan(T.size, n, prec, **kw) as p:
        got = p.nn_rows(torch.from_numpy(T).cuda(), torch.from_numpy(rows).cuda()).cpu().numpy()
    assert not np.isfinite(got[~valid]).any()
    ref, _ = oracle.nn_rows(T, n, rows[valid], znorm="window" if form == "window" else "global")
    # the Gram form's values are within its per-row bound (about 8 u n with u = 2^-11 here)
    tol = {"fp32": dict(rtol=RTOL, atol=1e-6), "tc_fp16": dict(rtol=1e-2, atol=8 * 2.0 ** -11 * n),
           "window": dict(rtol=1e-6, atol=1e-6)}[form]
    np.testing.assert_allclose(got[valid], ref, **tol)
