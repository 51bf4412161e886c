"""Batched search and the serving engine (dd_engine_*, dd_find_discord_batched).

Each request's result must equal its result when searched alone on a plan of its own. The
alone results are themselves checked against the oracle elsewhere; here a few requests are also
checked against the oracle directly."""
import math

import numpy as np
import pytest

import oracle
from paper_1901_00155_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _dd():
    import paper_1901_00155_gb300 as dd
    return dd


def _alone(dd, T, n, precision):
    with dd.Plan(T.size, n, precision) as p:
        return p.find_discord(torch.from_numpy(T).cuda())


@pytest.mark.parametrize("precision", ["fp32", "tc_fp16"])
def test_batched_equals_alone(precision):
    dd = _dd()
    specs = synth.workload_batch(seed=0, count=24)
    series = [synth.make_series(s)[0] for s in specs]
    dev = [torch.from_numpy(T).cuda() for T in series]
    got = dd.find_discord_batched(dev, [s.n for s in specs], precision)
    for T, s, r in zip(series, specs, got):
        a = _alone(dd, T, s.n, precision)
        assert (r.index, r.nn_distance) == (a.index, a.nn_distance), (s, r, a)
    for k in (0, 7):  # two checked against the definition directly
        i_ref, d2_ref = oracle.discord_brute(series[k], specs[k].n)
        assert got[k].index == i_ref
        assert got[k].nn_distance == pytest.approx(math.sqrt(d2_ref), rel=1e-4)


def test_batched_reports_each_series_error():
    dd = _dd()
    T, _ = synth.make_series(synth.workload_small())
    good = torch.from_numpy(T).cuda()
    short = good[:200].contiguous()  # N < 2n for n = 128
    got = dd.find_discord_batched([good, short, good], [128, 128, 128], "tc_fp16")
    assert isinstance(got[1], dd.DDError) and got[1].status == 1  # DD_EINVAL
    assert got[0].index == got[2].index == _alone(dd, T, 128, "tc_fp16").index


def test_engine_mix_equals_alone_host_and_device():
    """Requests of a serving trace, submitted together to 4 workers (host and device series
    mixed), give the results they give alone."""
    dd = _dd()
    trace = synth.serving_requests(seed=5, rate_per_s=200.0, duration_s=0.12, m_max=1 << 17)
    assert len(trace) >= 12
    series = [synth.make_series(s)[0] for _, s in trace]
    with dd.Engine(4, 1 << 17, 1024, "tc_fp16") as E:
        for k, ((_, s), T) in enumerate(zip(trace, series)):
            E.submit(torch.from_numpy(T).cuda() if k % 2 else T, s.n, id=k)
        done = E.drain()
        assert E.outstanding() == 0
    assert sorted(c.id for c in done) == list(range(len(trace)))
    for c in done:
        s = trace[c.id][1]
        a = _alone(dd, series[c.id], s.n, "tc_fp16")
        assert (c.result.index, c.result.nn_distance) == (a.index, a.nn_distance), (s, c, a)
        assert c.queue_ms >= 0.0 and c.service_ms > 0.0


def test_engine_admission_and_errors():
    dd = _dd()
    T, _ = synth.make_series(synth.workload_small())  # m = 8192
    with dd.Engine(2, 4096, 128, "fp32") as E:
        E.submit(T, 128, id=1)                         # host series longer than m_max -> ENOMEM
        E.submit(T[:4096].copy(), 2000, id=2)          # N < 2n -> EINVAL
        E.submit(T[:4096].copy(), 64, id=3)            # fits
        done = {c.id: c for c in E.drain()}
    assert isinstance(done[1].result, dd.DDError) and done[1].result.status == 2  # DD_ENOMEM
    assert isinstance(done[2].result, dd.DDError) and done[2].result.status == 1  # DD_EINVAL
    i_ref, d2_ref = oracle.discord_brute(T[:4096], 64)
    assert done[3].result.index == i_ref
    assert done[3].result.nn_distance == pytest.approx(math.sqrt(d2_ref), rel=1e-4)


def test_engine_destroy_with_queued_requests():
    dd = _dd()
    T, _ = synth.make_series(synth.workload_small())
    E = dd.Engine(1, T.size, 128, "fp32")
    for k in range(20):
        E.submit(T, 128, id=k)
    E.close()  # lets the running request finish and drops the queued ones


def test_engine_budget_admission_and_bypass():
    """Admission by device memory: the budget holds one plan of the large series at a time, so
    the second large request waits for the first while small ones, queued behind it, pass it.
    Every result equals its result alone."""
    dd = _dd()
    big = [synth.make_series(synth.SeriesSpec("rw", 1 << 18, 256, s, ("spike",)))[0] for s in (1, 2)]
    small = [synth.make_series(synth.SeriesSpec("sine", 8192, 64, 10 + k, ("burst",)))[0] for k in range(6)]
    fb = dd.Plan.footprint(1 << 18, 256, "tc_fp16")
    fs = dd.Plan.footprint(8192, 64, "tc_fp16")
    budget = fb + 4 * fs  # one large plan at a time, with room for small ones beside it
    with dd.Engine(4, 1 << 18, 256, "tc_fp16", budget=budget) as E:
        E.submit(torch.from_numpy(big[0]).cuda(), 256, id=100)
        E.submit(torch.from_numpy(big[1]).cuda(), 256, id=101)
        for k, T in enumerate(small):
            E.submit(torch.from_numpy(T).cuda(), 64, id=k)
        done = {c.id: c for c in E.drain()}
    assert sorted(done) == list(range(6)) + [100, 101]
    for k, T in enumerate(small):
        a = _alone(dd, T, 64, "tc_fp16")
        assert (done[k].result.index, done[k].result.nn_distance) == (a.index, a.nn_distance)
    for k, T in enumerate(big):
        a = _alone(dd, T, 256, "tc_fp16")
        assert (done[100 + k].result.index, done[100 + k].result.nn_distance) == (a.index, a.nn_distance)
    # the two large plans never held memory together: the second started after the first ended
    first, second = sorted((done[100], done[101]), key=lambda c: c.queue_ms)
    assert second.queue_ms >= first.queue_ms + first.service_ms - 1.0
    # and a small request queued behind the second large one started before it
    assert min(done[k].queue_ms for k in range(6)) < second.queue_ms


def test_engine_rejects_what_never_fits():
    dd = _dd()
    T, _ = synth.make_series(synth.workload_small())
    with dd.Engine(2, T.size, 128, "fp32", budget=dd.Plan.footprint(4096, 64) + 4 * 4096) as E:
        E.submit(T, 128, id=1)                    # its plan alone exceeds the budget -> ENOMEM
        E.submit(T[:4096].copy(), 64, id=2)       # fits
        done = {c.id: c for c in E.drain()}
    assert isinstance(done[1].result, dd.DDError) and done[1].result.status == 2
    assert done[2].result.index == _alone(dd, T[:4096].copy(), 64, "fp32").index
