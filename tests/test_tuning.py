"""Option autotuner (host logic): bucketing, selection of the fastest option set, unsupported
forms, the agreement check, and the JSON table.  The GPU timer is replaced by a fake here; the
real one is exercised in tests/test_gpu_tuning.py."""
import math

import pytest

from paper_1901_00155_gb300 import tuning


class Unsupported(Exception):
    pass


def test_bucket_and_key():
    assert tuning.bucket(1) == 2048 and tuning.bucket(2048) == 2048 and tuning.bucket(2049) == 4096
    assert tuning.bucket(1 << 20) == 1 << 20 and tuning.bucket((1 << 20) + 1) == 1 << 21
    assert tuning.bucket(1 << 40) == 1 << 31
    assert tuning.key(1000000, 256) == "n256/m1048576"
    with pytest.raises(ValueError):
        tuning.bucket(0)


def _fake(times, results, unsupported=()):
    calls = []

    def timer(opts, T, n, reps):
        calls.append((tuple(sorted(opts.items())), T, n, reps))
        k = (opts["precision"], opts["local_cols"])
        if k in unsupported:
            raise Unsupported(k)
        return times[k], results.get(k, (7, 2.5))[0], results.get(k, (7, 2.5))[1]
    return timer, calls


CANDS = [{"precision": p, "local_cols": lc} for p in ("tc_fp16", "fp32") for lc in (64, 128)]


def test_tune_picks_fastest_and_records_trials():
    times = {("tc_fp16", 64): 3.0, ("tc_fp16", 128): 1.5, ("fp32", 64): 9.0, ("fp32", 128): 8.0}
    timer, calls = _fake(times, {})
    series = lambda m, n, seed: ("series", m, n, seed)  # noqa: E731
    table = tuning.tune([(5000, 64), (1 << 20, 256)], CANDS, reps=2, seed=4, timer=timer, series=series,
                        unsupported=Unsupported)
    assert set(table["entries"]) == {"n64/m8192", "n256/m1048576"}
    e = table["entries"]["n64/m8192"]
    assert e["options"] == {"precision": "tc_fp16", "local_cols": 128} and e["ms"] == 1.5
    assert len(e["trials"]) == 4 and (e["index"], e["nn_distance"]) == (7, 2.5)
    assert all(c[1] == ("series", 5000, 64, 4) for c in calls[:4]) and all(c[3] == 2 for c in calls)
    assert tuning.lookup(table, 6000, 64) == {"precision": "tc_fp16", "local_cols": 128}
    assert tuning.lookup(table, 9000, 64) == {}      # another m bucket
    assert tuning.lookup(table, 6000, 128) == {}     # another n
    assert tuning.lookup({}, 6000, 64) == {}


def test_unsupported_forms_are_skipped_and_all_unsupported_raises():
    times = {("tc_fp16", 64): 1.0, ("tc_fp16", 128): 1.0, ("fp32", 64): 5.0, ("fp32", 128): 4.0}
    timer, _ = _fake(times, {}, unsupported={("tc_fp16", 64), ("tc_fp16", 128)})
    t = tuning.tune([(4096, 100000 // 64)], CANDS, timer=timer, series=lambda m, n, s: None,
                    unsupported=Unsupported)
    e = next(iter(t["entries"].values()))
    assert e["options"]["precision"] == "fp32" and e["ms"] == 4.0
    assert sum(1 for tr in e["trials"] if tr["ms"] is None) == 2
    timer2, _ = _fake(times, {}, unsupported=set(times))
    with pytest.raises(tuning.TuningError):
        tuning.tune([(4096, 8)], CANDS, timer=timer2, series=lambda m, n, s: None, unsupported=Unsupported)


def test_disagreeing_candidates_raise_and_ties_pass():
    times = {k: 1.0 for k in [("tc_fp16", 64), ("tc_fp16", 128), ("fp32", 64), ("fp32", 128)]}
    # a different index with an equal distance is accepted across forms (a tie)
    timer, _ = _fake(times, {("fp32", 64): (9, 2.5 * (1 + 1e-6)), ("fp32", 128): (9, 2.5)})
    tuning.tune([(4096, 8)], CANDS, timer=timer, series=lambda m, n, s: None, unsupported=Unsupported)
    # a different distance is a bug
    timer, _ = _fake(times, {("fp32", 128): (7, 2.6)})
    with pytest.raises(tuning.TuningError):
        tuning.tune([(4096, 8)], CANDS, timer=timer, series=lambda m, n, s: None, unsupported=Unsupported)
    with pytest.raises(ValueError):
        tuning.tune([(4096, 8)], [], timer=timer, series=lambda m, n, s: None, unsupported=Unsupported)


def test_table_round_trip(tmp_path):
    times = {("tc_fp16", 64): 2.0, ("tc_fp16", 128): 1.0, ("fp32", 64): 3.0, ("fp32", 128): 3.0}
    timer, _ = _fake(times, {})
    table = tuning.tune([(3000, 16)], CANDS, timer=timer, series=lambda m, n, s: None, unsupported=Unsupported)
    path = str(tmp_path / "tuned.json")
    tuning.save(table, path)
    back = tuning.load(path)
    assert back == table and tuning.lookup(back, 4000, 16)["local_cols"] == 128
    back["version"] = 99
    tuning.save(back, path)
    with pytest.raises(tuning.TuningError):
        tuning.load(path)
    assert tuning.lookup(back, 4000, 16) == {}


def test_default_candidates_cover_the_speed_options():
    c = tuning.DEFAULT_CANDIDATES
    assert len(c) == 27 and len({tuple(sorted(d.items())) for d in c}) == 27
    assert {d["precision"] for d in c} == {"tc_fp16", "tc_bf16", "fp32"}
    assert all(math.log2(d["local_cols"]).is_integer() and d["refine_k"] in (64, 128, 256) for d in c)


def test_candidates_are_valid_plan_options():
    """Every default candidate is an option set the library accepts (checked host-side)."""
    import paper_1901_00155_gb300 as dd
    for c in tuning.DEFAULT_CANDIDATES:
        dd._options(**c)
        assert dd.Plan.footprint(1 << 16, 256, **c) > 0


def test_batch_groups_follow_the_table():
    import paper_1901_00155_gb300 as dd
    table = {"version": tuning.TABLE_VERSION, "entries": {
        "n64/m4096": {"options": {"precision": "tc_fp16", "local_cols": 64, "refine_k": 64}},
        "n128/m65536": {"options": {"precision": "fp32", "local_cols": 256, "refine_k": 128}}}}
    ms = [3000, 50000, 4000, 9000, 60000]
    ns = [64, 128, 64, 64, 128]
    groups = dd.group_by_tuned_options(ms, ns, table, word_cols=256)
    assert [g[1] for g in groups] == [[0, 2], [1, 4], [3]]
    assert groups[0][0] == {"precision": "tc_fp16", "local_cols": 64, "refine_k": 64, "word_cols": 256}
    assert groups[1][0] == {"precision": "fp32", "local_cols": 256, "refine_k": 128, "word_cols": 256}
    assert groups[2][0] == {"precision": "fp32", "word_cols": 256}  # m=9000 has no entry
    assert dd.group_by_tuned_options(ms, ns, {}) == [({"precision": "fp32"}, [0, 1, 2, 3, 4])]
    assert dd.group_by_tuned_options(ms, ns, {}, "tc_bf16") == [({"precision": "tc_bf16"}, [0, 1, 2, 3, 4])]


def test_explicit_options_win_over_the_table():
    """A caller who names a precision (or any option) keeps it, whatever the table holds."""
    import paper_1901_00155_gb300 as dd
    table = {"version": tuning.TABLE_VERSION, "entries": {
        "n64/m4096": {"options": {"precision": "tc_fp16", "local_cols": 64, "refine_k": 64}}}}
    groups = dd.group_by_tuned_options([3000, 4000], [64, 64], table, "fp32", refine_k=32)
    assert groups == [({"precision": "fp32", "local_cols": 64, "refine_k": 32}, [0, 1])]
    groups = dd.group_by_tuned_options([3000], [64], table, "tc_bf16")
    assert groups[0][0]["precision"] == "tc_bf16"


def test_table_is_ignored_for_per_window_and_sharded_searches():
    """The tuner times globally normalised, unsharded searches only: a tensor-core entry must not
    reach a per-window search (which takes FP32 only) nor a shard of a search."""
    import paper_1901_00155_gb300 as dd
    table = {"version": tuning.TABLE_VERSION, "entries": {
        "n64/m4096": {"options": {"precision": "tc_fp16", "local_cols": 64, "refine_k": 64}}}}
    groups = dd.group_by_tuned_options([3000, 4000], [64, 64], table, znorm="window")
    assert groups == [({"precision": "fp32", "znorm": "window"}, [0, 1])]
    dd._options(**groups[0][0])  # a valid per-window option set
    groups = dd.group_by_tuned_options([3000], [64], table, shard_count=2, shard_index=1)
    assert groups == [({"precision": "fp32", "shard_count": 2, "shard_index": 1}, [0])]
    # the defaults (global, one shard) still use it
    groups = dd.group_by_tuned_options([3000], [64], table, znorm="global", shard_count=1)
    assert groups[0][0]["precision"] == "tc_fp16"


def test_same_form_candidates_must_agree_on_the_index():
    """Within one arithmetic form a different index is a bug even when the distances are close;
    across forms it is accepted as a tie of equal distances."""
    times = {k: 1.0 for k in [("tc_fp16", 64), ("tc_fp16", 128), ("fp32", 64), ("fp32", 128)]}
    timer, _ = _fake(times, {("tc_fp16", 128): (9, 2.5)})  # same form as ("tc_fp16", 64): index 7
    with pytest.raises(tuning.TuningError):
        tuning.tune([(4096, 8)], CANDS, timer=timer, series=lambda m, n, s: None, unsupported=Unsupported)
    a = tuning.Trial({"precision": "fp32"}, 1.0, 3, 2.0)
    b = tuning.Trial({"precision": "tc_bf16"}, 1.0, 4, 2.0 * (1 + 1e-6))
    assert tuning._agree(a, b, 1e-4)
    assert not tuning._agree(a, tuning.Trial({"precision": "fp32"}, 1.0, 4, 2.0), 1e-4)


# ---- fused batch schedules -------------------------------------------------------------------

def _fake_batch(times, disagree=None, unsupported=()):
    calls = []

    def timer(opts, series, ns, reps):
        calls.append((tuple(sorted(opts.items())), len(series), tuple(ns), reps))
        k = (opts["seg_cols"], opts["settle_min"])
        if k in unsupported:
            raise Unsupported(k)
        res = [(i, 1.0 + i) for i in range(len(series))]
        if disagree == k:
            res[0] = (5, 1.0)
        return times[k], res
    return timer, calls


BCANDS = [{"precision": "tc_fp16", "seg_cols": sc, "settle_min": st} for sc in (256, 512) for st in (4, 8)]


def _fake_series(mb, n, count, seed):
    return [("series", mb, n, k, seed) for k in range(count)]


def test_tune_batch_picks_fastest_schedule_per_class():
    times = {(256, 4): 5.0, (256, 8): 4.0, (512, 4): 3.0, (512, 8): 3.5}
    timer, calls = _fake_batch(times)
    t = tuning.tune_batch([(40000, 128), (3000, 64)], BCANDS, count=6, reps=2, timer=timer, batch=_fake_series,
                          unsupported=Unsupported)
    e = t["batch_entries"]
    assert set(e) == {"batch/n128/m65536", "batch/n64/m4096"}
    assert e["batch/n128/m65536"]["options"] == {"precision": "tc_fp16", "seg_cols": 512, "settle_min": 4}
    assert e["batch/n128/m65536"]["ms"] == 3.0 and len(e["batch/n128/m65536"]["trials"]) == 4
    assert all(c[1] == 6 and c[3] == 2 for c in calls)
    assert {c[2] for c in calls} == {(128,) * 6, (64,) * 6}


def test_tune_batch_rejects_disagreeing_schedules_and_skips_unsupported():
    times = {(256, 4): 5.0, (256, 8): 4.0, (512, 4): 3.0, (512, 8): 3.5}
    timer, _ = _fake_batch(times, disagree=(512, 8))
    with pytest.raises(tuning.TuningError):
        tuning.tune_batch([(4000, 64)], BCANDS, timer=timer, batch=_fake_series, unsupported=Unsupported)
    timer, _ = _fake_batch(times, unsupported={(512, 4)})
    t = tuning.tune_batch([(4000, 64)], BCANDS, timer=timer, batch=_fake_series, unsupported=Unsupported)
    e = t["batch_entries"]["batch/n64/m4096"]
    assert e["options"]["settle_min"] == 8 and e["options"]["seg_cols"] == 512
    assert [x["ms"] for x in e["trials"]].count(None) == 1
    timer, _ = _fake_batch(times, unsupported=set(times))
    with pytest.raises(tuning.TuningError):
        tuning.tune_batch([(4000, 64)], BCANDS, timer=timer, batch=_fake_series, unsupported=Unsupported)


def test_lookup_batch_uses_the_class_with_most_work(tmp_path):
    times = {(256, 4): 5.0, (256, 8): 4.0, (512, 4): 3.0, (512, 8): 3.5}
    timer, _ = _fake_batch(times)
    t = tuning.tune_batch([(40000, 128)], BCANDS, timer=timer, batch=_fake_series, unsupported=Unsupported)
    p = tmp_path / "t.json"
    tuning.save(t, str(p))
    t2 = tuning.load(str(p))
    # most work in n=128, m in (32768, 65536]
    assert tuning.lookup_batch(t2, [40000, 50000, 3000], [128, 128, 256]) == \
        {"precision": "tc_fp16", "seg_cols": 512, "settle_min": 4}
    # most work in a class without an entry
    assert tuning.lookup_batch(t2, [40000, 60000, 60000], [128, 256, 256]) == {}
    assert tuning.lookup_batch({}, [1000], [64]) == {}
    assert tuning.lookup(t2, 40000, 128) == {}  # single-series entries are separate


def test_lookup_batch_per_n():
    times = {(256, 4): 5.0, (256, 8): 4.0, (512, 4): 3.0, (512, 8): 3.5}
    timer, _ = _fake_batch(times)
    t = tuning.tune_batch([(40000, 128)], BCANDS, timer=timer, batch=_fake_series, unsupported=Unsupported)
    times2 = {(256, 4): 1.0, (256, 8): 4.0, (512, 4): 3.0, (512, 8): 3.5}
    timer2, _ = _fake_batch(times2)
    t = tuning.tune_batch([(3000, 64)], BCANDS, timer=timer2, batch=_fake_series, unsupported=Unsupported, table=t)
    per_n = tuning.lookup_batch_per_n(t, [40000, 3000, 2500, 5000, 9000], [128, 64, 64, 256, 128])
    assert per_n == {128: {"precision": "tc_fp16", "seg_cols": 512, "settle_min": 4},
                     64: {"precision": "tc_fp16", "seg_cols": 256, "settle_min": 4}}
