"""Option autotuner on the GPU: every candidate finds the oracle's discord, and the table's
winner is one of them (timing order is not asserted)."""
import math

import pytest

import oracle

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def test_tune_small_shape_against_oracle(tmp_path):
    from paper_1901_00155_gb300 import synth, tuning
    cands = [{"precision": "fp32", "local_cols": 128, "refine_k": 128},
             {"precision": "tc_fp16", "local_cols": 128, "refine_k": 64}]
    table = tuning.tune([(8192, 64)], cands, reps=2, seed=3)
    e = table["entries"]["n64/m8192"]
    assert e["options"] in cands and e["ms"] > 0
    assert all(t["ms"] is not None and t["ms"] > 0 for t in e["trials"])
    T, _ = synth.make_series(synth.SeriesSpec("rw", 8192, 64, 3, ("burst",)))
    i_ref, d2_ref = oracle.discord_brute(T, 64)
    assert e["nn_distance"] == pytest.approx(math.sqrt(d2_ref), rel=1e-4)
    if e["index"] != i_ref:
        nn, _ = oracle.nn_rows(T, 64, [e["index"]])
        assert nn[0] == pytest.approx(d2_ref, rel=1e-4)
    path = str(tmp_path / "t.json")
    tuning.save(table, path)
    assert tuning.lookup(tuning.load(path), 8000, 64) == e["options"]


def test_batched_with_table_matches_solo():
    import numpy as np

    import paper_1901_00155_gb300 as dd
    from paper_1901_00155_gb300 import synth, tuning
    table = {"version": tuning.TABLE_VERSION, "entries": {
        "n64/m8192": {"options": {"precision": "tc_fp16", "local_cols": 64, "refine_k": 64}}}}
    rng = np.random.default_rng(11)
    series = [np.cumsum(rng.standard_normal(m)).astype(np.float32) for m in (8000, 3000, 7000)]
    ns = [64, 64, 32]
    got = dd.find_discord_batched([torch.from_numpy(T).cuda() for T in series], ns, table=table)
    for T, n, g in zip(series, ns, got):
        i_ref, d2_ref = oracle.discord_brute(T, n)
        assert g.nn_distance == pytest.approx(math.sqrt(d2_ref), rel=1e-4)
        if g.index != i_ref:
            nn, _ = oracle.nn_rows(T, n, [g.index])
            assert nn[0] == pytest.approx(d2_ref, rel=1e-4)
    assert got[0].exact and not got[1].exact  # the tuned (tensor-core) and the default (FP32) forms


def test_tune_batch_class_against_oracle():
    """The fused batch's schedule tuner on one small class: every candidate schedule returns the
    same discords (the tuner checks), the winner is one of them, and a fused batched call with the
    table finds the oracle's discord of every series."""
    import paper_1901_00155_gb300 as dd
    from paper_1901_00155_gb300 import tuning
    cands = [{"precision": "tc_fp16", "seg_cols": 256, "settle_min": 4},
             {"precision": "tc_fp16", "seg_cols": 1024, "settle_min": 32}]
    table = tuning.tune_batch([(4096, 64)], cands, count=8, reps=2, seed=5)
    e = table["batch_entries"]["batch/n64/m4096"]
    assert e["options"] in cands and e["ms"] > 0 and e["count"] == 8
    series = tuning._default_batch(4096, 64, 8, 5)
    got = dd.find_discord_batched(series, [64] * 8, fused=True, table=table)
    for T, g in zip(series, got):
        Th = T.cpu().numpy()
        i_ref, d2_ref = oracle.discord_brute(Th, 64)
        assert g.exact and g.nn_distance == pytest.approx(math.sqrt(d2_ref), rel=1e-6)
        if g.index != i_ref:
            nn, _ = oracle.nn_rows(Th, 64, [g.index])
            assert nn[0] == pytest.approx(d2_ref, rel=1e-12)
