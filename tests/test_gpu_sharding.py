"""Sharded search on one GPU: the G shards run one after another on one device, and the host
merges them. The merged result must equal the unsharded search and the oracle.

Shard k of G keeps the rows at positions [k N / G, (k + 1) N / G) of the mean order. The shards
here are sized so that their boundaries fall inside the 128-row tiles of the band wave."""
import math

import numpy as np
import pytest

import oracle
from paper_1901_00155_gb300 import synth
from paper_1901_00155_gb300.sharding import merge

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _dd():
    import paper_1901_00155_gb300 as dd
    return dd


@pytest.mark.parametrize("precision", ["fp32", "tc_fp16", "tc_bf16"])
@pytest.mark.parametrize("G", [2, 3, 7])
def test_sharded_equals_unsharded_and_oracle(precision, G):
    dd = _dd()
    spec = synth.workload_small()
    T, _ = synth.make_series(spec)
    Td = torch.from_numpy(T).cuda()
    i_ref, d2_ref = oracle.discord_brute(T, spec.n)
    with dd.Plan(T.size, spec.n, precision) as p:
        whole = p.find_discord(Td)
    parts = []
    for k in range(G):
        with dd.Plan(T.size, spec.n, precision, shard_count=G, shard_index=k) as p:
            parts.append(p.find_discord(Td))
    r = merge(parts)
    assert r.index == whole.index == i_ref
    assert r.nn_distance == pytest.approx(math.sqrt(d2_ref), rel=1e-4 if precision == "fp32" else 1e-6)
    # the shard holding the discord finds it; every other shard reports a smaller distance
    assert sum(1 for x in parts if x.index == i_ref) == 1
    assert all(x.nn_distance <= r.nn_distance for x in parts)


def test_every_shard_answer_is_exact_and_the_best_is_the_discord():
    """Each shard returns the exact nn distance of the row it names. The shards partition the
    rows, so the largest shard answer is the series' discord."""
    dd = _dd()
    spec = synth.SeriesSpec(kind="sine", m=6000, n=64, seed=3, anomalies=("spike", "flat"))
    T, _ = synth.make_series(spec)
    Td = torch.from_numpy(T).cuda()
    nn2 = oracle.nn_profile(T, spec.n)
    G = 4
    seen = []
    for k in range(G):
        with dd.Plan(T.size, spec.n, "tc_fp16", shard_count=G, shard_index=k) as p:
            r = p.find_discord(Td)
        assert r.exact
        assert r.nn_distance == pytest.approx(math.sqrt(nn2[r.index]), rel=1e-9)
        seen.append(r)
    best = merge(seen)
    assert best.index == int(np.argmax(nn2))
    assert best.nn_distance == pytest.approx(math.sqrt(float(nn2.max())), rel=1e-9)
