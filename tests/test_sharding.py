"""Row sharding: the host merge rule and the all-gather among CPU ranks.

Every box here has one GPU. So the exchange step of a multi-GPU search is
tested among gloo ranks on the host (world sizes 2 and 3). Each rank computes
its own shard's discord with the oracle, which is the exact definition. The
ranks all-gather and merge, and every rank must then hold the series' discord.
"""
import math
import os
import socket

import numpy as np
import pytest

import oracle
from paper_1901_00155_gb300 import DiscordResult, synth
from paper_1901_00155_gb300.sharding import merge

torch = pytest.importorskip("torch")


def test_merge_takes_largest_distance_then_smallest_index():
    a = DiscordResult(7, 2.0, True, 10, 1)
    b = DiscordResult(3, 2.0, False, 5, 2)
    c = DiscordResult(1, 1.5, True, 1, 0)
    r = merge([a, c, b])
    assert (r.index, r.nn_distance) == (3, 2.0)
    assert r.exact is False and r.computed_pairs == 16 and r.candidates == 3
    assert merge([c]) == c
    with pytest.raises(ValueError):
        merge([])


def _shard_result(T, n, k, G):
    """The discord among the rows of shard k: a contiguous range of row
    indices (the merge does not depend on how the rows are split)."""
    N = T.size - n + 1
    rows = np.arange(N * k // G, N * (k + 1) // G)
    nn2, _ = oracle.nn_rows(T, n, rows)
    j = int(np.argmax(nn2))  # first maximiser = smallest index among ties
    return DiscordResult(int(rows[j]), math.sqrt(nn2[j]), True, int(rows.size), 0)


def _rank(rank, world, port, T, n, out_dir):
    import torch.distributed as dist
    from paper_1901_00155_gb300.sharding import allgather_discord
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)
    try:
        r = allgather_discord(_shard_result(T, n, rank, world))
        np.save(os.path.join(out_dir, f"r{rank}.npy"), np.array([r.index, r.nn_distance, r.computed_pairs]))
    finally:
        dist.destroy_process_group()


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


@pytest.mark.parametrize("world", [2, 3])
def test_gloo_allgather_merge_equals_global_discord(world, tmp_path):
    oracle.build()
    spec = synth.SeriesSpec(kind="rw", m=1500, n=32, seed=11, anomalies=("spike",))
    T, _ = synth.make_series(spec)
    i_ref, d2_ref = oracle.discord_brute(T, spec.n)
    torch.multiprocessing.spawn(_rank, args=(world, _free_port(), T, spec.n, str(tmp_path)), nprocs=world, join=True)
    for k in range(world):
        idx, d, pairs = np.load(tmp_path / f"r{k}.npy")
        assert int(idx) == i_ref
        assert d == pytest.approx(math.sqrt(d2_ref), rel=1e-12)
        assert int(pairs) == T.size - spec.n + 1  # every row lies in exactly one shard


def test_bad_shard_options_are_rejected():
    """Option validation happens before any device work (no GPU needed)."""
    import paper_1901_00155_gb300 as dd
    for sc, si in [(-1, 0), (2, 2), (3, -1), (0, 1)]:
        assert dd.Plan.footprint(8192, 128, "fp32", shard_count=sc, shard_index=si) == 0
    assert dd.Plan.footprint(8192, 128, "fp32", shard_count=3, shard_index=2) > 0
