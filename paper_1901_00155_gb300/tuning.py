"""Option autotuning for discord searches, keyed by (n, m bucket).

A search's options (arithmetic form, first-wave width, number of top rows fully scanned early)
change only how fast it reaches the discord, never which discord it returns (Algorithms 2-4 always
finish with exact distances of every row that can still win).  The tuner times every candidate
option set on a seeded synthetic series of each requested shape and keeps the fastest.  It also
checks that all candidates return the same discord (the same index and distance within 1e-4
relative for candidates of one arithmetic form; across forms, distances within 1e-4 relative, a
different index then being a tie); a disagreement is a bug, not a tuning result, and raises.

Entries are tuned on globally normalised, unsharded searches only, so a batch applies them only to
such searches, and options the caller passes explicitly always win over an entry.

Shapes are bucketed by m to the next power of two (2^11 .. 2^31), so one tuned entry serves every
series of that length class with the same n.  Tables are plain JSON.
"""
from __future__ import annotations

import json
import math
import os
from dataclasses import dataclass

M_MIN_BUCKET = 1 << 11
M_MAX_BUCKET = 1 << 31
TABLE_VERSION = 1

# Options the search exposes that change only its speed.
DEFAULT_CANDIDATES = tuple(
    {"precision": prec, "local_cols": lc, "refine_k": rk}
    for prec in ("tc_fp16", "tc_bf16", "fp32")
    for lc in (64, 128, 256)
    for rk in (64, 128, 256)
)


class TuningError(RuntimeError):
    pass


def bucket(m: int) -> int:
    """Smallest power of two >= m, clamped to [2^11, 2^31]."""
    if m < 1:
        raise ValueError("m must be positive")
    b = max(M_MIN_BUCKET, 1 << (int(m) - 1).bit_length())
    return min(b, M_MAX_BUCKET)


def key(m: int, n: int) -> str:
    return f"n{int(n)}/m{bucket(m)}"


@dataclass
class Trial:
    options: dict
    ms: float | None          # median time, None if the form is not supported for the shape
    index: int | None
    nn_distance: float | None


def _agree(a: Trial, b: Trial, rtol: float) -> bool:
    """Same discord.  Two option sets of the same arithmetic form take the same decisions, so they
    must return the same index and distances within rtol.  Across forms (FP32 vs a tensor-core
    form) a different index is accepted only as a tie: the distances agree within rtol."""
    same_dist = math.isclose(a.nn_distance, b.nn_distance, rel_tol=rtol, abs_tol=1e-9)
    if a.options.get("precision", "fp32") == b.options.get("precision", "fp32"):
        return a.index == b.index and same_dist
    return same_dist


def time_search(options: dict, T, n: int, reps: int = 3, warmup: int = 2):
    """Median CUDA-event time (ms) of dd_find_discord with `options` on the device series T, and
    its result.  Raises the library's DDError for unsupported option sets."""
    import statistics

    import torch

    from . import Plan

    with Plan(T.numel(), n, **options) as p:
        r = None
        for _ in range(warmup):
            r = p.find_discord(T)
        torch.cuda.synchronize()
        stream = torch.cuda.current_stream()
        ts = []
        for _ in range(reps):
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            r = p.find_discord(T)
            e1.record(stream)
            e1.synchronize()
            ts.append(e0.elapsed_time(e1))
    return statistics.median(ts), r.index, r.nn_distance


def _default_series(m: int, n: int, seed: int):
    """A seeded random walk with one sine burst: the benchmark workloads' structure."""
    import torch

    from . import synth

    spec = synth.SeriesSpec("rw", int(m), int(n), int(seed), ("burst",) if m >= 4 * n + 256 else ())
    T, _ = synth.make_series(spec)
    return torch.from_numpy(T).cuda()


def tune(shapes, candidates=None, reps: int = 3, seed: int = 0, timer=None, series=None, rtol: float = 1e-4,
         unsupported=None) -> dict:
    """Tune every (m, n) of `shapes`; returns a table {"version", "entries": {key: entry}}.

    timer(options, T, n, reps) -> (ms, index, nn_distance) times one option set (default: CUDA
    events around dd_find_discord); series(m, n, seed) builds the input (default: a seeded random
    walk on the device).  unsupported: the exception type a timer raises for option sets the shape
    does not support (default: the library's DDError).  Each entry holds the winning options, its
    time and every trial."""
    candidates = list(candidates if candidates is not None else DEFAULT_CANDIDATES)
    if not candidates:
        raise ValueError("no candidate option sets")
    timer = timer or time_search
    series = series or _default_series
    if unsupported is None:
        from . import DDError as unsupported  # noqa: N813
    entries = {}
    for m, n in shapes:
        T = series(m, n, seed)
        trials = []
        for opts in candidates:
            try:
                ms, idx, dist = timer(dict(opts), T, n, reps)
                trials.append(Trial(dict(opts), float(ms), int(idx), float(dist)))
            except unsupported:
                trials.append(Trial(dict(opts), None, None, None))
        ok = [t for t in trials if t.ms is not None]
        if not ok:
            raise TuningError(f"no candidate option set supports m={m} n={n}")
        ref = ok[0]
        for t in ok[1:]:
            if not _agree(ref, t, rtol):
                raise TuningError(f"option sets disagree on the discord of m={m} n={n}: {ref} vs {t}")
        best = min(ok, key=lambda t: t.ms)
        entries[key(m, n)] = {
            "m": int(m), "n": int(n), "options": best.options, "ms": best.ms,
            "index": best.index, "nn_distance": best.nn_distance,
            "trials": [{"options": t.options, "ms": t.ms} for t in trials],
        }
    return {"version": TABLE_VERSION, "entries": entries}


def lookup(table: dict, m: int, n: int) -> dict:
    """The tuned options for a series of length m and subsequence length n ({} if none)."""
    if not table or table.get("version") != TABLE_VERSION:
        return {}
    e = table.get("entries", {}).get(key(m, n))
    return dict(e["options"]) if e else {}


def save(table: dict, path: str) -> None:
    tmp = f"{path}.tmp{os.getpid()}"
    with open(tmp, "w") as f:
        json.dump(table, f, indent=1, sort_keys=True)
    os.replace(tmp, path)


def load(path: str) -> dict:
    with open(path) as f:
        table = json.load(f)
    if table.get("version") != TABLE_VERSION:
        raise TuningError(f"{path}: table version {table.get('version')} != {TABLE_VERSION}")
    return table
