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

The fused batch (dd_batch_*) has its own schedule: columns per work item of its full-scan waves
(seg_cols), the candidate count above which a series settles its candidates with direct FP32 full
scans before the FP64 rescoring (settle_min), the rows of those FP32 tiles (settle_rows), and the
tensor-core precision.  tune_batch times them
on a seeded batch of each (n, m bucket) class and keeps the fastest under "batch_entries"; every
candidate schedule must return the same discord for every series (exact FP64 rescoring: the same
index, distances within 1e-9 relative).
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


# Schedules of the fused batch that change only its speed.
BATCH_CANDIDATES = tuple(
    {"precision": "tc_fp16", "seg_cols": sc, "settle_min": st, "settle_rows": sr}
    for sc in (256, 512, 1024)
    for st in (4, 8, 16, 32)
    for sr in (32, 64, 128)
)


def batch_key(m: int, n: int) -> str:
    return f"batch/n{int(n)}/m{bucket(m)}"


def time_batch(options: dict, series, ns, reps: int = 3, warmup: int = 1):
    """Median wall time (ms) of a blocking dd_batch_search with `options` (the first call captures
    the graph and is not timed), and the per-series results [(index, nn_distance)]."""
    import statistics
    import time

    import torch

    from . import Batch

    opts = dict(options)
    prec = opts.pop("precision", "tc_fp16")
    with Batch(len(series), sum(int(t.numel()) for t in series), max(int(x) for x in ns), prec, **opts) as b:
        res = None
        for _ in range(warmup):
            res = b.search(series, ns)
        ts = []
        for _ in range(reps):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            res = b.search(series, ns)
            ts.append((time.perf_counter() - t0) * 1e3)
    return statistics.median(ts), [(r.index, r.nn_distance) for r in res]


def _default_batch(m_bucket: int, n: int, count: int, seed: int):
    """`count` seeded series of the class: m log-uniform in (m_bucket / 2, m_bucket], half random
    walks, half sine + noise, one injected anomaly each (the batch workload's structure)."""
    import numpy as np
    import torch

    from . import synth

    rng = np.random.default_rng(seed)
    lo = max(3 * int(n), m_bucket // 2 + 1)
    out = []
    for k in range(count):
        m = int(round(math.exp(rng.uniform(math.log(lo), math.log(m_bucket)))))
        kind = "rw" if k % 2 == 0 else "sine"
        anomaly = ("burst",) if kind == "rw" else ("phase",)
        spec = synth.SeriesSpec(kind, m, int(n), int(seed * 100003 + k), anomaly if m >= 4 * n + 256 else ())
        out.append(torch.from_numpy(synth.make_series(spec)[0]).cuda())
    return out


def _same_results(a, b, rtol: float) -> bool:
    return len(a) == len(b) and all(i == j and math.isclose(x, y, rel_tol=rtol, abs_tol=1e-12)
                                    for (i, x), (j, y) in zip(a, b))


def tune_batch(classes, candidates=None, count: int = 32, reps: int = 3, seed: int = 0, timer=None, batch=None,
               rtol: float = 1e-9, unsupported=None, table: dict | None = None) -> dict:
    """Tune the fused batch for every (m, n) class of `classes` (m is bucketed); returns `table`
    (or a new one) with "batch_entries" filled in.

    timer(options, series, ns, reps) -> (ms, results) times one schedule (default: time_batch);
    batch(m_bucket, n, count, seed) builds the class's series (default: _default_batch)."""
    candidates = list(candidates if candidates is not None else BATCH_CANDIDATES)
    if not candidates:
        raise ValueError("no candidate schedules")
    timer = timer or time_batch
    batch = batch or _default_batch
    if unsupported is None:
        from . import DDError as unsupported  # noqa: N813
    out = table if table is not None else {"version": TABLE_VERSION, "entries": {}}
    entries = out.setdefault("batch_entries", {})
    for m, n in classes:
        mb = bucket(m)
        series = batch(mb, n, count, seed)
        ns = [int(n)] * len(series)
        trials, ref = [], None
        for opts in candidates:
            try:
                ms, res = timer(dict(opts), series, ns, reps)
            except unsupported:
                trials.append({"options": dict(opts), "ms": None})
                continue
            if ref is None:
                ref = res
            elif not _same_results(ref, res, rtol):
                raise TuningError(f"batch schedules disagree on class n={n} m<={mb}: {opts}")
            trials.append({"options": dict(opts), "ms": float(ms)})
        ok = [t for t in trials if t["ms"] is not None]
        if not ok:
            raise TuningError(f"no candidate schedule supports class n={n} m<={mb}")
        best = min(ok, key=lambda t: t["ms"])
        entries[batch_key(mb, n)] = {"m_bucket": mb, "n": int(n), "count": len(series), "options": best["options"],
                                     "ms": best["ms"], "trials": trials}
    return out


def lookup_batch(table: dict, ms, ns) -> dict:
    """The tuned schedule for a batch: that of its (n, m bucket) class with the most work
    (sum of m n over the class's series); {} if that class has no entry."""
    if not table or table.get("version") != TABLE_VERSION or not len(ms):
        return {}
    work = {}
    for m, n in zip(ms, ns):
        k = batch_key(int(m), int(n))
        work[k] = work.get(k, 0) + int(m) * int(n)
    top = max(work, key=lambda k: (work[k], k))
    e = table.get("batch_entries", {}).get(top)
    return dict(e["options"]) if e else {}


def lookup_batch_per_n(table: dict, ms, ns) -> dict:
    """Per subsequence length n of a batch: the tuned schedule of the (n, m bucket) class with the
    most work among that n's series ({n: options}, only for classes with an entry)."""
    if not table or table.get("version") != TABLE_VERSION:
        return {}
    work = {}
    for m, n in zip(ms, ns):
        k = (int(n), batch_key(int(m), int(n)))
        work[k] = work.get(k, 0) + int(m) * int(n)
    out = {}
    for n in sorted({int(x) for x in ns}):
        top = max((k for k in work if k[0] == n), key=lambda k: (work[k], k[1]))
        e = table.get("batch_entries", {}).get(top[1])
        if e:
            out[n] = dict(e["options"])
    return out
