"""GB300-native time-series discord discovery (PhiDD / HOTSAX, arXiv:1901.00155).

Python binding of the C ABI in include/dd.h.  PyTorch supplies device memory
and streams; every step of the search runs in the library's sm_103a kernels.

    import torch, paper_1901_00155_gb300 as dd
    plan = dd.Plan(m=1 << 20, n=256)                 # FP32 form
    res = plan.find_discord(T_cuda)                  # -> DiscordResult(index, nn_distance, ...)

The package never falls back to the CPU: if libdd.so or a CUDA device is
missing, the calls raise.
"""
from __future__ import annotations

import ctypes
from dataclasses import dataclass

from . import _lib

__all__ = ["Plan", "Engine", "Batch", "Completion", "DiscordResult", "DDError", "find_discord", "find_discord_batched",
           "PRECISIONS"]

PRECISIONS = {"fp32": _lib.DD_FP32, "tc_fp16": _lib.DD_TC_FP16, "tc_bf16": _lib.DD_TC_BF16}
# "global": the whole series z-normalised (Eq. 2); "window": every subsequence on its own
ZNORMS = {"global": 0, "window": 1}


class DDError(RuntimeError):
    def __init__(self, status: int, what: str = ""):
        lib = _lib.load()
        msg = lib.dd_status_string(int(status)).decode()
        super().__init__(f"{what}: {msg} (status {status})" if what else f"{msg} (status {status})")
        self.status = int(status)


@dataclass
class DiscordResult:
    index: int
    nn_distance: float
    exact: bool
    computed_pairs: int
    candidates: int


def _torch():
    import torch
    return torch


def _stream_ptr(stream=None):
    torch = _torch()
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


def _check(st: int, what: str):
    if st != _lib.DD_OK:
        raise DDError(st, what)


def _options(precision="fp32", paa_w=4, alphabet=4, early_abandon=True, paa_mode=0, phase1_max=4096,
             refine_k=128, local_cols=64, word_cols=512, shard_count=1, shard_index=0, znorm="global",
             diag=False) -> _lib.Options:
    o = _lib.Options()
    _lib.load().dd_options_default(ctypes.byref(o))
    o.precision = PRECISIONS[precision] if isinstance(precision, str) else int(precision)
    o.paa_w = paa_w
    o.alphabet = alphabet
    o.early_abandon = 1 if early_abandon else 0
    o.paa_mode = paa_mode
    o.phase1_max = phase1_max
    o.refine_k = refine_k
    o.local_cols = local_cols
    o.word_cols = word_cols
    o.shard_count = shard_count
    o.shard_index = shard_index
    if znorm not in ZNORMS:
        raise ValueError(f"znorm must be one of {sorted(ZNORMS)}, not {znorm!r}")
    o.znorm = ZNORMS[znorm]
    o.diag = 1 if diag else 0
    return o


def _as_result(r: _lib.Result) -> DiscordResult:
    return DiscordResult(int(r.index), float(r.nn_distance), bool(r.exact), int(r.computed_pairs), int(r.candidates))


def _check_series(T, m):
    torch = _torch()
    if not isinstance(T, torch.Tensor) or not T.is_cuda or T.dtype != torch.float32 or not T.is_contiguous():
        raise TypeError("T must be a contiguous float32 CUDA tensor")
    if T.numel() != m:
        raise ValueError(f"series has {T.numel()} points, plan expects {m}")


class _DevArray:
    """Exposes a device pointer through __cuda_array_interface__ (zero copy)."""

    def __init__(self, ptr, shape, typestr):
        self.__cuda_array_interface__ = {"data": (int(ptr), False), "shape": tuple(shape), "typestr": typestr,
                                         "version": 3, "strides": None, "stream": None}


class Plan:
    """A device plan for series of length ``m`` and subsequence length ``n``."""

    def __init__(self, m: int, n: int, precision="fp32", workspace=None, **opts):
        self._lib = _lib.load()
        self.m, self.n = int(m), int(n)
        self.N = self.m - self.n + 1
        self.options = _options(precision, **opts)
        self._ptr = ctypes.c_void_p()
        ws_ptr, ws_bytes = None, 0
        if workspace is not None:
            ws_ptr, ws_bytes = ctypes.c_void_p(workspace.data_ptr()), workspace.numel() * workspace.element_size()
            self._ws = workspace
        _check(self._lib.dd_plan_create(ctypes.byref(self._ptr), self.m, self.n, ctypes.byref(self.options), ws_ptr,
                                        ws_bytes), "dd_plan_create")

    @staticmethod
    def footprint(m: int, n: int, precision="fp32", **opts) -> int:
        o = _options(precision, **opts)
        return int(_lib.load().dd_plan_footprint(int(m), int(n), ctypes.byref(o)))

    def close(self):
        if getattr(self, "_ptr", None) and self._ptr.value:
            self._lib.dd_plan_destroy(self._ptr)
            self._ptr = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def find_discord(self, T, stream=None) -> DiscordResult:
        _check_series(T, self.m)
        r = _lib.Result()
        _check(self._lib.dd_find_discord(self._ptr, ctypes.c_void_p(T.data_ptr()), ctypes.byref(r),
                                         _stream_ptr(stream)), "dd_find_discord")
        return _as_result(r)

    def find_discord_async(self, T, out_dev, stream=None):
        """Enqueue the search; out_dev: a CUDA uint8 tensor of >= 40 bytes receiving a dd_result_t."""
        _check_series(T, self.m)
        _check(self._lib.dd_find_discord_async(self._ptr, ctypes.c_void_p(T.data_ptr()),
                                               ctypes.c_void_p(out_dev.data_ptr()), _stream_ptr(stream)),
               "dd_find_discord_async")

    @staticmethod
    def decode_result(buf) -> DiscordResult:
        """Decode a dd_result_t from a host uint8 tensor / bytes."""
        raw = bytes(buf.cpu().numpy().tobytes()) if hasattr(buf, "cpu") else bytes(buf)
        r = _lib.Result.from_buffer_copy(raw[: ctypes.sizeof(_lib.Result)])
        if r.status != _lib.DD_OK:
            raise DDError(r.status, "dd_find_discord_async")
        return _as_result(r)

    def find_discord_host(self, T_host, stream=None) -> DiscordResult:
        """End-to-end: T_host is a host float32 array (numpy or CPU tensor, pinned or not)."""
        import numpy as np
        if hasattr(T_host, "numpy"):
            if T_host.is_cuda:
                raise TypeError("find_discord_host takes host memory")
            ptr, numel = T_host.data_ptr(), T_host.numel()
            if T_host.dtype != _torch().float32 or not T_host.is_contiguous():
                raise TypeError("T_host must be contiguous float32")
        else:
            arr = np.ascontiguousarray(T_host, dtype=np.float32)
            T_host = arr
            ptr, numel = arr.ctypes.data, arr.size
        if numel != self.m:
            raise ValueError(f"series has {numel} points, plan expects {self.m}")
        r = _lib.Result()
        _check(self._lib.dd_find_discord_host(self._ptr, ctypes.c_void_p(ptr), ctypes.byref(r), _stream_ptr(stream)),
               "dd_find_discord_host")
        return _as_result(r)

    def nn_profile(self, T, out=None, stream=None):
        """Exhaustive squared nearest-neighbour distances of every row (CUDA float32[N])."""
        torch = _torch()
        _check_series(T, self.m)
        if out is None:
            out = torch.empty(self.N, dtype=torch.float32, device=T.device)
        _check(self._lib.dd_nn_profile(self._ptr, ctypes.c_void_p(T.data_ptr()), ctypes.c_void_p(out.data_ptr()),
                                       _stream_ptr(stream)), "dd_nn_profile")
        return out

    def nn_profile_diag(self, T, out=None, index=None, stream=None):
        """Exhaustive nearest-neighbour profile by the diagonal recurrence (plans made with
        ``diag=True`` or ``znorm="window"``): the squared distance of every row to its argument
        (CUDA float32[N]) and, if ``index`` is True or a CUDA int32[N] tensor, the argument."""
        torch = _torch()
        _check_series(T, self.m)
        if out is None:
            out = torch.empty(self.N, dtype=torch.float32, device=T.device)
        if index is True:
            index = torch.empty(self.N, dtype=torch.int32, device=T.device)
        if index is not None and index is not False:
            if index.dtype != torch.int32 or not index.is_cuda or not index.is_contiguous() or index.numel() < self.N:
                raise TypeError(f"index must be a contiguous int32 CUDA tensor of at least {self.N} elements")
        if out.dtype != torch.float32 or not out.is_cuda or not out.is_contiguous() or out.numel() < self.N:
            raise TypeError(f"out must be a contiguous float32 CUDA tensor of at least {self.N} elements")
        ip = ctypes.c_void_p(index.data_ptr()) if index is not None and index is not False else None
        _check(self._lib.dd_nn_profile_diag(self._ptr, ctypes.c_void_p(T.data_ptr()), ctypes.c_void_p(out.data_ptr()),
                                            ip, _stream_ptr(stream)), "dd_nn_profile_diag")
        return (out, index) if ip is not None else out

    def nn_rows(self, T, rows, out=None, stream=None):
        """Exhaustive squared nearest-neighbour distances of the given rows (int32 CUDA tensor)."""
        torch = _torch()
        _check_series(T, self.m)
        if rows.dtype != torch.int32 or not rows.is_cuda or not rows.is_contiguous():
            raise TypeError("rows must be a contiguous int32 CUDA tensor")
        if out is None:
            out = torch.empty(rows.numel(), dtype=torch.float32, device=T.device)
        _check(self._lib.dd_nn_rows(self._ptr, ctypes.c_void_p(T.data_ptr()), ctypes.c_void_p(rows.data_ptr()),
                                    rows.numel(), ctypes.c_void_p(out.data_ptr()), _stream_ptr(stream)), "dd_nn_rows")
        return out

    def prep(self, T, stream=None) -> dict:
        """Run only the preparation stage; returns zero-copy CUDA views of its arrays."""
        torch = _torch()
        _check_series(T, self.m)
        _check(self._lib.dd_prep(self._ptr, ctypes.c_void_p(T.data_ptr()), _stream_ptr(stream)), "dd_prep")
        v = _lib.View()
        _check(self._lib.dd_plan_view(self._ptr, ctypes.byref(v)), "dd_plan_view")
        m, N, D = int(v.m), int(v.N), int(v.dict_size)

        def t(ptr, shape, typestr):
            return torch.as_tensor(_DevArray(ptr, shape, typestr), device=T.device)

        return {"stats": t(v.stats, (8,), "<f8"), "P1": t(v.P1, (m + 1,), "<f8"), "P2": t(v.P2, (m + 1,), "<f8"),
                "mu_w": t(v.mu_w, (N,), "<f8"), "c_w": t(v.c_w, (N,), "<f8"), "code": t(v.code, (N,), "<i4"),
                "freq_hist": t(v.freq_hist, (D,), "<i4"), "order": t(v.order, (N,), "<i4"),
                "word_start": t(v.word_start, (D,), "<i4"), "ncand": t(v.ncand, (1,), "<i4"),
                "t32": t(v.t32, (m,), "<f4")}

    def order_view(self, like) -> dict:
        """The mean-bucketed row order of the plan's last call (dd_plan_order_view): zero-copy
        CUDA views of sig, sigpos, mubin, binstart and the bin geometry (lo, 1/w) on the device of
        ``like``, plus the stride of the input order and the bin count."""
        torch = _torch()
        v = _lib.OrderView()
        _check(self._lib.dd_plan_order_view(self._ptr, ctypes.byref(v)), "dd_plan_order_view")
        N, bins = int(v.N), int(v.bins)

        def t(ptr, k):
            return torch.as_tensor(_DevArray(ptr, (k,), "<i4"), device=like.device)

        geom = torch.as_tensor(_DevArray(v.geom, (4,), "<f8"), device=like.device)
        return {"sig": t(v.sig, N), "sigpos": t(v.sigpos, N), "mubin": t(v.mubin, N),
                "binstart": t(v.binstart, bins + 1), "stride": int(v.stride), "bins": bins,
                "lo": geom[0], "inv_w": geom[3]}

    def bound_terms(self, like) -> dict:
        """Per-row terms of the Gram form's error bound F_i(D) = alpha_i + beta D + gam_i
        sqrt(max(D, 0) + q2_i) (dd_plan_bound_view), filled by the plan's last call: zero-copy
        CUDA views on the device of the tensor ``like``, plus beta."""
        torch = _torch()
        v = _lib.BoundView()
        _check(self._lib.dd_plan_bound_view(self._ptr, ctypes.byref(v)), "dd_plan_bound_view")
        N = int(v.N)

        def t(ptr):
            return torch.as_tensor(_DevArray(ptr, (N,), "<f4"), device=like.device)

        return {"alpha": t(v.alpha), "gam": t(v.gam), "q2": t(v.q2), "beta": float(v.beta)}

    def last_launches(self) -> int:
        return int(self._lib.dd_plan_last_launches(self._ptr))

    def find_discords(self, T, k: int, stream=None) -> list:
        """Top-k discords: each the largest nearest-neighbour distance among the subsequences at
        least n away from the previous ones (dd_find_discords); fewer than k when rows run out."""
        _check_series(T, self.m)
        out = (_lib.Result * int(k))()
        _check(self._lib.dd_find_discords(self._ptr, ctypes.c_void_p(T.data_ptr()), int(k), out,
                                          _stream_ptr(stream)), "dd_find_discords")
        return [_as_result(r) for r in out if r.index >= 0]

    def inject(self, what: int):
        """Fault injection for tests (dd_plan_inject): 1 = stall the next tensor-core launch."""
        _check(self._lib.dd_plan_inject(self._ptr, int(what)), "dd_plan_inject")

    def set_graph(self, enable: bool = True):
        """Replay searches from a captured CUDA graph (default) or enqueue them directly."""
        _check(self._lib.dd_plan_set_graph(self._ptr, 1 if enable else 0), "dd_plan_set_graph")

    def set_profiling(self, enable: bool = True):
        _check(self._lib.dd_plan_set_profiling(self._ptr, 1 if enable else 0), "dd_plan_set_profiling")

    def profile(self) -> dict:
        """Distance-kernel measurements of the last synchronous call (needs set_profiling)."""
        pr = _lib.Profile()
        _check(self._lib.dd_plan_get_profile(self._ptr, ctypes.byref(pr)), "dd_plan_get_profile")
        return {"dist_launches": int(pr.dist_launches), "precision": int(pr.precision), "dist_ms": float(pr.dist_ms),
                "computed_pairs": int(pr.computed_pairs), "call_ms": float(pr.call_ms)}

    def waves(self) -> list:
        """Waves of distance tiles of the last call: kind, rows, items run, pairs
        evaluated and (with set_profiling) duration in ms, else -1."""
        cap = 64
        buf = (_lib.Wave * cap)()
        nw = int(self._lib.dd_plan_get_waves(self._ptr, buf, cap))
        if nw < 0:
            _check(-nw, "dd_plan_get_waves")
        return [{"kind": _lib.WAVE_KINDS.get(int(w.kind), str(int(w.kind))), "rows": int(w.rows),
                 "items": int(w.items), "pairs": int(w.pairs), "ms": float(w.ms)} for w in buf[:min(nw, cap)]]


def probe_fma_rate(fp64: bool = False, stream=None) -> float:
    """Measured FMA lane operations per second of this device's CUDA cores, FP32 (default) or
    FP64 (dd_probe_fma_rate): a roofline denominator for the kernels off the tensor cores."""
    r = ctypes.c_double()
    _check(_lib.load().dd_probe_fma_rate(1 if fp64 else 0, ctypes.byref(r), _stream_ptr(stream)),
           "dd_probe_fma_rate")
    return float(r.value)


def find_discord(T, n: int, precision="fp32", stream=None, **opts) -> DiscordResult:
    """One-shot search (creates and destroys a plan)."""
    with Plan(T.numel(), n, precision, **opts) as p:
        return p.find_discord(T, stream)


# option values under which a tuning table applies: the tuner times globally normalised,
# unsharded searches only
_TUNED_ONLY = {"znorm": ("global",), "shard_count": (0, 1)}


def group_by_tuned_options(ms, ns, table, precision=None, **opts):
    """Split a batch by the options a tuning table (see tuning.py) gives each (m, n): returns
    [(options dict, [positions in the batch])], in first-appearance order.

    Options passed explicitly (``precision`` when not None, and every keyword) win over the
    table's; the table fills in only the rest.  Per-window (znorm="window") or sharded searches
    ignore the table, which was tuned on neither.  Series without an entry run with the explicit
    options, precision "fp32" unless one was given."""
    from . import tuning

    explicit = dict(opts)
    if precision is not None:
        explicit["precision"] = precision
    use_table = all(explicit.get(k, ok[0]) in ok for k, ok in _TUNED_ONLY.items())
    groups, where = [], {}
    for pos, (m, n) in enumerate(zip(ms, ns)):
        tuned = tuning.lookup(table, int(m), int(n)) if use_table else {}
        o = {"precision": "fp32", **tuned, **explicit}
        key = tuple(sorted(o.items()))
        if key not in where:
            where[key] = len(groups)
            groups.append((o, []))
        groups[where[key]][1].append(pos)
    return groups


def find_discord_batched(series, ns, precision=None, stream=None, table=None, fused=False, seg_cols=None,
                         settle_min=None, settle_rows=None, **opts):
    """Independent searches over CUDA float32 tensors of possibly different lengths.  With a
    tuning table, each series runs with the options tuned for its (n, m bucket), explicit options
    taking precedence: one batched call per distinct option set, results in the input order.
    ``precision`` defaults to "fp32" (with a table: to the tuned form).

    ``fused=True`` (tensor-core precisions only) searches the whole list with one fused batch
    (dd_batch_*: every step one launch over all series) instead of the engine's concurrent
    per-series searches; a table (tuning.tune_batch) then supplies each group's schedule
    (``seg_cols``, ``settle_min``, ``settle_rows``) from the (n, m bucket) class with the most work among that n's
    series, and the precision of the batch's dominant class; explicit arguments take precedence."""
    if fused:
        per_n = {}
        if table is not None:
            from . import tuning
            ms = [s.numel() for s in series]
            tuned = tuning.lookup_batch(table, ms, ns)
            precision = precision if precision is not None else tuned.get("precision")
            if seg_cols is None and settle_min is None and settle_rows is None:
                per_n = tuning.lookup_batch_per_n(table, ms, ns)
        if precision is None:
            precision = "tc_fp16"
        with Batch(len(series), sum(s.numel() for s in series), max(int(x) for x in ns), precision,
                   seg_cols=seg_cols, settle_min=settle_min, settle_rows=settle_rows, **opts) as b:
            for n_, o in per_n.items():
                b.set_schedule(n_, o.get("seg_cols"), o.get("settle_min"), o.get("settle_rows"))
            return b.search(series, ns, stream)
    if table is not None:
        results = [None] * len(series)
        for o, pos in group_by_tuned_options([s.numel() for s in series], ns, table, precision, **opts):
            prec = o.pop("precision")
            part = find_discord_batched([series[i] for i in pos], [ns[i] for i in pos], prec, stream, None, **o)
            for i, r in zip(pos, part):
                results[i] = r
        return results
    if precision is None:
        precision = "fp32"
    lib = _lib.load()
    k = len(series)
    ptrs = (ctypes.c_void_p * k)(*[ctypes.c_void_p(s.data_ptr()) for s in series])
    ms = (ctypes.c_int64 * k)(*[s.numel() for s in series])
    nn = (ctypes.c_int32 * k)(*[int(x) for x in ns])
    out = (_lib.Result * k)()
    for s in series:
        _check_series(s, s.numel())
    o = _options(precision, **opts)
    st = lib.dd_find_discord_batched(k, ptrs, ms, nn, ctypes.byref(o), out, _stream_ptr(stream))
    results = []
    for r in out:
        results.append(_as_result(r) if r.status == _lib.DD_OK else DDError(r.status, "batched item"))
    if st != _lib.DD_OK and all(isinstance(r, DDError) for r in results):
        raise DDError(st, "dd_find_discord_batched")
    return results


class Batch:
    """A fused batch plan (dd_batch_*): capacity ``max_series`` series of ``max_values`` values
    in total, subsequence lengths up to ``n_max``, tensor-core precision.  ``search`` runs every
    series with one launch per step of the search for all of them (per distinct n), captured into
    a CUDA graph that the next call with the same shapes replays; each result equals that of
    ``find_discord`` on the series alone."""

    def __init__(self, max_series: int, max_values: int, n_max: int, precision="tc_fp16", seg_cols=None,
                 settle_min=None, settle_rows=None, **opts):
        self._lib = _lib.load()
        self.options = _options(precision, **opts)
        cfg = _lib.BatchConfig()
        self._lib.dd_batch_config_default(ctypes.byref(cfg))
        if seg_cols is not None:
            cfg.seg_cols = int(seg_cols)
        if settle_min is not None:
            cfg.settle_min = int(settle_min)
        if settle_rows is not None:
            cfg.settle_rows = int(settle_rows)
        self.config = cfg
        self._ptr = ctypes.c_void_p()
        _check(self._lib.dd_batch_create(ctypes.byref(self._ptr), int(max_series), int(max_values), int(n_max),
                                         ctypes.byref(self.options), ctypes.byref(cfg)), "dd_batch_create")

    @staticmethod
    def footprint(max_series: int, max_values: int, n_max: int) -> int:
        return int(_lib.load().dd_batch_footprint(int(max_series), int(max_values), int(n_max)))

    def search(self, series, ns, stream=None) -> list:
        """Results in input order: DiscordResult, or DDError for a series that failed."""
        k = len(series)
        for s in series:
            _check_series(s, s.numel())
        ptrs = (ctypes.c_void_p * max(k, 1))(*[ctypes.c_void_p(s.data_ptr()) for s in series])
        ms = (ctypes.c_int64 * max(k, 1))(*[s.numel() for s in series])
        nn = (ctypes.c_int32 * max(k, 1))(*[int(x) for x in ns])
        out = (_lib.Result * max(k, 1))()
        st = self._lib.dd_batch_search(self._ptr, k, ptrs, ms, nn, out, _stream_ptr(stream))
        # a failure of the whole call marks every entry with its status
        if st in (_lib.DD_EBUSY, _lib.DD_ENOMEM, _lib.DD_ENOTSUP, _lib.DD_ECUDA) and all(r.status == st
                                                                                       for r in out[:k]):
            raise DDError(st, "dd_batch_search")
        return [_as_result(r) if r.status == _lib.DD_OK else DDError(r.status, "batch item") for r in out[:k]]

    def set_schedule(self, n: int, seg_cols=None, settle_min=None, settle_rows=None):
        """The schedule of the series with subsequence length n (all None: the batch's own)."""
        if seg_cols is None and settle_min is None and settle_rows is None:
            _check(self._lib.dd_batch_set_schedule(self._ptr, int(n), None), "dd_batch_set_schedule")
            return
        cfg = _lib.BatchConfig()
        ctypes.memmove(ctypes.byref(cfg), ctypes.byref(self.config), ctypes.sizeof(cfg))
        if seg_cols is not None:
            cfg.seg_cols = int(seg_cols)
        if settle_min is not None:
            cfg.settle_min = int(settle_min)
        if settle_rows is not None:
            cfg.settle_rows = int(settle_rows)
        _check(self._lib.dd_batch_set_schedule(self._ptr, int(n), ctypes.byref(cfg)), "dd_batch_set_schedule")

    def graph_replays(self) -> int:
        return int(self._lib.dd_batch_graph_replays(self._ptr))

    def close(self):
        if getattr(self, "_ptr", None) and self._ptr.value:
            self._lib.dd_batch_destroy(self._ptr)
            self._ptr = ctypes.c_void_p()

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


@dataclass
class Completion:
    id: int
    result: object      # DiscordResult, or DDError for a failed request
    queue_ms: float     # submission -> a worker took it
    service_ms: float   # a worker took it -> result on the host


class Engine:
    """Concurrent searches (dd_engine_*): ``workers`` host threads, each with its own
    CUDA stream, take requests from one queue and admit them against ``budget`` bytes of
    device memory (default: workers x the largest plan of m <= m_max, n <= n_max; smaller
    requests pass one that does not fit).  ``submit`` accepts
    a CUDA float32 tensor (already complete on its stream) or host data (numpy / CPU
    tensor; the worker copies it); the series is kept alive until its completion is
    polled."""

    def __init__(self, workers: int, m_max: int, n_max: int, precision="fp32", budget: int | None = None, **opts):
        self._lib = _lib.load()
        self.options = _options(precision, **opts)
        self._ptr = ctypes.c_void_p()
        _check(self._lib.dd_engine_create_budget(ctypes.byref(self._ptr), int(workers), ctypes.byref(self.options),
                                                 int(m_max), int(n_max), int(budget or 0)), "dd_engine_create")
        self._keep = {}
        self._next = 0

    def submit(self, T, n: int, id: int | None = None) -> int:
        import numpy as np
        if id is None:
            id = self._next
        self._next = max(self._next, int(id) + 1)
        if hasattr(T, "is_cuda") and T.is_cuda:
            if T.dtype != _torch().float32 or not T.is_contiguous():
                raise TypeError("T must be a contiguous float32 tensor")
            ptr, m, flags, keep = T.data_ptr(), T.numel(), _lib.DD_SERIES_DEVICE, T
        else:
            a = np.ascontiguousarray(T.numpy() if hasattr(T, "numpy") else T, dtype=np.float32)
            ptr, m, flags, keep = a.ctypes.data, a.size, _lib.DD_SERIES_HOST, a
        self._keep[int(id)] = keep
        _check(self._lib.dd_engine_submit(self._ptr, int(id), ctypes.c_void_p(ptr), int(m), int(n), flags),
               "dd_engine_submit")
        return int(id)

    def poll(self, max_items: int = 64, wait_ms: int = 0) -> list:
        buf = (_lib.Completion * max_items)()
        k = int(self._lib.dd_engine_poll(self._ptr, buf, max_items, int(wait_ms)))
        if k < 0:
            _check(-k, "dd_engine_poll")
        out = []
        for c in buf[:k]:
            self._keep.pop(int(c.id), None)
            r = c.result
            res = _as_result(r) if r.status == _lib.DD_OK else DDError(r.status, f"request {int(c.id)}")
            out.append(Completion(int(c.id), res, float(c.queue_ms), float(c.service_ms)))
        return out

    def outstanding(self) -> int:
        return int(self._lib.dd_engine_outstanding(self._ptr))

    def drain(self) -> list:
        """Waits for every outstanding request; returns their completions."""
        out = []
        while self.outstanding() > 0:
            out += self.poll(256, -1)
        return out

    def close(self):
        if getattr(self, "_ptr", None) and self._ptr.value:
            self._lib.dd_engine_destroy(self._ptr)
            self._ptr = ctypes.c_void_p()
            self._keep.clear()

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
