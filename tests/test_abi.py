"""The C-ABI library builds, loads and exports every symbol include/dd.h
declares; host-only entry points (no device work) behave as documented."""
import ctypes
import os
import re

import pytest

from paper_1901_00155_gb300 import _lib

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "dd.h")).read()
    return sorted(set(re.findall(r"DD_API\s+[\w\s\*]+?\b(dd_\w+)\s*\(", src)))


def test_header_declares_functions():
    names = _declared()
    assert "dd_find_discord" in names and "dd_plan_create" in names
    assert len(names) >= 14


def test_library_exports_every_declared_symbol():
    lib = _lib.load()
    for name in _declared():
        assert hasattr(lib, name), name
        assert name in _lib.SIGNATURES, f"binding lacks {name}"
    assert set(_lib.SIGNATURES) == set(_declared())


def test_struct_layouts():
    assert ctypes.sizeof(_lib.Options) == 64
    assert ctypes.sizeof(_lib.Result) == 40
    assert ctypes.sizeof(_lib.View) == 24 + 11 * 8
    assert ctypes.sizeof(_lib.Wave) == 32
    assert ctypes.sizeof(_lib.Completion) == 64
    assert ctypes.sizeof(_lib.BoundView) == 16 + 3 * 8
    assert ctypes.sizeof(_lib.OrderView) == 24 + 5 * 8
    assert ctypes.sizeof(_lib.BatchConfig) == 16


def test_options_default_and_footprint():
    lib = _lib.load()
    o = _lib.Options()
    lib.dd_options_default(ctypes.byref(o))
    assert (o.precision, o.paa_w, o.alphabet, o.early_abandon, o.paa_mode) == (0, 4, 4, 1, 0)
    fp = lib.dd_plan_footprint(1 << 20, 256, ctypes.byref(o))
    assert 32 << 20 < fp < 1 << 30
    assert lib.dd_plan_footprint(1000, 400, ctypes.byref(o)) == 0  # N < 2n
    assert lib.dd_plan_footprint(1000, 0, ctypes.byref(o)) == 0
    o.alphabet = 1
    assert lib.dd_plan_footprint(1 << 16, 64, ctypes.byref(o)) == 0
    lib.dd_options_default(ctypes.byref(o))
    o.reserved[2] = 1
    assert lib.dd_plan_footprint(1 << 16, 64, ctypes.byref(o)) == 0
    for field in ("znorm", "diag"):
        lib.dd_options_default(ctypes.byref(o))
        setattr(o, field, 2)
        assert lib.dd_plan_footprint(1 << 16, 64, ctypes.byref(o)) == 0


def test_window_and_diag_options():
    """Per-window plans and plans with the diagonal-recurrence workspace: footprints, and the
    combinations refused before any device work."""
    import paper_1901_00155_gb300 as dd
    lib = _lib.load()
    base = dd.Plan.footprint(1 << 16, 256)
    win = dd.Plan.footprint(1 << 16, 256, znorm="window")
    dg = dd.Plan.footprint(1 << 16, 256, diag=True)
    assert win == dg > base
    N = (1 << 16) - 255
    assert win - base >= N * (8 + 8 + 16 + 4 + 8 + 8 + 4 + 8)  # window stats, data, keys, bounds, FP64 results
    assert dd.Plan.footprint(1 << 16, 256, "tc_fp16", diag=True) > dd.Plan.footprint(1 << 16, 256, "tc_fp16")
    with pytest.raises(ValueError):
        dd.Plan.footprint(1 << 16, 256, znorm="per-window")
    p = ctypes.c_void_p()
    for kw in ({"precision": "tc_fp16", "znorm": "window"}, {"znorm": "window", "shard_count": 2}):
        o = dd._options(**kw)
        assert lib.dd_plan_create(ctypes.byref(p), 1 << 16, 256, ctypes.byref(o), None, 0) == _lib.DD_ENOTSUP
    o = dd._options(diag=True)
    assert lib.dd_plan_create(ctypes.byref(p), (1 << 26) + 300, 100, ctypes.byref(o), None, 0) == _lib.DD_ENOTSUP
    assert p.value is None
    assert lib.dd_nn_profile_diag(None, None, None, None, None) == _lib.DD_EINVAL


def test_status_strings():
    lib = _lib.load()
    assert lib.dd_status_string(0) == b"ok"
    assert b"NaN" in lib.dd_status_string(3)
    assert lib.dd_status_string(99) == b"unknown status"


def test_plan_create_rejects_bad_sizes_without_device_work():
    lib = _lib.load()
    p = ctypes.c_void_p()
    assert lib.dd_plan_create(ctypes.byref(p), 100, 40, None, None, 0) == _lib.DD_EINVAL
    assert lib.dd_plan_create(None, 100, 4, None, None, 0) == _lib.DD_EINVAL
    assert p.value is None
    assert lib.dd_find_discord(None, None, None, None) == _lib.DD_EINVAL


def test_product_path_does_not_import_oracle():
    pkg = os.path.join(ROOT, "paper_1901_00155_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h")):
                txt = open(os.path.join(dirpath, f)).read()
                assert "import oracle" not in txt and "from oracle" not in txt, f
                assert "dd_oracle" not in txt, f


def test_new_entry_points_reject_bad_arguments_without_device_work():
    """Null handles and bad arguments are refused before any CUDA call."""
    lib = _lib.load()
    assert lib.dd_plan_get_waves(None, None, 0) == -_lib.DD_EINVAL
    assert lib.dd_plan_set_graph(None, 1) == _lib.DD_EINVAL
    assert lib.dd_plan_inject(None, 1) == _lib.DD_EINVAL
    assert lib.dd_find_discords(None, None, 3, None, None) == _lib.DD_EINVAL
    e = ctypes.c_void_p()
    assert lib.dd_engine_create(ctypes.byref(e), 0, None, 8192, 128) == _lib.DD_EINVAL   # no workers
    assert lib.dd_engine_create(ctypes.byref(e), 65, None, 8192, 128) == _lib.DD_EINVAL  # too many
    assert lib.dd_engine_create(ctypes.byref(e), 2, None, 100, 40) == _lib.DD_EINVAL     # N < 2n
    assert lib.dd_engine_create(None, 2, None, 8192, 128) == _lib.DD_EINVAL
    assert e.value is None
    assert lib.dd_engine_submit(None, 0, None, 10, 2, 0) == _lib.DD_EINVAL
    assert lib.dd_engine_poll(None, None, 0, 0) == -_lib.DD_EINVAL
    assert lib.dd_engine_outstanding(None) == 0
    lib.dd_engine_destroy(None)
    opts = _lib.Options()
    lib.dd_options_default(ctypes.byref(opts))
    assert opts.shard_count == 0 and opts.shard_index == 0
    assert lib.dd_find_discord_batched(-1, None, None, None, None, None, None) == _lib.DD_EINVAL
    assert lib.dd_find_discord_batched(0, None, None, None, None, None, None) == _lib.DD_OK


def test_sharded_footprint_matches_unsharded():
    """Sharding selects rows; the plan's device footprint does not change."""
    import paper_1901_00155_gb300 as dd
    for prec in ("fp32", "tc_fp16"):
        a = dd.Plan.footprint(1 << 16, 256, prec)
        assert a > 0 and dd.Plan.footprint(1 << 16, 256, prec, shard_count=4, shard_index=3) == a


def test_batch_entry_points_reject_bad_arguments_without_device_work():
    """The fused batch: defaults, footprint limits and argument checks before any CUDA call."""
    lib = _lib.load()
    cfg = _lib.BatchConfig()
    lib.dd_batch_config_default(ctypes.byref(cfg))
    assert cfg.seg_cols == 512 and cfg.settle_min == 4 and cfg.settle_rows == 64 and list(cfg.reserved) == [0]
    fp = lib.dd_batch_footprint(512, 10_200_000, 256)
    assert 10 << 30 < fp < 16 << 30  # two 16-bit operand matrices of ~10.4 M rows x 256 dominate
    assert lib.dd_batch_footprint(0, 1000, 64) == 0
    assert lib.dd_batch_footprint(4, 0, 64) == 0
    assert lib.dd_batch_footprint(4, 1000, 0) == 0
    assert lib.dd_batch_footprint(4, 1000, 70000) == 0
    assert lib.dd_batch_footprint(4, 1 << 30, 64) == 0  # beyond 2^30 rows
    b = ctypes.c_void_p()
    o = _lib.Options()
    lib.dd_options_default(ctypes.byref(o))
    assert lib.dd_batch_create(ctypes.byref(b), 4, 1000, 64, ctypes.byref(o), None) == _lib.DD_ENOTSUP  # FP32
    o.precision = 1
    o.znorm = 1
    assert lib.dd_batch_create(ctypes.byref(b), 4, 1000, 64, ctypes.byref(o), None) == _lib.DD_ENOTSUP
    o.znorm = 0
    for bad in (0, 100, 1 << 17):
        cfg.seg_cols = bad
        assert lib.dd_batch_create(ctypes.byref(b), 4, 1000, 64, ctypes.byref(o), ctypes.byref(cfg)) == \
            _lib.DD_EINVAL
    lib.dd_batch_config_default(ctypes.byref(cfg))
    cfg.settle_min = -1
    assert lib.dd_batch_create(ctypes.byref(b), 4, 1000, 64, ctypes.byref(o), ctypes.byref(cfg)) == _lib.DD_EINVAL
    for bad in (0, 16, 96, 256):
        lib.dd_batch_config_default(ctypes.byref(cfg))
        cfg.settle_rows = bad
        assert lib.dd_batch_create(ctypes.byref(b), 4, 1000, 64, ctypes.byref(o), ctypes.byref(cfg)) == \
            _lib.DD_EINVAL
    lib.dd_batch_config_default(ctypes.byref(cfg))
    cfg.reserved[0] = 3
    assert lib.dd_batch_create(ctypes.byref(b), 4, 1000, 64, ctypes.byref(o), ctypes.byref(cfg)) == _lib.DD_EINVAL
    assert lib.dd_batch_create(None, 4, 1000, 64, ctypes.byref(o), None) == _lib.DD_EINVAL
    assert lib.dd_batch_create(ctypes.byref(b), 0, 1000, 64, ctypes.byref(o), None) == _lib.DD_EINVAL
    assert b.value is None
    assert lib.dd_batch_search(None, 1, None, None, None, None, None) == _lib.DD_EINVAL
    assert lib.dd_batch_graph_replays(None) == -1
    assert lib.dd_batch_set_schedule(None, 64, None) == _lib.DD_EINVAL
    lib.dd_batch_destroy(None)
