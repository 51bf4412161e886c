"""FP64 CPU oracle for discord discovery -- TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and the benchmark's
``cpu_baseline`` / reference leg may import this package.  The product path
(the CUDA library and its Python binding) never imports or calls it, and the
two share no code.

The arithmetic lives in ``dd_oracle.c`` (plain C99 + OpenMP, compiled by
:func:`build`); this module only marshals numpy arrays through ctypes.
Functions and the passages of the paper they follow:

* :func:`znorm`          -- Eq. 2
* :func:`nn_rows`        -- Section 2.1 (non-self match) + Eq. 1, brute force
* :func:`nn_profile`     -- the same for every subsequence
* :func:`discord_brute`  -- Section 2.1 "discord" definition ("O1")
* :func:`window_stats`   -- rows of the subsequence matrix, Eq. 5
* :func:`breakpoints`    -- SAX breakpoints, text after Eq. 4
* :func:`sax`            -- Eq. 3 + Eq. 4 + Eq. 9
* :func:`index`          -- Eq. 7, Eq. 8, Eq. 10
* :func:`hotsax`         -- Algorithms 2-4 on the CPU ("O2")
* :func:`window_mu_sigma`, :func:`dist2` and ``znorm="window"`` in
  :func:`nn_rows` / :func:`nn_profile` / :func:`discord_brute` /
  :func:`discords_brute` -- the per-window z-normalised variant (every
  subsequence normalised on its own, a constant one to the zero vector; one
  reading of Algorithm 2's Znormalize step)
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "dd_oracle.c")
_OUT_DIR = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_OUT_DIR, "libdd_oracle.so")
_lock = threading.Lock()
_lib = None

OK, EINVAL, ENOMEM, ENONFINITE = 0, 1, 2, 3


class OracleError(RuntimeError):
    def __init__(self, code: int, what: str):
        super().__init__(f"oracle {what} failed with status {code}")
        self.code = code


def build(force: bool = False) -> str:
    """Compile dd_oracle.c into a shared library (idempotent)."""
    os.makedirs(_OUT_DIR, exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    cmd = ["gcc", "-std=gnu99", "-O2", "-fopenmp", "-ffp-contract=off", "-fPIC", "-shared",
           "-o", tmp, _SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        build()
        lib = ctypes.CDLL(_LIB_PATH)
        P = ctypes.c_void_p
        i64, i32 = ctypes.c_int64, ctypes.c_int32
        sig = {
            "dd_oracle_threads": ([], ctypes.c_int),
            "dd_oracle_znorm": ([P, i64, P, P, P], ctypes.c_int),
            "dd_oracle_nn_rows": ([P, i64, i32, P, i64, P, P], ctypes.c_int),
            "dd_oracle_nn_profile": ([P, i64, i32, P], ctypes.c_int),
            "dd_oracle_discord_brute": ([P, i64, i32, P, P], ctypes.c_int),
            "dd_oracle_window_stats": ([P, i64, i32, P, P], ctypes.c_int),
            "dd_oracle_breakpoints": ([i32, P], ctypes.c_int),
            "dd_oracle_sax": ([P, i64, i32, i32, i32, i32, P, P], ctypes.c_int),
            "dd_oracle_index": ([P, i64, i32, P, P, P, P, P], ctypes.c_int),
            "dd_oracle_hotsax": ([P, i64, i32, i32, i32, i32, P, P, P], ctypes.c_int),
            "dd_oracle_window_mu_sigma": ([P, i64, i32, P, P], ctypes.c_int),
            "dd_oracle_dist2": ([P, i64, i32, i32, i64, i64, P], ctypes.c_int),
            "dd_oracle_nn_rows_w": ([P, i64, i32, P, i64, P, P], ctypes.c_int),
            "dd_oracle_nn_profile_w": ([P, i64, i32, P], ctypes.c_int),
        }
        for name, (args, res) in sig.items():
            f = getattr(lib, name)
            f.argtypes = args
            f.restype = res
        _lib = lib
        return lib


def _f32(T) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(T, dtype=np.float32))


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def _chk(st: int, what: str):
    if st != OK:
        raise OracleError(st, what)


def threads() -> int:
    return int(_load().dd_oracle_threads())


def znorm(T):
    """Eq. 2 -> (t_hat float64[m], mu, sigma)."""
    T = _f32(T)
    out = np.empty(T.size, dtype=np.float64)
    mu, sg = ctypes.c_double(), ctypes.c_double()
    _chk(_load().dd_oracle_znorm(_ptr(T), T.size, _ptr(out), ctypes.byref(mu), ctypes.byref(sg)), "znorm")
    return out, mu.value, sg.value


def _znorm_code(znorm: str) -> int:
    if znorm not in ("global", "window"):
        raise ValueError(f"znorm must be 'global' or 'window', not {znorm!r}")
    return 0 if znorm == "global" else 1


def nn_rows(T, n: int, rows, znorm: str = "global"):
    """Squared nearest non-self-match distance (and its argument) of the given rows."""
    T = _f32(T)
    rows = np.ascontiguousarray(np.asarray(rows, dtype=np.int64))
    nn2 = np.empty(rows.size, dtype=np.float64)
    arg = np.empty(rows.size, dtype=np.int64)
    f = _load().dd_oracle_nn_rows if _znorm_code(znorm) == 0 else _load().dd_oracle_nn_rows_w
    _chk(f(_ptr(T), T.size, n, _ptr(rows), rows.size, _ptr(nn2), _ptr(arg)), "nn_rows")
    return nn2, arg


def nn_profile(T, n: int, znorm: str = "global") -> np.ndarray:
    """Squared nearest non-self-match distance of every subsequence (float64[N])."""
    T = _f32(T)
    N = T.size - n + 1
    out = np.empty(max(N, 0), dtype=np.float64)
    f = _load().dd_oracle_nn_profile if _znorm_code(znorm) == 0 else _load().dd_oracle_nn_profile_w
    _chk(f(_ptr(T), T.size, n, _ptr(out)), "nn_profile")
    return out


def discord_brute(T, n: int, znorm: str = "global"):
    """O1: (index, nn^2) of the discord; ties -> smallest index."""
    T = _f32(T)
    if _znorm_code(znorm) == 1:
        nn2 = nn_profile(T, n, znorm)
        i = int(np.argmax(nn2))  # first maximiser = smallest index
        return i, float(nn2[i])
    idx, d2 = ctypes.c_int64(), ctypes.c_double()
    _chk(_load().dd_oracle_discord_brute(_ptr(T), T.size, n, ctypes.byref(idx), ctypes.byref(d2)), "discord_brute")
    return int(idx.value), float(d2.value)


def window_mu_sigma(T, n: int):
    """Per-window mean and population sigma of the input series (two-pass FP64)."""
    T = _f32(T)
    N = T.size - n + 1
    mu = np.empty(max(N, 0), dtype=np.float64)
    sg = np.empty(max(N, 0), dtype=np.float64)
    _chk(_load().dd_oracle_window_mu_sigma(_ptr(T), T.size, n, _ptr(mu), _ptr(sg)), "window_mu_sigma")
    return mu, sg


def dist2(T, n: int, i: int, j: int, znorm: str = "global") -> float:
    """Squared distance between subsequences i and j under either normalisation."""
    T = _f32(T)
    out = ctypes.c_double()
    _chk(_load().dd_oracle_dist2(_ptr(T), T.size, n, _znorm_code(znorm), int(i), int(j), ctypes.byref(out)),
         "dist2")
    return float(out.value)


def discords_brute(T, n: int, k: int, znorm: str = "global"):
    """Top-k discords by definition: repeatedly the largest nearest non-self-match distance
    (first maximiser = smallest index), among subsequences at least n away from those already
    chosen.  Returns [(index, nn2)]."""
    nn2 = nn_profile(T, n, znorm)
    allowed = np.ones(nn2.size, dtype=bool)
    out = []
    for _ in range(k):
        if not allowed.any():
            break
        cand = np.where(allowed, nn2, -np.inf)
        i = int(np.argmax(cand))
        out.append((i, float(nn2[i])))
        allowed[max(0, i - n + 1):min(nn2.size, i + n)] = False
    return out


def window_stats(T, n: int):
    """(mu_w, c_w) float64[N]: mean and centred sum of squares of each row."""
    T = _f32(T)
    N = T.size - n + 1
    mu = np.empty(N, dtype=np.float64)
    c = np.empty(N, dtype=np.float64)
    _chk(_load().dd_oracle_window_stats(_ptr(T), T.size, n, _ptr(mu), _ptr(c)), "window_stats")
    return mu, c


def breakpoints(A: int) -> np.ndarray:
    out = np.empty(A - 1, dtype=np.float64)
    _chk(_load().dd_oracle_breakpoints(A, _ptr(out)), "breakpoints")
    return out


def sax(T, n: int, w: int = 4, A: int = 4, paa_mode: int = 0, want_paa: bool = False):
    """Word code per row (int32[N]) and optionally the PAA values (float64[N, w])."""
    T = _f32(T)
    N = T.size - n + 1
    code = np.empty(N, dtype=np.int32)
    paa = np.empty((N, w), dtype=np.float64) if want_paa else None
    _chk(_load().dd_oracle_sax(_ptr(T), T.size, n, w, A, paa_mode, _ptr(code),
                               _ptr(paa) if want_paa else None), "sax")
    return (code, paa) if want_paa else code


def index(code, dict_size: int):
    """(freq int64[N], cand int64[k], offsets int64[dict+1], members int64[N])."""
    code = np.ascontiguousarray(np.asarray(code, dtype=np.int32))
    N = code.size
    freq = np.empty(N, dtype=np.int64)
    cand = np.empty(N, dtype=np.int64)
    nc = ctypes.c_int64()
    offs = np.empty(dict_size + 1, dtype=np.int64)
    mem = np.empty(N, dtype=np.int64)
    _chk(_load().dd_oracle_index(_ptr(code), N, dict_size, _ptr(freq), _ptr(cand), ctypes.byref(nc),
                                 _ptr(offs), _ptr(mem)), "index")
    return freq, cand[: nc.value].copy(), offs, mem


def hotsax(T, n: int, w: int = 4, A: int = 4, paa_mode: int = 0):
    """O2: (index, nn^2, evaluated pairs) from Algorithms 2-4 on the CPU."""
    T = _f32(T)
    idx, d2, ev = ctypes.c_int64(), ctypes.c_double(), ctypes.c_int64()
    _chk(_load().dd_oracle_hotsax(_ptr(T), T.size, n, w, A, paa_mode, ctypes.byref(idx), ctypes.byref(d2),
                                  ctypes.byref(ev)), "hotsax")
    return int(idx.value), float(d2.value), int(ev.value)
