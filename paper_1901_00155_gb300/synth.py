"""Seeded synthetic time series shaped like the discord-search workloads.

The paper measures on real series (SCD-1M / SCD-10M, Section 4, Table 2) that
are not available here; these generators stand in for them.  They hold none of
the method's arithmetic (no normalisation, no distances, no SAX) and are the
only module shared by the oracle side and the CUDA side of the tests and the
benchmark.

Series kinds
  * ``"rw"``   random walk: cumulative sum of N(0, 1) steps.
  * ``"sine"`` sin(2*pi*k/200) + N(0, 0.1^2) noise.

Anomaly kinds (inserted at seeded, non-overlapping offsets that lie at least
2n apart and at least n from either end):
  * ``"burst"``  T[o+k] += 3*sin(2*pi*k/32) for k < 128
  * ``"flat"``   T[o:o+n] = T[o]
  * ``"spike"``  T[o] += 20 (random walk) or += 3 (sine)
  * ``"phase"``  sine: the sine component over [o, o+n) is shifted by pi;
                 random walk: the segment [o, o+n) is reversed in time.

All outputs are float32 numpy arrays.  numpy's PCG64 ``default_rng(seed)`` is
the only source of randomness.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

SINE_PERIOD = 200.0
SINE_NOISE = 0.1
BURST_LEN = 128
BURST_PERIOD = 32.0
BURST_AMP = 3.0


@dataclass(frozen=True)
class SeriesSpec:
    kind: str            # "rw" | "sine"
    m: int
    n: int
    seed: int
    anomalies: tuple = field(default_factory=tuple)

    def name(self) -> str:
        an = "+".join(self.anomalies) if self.anomalies else "none"
        return f"{self.kind}_m{self.m}_n{self.n}_s{self.seed}_{an}"


def _offsets(rng: np.random.Generator, m: int, n: int, count: int) -> list[int]:
    """Seeded offsets, pairwise >= 2n apart and >= n from both ends."""
    if count == 0:
        return []
    span = max(BURST_LEN, n)
    lo, hi = n, m - span - n
    if hi <= lo:
        raise ValueError("series too short for the requested anomalies")
    out: list[int] = []
    for _ in range(10000):
        o = int(rng.integers(lo, hi))
        if all(abs(o - p) >= 2 * n + span for p in out):
            out.append(o)
            if len(out) == count:
                return sorted(out)
    raise ValueError("could not place anomalies; series too short")


def make_series(spec: SeriesSpec) -> tuple[np.ndarray, list[int]]:
    """Return (T float32[m], anomaly offsets)."""
    rng = np.random.default_rng(spec.seed)
    m, n = spec.m, spec.n
    k = np.arange(m, dtype=np.float64)
    if spec.kind == "rw":
        base = np.cumsum(rng.standard_normal(m))
        sine = None
    elif spec.kind == "sine":
        sine = np.sin(2.0 * math.pi * k / SINE_PERIOD)
        base = sine + SINE_NOISE * rng.standard_normal(m)
    else:
        raise ValueError(f"unknown series kind {spec.kind!r}")
    offs = _offsets(rng, m, n, len(spec.anomalies))
    t = base.copy()
    for kind, o in zip(spec.anomalies, offs):
        if kind == "burst":
            kk = np.arange(BURST_LEN, dtype=np.float64)
            t[o:o + BURST_LEN] += BURST_AMP * np.sin(2.0 * math.pi * kk / BURST_PERIOD)
        elif kind == "flat":
            t[o:o + n] = t[o]
        elif kind == "spike":
            t[o] += 20.0 if spec.kind == "rw" else 3.0
        elif kind == "phase":
            if sine is not None:
                t[o:o + n] -= 2.0 * sine[o:o + n]
            else:
                t[o:o + n] = t[o:o + n][::-1].copy()
        else:
            raise ValueError(f"unknown anomaly kind {kind!r}")
    return t.astype(np.float32), offs


def random_small(rng: np.random.Generator, m: int, kind: str | None = None) -> np.ndarray:
    """Small adversarial-ish float32 series for brute-force parity sweeps.

    Mixes random walks, sines, plateaus with exact repeats (ties) and integer
    valued data, so that exact ties and constant windows occur.
    """
    kinds = ["rw", "sine", "ints", "plateau", "repeat", "gauss"]
    kind = kind or kinds[int(rng.integers(len(kinds)))]
    if kind == "rw":
        t = np.cumsum(rng.standard_normal(m))
    elif kind == "sine":
        p = float(rng.uniform(4, 40))
        t = np.sin(2 * math.pi * np.arange(m) / p) + 0.05 * rng.standard_normal(m)
    elif kind == "ints":
        t = rng.integers(-3, 4, size=m).astype(np.float64)
    elif kind == "plateau":
        t = np.repeat(rng.integers(0, 3, size=m // 4 + 1), 4)[:m].astype(np.float64)
    elif kind == "repeat":
        p = int(rng.integers(2, 9))
        unit = rng.integers(-2, 3, size=p).astype(np.float64)
        t = np.tile(unit, m // p + 1)[:m]
        t[int(rng.integers(m))] += float(rng.integers(1, 5))
    else:
        t = rng.standard_normal(m)
    return np.asarray(t, dtype=np.float32)


# Workloads of the discord benchmark suite (sizes and structure of the paper's
# experiments, Section 4: series of length ~1e6, subsequence lengths 64..2048).
def workload_small() -> SeriesSpec:
    """Random walk, m=8192, n=128, one sine burst."""
    return SeriesSpec("rw", 8192, 128, 0, ("burst",))


def workloads_medium() -> list[SeriesSpec]:
    """Random walk and sine+noise, m=262144, n in {128,256,512}, three anomalies."""
    out = []
    for kind in ("rw", "sine"):
        for n in (128, 256, 512):
            for seed in (0, 1):
                out.append(SeriesSpec(kind, 262144, n, seed, ("flat", "spike", "phase")))
    return out


def workload_large(seed: int = 0) -> SeriesSpec:
    """Random walk, m=2^20, n=256, five anomalies."""
    return SeriesSpec("rw", 1 << 20, 256, seed, ("burst", "flat", "spike", "phase", "burst"))


def _log_uniform_int(rng: np.random.Generator, lo: int, hi: int) -> int:
    return int(round(math.exp(rng.uniform(math.log(lo), math.log(hi)))))


def workload_batch(seed: int = 0, count: int = 512) -> list[SeriesSpec]:
    """Many uneven series for batched search: m log-uniform in [2048, 65536],
    n in {64, 128, 256}, random walk and sine alternating, one anomaly each
    (kind drawn from the four)."""
    rng = np.random.default_rng(seed)
    kinds = ("burst", "flat", "spike", "phase")
    out = []
    for k in range(count):
        m = _log_uniform_int(rng, 2048, 65536)
        n = int(rng.choice([64, 128, 256]))
        an = (kinds[int(rng.integers(0, 4))],)
        out.append(SeriesSpec("rw" if k % 2 == 0 else "sine", m, n, seed * 100003 + k, an))
    return out


def serving_requests(seed: int = 0, rate_per_s: float = 200.0, duration_s: float = 20.0,
                     m_max: int = 1 << 20) -> list[tuple[float, SeriesSpec]]:
    """A serving trace: Poisson arrivals at `rate_per_s` over `duration_s`
    seconds; each request a series with m log-uniform in [4096, m_max],
    n in {64, 128, 256, 512, 1024}, random walk or sine, one anomaly."""
    rng = np.random.default_rng(seed)
    kinds = ("burst", "flat", "spike", "phase")
    t = 0.0
    out = []
    k = 0
    while True:
        t += float(rng.exponential(1.0 / rate_per_s))
        if t >= duration_s:
            return out
        m = _log_uniform_int(rng, 4096, m_max)
        n = int(rng.choice([64, 128, 256, 512, 1024]))
        an = (kinds[int(rng.integers(0, 4))],)
        out.append((t, SeriesSpec("rw" if rng.integers(0, 2) == 0 else "sine", m, n, seed * 1000003 + k, an)))
        k += 1
