"""Pins for the FP64 oracle (CPU only).

Every oracle function is checked against something other than itself:
hand-worked examples (tests/golden), closed forms, exact integer brute force,
invariants of the definitions, and the agreement of two different algorithms
(brute force O1 and CPU HOTSAX O2) bit for bit.
"""
import math
import os
from fractions import Fraction

import numpy as np
import pytest

import oracle
from paper_1901_00155_gb300 import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _hand_examples():
    out = []
    with open(os.path.join(GOLDEN, "hand_examples.txt")) as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            T, n, idx, dist, mu, var = [x.strip() for x in line.split("|")]
            out.append((np.array([float(v) for v in T.split(",")], dtype=np.float32), int(n), int(idx),
                        float(dist), float(mu), float(var)))
    return out


@pytest.mark.parametrize("case", _hand_examples(), ids=lambda c: f"m{c[0].size}_n{c[1]}")
def test_hand_examples_brute(case):
    T, n, idx, dist, mu, var = case
    i, d2 = oracle.discord_brute(T, n)
    assert i == idx
    assert math.sqrt(d2) == pytest.approx(dist, rel=1e-14, abs=1e-15)
    _, mu_o, sg_o = oracle.znorm(T)
    assert mu_o == pytest.approx(mu, rel=1e-15)
    assert sg_o * sg_o == pytest.approx(var, rel=1e-14, abs=1e-300)


@pytest.mark.parametrize("case", _hand_examples(), ids=lambda c: f"m{c[0].size}_n{c[1]}")
def test_hand_examples_hotsax(case):
    T, n, idx, dist, _, _ = case
    i, d2, _ = oracle.hotsax(T, n, w=min(4, n), A=4)
    assert i == idx
    assert math.sqrt(d2) == pytest.approx(dist, rel=1e-14, abs=1e-15)


def _exact_profile_int(T, n):
    """Exact rational brute force for integer series: raw squared distances in
    integers; normalised nn^2 = raw / sigma^2 (Eq. 2 is affine, so the argmax is
    that of the raw distances).  Returns (raw nn^2 per row, sigma^2)."""
    t = [int(v) for v in T]
    m = len(t)
    N = m - n + 1
    raw = []
    for i in range(N):
        mn = None
        for j in range(N):
            if abs(i - j) < n:
                continue
            s = sum((t[i + k] - t[j + k]) ** 2 for k in range(n))
            if mn is None or s < mn:
                mn = s
        raw.append(mn)
    mu = Fraction(sum(t), m)
    var = Fraction(sum(v * v for v in t), m) - mu * mu
    return raw, var


def test_exact_integer_brute_force():
    """Exact arithmetic fixes the maximum; where several rows tie exactly, the
    FP64 rounding of Eq. 2 may order them either way, so the oracle's index must
    be one of the exact maximisers (and the first one when there is no tie)."""
    rng = np.random.default_rng(1234)
    ties = 0
    for trial in range(150):
        n = int(rng.integers(1, 6))
        m = int(rng.integers(3 * n - 1, 3 * n + 20))
        T = rng.integers(-4, 5, size=m).astype(np.float32)
        raw, var = _exact_profile_int(T, n)
        mx = max(raw)
        winners = [i for i, r in enumerate(raw) if r == mx]
        enn2 = Fraction(0) if var == 0 else Fraction(mx) / var
        i, d2 = oracle.discord_brute(T, n)
        assert i in winners, (trial, T.tolist(), n)
        if len(winners) == 1 or var == 0:
            assert i == winners[0]
        else:
            ties += 1
        assert d2 == pytest.approx(float(enn2), rel=1e-12, abs=1e-12)
        nn = oracle.nn_profile(T, n)
        exact = [0.0 if var == 0 else float(Fraction(r) / var) for r in raw]
        np.testing.assert_allclose(nn, exact, rtol=1e-12, atol=1e-12)
    assert ties > 0  # the sweep does exercise exact ties


def test_discord_dominates_profile():
    rng = np.random.default_rng(7)
    for _ in range(20):
        T = synth.random_small(rng, 300)
        n = int(rng.integers(2, 30))
        nn = oracle.nn_profile(T, n)
        i, d2 = oracle.discord_brute(T, n)
        assert d2 == nn[i]
        assert np.all(nn <= d2)
        assert np.all(nn[:i] < d2)  # ties resolve to the smallest index


def test_affine_invariance_bitwise():
    """T -> 2T and T -> -T leave the normalised series, hence the whole
    nearest-neighbour profile, unchanged bit for bit (mu, sigma scale exactly)."""
    rng = np.random.default_rng(11)
    for _ in range(10):
        T = synth.random_small(rng, 257)
        n = int(rng.integers(2, 40))
        nn = oracle.nn_profile(T, n)
        assert np.array_equal(nn, oracle.nn_profile(2.0 * T, n))
        assert np.array_equal(nn, oracle.nn_profile(-T, n))


def test_affine_invariance_general():
    rng = np.random.default_rng(12)
    for _ in range(10):
        T = np.cumsum(rng.standard_normal(400)).astype(np.float32)
        n = int(rng.integers(4, 40))
        T2 = (T.astype(np.float64) * 0.37 + 5.0).astype(np.float32)
        i1, d1 = oracle.discord_brute(T, n)
        i2, d2 = oracle.discord_brute(T2, n)
        assert d2 == pytest.approx(d1, rel=1e-5)
        if i1 != i2:
            nn = oracle.nn_profile(T, n)
            assert nn[i2] == pytest.approx(d1, rel=1e-5)


def test_time_reversal():
    rng = np.random.default_rng(13)
    for _ in range(10):
        T = np.cumsum(rng.standard_normal(300)).astype(np.float32)
        n = int(rng.integers(3, 30))
        nn = oracle.nn_profile(T, n)
        nr = oracle.nn_profile(T[::-1].copy(), n)
        np.testing.assert_allclose(nr[::-1], nn, rtol=1e-12, atol=1e-12)


def test_periodic_spike_closed_form():
    """A periodic series whose every window has an exact copy >= n away, with
    one unit spike: windows holding the spike have raw NN^2 exactly 1 (their
    spike-free copy), all others 0.  Discord = first window holding the spike,
    nn^2 = 1 / sigma^2 with sigma^2 from Eq. 2 in exact arithmetic."""
    rng = np.random.default_rng(5)
    for P, n in [(7, 5), (12, 12), (9, 4), (16, 10)]:
        unit = 3 * rng.permutation(P)
        reps = 12
        t = np.tile(unit, reps).astype(np.int64)
        m = t.size
        o = m // 2 + 1
        t[o] += 1
        T = t.astype(np.float32)
        tl = [int(v) for v in t]
        mu = Fraction(sum(tl), m)
        var = Fraction(sum(v * v for v in tl), m) - mu * mu
        nn = oracle.nn_profile(T, n)
        N = m - n + 1
        holds = np.array([(i <= o < i + n) for i in range(N)])
        np.testing.assert_allclose(nn[holds], float(1 / var), rtol=1e-12)
        assert np.all(np.abs(nn[~holds]) <= 1e-12)
        i, d2 = oracle.discord_brute(T, n)
        assert i == o - n + 1
        assert d2 == pytest.approx(float(1 / var), rel=1e-12)


def test_nn_rows_matches_profile_and_arg():
    rng = np.random.default_rng(3)
    T = np.cumsum(rng.standard_normal(500)).astype(np.float32)
    n = 17
    nn = oracle.nn_profile(T, n)
    rows = np.array([0, 5, 100, 483])
    r, arg = oracle.nn_rows(T, n, rows)
    assert np.array_equal(r, nn[rows])
    assert np.all(np.abs(arg - rows) >= n)


def test_o1_equals_o2_bitwise():
    """CPU HOTSAX (Algorithms 2-4, abandon + SAX ordering) returns the brute
    force's discord bit for bit on many tiny series."""
    rng = np.random.default_rng(2024)
    count = 0
    for trial in range(1000):
        n = int(rng.choice([1, 2, 3, 8, 16]))
        m = int(rng.integers(3 * n - 1, 3 * n + 90))
        T = synth.random_small(rng, m)
        w = min(4, n)
        mode = int(trial % 2)
        i1, d1 = oracle.discord_brute(T, n)
        i2, d2, _ = oracle.hotsax(T, n, w=w, A=4, paa_mode=mode)
        assert (i1, d1) == (i2, d2), (trial, n, m)
        count += 1
    assert count == 1000


def test_o2_prunes():
    """HOTSAX evaluates far fewer pairs than the brute force on a random walk."""
    T, _ = synth.make_series(synth.SeriesSpec("rw", 4096, 64, 0, ("burst",)))
    i1, d1 = oracle.discord_brute(T, 64)
    i2, d2, ev = oracle.hotsax(T, 64)
    assert (i1, d1) == (i2, d2)
    N = T.size - 64 + 1
    assert ev < 0.25 * N * (N - 64)


def test_invalid_inputs():
    with pytest.raises(oracle.OracleError) as e:
        oracle.discord_brute(np.zeros(10, np.float32), 4)  # N = 7 < 2n
    assert e.value.code == oracle.EINVAL
    T = np.arange(50, dtype=np.float32)
    T[7] = np.nan
    with pytest.raises(oracle.OracleError) as e:
        oracle.discord_brute(T, 4)
    assert e.value.code == oracle.ENONFINITE
    T[7] = np.inf
    with pytest.raises(oracle.OracleError) as e:
        oracle.hotsax(T, 4)
    assert e.value.code == oracle.ENONFINITE


# ---------------------------------------------------------------- SAX pins

def _golden_breakpoints():
    rows, q3 = {}, None
    with open(os.path.join(GOLDEN, "sax_breakpoints.txt")) as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            k, v = [x.strip() for x in line.split("|")]
            if k == "Q3":
                q3 = float(v)
            else:
                rows[int(k)] = [float(x) for x in v.split()]
    return rows, q3


def test_breakpoints_table():
    rows, q3 = _golden_breakpoints()
    for A, ref in rows.items():
        b = oracle.breakpoints(A)
        np.testing.assert_allclose(b, ref, atol=0.005 + 1e-12)
        assert np.all(np.diff(b) > 0)
    b4 = oracle.breakpoints(4)
    assert b4[2] == pytest.approx(q3, abs=1e-13)
    assert b4[0] == -b4[2] and b4[1] == 0.0


def test_paa_sax_ramp_closed_form():
    """An increasing ramp: every window z-normalised is the same centred ramp;
    for n=8, w=4 the segment means of k are 0.5,2.5,4.5,6.5, centred -3,-1,1,3,
    divided by sqrt(63/12) -> letters (0,1,2,3) -> code 27.  A decreasing ramp
    gives (3,2,1,0) -> 228; a constant series gives zeros -> (2,2,2,2) -> 170."""
    T = np.arange(64, dtype=np.float32)
    code, paa = oracle.sax(T, 8, 4, 4, paa_mode=0, want_paa=True)
    sd = math.sqrt(63.0 / 12.0)
    np.testing.assert_allclose(paa, np.tile(np.array([-3, -1, 1, 3]) / sd, (code.size, 1)), rtol=1e-12)
    assert np.all(code == 27)
    assert np.all(oracle.sax(T[::-1].copy(), 8, 4, 4) == 228)
    assert np.all(oracle.sax(np.full(40, 3.0, np.float32), 8, 4, 4) == 170)


def test_paa_literal_mode_closed_form():
    """Mode 1 takes the globally normalised values: for T = 0..m-1,
    t^_k = (k - (m-1)/2) / sigma with sigma^2 = (m^2 - 1)/12."""
    m, n, w = 40, 8, 4
    T = np.arange(m, dtype=np.float32)
    _, paa = oracle.sax(T, n, w, 4, paa_mode=1, want_paa=True)
    sg = math.sqrt((m * m - 1) / 12.0)
    for i in (0, 7, 32):
        seg = np.array([i + 0.5, i + 2.5, i + 4.5, i + 6.5])
        np.testing.assert_allclose(paa[i], (seg - (m - 1) / 2) / sg, rtol=1e-12)


def test_sax_uneven_segments():
    """n not divisible by w: segment s is [floor(s n/w), floor((s+1) n/w))."""
    T = np.arange(30, dtype=np.float32)
    n, w = 10, 4  # segments [0,2) [2,5) [5,7) [7,10)
    _, paa = oracle.sax(T, n, w, 4, paa_mode=0, want_paa=True)
    k = np.arange(10.0)
    sd = k.std()
    ref = np.array([k[0:2].mean(), k[2:5].mean(), k[5:7].mean(), k[7:10].mean()]) - k.mean()
    np.testing.assert_allclose(paa[3], ref / sd, rtol=1e-12)


def test_index_hand_example():
    code = np.array([3, 1, 3, 2, 1, 3], dtype=np.int32)
    freq, cand, offs, mem = oracle.index(code, 4)
    assert freq.tolist() == [3, 2, 3, 1, 2, 3]
    assert cand.tolist() == [3]
    assert offs.tolist() == [0, 0, 2, 3, 6]
    assert mem.tolist() == [1, 4, 3, 0, 2, 5]


def test_index_properties():
    rng = np.random.default_rng(9)
    for _ in range(20):
        N = int(rng.integers(1, 2000))
        code = rng.integers(0, 256, size=N).astype(np.int32)
        freq, cand, offs, mem = oracle.index(code, 256)
        assert offs[-1] == N and offs[0] == 0 and np.all(np.diff(offs) >= 0)
        assert np.array_equal(np.sort(mem), np.arange(N))
        for h in range(256):
            seg = mem[offs[h]:offs[h + 1]]
            assert np.all(code[seg] == h)
            assert np.all(np.diff(seg) > 0)
        cnt = np.bincount(code, minlength=256)
        assert np.array_equal(freq, cnt[code])
        fmin = freq.min()
        assert np.array_equal(cand, np.nonzero(freq == fmin)[0])


# ----------------------------------------------------- normalisation pins

def test_window_stats_ramp_closed_form():
    """For T = 0..m-1: t^ is a ramp of slope 1/sigma, sigma^2 = (m^2-1)/12, so
    mu_i = (i + (n-1)/2 - (m-1)/2)/sigma and c_i = n(n^2-1)/12 / sigma^2."""
    m, n = 100, 9
    T = np.arange(m, dtype=np.float32)
    mu, c = oracle.window_stats(T, n)
    sg = math.sqrt((m * m - 1) / 12.0)
    i = np.arange(m - n + 1)
    np.testing.assert_allclose(mu, (i + (n - 1) / 2 - (m - 1) / 2) / sg, rtol=1e-12, atol=1e-14)
    np.testing.assert_allclose(c, n * (n * n - 1) / 12.0 / sg ** 2, rtol=1e-12)


def test_znorm_closed_form():
    T = np.array([1, 2, 3, 4], dtype=np.float32)
    t, mu, sg = oracle.znorm(T)
    assert mu == 2.5 and sg == pytest.approx(math.sqrt(1.25), rel=1e-15)
    np.testing.assert_allclose(t, (np.array([1, 2, 3, 4]) - 2.5) / math.sqrt(1.25), rtol=1e-15)
    t0, _, s0 = oracle.znorm(np.full(5, 2.0, np.float32))
    assert s0 == 0.0 and np.all(t0 == 0.0)


def _topk_examples():
    out = []
    with open(os.path.join(GOLDEN, "topk_examples.txt")) as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            T, n, k, picks, var = [x.strip() for x in line.split("|")]
            want = [(int(a), float(b)) for a, b in (p.split(":") for p in picks.split(","))]
            out.append((np.array([float(v) for v in T.split(",")], dtype=np.float32), int(n), int(k), want,
                        float(var)))
    return out


@pytest.mark.parametrize("case", _topk_examples(), ids=lambda c: f"m{c[0].size}_n{c[1]}")
def test_discords_brute_hand_examples(case):
    """Top-k pinned to hand-worked values: an overlapping row with the second-largest nn is
    skipped, a row exactly n away stays allowed, and nearest neighbours keep the earlier
    discords as candidates."""
    T, n, k, want, var = case
    got = oracle.discords_brute(T, n, k)
    assert [g[0] for g in got] == [w[0] for w in want]
    for (_, d2), (_, d) in zip(got, want):
        assert math.sqrt(d2) == pytest.approx(d, rel=1e-14, abs=1e-15)
    _, _, sg = oracle.znorm(T)
    assert sg * sg == pytest.approx(var, rel=1e-14)


def test_discords_brute_definition():
    """Top-k discords: the first is the discord; every later one is the largest nn among the
    subsequences at least n from all earlier ones (rechecked by a plain loop); distances do not
    increase; chosen indices are pairwise at least n apart."""
    rng = np.random.default_rng(77)
    for trial in range(20):
        n = int(rng.choice([2, 3, 5, 8]))
        T = np.cumsum(rng.standard_normal(int(rng.integers(6 * n, 6 * n + 60)))).astype(np.float32)
        k = 4
        got = oracle.discords_brute(T, n, k)
        i0, d0 = oracle.discord_brute(T, n)
        assert got[0][0] == i0 and got[0][1] == d0
        nn2 = oracle.nn_profile(T, n)
        chosen = []
        for idx, v in got:
            best = None
            for i in range(nn2.size):
                if any(abs(i - c) < n for c in chosen):
                    continue
                if best is None or nn2[i] > nn2[best]:
                    best = i
            assert idx == best and v == nn2[best]
            chosen.append(idx)
        assert all(a[1] >= b[1] for a, b in zip(got, got[1:]))
        assert all(abs(a - b) >= n for x, a in enumerate(chosen) for b in chosen[x + 1:])
