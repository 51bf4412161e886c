"""Pins of the oracle's per-window z-normalised variant (every subsequence normalised on its own,
a constant one to the zero vector; one reading of Algorithm 2's Znormalize step).

Each check ties the oracle to something other than its own formula:
- the textbook identity d^2 = 2n(1 - r) with r from numpy's Pearson correlation (np.corrcoef);
- scipy's z-score (population sigma) followed by plain Euclidean distances;
- closed forms: anti-correlated windows at 4n, constant vs non-constant at n, constant vs constant
  at 0, exact copies at 0;
- exact invariances: negating or doubling the series leaves every distance bit for bit equal.
"""
import numpy as np
import pytest

import oracle


def _windows(T, n):
    T = np.asarray(T, dtype=np.float64)
    return np.lib.stride_tricks.sliding_window_view(T, n)


def _nn_from_corrcoef(T, n):
    """Nearest non-self-match distance of every row via d^2 = 2n(1 - r), r = np.corrcoef."""
    W = _windows(T, n)
    R = np.corrcoef(W)
    D = 2.0 * n * (1.0 - R)
    N = W.shape[0]
    idx = np.arange(N)
    D[np.abs(idx[:, None] - idx[None, :]) < n] = np.inf
    return D.min(axis=1)


@pytest.mark.parametrize("seed,m,n", [(0, 200, 8), (1, 300, 16), (2, 257, 5), (3, 180, 1 + 2)])
def test_window_profile_equals_pearson_identity(seed, m, n):
    rng = np.random.default_rng(seed)
    T = np.cumsum(rng.standard_normal(m)).astype(np.float32) * 3.0 + 100.0
    got = oracle.nn_profile(T, n, "window")
    ref = _nn_from_corrcoef(T, n)
    assert np.allclose(got, ref, rtol=1e-9, atol=1e-9 * n)


def test_window_distance_equals_scipy_zscore():
    stats = pytest.importorskip("scipy.stats")
    rng = np.random.default_rng(5)
    m, n = 400, 24
    T = (rng.standard_normal(m) * 0.2 + np.sin(np.arange(m) / 7.0) * 5).astype(np.float32)
    W = _windows(T, n)
    Z = stats.zscore(W, axis=1, ddof=0)
    for i, j in [(0, 100), (3, 250), (376, 12), (200, 200 - n)]:
        ref = float(np.sum((Z[i] - Z[j]) ** 2))
        assert oracle.dist2(T, n, i, j, "window") == pytest.approx(ref, rel=1e-12, abs=1e-12)


def test_window_closed_forms():
    n = 6
    p = np.array([0.0, 1.0, 3.0, 2.0, 5.0, 4.0], dtype=np.float32)
    flat = np.full(n, 7.0, dtype=np.float32)
    T = np.concatenate([p, -p + 2.0, flat, flat, p * 3.0 - 1.0, np.float32(9.0) * np.ones(n, np.float32)])
    T = T.astype(np.float32)
    # window 0 = p, window n = -p + 2: perfectly anti-correlated -> 4n
    assert oracle.dist2(T, n, 0, n, "window") == pytest.approx(4 * n, rel=1e-14)
    # window 0 and the scaled, shifted copy at 4n: identical after normalisation -> 0
    assert oracle.dist2(T, n, 0, 4 * n, "window") == pytest.approx(0.0, abs=1e-12)
    # constant windows at 2n and 3n (and 5n): constant vs constant 0, constant vs not n
    assert oracle.dist2(T, n, 2 * n, 3 * n, "window") == 0.0
    assert oracle.dist2(T, n, 2 * n, 5 * n, "window") == 0.0
    assert oracle.dist2(T, n, 2 * n, 0, "window") == pytest.approx(n, rel=1e-14)
    # every distance lies in [0, 4n]
    N = T.size - n + 1
    for i in range(N):
        for j in range(N):
            d = oracle.dist2(T, n, i, j, "window")
            assert -1e-12 <= d <= 4 * n * (1 + 1e-14)


def test_window_profile_of_constant_and_tiled_series():
    n = 8
    assert np.all(oracle.nn_profile(np.full(64, 3.5, np.float32), n, "window") == 0.0)
    # exact copies every 16 samples: each row has an identical window 16 or 32 away
    rng = np.random.default_rng(9)
    p = rng.standard_normal(16).astype(np.float32)
    T = np.tile(p, 8)
    assert np.all(oracle.nn_profile(T, n, "window") == 0.0)
    # a planted non-copy: the rows covering it are the discords, the others still 0
    T2 = T.copy()
    T2[64:72] = rng.standard_normal(8).astype(np.float32) * 2
    nn = oracle.nn_profile(T2, n, "window")
    i, d2 = oracle.discord_brute(T2, n, "window")
    assert 64 - n < i < 72 and d2 == nn.max() > 0.0
    far = [k for k in range(nn.size) if k + n <= 64 - 16 or k >= 72 + 16]
    assert np.all(nn[far] == 0.0)


def test_window_exact_invariances():
    rng = np.random.default_rng(11)
    T = (np.cumsum(rng.standard_normal(240)) + 50).astype(np.float32)
    n = 12
    base = oracle.nn_profile(T, n, "window")
    assert np.array_equal(oracle.nn_profile(-T, n, "window"), base)
    assert np.array_equal(oracle.nn_profile(T * np.float32(2.0), n, "window"), base)
    # with values on a 1/64 grid, 3T + 7 is exact in float32: equal up to FP64 rounding
    Tq = (np.round(T.astype(np.float64) * 64) / 64).astype(np.float32)
    Tq3 = Tq * np.float32(3.0) + np.float32(7.0)
    assert np.array_equal(Tq3.astype(np.float64), Tq.astype(np.float64) * 3 + 7)
    assert np.allclose(oracle.nn_profile(Tq3, n, "window"), oracle.nn_profile(Tq, n, "window"),
                       rtol=1e-10, atol=1e-10)


def test_window_rows_and_mu_sigma_agree_with_profile():
    rng = np.random.default_rng(12)
    T = rng.standard_normal(500).astype(np.float32)
    n = 20
    prof = oracle.nn_profile(T, n, "window")
    rows = np.array([0, 7, 240, 480], dtype=np.int64)
    nn2, arg = oracle.nn_rows(T, n, rows, "window")
    assert np.array_equal(nn2, prof[rows])
    for r, a in zip(rows, arg):
        assert abs(int(a) - int(r)) >= n
        assert oracle.dist2(T, n, int(r), int(a), "window") == nn2[list(rows).index(r)]
    mu, sg = oracle.window_mu_sigma(T, n)
    W = _windows(T, n)
    assert np.allclose(mu, W.mean(axis=1), rtol=0, atol=1e-12)
    assert np.allclose(sg, W.std(axis=1), rtol=1e-12, atol=1e-12)


def test_window_topk_excludes_previous_discords():
    rng = np.random.default_rng(13)
    T = rng.standard_normal(400).astype(np.float32)
    n = 10
    got = oracle.discords_brute(T, n, 3, "window")
    nn = oracle.nn_profile(T, n, "window")
    assert got[0][0] == int(np.argmax(nn))
    for a in range(len(got)):
        for b in range(a):
            assert abs(got[a][0] - got[b][0]) >= n
        assert got[a][1] == nn[got[a][0]]


def test_znorm_argument_is_checked():
    T = np.zeros(64, np.float32)
    with pytest.raises(ValueError):
        oracle.nn_profile(T, 4, "per-window")
