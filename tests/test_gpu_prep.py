"""Preparation stage on the GPU (Eq. 2 normalisation, FP64 prefix sums, row
statistics, PAA/SAX words, Freq / Cand / Index_Word) against the FP64 oracle,
through the C ABI."""
import numpy as np
import pytest

import oracle
from paper_1901_00155_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

BAND = 1e-9  # PAA values this close to a breakpoint may take either letter


def _prep(T, n, **opts):
    import paper_1901_00155_gb300 as dd
    Td = torch.from_numpy(T).cuda()
    p = dd.Plan(T.size, n, **opts)
    v = p.prep(Td)
    out = {k: t.cpu().numpy().copy() for k, t in v.items()}
    torch.cuda.synchronize()
    p.close()
    return out


CASES = [("rw", 8192, 128, 0), ("sine", 5000, 100, 1), ("rw", 3 * 64 - 1, 64, 2), ("rw", 20000, 7, 3),
         ("sine", 70001, 256, 4)]


@pytest.mark.parametrize("kind,m,n,seed", CASES)
@pytest.mark.parametrize("paa_mode", [0, 1])
def test_prep_matches_oracle(kind, m, n, seed, paa_mode):
    rng = np.random.default_rng(seed)
    T = synth.random_small(rng, m, kind)
    g = _prep(T, n, paa_mode=paa_mode)
    th, mu, sg = oracle.znorm(T)
    # Eq. 2
    assert g["stats"][0] == pytest.approx(mu, rel=1e-12, abs=1e-12)
    assert g["stats"][1] == pytest.approx(sg, rel=1e-12)
    np.testing.assert_allclose(g["t32"], th.astype(np.float32), rtol=2e-7, atol=1e-30)
    # FP64 prefix sums
    ref1 = np.concatenate([[0.0], np.cumsum(th)])
    ref2 = np.concatenate([[0.0], np.cumsum(th * th)])
    np.testing.assert_allclose(g["P1"], ref1, rtol=1e-12, atol=1e-9)
    np.testing.assert_allclose(g["P2"], ref2, rtol=1e-12, atol=1e-9)
    # rows of the subsequence matrix (Eq. 5)
    muw, cw = oracle.window_stats(T, n)
    np.testing.assert_allclose(g["mu_w"], muw, rtol=1e-10, atol=1e-11)
    np.testing.assert_allclose(g["c_w"], cw, rtol=1e-8, atol=1e-12 * (1.0 + ref2[-1]))
    # SAX words (Eq. 3, 4, 9): identical except within the rounding band
    w = min(4, n)
    code, paa = oracle.sax(T, n, w, 4, paa_mode=paa_mode, want_paa=True)
    beta = oracle.breakpoints(4)
    amb = np.any(np.abs(paa[:, :, None] - beta[None, None, :]) < BAND, axis=(1, 2))
    if paa_mode == 0:
        amb |= cw <= 1e-10 * (1.0 + ref2[-1])
    gc = g["code"]
    assert np.array_equal(gc[~amb], code[~amb])
    assert amb.mean() < 0.01
    # Freq histogram, word order = Index_Word, Cand
    D = 4 ** w
    hist = np.bincount(gc, minlength=D)
    assert np.array_equal(g["freq_hist"][:D], hist)
    freq, cand, offs, mem = oracle.index(gc, D)
    ws = g["word_start"][:D]
    order = g["order"]
    for h in range(D):
        seg = order[ws[h]:ws[h] + hist[h]]
        assert np.array_equal(seg, mem[offs[h]:offs[h + 1]]), h
    nonempty = [h for h in range(D) if hist[h] > 0]
    keyed = sorted(nonempty, key=lambda h: (hist[h], h))
    assert [int(ws[h]) for h in keyed] == list(np.cumsum([0] + [hist[h] for h in keyed])[:-1])
    assert int(g["ncand"][0]) == cand.size
    assert np.array_equal(np.sort(order[:cand.size]), cand)
    assert np.array_equal(np.sort(order), np.arange(T.size - n + 1))


def test_prep_rejects_nonfinite():
    import paper_1901_00155_gb300 as dd
    T = np.cumsum(np.random.default_rng(0).standard_normal(1000)).astype(np.float32)
    T[500] = np.inf
    with dd.Plan(T.size, 16) as p:
        with pytest.raises(dd.DDError) as e:
            p.prep(torch.from_numpy(T).cuda())
    assert e.value.status == 3
