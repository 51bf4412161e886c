"""The mean-bucketed row order every search wave visits columns in, checked bit for bit.

The order is integer work, so the bar is exact equality with a plain NumPy restatement:
  * each row's bin is clamp(floor((mu_i - lo) * (1 / w)), 0, bins - 1), recomputed in FP64 from the
    plan's own mu_i (Eq. 5 rows) and bin geometry (lo = min t^, w = (max t^ - lo) / bins, Eq. 2);
  * sig is the stable sort by bin of the rows taken in the order e -> (e * stride) mod N
    (NumPy's stable argsort);
  * sigpos is its inverse, and binstart[b] counts the rows in bins below b (binstart[bins] = N).
The pruning bound d^2(i, j) >= n (mu_i - mu_j)^2 that the search applies over this order is only
admissible if bins and positions agree exactly.
"""
import numpy as np
import pytest

from paper_1901_00155_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _cases():
    rng = np.random.default_rng(77)
    out = [("random_walk_m8192_n128", np.cumsum(rng.standard_normal(8192)).astype(np.float32), 128),
           ("sine_m20000_n64", (np.sin(2 * np.pi * np.arange(20000) / 200.0)
                                + 0.1 * rng.standard_normal(20000)).astype(np.float32), 64)]
    flat = np.cumsum(rng.standard_normal(30000))
    flat[5000:9000] = flat[5000]  # a long run of equal means: one crowded bin
    out.append(("flat_stretch_m30000_n100", flat.astype(np.float32), 100))
    spec = synth.workload_large(0)
    T, _ = synth.make_series(spec)
    out.append(("random_walk_m1048576_n256", T, spec.n))
    return out


CASES = _cases()


@pytest.mark.parametrize("prec", ["fp32", "tc_fp16"])
@pytest.mark.parametrize("case", CASES, ids=[c[0] for c in CASES])
def test_mean_order_exact(case, prec):
    import paper_1901_00155_gb300 as dd
    name, T, n = case
    Td = torch.from_numpy(T).cuda()
    with dd.Plan(T.size, n, prec) as p:
        v = p.prep(Td)
        o = p.order_view(Td)
        torch.cuda.synchronize()
        mu = v["mu_w"].cpu().numpy()
        sig = o["sig"].cpu().numpy().astype(np.int64)
        sigpos = o["sigpos"].cpu().numpy().astype(np.int64)
        mubin = o["mubin"].cpu().numpy().astype(np.int64)
        binstart = o["binstart"].cpu().numpy().astype(np.int64)
        lo, inv_w = float(o["lo"].item()), float(o["inv_w"].item())
        stride, bins = o["stride"], o["bins"]
    N = T.size - n + 1
    assert sig.size == N and bins == 4096
    # bins, in FP64 exactly as defined (floor of the scaled offset, clamped to the end bins)
    b = np.floor((mu - lo) * inv_w)
    want_bin = np.where(b >= 0, np.where(b < bins, b, bins - 1), 0).astype(np.int64)
    assert np.array_equal(mubin, want_bin), name
    # stable counting sort of the rows in the stride order
    rows_in = (np.arange(N, dtype=np.int64) * stride) % N
    assert np.unique(rows_in).size == N  # the stride is coprime with N
    want_sig = rows_in[np.argsort(want_bin[rows_in], kind="stable")]
    assert np.array_equal(sig, want_sig), name
    assert np.array_equal(sigpos[sig], np.arange(N))
    want_start = np.concatenate([[0], np.cumsum(np.bincount(want_bin, minlength=bins))])
    assert np.array_equal(binstart, want_start), name
