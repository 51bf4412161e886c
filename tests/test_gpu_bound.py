"""The tensor-core Gram form's per-row error bound, row by row, against the FP64 oracle.

Algorithm 4 abandons a row once a distance falls below the best-so-far; in the Gram form the
library does so only when the row's rigorous upper bound D + F_i(D) is below a proven lower bound,
with F_i(D) = alpha_i + beta D + gam_i sqrt(max(D, 0) + q2_i) (dd_plan_bound_view).  If alpha_i or
gam_i were too small, the returned index could be wrong on unlucky inputs only, so every row of the
exhaustive Gram profile D_i is checked here against the oracle's exact nn^2_i:

    D_i - F_i(D_i) - gam_i^2  <=  nn^2_i  <=  D_i + F_i(D_i)

on inputs chosen to stress the bound: near-duplicate windows (nn^2 near 0), large mean offsets
(the n (mu_i - mu_j)^2 term dominates), noisy sine at n = 1024 (long accumulations), flat stretches
(constant windows, c_i = 0) and random walks.  The ratio |D_i - nn^2_i| / F_i(D_i) (at most 1 if
the bound holds; its complement is the margin) is printed for the record.
"""
import numpy as np
import pytest

import oracle

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _cases():
    rng = np.random.default_rng(606)
    out = []
    base = np.sin(2 * np.pi * np.arange(3000) / 50.0)
    out.append(("near_duplicates", (base + 1e-4 * rng.standard_normal(3000)).astype(np.float32), 100))
    out.append(("mean_offsets", np.cumsum(rng.standard_normal(4000) + 2.0).astype(np.float32), 64))
    sine = np.sin(2 * np.pi * np.arange(6000) / 200.0) + 0.1 * rng.standard_normal(6000)
    out.append(("sine_noise_n1024", sine.astype(np.float32), 1024))
    out.append(("random_walk_n256", np.cumsum(rng.standard_normal(5000)).astype(np.float32), 256))
    out.append(("random_walk_n16", np.cumsum(rng.standard_normal(3000)).astype(np.float32), 16))
    flat = np.cumsum(rng.standard_normal(4000))
    flat[1000:1600] = flat[1000]
    flat[2500:2900] = flat[2500]
    flat[3200] += 15.0
    out.append(("flat_stretches", flat.astype(np.float32), 128))
    return out


CASES = _cases()


@pytest.mark.parametrize("prec", ["tc_fp16", "tc_bf16"])
@pytest.mark.parametrize("case", CASES, ids=[c[0] for c in CASES])
def test_every_row_within_its_bound(prec, case):
    import paper_1901_00155_gb300 as dd
    name, T, n = case
    Td = torch.from_numpy(T).cuda()
    with dd.Plan(T.size, n, prec) as p:
        D = p.nn_profile(Td).cpu().numpy().astype(np.float64)
        b = p.bound_terms(Td)
        torch.cuda.synchronize()
        alpha = b["alpha"].cpu().numpy().astype(np.float64)
        gam = b["gam"].cpu().numpy().astype(np.float64)
        q2 = b["q2"].cpu().numpy().astype(np.float64)
        beta = float(b["beta"])
    exact = oracle.nn_profile(T, n)
    F = alpha + beta * D + gam * np.sqrt(np.maximum(D, 0.0) + q2)
    assert np.all(F > 0) and np.all(np.isfinite(F))
    upper = D + F
    lower = D - F - gam * gam
    bad_u = np.nonzero(exact > upper)[0]
    bad_l = np.nonzero(exact < lower)[0]
    assert bad_u.size == 0, (name, prec, bad_u[:5], exact[bad_u[:5]], upper[bad_u[:5]])
    assert bad_l.size == 0, (name, prec, bad_l[:5], exact[bad_l[:5]], lower[bad_l[:5]])
    ratio = np.abs(D - exact) / F
    i = int(np.argmax(ratio))
    print(f"\nbound {prec} {name}: max |D - nn2| / F = {ratio[i]:.3e} at row {i} "
          f"(D {D[i]:.6g}, nn2 {exact[i]:.6g}, F {F[i]:.3e}); median F / nn2 = "
          f"{np.median(F / np.maximum(exact, 1e-30)):.3e}")
