"""dd_nn_profile_static: the allocation-free profile entry point.

Some callers cannot allocate device memory when they need a result (their
device memory is already fully handed to another allocator, or an allocation
would stall a latency-critical loop).  This entry point serves them from a
fixed scratch array inside the library.  The test calls it through the C ABI
twice in a row, on two different series, and checks each result against the
FP64 oracle's nearest-neighbour profile and against the plan-based
dd_nn_profile, within the FP32 form's tolerance.  It lives in its
own file, collected last, and passes both alone and after the other tests.
"""
import ctypes

import numpy as np
import pytest

import oracle
from paper_1901_00155_gb300 import _lib

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

RTOL = 1e-4


def _static(lib, Td, n, out, stream):
    return lib.dd_nn_profile_static(ctypes.c_void_p(Td.data_ptr()), Td.numel(), n, ctypes.c_void_p(out.data_ptr()),
                                    ctypes.c_void_p(stream.cuda_stream))


def test_static_profile_matches_plan_profile_twice():
    import paper_1901_00155_gb300 as dd
    lib = _lib.load()
    stream = torch.cuda.current_stream()
    rng = np.random.default_rng(31)
    cases = [(np.cumsum(rng.standard_normal(9000)).astype(np.float32), 100),
             (np.sin(np.arange(4000) / 7.0).astype(np.float32) + 0.05 * rng.standard_normal(4000).astype(np.float32),
              17)]
    for T, n in cases:  # two calls in a row, different sizes
        Td = torch.from_numpy(T).cuda()
        N = T.size - n + 1
        out = torch.full((N,), -1.0, dtype=torch.float32, device="cuda")
        assert _static(lib, Td, n, out, stream) == _lib.DD_OK
        with dd.Plan(T.size, n) as p:
            ref = p.nn_profile(Td)
        torch.cuda.synchronize()
        got, want = out.cpu().numpy(), ref.cpu().numpy()
        np.testing.assert_allclose(got, want, rtol=RTOL, atol=1e-6 * max(1.0, float(want.max())))
        exact = oracle.nn_profile(T, n)
        np.testing.assert_allclose(got, exact, rtol=RTOL, atol=1e-5 * max(1.0, float(exact.max())))


def test_static_profile_rejects_oversized_series():
    lib = _lib.load()
    big = torch.zeros((1 << 18) + 1, dtype=torch.float32, device="cuda")
    out = torch.empty(1 << 18, dtype=torch.float32, device="cuda")
    assert _static(lib, big, 64, out, torch.cuda.current_stream()) == _lib.DD_EINVAL
    small = torch.zeros(100, dtype=torch.float32, device="cuda")
    assert _static(lib, small, 40, out, torch.cuda.current_stream()) == _lib.DD_EINVAL  # N < 2n
