"""The allocation-free reproducible dot (bd_dot_exact_noalloc), through the C ABI.

This entry point serves callers that cannot allocate device memory: hosts
whose device memory belongs to another allocator, and latency-critical loops
in which cudaMalloc would synchronise the device.  Its scratch is a static device array shared by every
call, so the test makes two calls in a row with different inputs: the second
must not see anything left over from the first.  The file is named so that
pytest collects it last.
"""
import ctypes

import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def B():
    import torch

    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    from paper_2311_13914_gb300 import _build, binding

    _build.build()
    return binding


def test_noalloc_dot_equals_allocating_dot_twice_in_a_row(B):
    import torch

    rng = np.random.default_rng(31)
    stream = torch.cuda.current_stream()
    out = torch.zeros(1, dtype=torch.float64, device="cuda")
    # a large cancelling sum, then a short one with a different magnitude range
    inputs = [
        (rng.standard_normal(200003) * np.exp(rng.uniform(-40, 40, 200003)),
         rng.standard_normal(200003)),
        (rng.standard_normal(37), rng.standard_normal(37) * 1e-7),
    ]
    for x, y in inputs:
        want = B.bd_dot_exact(x, y)  # the allocating entry point, host arrays
        B.bd_dot_exact_noalloc(torch.tensor(x, device="cuda"), torch.tensor(y, device="cuda"), out,
                               stream=stream)
        stream.synchronize()
        got = out.item()
        # same tolerance as the other reproducible-dot tests: bit for bit
        assert np.float64(got).view(np.uint64) == np.float64(want).view(np.uint64)


def test_noalloc_dot_rejects_sizes_beyond_its_maximum(B):
    import torch

    x = torch.zeros(4, dtype=torch.float64, device="cuda")
    out = torch.zeros(1, dtype=torch.float64, device="cuda")
    p = ctypes.c_void_p
    st = B.lib().bd_dot_exact_noalloc(p(x.data_ptr()), p(x.data_ptr()), 2**31, p(out.data_ptr()),
                                      None)
    assert st == B.BD_ERANGE
    st = B.lib().bd_dot_exact_noalloc(p(x.data_ptr()), p(x.data_ptr()), -1, p(out.data_ptr()), None)
    assert st == B.BD_EINVAL
    with pytest.raises(ValueError):
        B.bd_dot_exact_noalloc(x, x, torch.zeros(0, dtype=torch.float64, device="cuda"))
