"""The allocation-free inner product (ndmg_dot_noalloc) through the C ABI,
against an FP64 NumPy dot of the host copies and against the handle's inner
product (ndmg_dot).

Some callers cannot allocate device memory (an allocator that owns every
device byte, or a place where cudaMalloc's possible device synchronisation is
not acceptable); ndmg_dot_noalloc serves them from a fixed device array inside
the library.  Collected last so that a stop-at-first-failure run has already
run every other test."""
import ctypes

import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu

try:
    from paper_2205_05840_gb300 import ndmg
except ImportError:
    if torch.cuda.is_available():
        raise
    pytest.skip("library not built and no GPU here", allow_module_level=True)


def _noalloc(dtype_code, x, y, n, stream):
    out = ctypes.c_double(float("nan"))
    st = ndmg._lib.ndmg_dot_noalloc(dtype_code, x.data_ptr(), y.data_ptr(), n, ctypes.byref(out), stream)
    return st, out.value


def test_noalloc_dot_matches_numpy_and_handle_dot_two_calls():
    S = ndmg.Solver(32, n_coarsest=4)
    N = S.num_dofs()
    stream = S.stream.cuda_stream
    # two FP64 calls in a row (the second reuses the array the first left
    # behind), then an FP32 call
    for call, (dtype, code) in enumerate(((torch.float64, ndmg.F64), (torch.float64, ndmg.F64),
                                          (torch.float32, ndmg.F32))):
        g = np.random.default_rng(10 + call)
        xh = g.standard_normal(N)
        yh = g.standard_normal(N)
        x = torch.tensor(xh, dtype=dtype, device="cuda")
        y = torch.tensor(yh, dtype=dtype, device="cuda")
        torch.cuda.synchronize()
        st, got = _noalloc(code, x, y, N, stream)
        assert st == ndmg.OK
        # FP64 dot of exactly the values on the device (FP32 entries are exact in FP64)
        ref_np = float(np.dot(x.cpu().double().numpy(), y.cpu().double().numpy()))
        ref_h = S.dot(x, y)
        scale = float(np.linalg.norm(x.cpu().double().numpy()) * np.linalg.norm(y.cpu().double().numpy()))
        # both sides accumulate N products in FP64 in different orders: random
        # data keeps the difference near sqrt(N) eps |x||y| ~ 7e-14 |x||y|
        tol = 1e-12 * scale
        assert abs(got - ref_np) <= tol, (call, got, ref_np)
        assert abs(got - ref_h) <= tol, (call, got, ref_h)


def test_noalloc_dot_limits():
    x = torch.zeros(8, dtype=torch.float64, device="cuda")
    st, got = _noalloc(ndmg.F64, x, x, 0, None)
    assert st == ndmg.OK and got == 0.0
    st, _ = _noalloc(ndmg.F64, x, x, 67_108_864 + 1, None)      # beyond the static scratch
    assert st == ndmg.INVALID_ARG
    st, _ = _noalloc(7, x, x, 8, None)
    assert st == ndmg.INVALID_ARG
