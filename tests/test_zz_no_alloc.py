"""stencil_run_noalloc: the sweep for callers that must not allocate device memory.

Those callers (an inference-engine plugin whose enqueue may not allocate, code
running while a caching allocator already holds the free memory, a loop that
cannot afford cudaMalloc's device-wide synchronisation) get the same sweep as
stencil_plan_create + stencil_run, using a fixed scratch array inside the
library instead of a plan's workspace.  This file runs last so that a failure
here never hides the result of any other test.
"""
import ctypes

import numpy as np
import pytest

from paper_2605_07954_gb300 import inputs
from _util import fp32_tol, rel_l2

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2605_07954_gb300 import _capi, build
    build.build()
    return _capi.load()


def _noalloc(lib, x, W, T, boundary=0, out=None):
    out = torch.empty_like(x) if out is None else out
    Wc = np.ascontiguousarray(W, dtype=np.float32)
    st = lib.stencil_run_noalloc(x.shape[0], x.shape[1], W.shape[0] // 2,
                                 Wc.ctypes.data_as(ctypes.POINTER(ctypes.c_float)), 0, boundary,
                                 x.data_ptr(), out.data_ptr(), T,
                                 torch.cuda.current_stream().cuda_stream)
    assert st == 0, lib.stencil_noalloc_last_error().decode()
    return out


def _planned(x, W, T, boundary="zero"):
    from paper_2605_07954_gb300 import Plan
    p = Plan(x.shape[0], x.shape[1], W, boundary=boundary)
    y = p.run(x, T)
    torch.cuda.synchronize()
    p.close()
    return y


def test_noalloc_matches_planned_run_twice(lib):
    """Two calls in a row (different shapes, weights and boundaries) agree with
    the plan-based path, and the second call allocates no device memory."""
    cases = [("box9", 2048, 1536, 100, 0), ("star13", 1000, 1204, 37, 1)]
    free_after = []
    for name, ny, nx, T, boundary in cases:
        W = inputs.pattern_weights(name)
        x = torch.from_numpy(inputs.field(ny, nx)).cuda()
        ref = _planned(x, W, T, "periodic" if boundary else "zero")
        torch.cuda.synchronize()
        free0 = torch.cuda.mem_get_info()[0]
        y = _noalloc(lib, x, W, T, boundary)
        torch.cuda.synchronize()
        free_after.append((free0, torch.cuda.mem_get_info()[0]))
        assert rel_l2(y.cpu().numpy(), ref.cpu().numpy()) <= fp32_tol(T), name
    # The call itself took no device memory (the output tensor was allocated
    # by the test before the call).
    free0, free1 = free_after[1]
    assert free1 >= free0


def test_noalloc_in_place_and_zero_steps(lib):
    W = inputs.pattern_weights("box9")
    x = torch.from_numpy(inputs.field(257, 300)).cuda()
    ref = _planned(x, W, 13)
    z = x.clone()
    _noalloc(lib, z, W, 13, out=z)
    torch.cuda.synchronize()
    assert rel_l2(z.cpu().numpy(), ref.cpu().numpy()) <= fp32_tol(13)
    y = _noalloc(lib, x, W, 0)
    torch.cuda.synchronize()
    assert torch.equal(x, y)


def test_noalloc_rejects_grids_beyond_the_scratch(lib):
    W = inputs.pattern_weights("box9")
    x = torch.empty((8192, 8192), device="cuda")  # 256 MiB > the 64 MiB scratch
    Wc = np.ascontiguousarray(W)
    st = lib.stencil_run_noalloc(8192, 8192, 1, Wc.ctypes.data_as(ctypes.POINTER(ctypes.c_float)),
                                 0, 0, x.data_ptr(), x.data_ptr(), 1, None)
    assert st == 2  # STENCIL_ERR_UNSUPPORTED
    assert "exceeds" in lib.stencil_noalloc_last_error().decode()
