"""stencil_run_noalloc: the sweep for callers that must not allocate device memory.

Those callers (an inference-engine plugin whose enqueue may not allocate, code
running while a caching allocator already holds the free memory, a loop that
cannot afford cudaMalloc's device-wide synchronisation) get the same sweep as
stencil_plan_create + stencil_run, using a fixed scratch array inside the
library instead of a plan's workspace.  This file runs last so that a failure
here never hides the result of any other test.

Device memory is measured with cudaMemGetInfo around the calls.  The first
call on a device may take up to STENCIL_NOALLOC_MAX_BYTES (under CUDA's lazy
module loading it loads the module that holds the scratch array); every later
call takes nothing.
"""
import ctypes

import numpy as np
import pytest

from paper_2605_07954_gb300 import inputs
from _util import fp32_tol, rel_l2

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

MAX_BYTES = 64 << 20  # STENCIL_NOALLOC_MAX_BYTES
DT = {torch.float32: 0, torch.bfloat16: 1, torch.float16: 2}


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
                                 Wc.ctypes.data_as(ctypes.POINTER(ctypes.c_float)), DT[x.dtype],
                                 boundary, x.data_ptr(), out.data_ptr(), T,
                                 torch.cuda.current_stream().cuda_stream)
    assert st == 0, lib.stencil_noalloc_last_error().decode()
    return out


def _planned(x, W, T, boundary="zero", **opts):
    from paper_2605_07954_gb300 import Plan
    dt = {torch.float32: "f32", torch.bfloat16: "bf16", torch.float16: "f16"}[x.dtype]
    p = Plan(x.shape[0], x.shape[1], W, dtype=dt, boundary=boundary, **opts)
    y = p.run(x, T)
    torch.cuda.synchronize()
    p.close()
    return y


def _free():
    torch.cuda.synchronize()
    return torch.cuda.mem_get_info()[0]


def test_first_call_sets_up_the_scratch(lib):
    """A T = 0 call is the per-device warm-up: it copies in to out and takes at
    most the documented scratch size of device memory; a second one takes none."""
    x = torch.from_numpy(inputs.field(64, 96)).cuda()
    y = torch.empty_like(x)
    free0 = _free()
    _noalloc(lib, x, inputs.pattern_weights("box9"), 0, out=y)
    free1 = _free()
    assert torch.equal(x, y)
    assert 0 <= free0 - free1 <= MAX_BYTES + (8 << 20), (free0, free1)
    _noalloc(lib, x, inputs.pattern_weights("box9"), 0, out=y)
    assert _free() >= free1


def test_noalloc_matches_oracle_and_planned_run_twice(lib, oracle):
    """Two calls in a row (different shapes, weights and boundaries) agree with
    the FP64 oracle and with the plan-based path, and neither call allocates
    device memory (the output tensor is allocated by the test beforehand)."""
    cases = [("box9", 1024, 1536, 100, 0), ("star13", 1000, 1204, 37, 1)]
    for name, ny, nx, T, boundary in cases:
        W = inputs.pattern_weights(name)
        u0 = inputs.field(ny, nx)
        x = torch.from_numpy(u0).cuda()
        bname = "periodic" if boundary else "zero"
        ref = _planned(x, W, T, bname)
        out = torch.empty_like(x)
        free0 = _free()
        y = _noalloc(lib, x, W, T, boundary, out=out)
        assert _free() >= free0, name
        got = y.cpu().numpy()
        assert rel_l2(got, ref.cpu().numpy()) <= fp32_tol(T), name
        assert rel_l2(got, oracle.sweep_f64(u0, W, T, bname)) <= fp32_tol(T), name


def test_noalloc_bf16_storage(lib, oracle):
    """BF16 storage: bit-identical to the streaming plan with the same depth and
    CTA size, and within the BF16 gate of the FP64 oracle."""
    W = inputs.pattern_weights("box9")
    u0 = inputs.field(512, 768)
    x = torch.from_numpy(u0).to(torch.bfloat16).cuda()
    T = 50
    ref = _planned(x, W, T, kernel="stream", tb_depth=8, threads=128)
    y = _noalloc(lib, x, W, T)
    torch.cuda.synchronize()
    assert torch.equal(y, ref)
    assert rel_l2(y.float().cpu().numpy(), oracle.sweep_f64(u0, W, T)) <= 1e-2


def test_noalloc_in_place_and_zero_steps(lib, oracle):
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


def test_noalloc_in_place_staging_path(lib, oracle):
    """Box-49 runs one step per launch, so in == out with an odd T cannot be
    split into an even number of launches: the input is staged in the scratch
    array first.  The result still matches the oracle."""
    W = inputs.pattern_weights("box49")
    u0 = inputs.field(300, 400)
    z = torch.from_numpy(u0).cuda()
    T = 5
    free0 = _free()
    _noalloc(lib, z, W, T, out=z)
    assert _free() >= free0
    assert rel_l2(z.cpu().numpy(), oracle.sweep_f64(u0, W, T)) <= fp32_tol(T)


def test_noalloc_rejects_grids_beyond_the_scratch(lib):
    W = inputs.pattern_weights("box9")
    x = torch.empty((8192, 8192), device="cuda")  # 256 MiB > the 64 MiB scratch
    Wc = np.ascontiguousarray(W)
    st = lib.stencil_run_noalloc(8192, 8192, 1, Wc.ctypes.data_as(ctypes.POINTER(ctypes.c_float)),
                                 0, 0, x.data_ptr(), x.data_ptr(), 1, None)
    assert st == 2  # STENCIL_ERR_UNSUPPORTED
    assert "exceeds" in lib.stencil_noalloc_last_error().decode()
