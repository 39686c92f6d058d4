"""The TMA-fed streaming kernel (rows brought in by cp.async.bulk.tensor copies
into an mbarrier-completed ring; the copy engine's zero fill is the zero halo
of Sec. IV-A).  Same arithmetic as the cp.async-fed kernel, so every result
must be bit-identical to it, and exact on dyadic data."""
import numpy as np
import pytest

from paper_2605_07954_gb300 import inputs
from _util import fp32_tol, rel_l2

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2605_07954_gb300 import build
    build.build()


def _run(u0, W, T, load, **kw):
    from paper_2605_07954_gb300 import Plan
    x = torch.from_numpy(np.ascontiguousarray(u0, dtype=np.float32)).cuda()
    p = Plan(x.shape[0], x.shape[1], W, kernel="stream", load=load, **kw)
    y = p.run(x, T)
    torch.cuda.synchronize()
    p.status()
    info = p.info()
    p.close()
    return y, info


@pytest.mark.parametrize("name,k", [("heat5", 8), ("box9", 8), ("box9", 3), ("star13", 2), ("star13", 3),
                                    ("star13", 4), ("box49", 1), ("box49", 2)])
@pytest.mark.parametrize("ny,nx,threads", [(1000, 1024, 128), (301, 516, 64), (77, 2052, 256), (9, 12, 32)])
def test_tma_bitwise_equals_cp_async(name, k, ny, nx, threads):
    W = inputs.pattern_weights(name)
    u0 = inputs.field(ny, nx)
    T = 2 * k + 1
    a, ia = _run(u0, W, T, "tma", tb_depth=k, threads=threads)
    b, ib = _run(u0, W, T, "cp_async", tb_depth=k, threads=threads)
    assert ia["load"] == 2 and ib["load"] == 1
    assert torch.equal(a, b), (name, k, ny, nx, threads)


@pytest.mark.parametrize("r", [1, 2, 3])
def test_tma_radius2_and_in_place(oracle, r):
    rng = np.random.default_rng(r)
    d = 2 * r + 1
    W = (rng.uniform(size=(d, d)) / (d * d)).astype(np.float32)
    u0 = inputs.field(333, 644)
    from paper_2605_07954_gb300 import Plan
    x = torch.from_numpy(u0).cuda()
    p = Plan(333, 644, W, kernel="stream", load="tma")
    p.run(x, 7, out=x)  # in place: an odd launch count is split
    torch.cuda.synchronize()
    p.status()
    assert rel_l2(x.cpu().numpy(), oracle.sweep_f64(u0, W, 7)) <= fp32_tol(7)
    p.close()


def test_tma_dyadic_exact(oracle):
    """Weights k/8 (k <= 2), inputs m/256: after T steps every value is an
    integer over 8^T * 256 of at most (2 (2r+1)^2)^T * 255, under 2^24 for
    T = 3 at r = 1 and T = 2 at r = 3, so FP32 is exact."""
    rng = np.random.default_rng(5)
    for r, T in ((1, 3), (3, 2)):
        d = 2 * r + 1
        W = (rng.integers(0, 3, size=(d, d)) / 8.0).astype(np.float32)
        u0 = (rng.integers(0, 256, size=(130, 260)) / 256.0).astype(np.float32)
        y, _ = _run(u0, W, T, "tma")
        assert np.array_equal(y.cpu().numpy().astype(np.float64), oracle.sweep_f64(u0, W, T))


def test_tma_unsupported_layouts_rejected():
    from paper_2605_07954_gb300 import Plan, StencilError
    W = inputs.pattern_weights("box9")
    for kw in (dict(dtype="bf16"), dict(boundary="periodic"), dict(ny=64, nx=66)):
        args = dict(ny=64, nx=64)
        args.update({k: v for k, v in kw.items() if k in ("ny", "nx")})
        opts = {k: v for k, v in kw.items() if k not in ("ny", "nx")}
        with pytest.raises(StencilError):
            Plan(args["ny"], args["nx"], W, kernel="stream", load="tma", **opts)


def test_tma_unaligned_source_uses_cp_async_path():
    """A source that is not 16-byte aligned has no tensor map: the launch runs
    the cp.async kernel with the same arithmetic."""
    W = inputs.pattern_weights("star13")
    u0 = inputs.field(200, 256)
    from paper_2605_07954_gb300 import Plan
    buf = torch.zeros(200 * 256 + 1, device="cuda")
    x = buf[1:].view(200, 256)
    x.copy_(torch.from_numpy(u0))
    p = Plan(200, 256, W, kernel="stream", load="tma")
    y = p.run(x, 5)
    torch.cuda.synchronize()
    p.status()
    ref, _ = _run(u0, W, 5, "cp_async")
    assert torch.equal(y, ref)
    p.close()


def test_tma_expired_wait_reports_timeout_and_device_recovers():
    """CTA 0 waits for bytes its first row never brings (test hook): the wait
    runs out after 100 ms, the plan reports STENCIL_ERR_TIMEOUT, and a normal
    plan afterwards gives the right result."""
    from paper_2605_07954_gb300 import Plan, StencilError
    W = inputs.pattern_weights("box9")
    u0 = inputs.field(512, 512)
    x = torch.from_numpy(u0).cuda()
    p = Plan(512, 512, W, kernel="stream", load="tma", tb_depth=8, timeout_ms=100, debug_withhold=1)
    p.run(x, 8)
    with pytest.raises(StencilError) as e:
        p.status()
    assert "TIMEOUT" in str(e.value)
    p.close()
    y, _ = _run(u0, W, 8, "tma", tb_depth=8)
    z, _ = _run(u0, W, 8, "cp_async", tb_depth=8)
    assert torch.equal(y, z)
