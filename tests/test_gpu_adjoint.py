"""GPU tests of the adjoint (stencil_adjoint) and the autograd Function.

The adjoint is checked against the FP64 oracle's gradient (which the CPU pins
check against finite differences), by the dot test <A^T x, y> = <x, (A^T)' y>,
and for exact independence of the checkpoint interval.
"""
import numpy as np
import pytest

from paper_2605_07954_gb300 import inputs
from _util import rel_l2

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2605_07954_gb300 import build
    build.build()


def _grads(u0, W, T, gT, boundary="zero", ckpt=0, **plan_opts):
    from paper_2605_07954_gb300 import Plan, adjoint
    p = Plan(u0.shape[0], u0.shape[1], W, boundary=boundary, **plan_opts)
    gu, gw = adjoint(p, torch.from_numpy(np.ascontiguousarray(u0, dtype=np.float32)).cuda(),
                     torch.from_numpy(np.ascontiguousarray(gT, dtype=np.float32)).cuda(), T, ckpt)
    torch.cuda.synchronize()
    p.close()
    return gu.cpu().numpy().astype(np.float64), gw.cpu().numpy()


@pytest.mark.parametrize("boundary", ["zero", "periodic"])
@pytest.mark.parametrize("name", ["heat5", "box9", "star13", "asym2"])
def test_gradients_match_oracle(oracle, name, boundary):
    """64x64, 32 steps, L = 0.5 ||u_T - target||^2: both gradients vs the FP64 oracle."""
    if name == "asym2":
        rng = np.random.default_rng(41)
        W = (rng.uniform(-1, 1, size=(5, 5)) / 12.5).astype(np.float32)
    else:
        W = inputs.pattern_weights(name)
    u0 = inputs.field(64, 64)
    target = inputs.field(64, 64, stream=inputs.STREAM_TARGET)
    T = 32
    uT = oracle.sweep_f64(u0, W, T, boundary)
    gT = (uT - target).astype(np.float32)
    ref_u, ref_w = oracle.adjoint_f64(u0, W, T, gT.astype(np.float64), boundary)
    gu, gw = _grads(u0, W, T, gT, boundary)
    assert rel_l2(gu, ref_u) <= 1e-4
    fp = np.abs(W) > 0
    assert rel_l2(gw[fp], ref_w[fp]) <= 1e-4
    assert rel_l2(gw, ref_w) <= 1e-4


@pytest.mark.parametrize("boundary", ["zero", "periodic"])
@pytest.mark.parametrize("shape", [(70, 132), (5, 8), (129, 260), (64, 4), (300, 520)])
@pytest.mark.parametrize("name", ["heat5", "box9"])
def test_row_streamed_step_ragged_shapes(oracle, name, shape, boundary):
    """Radius 1 with widths that are a multiple of 4 takes the row-streaming
    reverse step: 128-column strips and 64-row tiles that the shapes cut
    unevenly, strips wider than the grid, grids shorter than a warp's rows;
    both gradients against the FP64 oracle."""
    W = inputs.pattern_weights(name)
    u0 = inputs.field(*shape)
    target = inputs.field(*shape, stream=inputs.STREAM_TARGET)
    T = 12
    uT = oracle.sweep_f64(u0, W, T, boundary)
    gT = (uT - target).astype(np.float32)
    ref_u, ref_w = oracle.adjoint_f64(u0, W, T, gT.astype(np.float64), boundary)
    gu, gw = _grads(u0, W, T, gT, boundary)
    assert rel_l2(gu, ref_u) <= 1e-5
    assert rel_l2(gw, ref_w) <= 1e-5


def test_checkpoint_interval_does_not_change_bits():
    W = inputs.pattern_weights("box9")
    u0 = inputs.field(100, 130)
    gT = inputs.field(100, 130, stream=inputs.STREAM_TARGET)
    T = 37
    base = _grads(u0, W, T, gT, ckpt=0)
    for c in (1, 5, 36, 37, 100):
        other = _grads(u0, W, T, gT, ckpt=c)
        assert np.array_equal(base[0], other[0]) and np.array_equal(base[1], other[1]), c
    # and, on the streaming kernel, neither on the forward plan's temporal-blocking
    # depth (the default plan of this small grid is the cluster-resident kernel,
    # whose per-point summation order is its own)
    stream = _grads(u0, W, T, gT, kernel="stream")
    for k in (1, 2, 8):
        other = _grads(u0, W, T, gT, tb_depth=k)
        assert np.array_equal(stream[0], other[0]) and np.array_equal(stream[1], other[1]), k
    assert rel_l2(stream[0], base[0]) <= 1e-5 and rel_l2(stream[1], base[1]) <= 1e-5


@pytest.mark.parametrize("boundary", ["zero", "periodic"])
def test_dot_test(boundary):
    """<A^T x, y> = <x, (A^T)' y> for the T-step operator, in FP32 to 1e-5."""
    from paper_2605_07954_gb300 import Plan
    rng = np.random.default_rng(43)
    W = (rng.uniform(-1, 1, size=(7, 7)) / 20).astype(np.float32)
    x = rng.normal(size=(300, 257)).astype(np.float32)
    y = rng.normal(size=(300, 257)).astype(np.float32)
    T = 20
    p = Plan(300, 257, W, boundary=boundary)
    Ax = p.run(torch.from_numpy(x).cuda(), T).cpu().numpy().astype(np.float64)
    p.close()
    ATy, _ = _grads(np.zeros_like(x), W, T, y, boundary)
    lhs, rhs = float(np.vdot(Ax, y)), float(np.vdot(x.astype(np.float64), ATy))
    assert abs(lhs - rhs) <= 1e-5 * max(abs(lhs), np.linalg.norm(Ax) * np.linalg.norm(y) * 1e-3)


def test_autograd_function_matches_adjoint(oracle):
    from paper_2605_07954_gb300 import StencilFn
    W = torch.from_numpy(inputs.heat_weights(0.2).astype(np.float64)).requires_grad_()
    u0 = torch.from_numpy(inputs.field(64, 64)).cuda().requires_grad_()
    target = torch.from_numpy(inputs.field(64, 64, stream=inputs.STREAM_TARGET)).cuda()
    uT = StencilFn.apply(u0, W, 32)
    loss = 0.5 * ((uT - target) ** 2).sum()
    loss.backward()
    gT = (uT.detach() - target).cpu().numpy().astype(np.float64)
    ref_u, ref_w = oracle.adjoint_f64(u0.detach().cpu().numpy(), W.detach().numpy(), 32, gT)
    assert rel_l2(u0.grad.cpu().numpy(), ref_u) <= 1e-4
    assert W.grad.dtype == torch.float64 and W.grad.device.type == "cpu"
    assert rel_l2(W.grad.numpy(), ref_w) <= 1e-4


def test_autograd_loop_reuses_plans(oracle):
    """A training loop: StencilFn with new weights every iteration.  Each
    iteration's gradients match the oracle's, and after the first iteration no
    device memory is taken (the cached plan and its adjoint scratch are reused
    with the new weights)."""
    from paper_2605_07954_gb300 import StencilFn
    u0 = torch.from_numpy(inputs.field(96, 80)).cuda().requires_grad_()
    target = torch.from_numpy(inputs.field(96, 80, stream=inputs.STREAM_TARGET)).cuda()
    rng = np.random.default_rng(3)
    free = []
    for it in range(4):
        Wn = rng.uniform(0.05, 0.2, size=(3, 3))
        W = torch.from_numpy(Wn).requires_grad_()
        u0.grad = None
        uT = StencilFn.apply(u0, W, 16)
        loss = 0.5 * ((uT - target) ** 2).sum()
        loss.backward()
        torch.cuda.synchronize()
        free.append(torch.cuda.mem_get_info()[0])
        gT = (uT.detach() - target).cpu().numpy().astype(np.float64)
        ref_u, ref_w = oracle.adjoint_f64(u0.detach().cpu().numpy(), W.detach().numpy().astype(np.float32),
                                          16, gT)
        assert rel_l2(u0.grad.cpu().numpy(), ref_u) <= 1e-4, it
        assert rel_l2(W.grad.numpy(), ref_w) <= 1e-4, it
    assert free[-1] >= free[1], free


def test_weight_gradient_into_host_memory():
    """grad_w may be host memory: the call synchronises and writes the same
    values as into device memory."""
    import ctypes
    from paper_2605_07954_gb300 import Plan, _capi
    W = inputs.pattern_weights("box9")
    u0 = torch.from_numpy(inputs.field(70, 90)).cuda()
    gT = torch.from_numpy(inputs.field(70, 90, stream=inputs.STREAM_TARGET)).cuda()
    p = Plan(70, 90, W)
    lib = _capi.load()
    st = torch.cuda.current_stream().cuda_stream
    gu = torch.empty_like(u0)
    gw_dev = torch.empty((3, 3), dtype=torch.float64, device="cuda")
    assert lib.stencil_adjoint(p.handle, u0.data_ptr(), gT.data_ptr(), 12, gu.data_ptr(),
                               gw_dev.data_ptr(), 0, st) == 0
    for host in (np.zeros(9), torch.zeros(9, dtype=torch.float64).pin_memory().numpy()):
        assert lib.stencil_adjoint(p.handle, u0.data_ptr(), gT.data_ptr(), 12, gu.data_ptr(),
                                   host.ctypes.data_as(ctypes.c_void_p), 0, st) == 0
        assert np.array_equal(host, gw_dev.cpu().numpy().ravel())
    p.close()


def test_set_weights_keeps_the_footprint():
    from paper_2605_07954_gb300 import Plan, StencilError
    p = Plan(64, 64, inputs.heat_weights(0.2))
    p.set_weights(inputs.heat_weights(0.1))  # still a 5-point star
    with pytest.raises(StencilError):
        p.set_weights(inputs.pattern_weights("box9"))  # a box: another kernel
    p.close()


def test_fullsize_heat_4096_T512_window(oracle):
    """The 4096^2, 512-step Heat workload: the corner window of dL/du0 against
    the FP64 oracle on its exact light cone, and the dot test at full size."""
    from paper_2605_07954_gb300 import Plan, adjoint
    n, T = 4096, 512
    W = inputs.heat_weights(0.2)
    u0 = inputs.field(n, n)
    target = inputs.field(n, n, stream=inputs.STREAM_TARGET)
    p = Plan(n, n, W)
    x = torch.from_numpy(u0).cuda()
    uT = p.run(x, T)
    gT = uT - torch.from_numpy(target).cuda()
    gu, gw = adjoint(p, x, gT, T)
    torch.cuda.synchronize()
    # window [0, b)^2 of lambda_0 needs lambda_T on [0, b + T), which needs u_0 on [0, b + 2T)
    b = 24
    m1, m2 = b + T, b + 2 * T
    uT_ref = oracle.sweep_f64(u0[:m2, :m2], W, T)[:m1, :m1]
    gT_ref = uT_ref - target[:m1, :m1]
    lam0_ref, _ = oracle.adjoint_f64(np.zeros((m1, m1)), W, T, gT_ref)
    e = rel_l2(gu[:b, :b].cpu().numpy(), lam0_ref[:b, :b])
    print(f"4096^2 T=512 corner window dL/du0 relL2={e:.3e}")
    assert e <= 1e-4
    # dot test of the full-size operator: <A^T x, y> = <x, (A^T)' y>
    yv = gT
    Ax = uT
    zero = torch.zeros_like(x)
    ATy, _ = adjoint(p, zero, yv, T)
    lhs = float(torch.dot(Ax.double().flatten(), yv.double().flatten()))
    rhs = float(torch.dot(x.double().flatten(), ATy.double().flatten()))
    assert abs(lhs - rhs) <= 1e-5 * abs(lhs)
    p.close()
