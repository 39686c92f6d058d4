"""Periodic convergence checks (stencil_run_residual): residuals ||u_t - u_{t-1}||_2
after every m-th step against the FP64 oracle, and the final state bit-identical
to stencil_run."""
import numpy as np
import pytest

from paper_2605_07954_gb300 import inputs

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2605_07954_gb300 import build
    build.build()


@pytest.mark.parametrize("name,boundary", [("box9", "zero"), ("star13", "periodic"), ("heat5", "zero")])
@pytest.mark.parametrize("T,m", [(23, 5), (10, 1), (4, 9), (24, 8)])
def test_residuals_match_oracle(oracle, name, boundary, T, m):
    from paper_2605_07954_gb300 import Plan
    W = inputs.pattern_weights(name)
    # periodic widths that are multiples of 4 keep results independent of the
    # launch depths (see test_depth_does_not_change_bits)
    nx = 256 if boundary == "periodic" else 257
    u0 = inputs.field(130, nx)
    p = Plan(130, nx, W, boundary=boundary)
    x = torch.from_numpy(u0).cuda()
    y, res = p.run_residual(x, T, m)
    ref_final = p.run(x, T)
    torch.cuda.synchronize()
    assert torch.equal(y, ref_final)
    assert res.numel() == T // m
    states = [u0.astype(np.float64)]
    for t in range(T):
        states.append(oracle.sweep_f64(states[-1], W, 1, boundary))
    want = [np.linalg.norm(states[t] - states[t - 1]) for t in range(m, T + 1, m)]
    np.testing.assert_allclose(res.cpu().numpy(), want, rtol=2e-4)
    p.close()


def test_fullsize_residuals_nonincreasing():
    """8192^2 Box-9 (non-negative weights summing to 1, zero boundary): the
    step operator is a contraction, so the residual never grows."""
    from paper_2605_07954_gb300 import Plan
    W = inputs.pattern_weights("box9")
    p = Plan(8192, 8192, W)
    x = torch.from_numpy(inputs.field(8192, 8192)).cuda()
    y, res = p.run_residual(x, 1000, 100)
    ref = p.run(x, 1000)
    torch.cuda.synchronize()
    assert torch.equal(y, ref)
    r = res.cpu().numpy()
    assert len(r) == 10 and np.all(r > 0)
    assert np.all(r[1:] <= r[:-1] * (1 + 1e-6))
    p.close()
