"""The separable (low-rank) form of the step: compute = "lowrank".

The weights are factored by an SVD, W = sum_k c_k v_k^T, and each step runs
as row passes and column passes (the low-rank stencil idea the paper cites in
its related work, Sec. II-D).  For weights of exact rank 1..3 the result is
the oracle's up to the FP32 rounding of the factors; a forced lower rank
gives the truncated SVD's operator.
"""
import numpy as np
import pytest

from paper_2605_07954_gb300 import inputs
from _util import rel_l2

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2605_07954_gb300 import build
    build.build()


def _rank_weights(r, rho, seed):
    """A (2r+1)^2 FP32 weight array of exact rank rho (sum of rho outer products), sum 1."""
    rng = np.random.default_rng(seed)
    d = 2 * r + 1
    w = sum(np.outer(rng.uniform(0.1, 1.0, d), rng.uniform(0.1, 1.0, d)) for _ in range(rho))
    return (w / w.sum()).astype(np.float32)


def _run(u0, W, T, boundary="zero", **kw):
    from paper_2605_07954_gb300 import Plan
    x = torch.from_numpy(u0).cuda()
    p = Plan(u0.shape[0], u0.shape[1], W, boundary=boundary, compute="lowrank", **kw)
    y = p.run(x, T)
    torch.cuda.synchronize()
    p.status()
    info = p.info()
    p.close()
    return y.cpu().numpy(), info


@pytest.mark.parametrize("r,rho", [(1, 1), (1, 2), (2, 2), (3, 1), (3, 2), (3, 3)])
@pytest.mark.parametrize("boundary", ["zero", "periodic"])
def test_exact_low_rank_matches_oracle(oracle, r, rho, boundary):
    W = _rank_weights(r, rho, seed=10 * r + rho)
    u0 = inputs.field(301, 517)
    T = 8
    got, info = _run(u0, W, T, boundary)
    assert info["rank"] == rho and info["kernel"] == 7
    assert rel_l2(got, oracle.sweep_f64(u0, W, T, boundary)) <= 1e-6


def test_full_rank_box49_is_exact_to_fp32(oracle):
    """Random 7x7 weights have rank 7: seven terms reproduce them to FP32 rounding."""
    W = inputs.pattern_weights("box49")
    u0 = inputs.field(260, 384)
    got, info = _run(u0, W, 6)
    assert info["rank"] == 7
    assert rel_l2(got, oracle.sweep_f64(u0, W, 6)) <= 1e-6


def test_forced_rank_is_the_truncated_svd(oracle):
    """rank = 1 on rank-3 weights: the operator of the best rank-1 approximation."""
    W = _rank_weights(3, 3, seed=4)
    U, s, Vt = np.linalg.svd(W.astype(np.float64))
    W1 = s[0] * np.outer(U[:, 0], Vt[0])
    u0 = inputs.field(200, 256)
    got, info = _run(u0, W, 5, rank=1)
    assert info["rank"] == 1
    assert rel_l2(got, oracle.sweep_f64(u0, W1, 5)) <= 1e-6
    # ... which is not the full operator
    assert rel_l2(got, oracle.sweep_f64(u0, W, 5)) > 1e-4


def test_in_place_odd_steps_and_tiny_grids(oracle):
    W = _rank_weights(3, 2, seed=7)
    for ny, nx in ((5, 3), (1, 130), (129, 1)):
        u0 = inputs.field(ny, nx)
        from paper_2605_07954_gb300 import Plan
        x = torch.from_numpy(u0).cuda()
        p = Plan(ny, nx, W, compute="lowrank")
        p.run(x, 3, out=x)
        torch.cuda.synchronize()
        assert rel_l2(x.cpu().numpy(), oracle.sweep_f64(u0, W, 3)) <= 1e-6, (ny, nx)
        p.close()
