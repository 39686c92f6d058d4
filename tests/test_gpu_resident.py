"""GPU tests of the cluster-resident kernel (small grids held in the shared
memory of one thread-block cluster, every step of a run in one launch).

Against the FP64 oracle for every footprint, both boundaries and the three
storage types, on shapes that give one to sixteen CTAs per cluster, slabs of
uneven height, and widths that are not multiples of anything; bit-exact on
dyadic data; in-place runs; launch counts; and the streaming kernel and the
resident kernel agreeing to FP32 rounding on the same plan shapes.
"""
import numpy as np
import pytest

from paper_2605_07954_gb300 import inputs
from _util import fp32_elem_tol, fp32_tol, rel_l2, rel_linf

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

TDT = {"f32": torch.float32, "bf16": torch.bfloat16, "f16": torch.float16}


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2605_07954_gb300 import build
    build.build()


def _weights(name):
    if name == "box25":  # radius 2, asymmetric, with holes
        rng = np.random.default_rng(25)
        W = rng.random((5, 5)).astype(np.float32)
        W[rng.random((5, 5)) < 0.3] = 0.0
        return (W / W.sum()).astype(np.float32)
    return inputs.pattern_weights(name)


def _run(u0, W, T, boundary="zero", dtype="f32", **opts):
    from paper_2605_07954_gb300 import Plan
    x = torch.from_numpy(np.ascontiguousarray(u0, dtype=np.float32)).to("cuda", TDT[dtype])
    p = Plan(u0.shape[0], u0.shape[1], W, dtype=dtype, boundary=boundary, **opts)
    info = p.info()
    y = p.run(x, T)
    torch.cuda.synchronize()
    p.status()
    launches = p.launches(T)
    p.close()
    return y.float().cpu().numpy().astype(np.float64), info, launches


@pytest.mark.parametrize("name", ["heat5", "box9", "star13", "box49", "box25"])
@pytest.mark.parametrize("boundary", ["zero", "periodic"])
@pytest.mark.parametrize("shape", [(130, 517), (64, 64), (300, 7), (9, 400), (17, 33), (512, 512)])
def test_parity_fp32(oracle, name, boundary, shape):
    W = _weights(name)
    u0 = inputs.field(*shape)
    T = 23
    got, info, launches = _run(u0, W, T, boundary, kernel="resident")
    assert info["kernel"] == 6 and info["tb_depth"] == 0 and launches == 1
    ref = oracle.sweep_f64(u0, W, T, boundary)
    taps = int(np.count_nonzero(W))
    assert rel_l2(got, ref) <= fp32_tol(T)
    assert rel_linf(got, ref) <= fp32_elem_tol(T, taps)


def test_cluster_sizes_cover_one_to_sixteen():
    """The largest usable cluster is taken: 16 for tall grids, fewer when the
    slabs would get shorter than the radius."""
    from paper_2605_07954_gb300 import Plan
    W = inputs.pattern_weights("box49")
    assert Plan(512, 512, W, kernel="resident").info()["ctas"] == 16
    assert Plan(20, 64, W, kernel="resident").info()["ctas"] in (4, 8)
    assert Plan(3, 64, W, kernel="resident").info()["ctas"] == 1
    i = Plan(4, 64, W, kernel="resident", boundary="periodic").info()
    assert i["ctas"] == 1 and i["tile_rows"] == 4


@pytest.mark.parametrize("dtype,gate", [("bf16", 1e-2), ("f16", 5e-3)])
def test_reduced_precision_storage(oracle, dtype, gate):
    W = inputs.pattern_weights("box9")
    u0 = inputs.field(200, 333)
    got, info, _ = _run(u0, W, 50, dtype=dtype, kernel="resident")
    assert info["kernel"] == 6
    assert rel_l2(got, oracle.sweep_f64(u0, W, 50)) <= gate


@pytest.mark.parametrize("boundary", ["zero", "periodic"])
def test_dyadic_bitwise(oracle, boundary):
    """Weights in {0, 1/8} and a 0/1 field: after T steps every value is a
    multiple of 8^-T below 49^T / 8^T, exact in FP32 for T <= 3."""
    rng = np.random.default_rng(3)
    W = np.where(rng.random((7, 7)) < 0.6, 0.125, 0.0).astype(np.float32)
    u0 = (rng.random((150, 211)) < 0.5).astype(np.float32)
    got, _, _ = _run(u0, W, 3, boundary, kernel="resident")
    assert np.array_equal(got, oracle.sweep_f64(u0, W, 3, boundary))


def test_in_place_and_zero_steps():
    from paper_2605_07954_gb300 import Plan
    W = inputs.pattern_weights("star13")
    u0 = inputs.field(257, 300)
    p = Plan(257, 300, W, kernel="resident")
    x = torch.from_numpy(u0).cuda()
    y = p.run(x, 11)
    z = x.clone()
    p.run(z, 11, out=z)
    w = p.run(x, 0)
    torch.cuda.synchronize()
    assert torch.equal(y, z) and torch.equal(w, x)
    assert p.launches(0) == 0 and p.launches(11) == 1
    p.close()


def test_matches_streaming_kernel():
    """The same plan shape on the streaming kernel: same operation, other
    summation order, so equal to FP32 rounding."""
    W = inputs.pattern_weights("box9")
    u0 = inputs.field(333, 480)
    a, ia, _ = _run(u0, W, 100, kernel="resident")
    b, ib, _ = _run(u0, W, 100, kernel="stream")
    assert ia["kernel"] == 6 and ib["kernel"] == 2
    assert rel_l2(a, b) <= 2 * fp32_tol(100)


def test_default_choice_and_autotune(oracle):
    """kernel = AUTO picks the resident kernel for grids that fit one cluster
    (unless a streaming-kernel option is set); autotuning keeps whichever is
    faster, and either result matches the oracle."""
    from paper_2605_07954_gb300 import Plan
    W = inputs.pattern_weights("heat5")
    assert Plan(512, 512, W).info()["kernel"] == 6
    assert Plan(512, 512, W, tb_depth=4).info()["kernel"] == 2
    assert Plan(4096, 4096, W).info()["kernel"] == 2
    u0 = inputs.field(512, 512)
    got, info, _ = _run(u0, W, 100, autotune=True)
    print("autotuned 512^2 Heat:", info["kernel"], info["ctas"])
    assert rel_l2(got, oracle.sweep_f64(u0, W, 100)) <= fp32_tol(100)


def test_rejects_grids_that_do_not_fit():
    from paper_2605_07954_gb300 import Plan, StencilError
    with pytest.raises(StencilError, match="UNSUPPORTED"):
        Plan(2048, 2048, inputs.pattern_weights("box9"), kernel="resident")


@pytest.mark.parametrize("name,kb", [("heat5", 2), ("box9", 4), ("box9", 8), ("star13", 2), ("box25", 2)])
@pytest.mark.parametrize("boundary", ["zero", "periodic"])
def test_blocked_exchange_depths(oracle, name, kb, boundary):
    """kb steps per halo exchange (slabs with kb*R-deep halos, redundant rows
    recomputed, double-buffered mailboxes): the same results, for step counts
    that are and are not multiples of kb."""
    W = _weights(name)
    u0 = inputs.field(260, 300)
    for T in (kb * 3, kb * 3 + 1):
        got, info, launches = _run(u0, W, T, boundary, kernel="resident", tb_depth=kb)
        assert info["kernel"] == 6 and launches == 1
        ref = oracle.sweep_f64(u0, W, T, boundary)
        assert rel_l2(got, ref) <= fp32_tol(T)
        assert rel_linf(got, ref) <= fp32_elem_tol(T, int(np.count_nonzero(W)))
    # bit-identical to one step per exchange: the per-point arithmetic is the same
    a, _, _ = _run(u0, W, 3 * kb + 1, boundary, kernel="resident", tb_depth=kb)
    b, _, _ = _run(u0, W, 3 * kb + 1, boundary, kernel="resident")
    assert np.array_equal(a, b)
