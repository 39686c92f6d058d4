"""GPU tests of the 7x7 box on tensor cores (TF32 / BF16 warp MMAs, FP32 accumulate)
and of the precision variants of the 16384^2, 200-step Box-49 workload.

One step with dyadic data is exact on every engine, so it must match the
oracle bit for bit: that pins the Toeplitz band, the fragment layouts and the
row/column offsets.  Multi-step results are compared with the FP64 oracle and
their relative L2 / L-infinity errors are printed (reported, not gated
tightly: TF32 keeps 11 significand bits, BF16 8).
"""
import numpy as np
import pytest

from paper_2605_07954_gb300 import inputs
from _util import fp32_tol, rel_l2, rel_linf

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

ENGINES = [("tc_tf32", "f32"), ("tc_bf16", "bf16"), ("tc_bf16", "f32"), ("tc_tf32", "bf16"),
           ("tc_3xtf32", "f32")]


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2605_07954_gb300 import build
    build.build()


def _run(u0, W, T, compute, dtype, boundary="zero"):
    from paper_2605_07954_gb300 import Plan
    tdt = {"f32": torch.float32, "bf16": torch.bfloat16}[dtype]
    x = torch.from_numpy(np.ascontiguousarray(u0, dtype=np.float32)).to("cuda", tdt)
    p = Plan(u0.shape[0], u0.shape[1], W, dtype=dtype, boundary=boundary, compute=compute)
    info = p.info()
    y = p.run(x, T)
    torch.cuda.synchronize()
    p.status()
    p.close()
    return y.float().cpu().numpy().astype(np.float64), info


@pytest.mark.parametrize("compute,dtype", ENGINES)
@pytest.mark.parametrize("shape", [(131, 260), (256, 384), (77, 130)])
@pytest.mark.parametrize("boundary", ["zero", "periodic"])
def test_one_step_dyadic_exact(oracle, compute, dtype, shape, boundary):
    """Inputs m/256 (m < 256) and weights k/8 (k < 4) are exact in TF32 and BF16,
    and every partial sum of one step fits FP32: the result is exact."""
    rng = np.random.default_rng(shape[0] + shape[1])
    W = (rng.integers(0, 4, size=(7, 7)) / 8.0).astype(np.float32)
    W[rng.random((7, 7)) < 0.3] = 0.0  # asymmetric, with holes
    u0 = (rng.integers(0, 256, size=shape) / 256.0).astype(np.float32)
    got, info = _run(u0, W, 1, compute, dtype, boundary)
    assert info["kernel"] in (3, 5)  # warp MMAs, or tcgen05 where it applies
    ref = oracle.sweep_f64(u0, W, 1, boundary)
    if dtype == "bf16":  # the stored result is rounded to BF16
        ref = torch.from_numpy(ref.astype(np.float32)).bfloat16().float().numpy()
    assert np.array_equal(got, ref)


@pytest.mark.parametrize("compute,dtype,gate", [("tc_tf32", "f32", 2e-3), ("tc_bf16", "bf16", 2e-2),
                                                ("tc_bf16", "f32", 2e-2), ("tc_tf32", "bf16", 2e-2),
                                                ("tc_3xtf32", "f32", 1e-5)])
def test_multistep_error_vs_oracle(oracle, compute, dtype, gate):
    W = inputs.pattern_weights("box49")
    u0 = inputs.field(300, 517)
    T = 20
    ref = oracle.sweep_f64(u0, W, T)
    got, _ = _run(u0, W, T, compute, dtype)
    e2, ei = rel_l2(got, ref), rel_linf(got, ref)
    print(f"{compute}/{dtype} 300x517 T={T}: relL2={e2:.3e} relLinf={ei:.3e}")
    assert e2 <= gate


@pytest.mark.parametrize("compute,dtype", [("tc_tf32", "f32"), ("tc_bf16", "bf16"), ("tc_3xtf32", "f32")])
@pytest.mark.parametrize("boundary", ["zero", "periodic"])
def test_pipelined_equals_single_tile_kernel(compute, dtype, boundary):
    """The persistent double-buffered kernel (aligned rows) and the one-tile-per-CTA
    kernel (taken when the rows are not 16-byte aligned) give the same bits over
    several steps: keeping the state TF32-rounded between launches rounds each
    step's input exactly once, as rounding at load does."""
    from paper_2605_07954_gb300 import Plan
    W = inputs.pattern_weights("box49")
    u0 = inputs.field(300, 520)
    tdt = {"f32": torch.float32, "bf16": torch.bfloat16}[dtype]
    p = Plan(300, 520, W, dtype=dtype, boundary=boundary, compute=compute, kernel="tc_warp")
    x = torch.from_numpy(u0).to("cuda", tdt)
    a = p.run(x, 7)
    # the same grid at an offset of one element: rows are no longer 16-byte aligned
    buf = torch.empty(300 * 520 + 1, dtype=tdt, device="cuda")
    xs = buf[1:].view(300, 520)
    xs.copy_(x)
    obuf = torch.empty_like(buf)
    ys = obuf[1:].view(300, 520)
    p.run(xs, 7, out=ys)
    torch.cuda.synchronize()
    assert torch.equal(a, ys)
    p.close()


def test_rejects_unsupported():
    from paper_2605_07954_gb300 import Plan, StencilError
    with pytest.raises(StencilError, match="UNSUPPORTED"):
        Plan(64, 64, inputs.pattern_weights("box9"), compute="tc_tf32")
    with pytest.raises(StencilError, match="UNSUPPORTED"):
        Plan(64, 64, inputs.pattern_weights("box49"), dtype="f16", compute="tc_bf16")
    with pytest.raises(StencilError, match="UNSUPPORTED"):
        Plan(300, 392, inputs.pattern_weights("box49"), dtype="bf16", compute="tc_3xtf32")
    with pytest.raises(StencilError, match="UNSUPPORTED"):
        Plan(300, 392, inputs.pattern_weights("box49"), compute="tc_3xtf32", kernel="tc_umma")


VARIANTS = [("fp32", "f32", 1e-5), ("fp32", "bf16", 1e-2), ("tc_tf32", "f32", 5e-2),
            ("tc_bf16", "bf16", 5e-2), ("tc_3xtf32", "f32", 1e-5)]


@pytest.mark.parametrize("compute,dtype,gate", VARIANTS)
def test_box49_16384_T200_variants(oracle, compute, dtype, gate):
    """The 16384^2, 200-step Box-49 workload on each engine: the corner window
    and an interior window against their exact light cones in FP64."""
    n, T, b = 16384, 200, 24
    W = inputs.pattern_weights("box49")
    u0 = inputs.field(n, n)
    got, info = _run(u0, W, T, compute, dtype)
    m = 3 * T
    errs = []
    for (y0, x0) in ((0, 0), (n // 2 + 5, n // 3 - 7)):
        a0, b0 = max(0, y0 - m), max(0, x0 - m)
        sub = oracle.sweep_f64(u0[a0:y0 + b + m, b0:x0 + b + m], W, T)
        ref = sub[y0 - a0:y0 - a0 + b, x0 - b0:x0 - b0 + b]
        g = got[y0:y0 + b, x0:x0 + b]
        errs.append((rel_l2(g, ref), rel_linf(g, ref)))
    print(f"box49 16384^2 T=200 {compute}/{dtype}: corner relL2={errs[0][0]:.3e} "
          f"relLinf={errs[0][1]:.3e}; interior relL2={errs[1][0]:.3e} relLinf={errs[1][1]:.3e}")
    assert max(e[0] for e in errs) <= gate
    assert got.min() >= -1e-3 and got.max() <= u0.max() * (1 + 1e-2)


def test_3xtf32_recovers_fp32_accuracy(oracle):
    """Splitting operands into TF32 hi + lo parts brings the tensor-core error
    from TF32 level down to that of the FP32 CUDA-core path (same order of
    magnitude), 20 steps of Box-49 on a random field."""
    W = inputs.pattern_weights("box49")
    u0 = inputs.field(300, 520)
    T = 20
    ref = oracle.sweep_f64(u0, W, T)
    errs = {c: rel_l2(_run(u0, W, T, c, "f32")[0], ref) for c in ("fp32", "tc_tf32", "tc_3xtf32")}
    print("relL2 after 20 steps:", {k: f"{v:.2e}" for k, v in errs.items()})
    assert errs["tc_3xtf32"] <= 1e-2 * errs["tc_tf32"]
    assert errs["tc_3xtf32"] <= max(20 * errs["fp32"], 1e-6)
