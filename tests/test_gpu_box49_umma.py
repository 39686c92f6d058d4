"""GPU tests of the tcgen05 engine for the 7x7 box (TMA-staged operands,
tensor-memory accumulators): engine selection, exactness on dyadic data, and
agreement with the FP64 oracle and with the warp-MMA engine on random data.

With inputs in {0, 1} and weights in {0, 1/8}, one step gives multiples of 1/8
up to 49/8 (exact in BF16 and TF32) and two steps multiples of 1/64 up to
2401/64 (exact in FP32).  Every partial sum is then exact, so the result is
the oracle's FP64 value, rounded once to the storage type: a wrong Toeplitz
band, plane index, descriptor offset, TMEM column or tile coordinate fails it.
The shapes span several tiles with ragged right and bottom edges, and the
largest one gives each persistent CTA enough tiles to cycle its staging ring
and both accumulators several times.
"""
import numpy as np
import pytest

from paper_2605_07954_gb300 import inputs
from _util import rel_l2

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

TDT = {"f32": "float32", "bf16": "bfloat16"}
# N = 16, 32, 64: one weight row per MMA; 96, 128: three or four rows per MMA
NTS = [("tc_bf16", "bf16", 16), ("tc_bf16", "bf16", 32), ("tc_bf16", "bf16", 64),
       ("tc_bf16", "bf16", 96), ("tc_bf16", "bf16", 128),
       ("tc_tf32", "f32", 16), ("tc_tf32", "f32", 32), ("tc_tf32", "f32", 96), ("tc_tf32", "f32", 128)]


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2605_07954_gb300 import build
    build.build()


def _dyadic(shape, seed):
    rng = np.random.default_rng(seed)
    W = np.where(rng.random((7, 7)) < 0.7, 0.125, 0.0).astype(np.float32)
    u0 = (rng.random(shape) < 0.5).astype(np.float32)
    return u0, W


def _plan(shape, W, compute, dtype, kernel="tc", mma_n=0, boundary="zero"):
    from paper_2605_07954_gb300 import Plan
    return Plan(shape[0], shape[1], W, dtype=dtype, boundary=boundary, compute=compute,
                kernel=kernel, mma_n=mma_n)


def _to_dev(u0, dtype):
    return torch.from_numpy(np.ascontiguousarray(u0, dtype=np.float32)).to(
        "cuda", getattr(torch, TDT[dtype]))


def _round_like(ref, dtype):
    t = torch.from_numpy(ref.astype(np.float32))
    if dtype == "bf16":
        t = t.bfloat16().float()
    return t.numpy().astype(np.float64)


def test_engine_selection():
    from paper_2605_07954_gb300 import StencilError
    W = inputs.pattern_weights("box49")
    p = _plan((300, 392), W, "tc_bf16", "bf16", kernel="tc_umma")
    i = p.info()
    assert i["kernel"] == 5 and i["mma_n"] in (16, 32, 64, 96, 128) and i["threads"] == 192
    assert 1 <= i["ctas"] <= torch.cuda.get_device_properties(0).multi_processor_count
    p.close()
    p = _plan((300, 392), W, "tc_bf16", "bf16")  # default: the faster engine as measured
    assert p.info()["kernel"] in (3, 5)
    p.close()
    # the warp-MMA engine on request, for periodic grids, FP32 storage with BF16
    # MMAs, short grids and rows that are not a multiple of 16 bytes
    for shape, compute, dtype, kernel, boundary in [
            ((300, 392), "tc_bf16", "bf16", "tc_warp", "zero"),
            ((300, 392), "tc_bf16", "bf16", "tc", "periodic"),
            ((300, 392), "tc_bf16", "f32", "tc", "zero"),
            ((133, 392), "tc_bf16", "bf16", "tc", "zero"),
            ((300, 120), "tc_bf16", "bf16", "tc", "zero"),
            ((300, 390), "tc_bf16", "bf16", "tc", "zero"),
            ((300, 390), "tc_tf32", "f32", "tc", "zero")]:
        p = _plan(shape, W, compute, dtype, kernel=kernel, boundary=boundary)
        i = p.info()
        assert i["kernel"] == 3 and i["mma_n"] == 0, (shape, compute, dtype, kernel, boundary)
        p.close()
        if kernel == "tc":
            with pytest.raises(StencilError, match="UNSUPPORTED"):
                _plan(shape, W, compute, dtype, kernel="tc_umma", boundary=boundary)
    with pytest.raises(StencilError, match="UNSUPPORTED"):
        _plan((300, 392), W, "tc_tf32", "f32", kernel="tc_umma", mma_n=64)
    p = _plan((300, 392), W, "tc_tf32", "f32", kernel="tc", mma_n=64)  # not instantiated: warp MMAs
    assert p.info()["kernel"] == 3
    p.close()
    for nt, rows in ((64, 128), (96, 126), (128, 125)):
        p = _plan((300, 392), W, "tc_bf16", "bf16", kernel="tc_umma", mma_n=nt)
        assert p.info()["tile_rows"] == rows
        p.close()


@pytest.mark.parametrize("compute,dtype,nt", NTS)
@pytest.mark.parametrize("shape", [(134, 136), (300, 392), (517, 1288), (4100, 4104)])
def test_dyadic_exact(oracle, compute, dtype, nt, shape):
    u0, W = _dyadic(shape, shape[0] * 7 + shape[1])
    p = _plan(shape, W, compute, dtype, kernel="tc_umma", mma_n=nt)
    assert p.info()["mma_n"] == nt
    x = _to_dev(u0, dtype)
    # TF32: the first step of a run is the warp-MMA engine's, the second tcgen05's
    for T in ((1, 2) if dtype == "bf16" else (2,)):
        got = p.run(x, T).float().cpu().numpy().astype(np.float64)
        ref = _round_like(oracle.sweep_f64(u0, W, T), dtype)
        bad = np.argwhere(got != ref)
        assert bad.size == 0, f"T={T}: {len(bad)} mismatches, first at {bad[:4].tolist()}"
    torch.cuda.synchronize()
    p.status()
    p.close()


@pytest.mark.parametrize("compute,dtype,nt", NTS)
def test_random_field_vs_oracle_and_warp_engine(oracle, compute, dtype, nt):
    """Box-49 weights, a random field, 12 steps: the tcgen05 engine's error
    against FP64 is that of the warp-MMA engine (same operand rounding; only
    the FP32 accumulation order differs)."""
    shape, T = (300, 520), 12
    W = inputs.pattern_weights("box49")
    u0 = inputs.field(*shape)
    ref = oracle.sweep_f64(u0, W, T)
    x = _to_dev(u0, dtype)
    pu = _plan(shape, W, compute, dtype, kernel="tc_umma", mma_n=nt)
    pw = _plan(shape, W, compute, dtype, kernel="tc_warp")
    gu = pu.run(x, T).float().cpu().numpy()
    gw = pw.run(x, T).float().cpu().numpy()
    torch.cuda.synchronize()
    pu.status()
    eu, ew = rel_l2(gu, ref), rel_l2(gw, ref)
    print(f"{compute}/{dtype} N={nt}: tcgen05 relL2={eu:.3e}, warp MMA relL2={ew:.3e}, "
          f"between engines {rel_l2(gu, gw):.3e}")
    assert eu <= 1.25 * ew + 1e-7
    assert rel_l2(gu, gw) <= (2e-3 if dtype == "bf16" else 2e-4)
    pu.close()
    pw.close()


@pytest.mark.parametrize("compute,dtype", [("tc_bf16", "bf16"), ("tc_tf32", "f32")])
def test_in_place_and_odd_launch_counts(oracle, compute, dtype):
    shape = (260, 264)
    u0, W = _dyadic(shape, 5)
    p = _plan(shape, W, compute, dtype, kernel="tc_umma")
    x = _to_dev(u0, dtype)
    y = p.run(x, 2)
    x2 = x.clone()
    p.run(x2, 2, out=x2)  # in == out
    torch.cuda.synchronize()
    assert torch.equal(x2, y)
    assert np.array_equal(y.float().cpu().numpy().astype(np.float64),
                          _round_like(oracle.sweep_f64(u0, W, 2), dtype))
    p.status()
    p.close()


@pytest.mark.parametrize("compute,dtype", [("tc_bf16", "bf16"), ("tc_tf32", "f32")])
def test_autotune_picks_an_engine_and_stays_exact(oracle, compute, dtype):
    """Autotuning times the warp-MMA engine and each tcgen05 width on the first
    run; whichever it keeps, dyadic two-step results stay exact."""
    shape = (1030, 1160)
    u0, W = _dyadic(shape, 11)
    from paper_2605_07954_gb300 import Plan
    p = Plan(shape[0], shape[1], W, dtype=dtype, compute=compute, autotune=True)
    x = _to_dev(u0, dtype)
    got = p.run(x, 2).float().cpu().numpy().astype(np.float64)
    i = p.info()
    print(f"{compute}/{dtype} autotuned: kernel={i['kernel']} mma_n={i['mma_n']}")
    assert (i["kernel"], i["mma_n"] > 0) in ((3, False), (5, True))
    assert np.array_equal(got, _round_like(oracle.sweep_f64(u0, W, 2), dtype))
    p.status()
    p.close()


@pytest.mark.parametrize("nt", [64, 96])
def test_expired_wait_reports_timeout_and_device_recovers(oracle, nt):
    """Failure detection without a fault: with the test hook, CTA 0 never
    signals its first accumulator, so its epilogue wait runs out after
    timeout_ms; the kernel drains its own copies and MMAs, frees its tensor
    memory and returns, the plan reports TIMEOUT, and the device then runs a
    normal plan with exact results.  N = 64: one weight row per MMA; N = 96:
    row groups, whose MMA warp is then blocked on a later accumulator."""
    from paper_2605_07954_gb300 import Plan, StencilError
    shape = (300, 392)
    u0, W = _dyadic(shape, 17)
    x = _to_dev(u0, "bf16")
    bad = Plan(shape[0], shape[1], W, dtype="bf16", compute="tc_bf16", kernel="tc_umma",
               timeout_ms=100, debug_withhold=1, mma_n=nt)
    bad.run(x, 1)
    torch.cuda.synchronize()
    with pytest.raises(StencilError, match="TIMEOUT"):
        bad.status()
    bad.close()
    good = _plan(shape, W, "tc_bf16", "bf16", kernel="tc_umma", mma_n=nt)
    got = good.run(x, 2).float().cpu().numpy().astype(np.float64)
    torch.cuda.synchronize()
    good.status()
    assert np.array_equal(got, _round_like(oracle.sweep_f64(u0, W, 2), "bf16"))
    good.close()
