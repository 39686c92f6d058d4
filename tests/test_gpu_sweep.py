"""GPU parity of the CUDA sweep (through the C ABI) against the CPU oracle.

Every comparison runs both sides on the same seeded inputs.  Small grids
span several CTA tiles and ragged tails in both directions; the full-size
workloads (8192^2 Box-9 / Star-13 with the benchmark's launch configuration)
are checked on sampled windows through the light cone, and through closed
forms and invariants that hold at any size.
"""
import numpy as np
import pytest

from paper_2605_07954_gb300 import inputs
from _util import fp32_elem_tol, fp32_tol, rel_l2, rel_linf

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2605_07954_gb300 import build
    build.build()


def _plan(*a, **k):
    from paper_2605_07954_gb300 import Plan
    return Plan(*a, **k)


def _gpu_run(u0, W, T, boundary="zero", dtype="f32", **opts):
    tdt = {"f32": torch.float32, "bf16": torch.bfloat16, "f16": torch.float16}[dtype]
    x = torch.from_numpy(np.ascontiguousarray(u0, dtype=np.float32)).to("cuda", tdt)
    p = _plan(u0.shape[0], u0.shape[1], W, dtype=dtype, boundary=boundary, **opts)
    y = p.run(x, T)
    torch.cuda.synchronize()
    p.status()
    info = p.info()
    p.close()
    return y.float().cpu().numpy().astype(np.float64), info


def _taps(W):
    return int(np.count_nonzero(W))


PATTERNS = ["heat5", "box9", "star13", "box49"]


@pytest.mark.parametrize("name", PATTERNS)
@pytest.mark.parametrize("boundary", ["zero", "periodic"])
@pytest.mark.parametrize("shape", [(67, 203), (130, 516)])
def test_parity_small_auto(oracle, name, boundary, shape):
    W = inputs.pattern_weights(name)
    u0 = inputs.field(*shape)
    T = 23
    ref = oracle.sweep_f64(u0, W, T, boundary)
    got, info = _gpu_run(u0, W, T, boundary)
    assert rel_l2(got, ref) <= fp32_tol(T), info
    assert rel_linf(got, ref) <= fp32_elem_tol(T, _taps(W)), info


# Depths the streaming kernel is instantiated for, per (radius, shape).
DEPTHS = {(1, "box"): [1, 2, 3, 4, 6, 8], (1, "star"): [1, 2, 3, 4, 6, 8],
          (3, "box"): [1, 2], (3, "star"): [1, 2, 3, 4]}


@pytest.mark.parametrize("name", PATTERNS)
@pytest.mark.parametrize("k", [1, 2, 3, 4, 6, 8])
@pytest.mark.parametrize("threads,tile_rows", [(32, 7), (64, 33)])
def test_parity_depths_small_tiles(oracle, name, k, threads, tile_rows):
    """Forced small CTAs and odd tile heights: many tiles, ragged last strip/tile.
    T = 2k + 5 also exercises the remainder launches (greedy split of T mod k)."""
    shape, r = inputs.PATTERNS[name]
    if k not in DEPTHS[(r, shape)] or 4 * threads - 2 * ((r * k + 3) // 4 * 4) < 4:
        pytest.skip("configuration outside the instantiated range")
    W = inputs.pattern_weights(name)
    u0 = inputs.field(45, 150 if threads == 32 else 601)
    T = 2 * k + 5
    ref = oracle.sweep_f64(u0, W, T)
    got, info = _gpu_run(u0, W, T, tb_depth=k, threads=threads, tile_rows=tile_rows)
    assert info["tb_depth"] == k and info["ctas"] > 4
    assert rel_l2(got, ref) <= fp32_tol(T), info
    assert rel_linf(got, ref) <= fp32_elem_tol(T, _taps(W)), info


@pytest.mark.parametrize("name", ["heat5", "box9", "star13"])
def test_parity_asymmetric_weights(oracle, name):
    """Signed, asymmetric weights catch a flipped or transposed offset."""
    shape, r = inputs.PATTERNS[name]
    rng = np.random.default_rng(17)
    W = (rng.uniform(-1, 1, size=(2 * r + 1, 2 * r + 1)) * inputs.footprint(shape, r))
    W = (W / np.abs(W).sum()).astype(np.float32)
    u0 = inputs.field(77, 260)
    for boundary in ("zero", "periodic"):
        ref = oracle.sweep_f64(u0, W, 9, boundary)
        got, info = _gpu_run(u0, W, 9, boundary)
        assert rel_l2(got, ref) <= fp32_tol(9), (boundary, info)


@pytest.mark.parametrize("kernel", ["naive", "stream"])
@pytest.mark.parametrize("r,T", [(1, 5), (3, 2)])
def test_dyadic_bitwise(oracle, kernel, r, T):
    """Weights in {0, 1/8} and inputs m/256: after T steps every value is
    n / 2^(3T+8) with 0 <= n <= (2r+1)^(2T) * 255 < 2^24, so every FP32
    product and partial sum is exact and the GPU result equals the oracle
    bit for bit."""
    rng = np.random.default_rng(5)
    d = 2 * r + 1
    assert d ** (2 * T) * 255 < 2 ** 24
    W = (rng.integers(0, 2, size=(d, d)) / 8.0).astype(np.float32)
    u0 = (rng.integers(0, 256, size=(61, 133)) / 256.0).astype(np.float32)
    ref = oracle.sweep_f64(u0, W, T)
    got, _ = _gpu_run(u0, W, T, kernel=kernel, tb_depth=(0 if kernel == "naive" else 2))
    assert np.array_equal(got, ref)


@pytest.mark.parametrize("shape", [(1, 1), (1, 37), (29, 1), (2, 3), (5, 6)])
@pytest.mark.parametrize("boundary", ["zero", "periodic"])
def test_degenerate_shapes(oracle, shape, boundary):
    """Grids smaller than the stencil and the halo (periodic wraps several times)."""
    for name in ("heat5", "star13", "box49"):
        W = inputs.pattern_weights(name)
        u0 = inputs.field(*shape)
        ref = oracle.sweep_f64(u0, W, 6, boundary)
        got, info = _gpu_run(u0, W, 6, boundary)
        assert rel_l2(got, ref) <= fp32_tol(6), (name, info)


def test_unaligned_width_scalar_path(oracle):
    """nx not a multiple of 4 takes the element-wise load/store path."""
    W = inputs.pattern_weights("box9")
    for nx in (201, 202, 203):
        u0 = inputs.field(40, nx)
        ref = oracle.sweep_f64(u0, W, 17)
        got, _ = _gpu_run(u0, W, 17)
        assert rel_l2(got, ref) <= fp32_tol(17)


def test_T0_aliasing_and_launch_counts(oracle):
    from paper_2605_07954_gb300 import Plan
    W = inputs.pattern_weights("box9")
    u0 = inputs.field(50, 64)
    x = torch.from_numpy(u0).cuda()
    for k in (1, 3, 8):
        p = Plan(50, 64, W, tb_depth=k)
        assert p.launches(0) == 0 and p.launches(1) == 1
        assert p.launches(17) == -(-17 // k)
        y = p.run(x, 0)
        assert torch.equal(y, x)
        for T in (1, 2, 5, 16, 17):
            ref = oracle.sweep_f64(u0, W, T)
            z = x.clone()
            p.run(z, T, out=z)   # in == out
            torch.cuda.synchronize()
            assert rel_l2(z.cpu().numpy(), ref) <= fp32_tol(T), (k, T)
            # the unaliased run gives the same bits
            y = p.run(x, T)
            torch.cuda.synchronize()
            assert torch.equal(y, z), (k, T)
        p.status()
        p.close()
    assert torch.equal(x, torch.from_numpy(u0).cuda())  # the input was never written


def test_run_host_matches_device_path():
    W = inputs.pattern_weights("star13")
    u0 = inputs.field(300, 412)
    p = _plan(300, 412, W)
    a = p.run_host(u0, 11)
    b = p.run(torch.from_numpy(u0).cuda(), 11).cpu().numpy()
    assert np.array_equal(a, b)
    p.close()


@pytest.mark.parametrize("dtype,gate", [("bf16", 1e-2), ("f16", 2e-3)])
@pytest.mark.parametrize("name", ["box9", "star13"])
def test_reduced_precision_storage(oracle, dtype, gate, name):
    """BF16/FP16 storage with FP32 arithmetic vs the FP64 oracle on the FP32 field."""
    W = inputs.pattern_weights(name)
    u0 = inputs.field(256, 384)
    T = 50
    ref = oracle.sweep_f64(u0, W, T)
    got, _ = _gpu_run(u0, W, T, dtype=dtype)
    e = rel_l2(got, ref)
    print(f"{dtype} {name} relL2={e:.3e}")
    assert e <= gate


# ---- full-size workloads -------------------------------------------------------------

def _window_check(oracle, u0, got, W, T, y0, y1, x0, x1):
    """Exact FP64 values on [y0,y1) x [x0,x1) from the light cone of the window."""
    r = W.shape[0] // 2
    m = r * T
    ny, nx = u0.shape
    a0, a1 = max(0, y0 - m), min(ny, y1 + m)
    b0, b1 = max(0, x0 - m), min(nx, x1 + m)
    sub = oracle.sweep_f64(u0[a0:a1, b0:b1], W, T)
    ref = sub[y0 - a0:y1 - a0, x0 - b0:x1 - b0]
    g = got[y0:y1, x0:x1]
    return rel_l2(g, ref), rel_linf(g, ref)


def _bench_plan_run(name, n, T, boundary="zero", u0=None, W=None):
    W = inputs.pattern_weights(name) if W is None else W
    u0 = inputs.field(n, n) if u0 is None else u0
    got, info = _gpu_run(u0, W, T, boundary)
    return u0, W, got, info


@pytest.mark.parametrize("name", ["box9", "star13"])
def test_fullsize_8192_windows(oracle, name):
    """8192^2, the benchmark's plan; a few launches, windows at corners, edges, centre."""
    n = 8192
    shape, r = inputs.PATTERNS[name]
    from paper_2605_07954_gb300 import Plan
    k = Plan(64, 64, inputs.pattern_weights(name), kernel="stream").info()["tb_depth"]
    T = 3 * k + 1
    u0, W, got, info = _bench_plan_run(name, n, T)
    b = 48
    for (y0, x0) in ((0, 0), (0, n - b), (n - b, 0), (n - b, n - b), (n // 2 - 7, n // 3 + 5),
                     (info["tile_rows"] - b // 2, info["tile_cols"] - b // 2)):
        l2, linf = _window_check(oracle, u0, got, W, T, y0, y0 + b, x0, x0 + b)
        assert l2 <= fp32_tol(T) and linf <= fp32_elem_tol(T, _taps(W)), (y0, x0, l2, linf, info)


def test_fullsize_box9_T1000_corner(oracle):
    """8192^2 Box-9, 1000 steps (the benchmark workload): the corner window
    against its exact light cone in FP64, plus the maximum principle."""
    u0, W, got, info = _bench_plan_run("box9", 8192, 1000)
    l2, linf = _window_check(oracle, u0, got, W, 1000, 0, 40, 0, 40)
    print(f"box9 T=1000 corner relL2={l2:.3e} relLinf={linf:.3e}")
    assert l2 <= fp32_tol(1000)
    assert got.min() >= 0.0 and got.max() <= u0.max() * (1 + 1e-5)


@pytest.mark.parametrize("name", ["box9", "star13"])
def test_fullsize_T1000_fourier_periodic(name):
    """8192^2 periodic, 1000 steps: a Fourier mode decays by |lam|^T, phase T*arg(lam)."""
    n, T = 8192, 1000
    W = inputs.pattern_weights(name).astype(np.float64)
    r = W.shape[0] // 2
    p, q = 3, 5
    i = np.arange(n)[:, None]
    j = np.arange(n)[None, :]
    theta = 2 * np.pi * (p * i / n + q * j / n)
    lam = sum(W[dy + r, dx + r] * np.exp(2j * np.pi * (p * dy + q * dx) / n)
              for dy in range(-r, r + 1) for dx in range(-r, r + 1))
    u0 = np.cos(theta).astype(np.float32)
    _, _, got, info = _bench_plan_run(name, n, T, "periodic", u0=u0, W=W.astype(np.float32))
    want = np.abs(lam) ** T * np.cos(theta + T * np.angle(lam))
    e = rel_l2(got, want)
    print(f"{name} periodic Fourier T=1000 relL2={e:.3e}")
    assert e <= 1e-5


def test_fullsize_T1000_sine_mode_zero_boundary():
    """8192^2 zero boundary, 1000 steps, axis-symmetric 3x3 weights (the Box-9
    kernel): sine modes are exact eigenvectors."""
    n, T = 8192, 1000
    W = np.array([[0.05, 0.15, 0.05], [0.15, 0.2, 0.15], [0.05, 0.15, 0.05]], dtype=np.float32)
    Wd = W.astype(np.float64)
    p, q = 2, 3
    i = np.arange(n)[:, None]
    j = np.arange(n)[None, :]
    sy = np.sin(np.pi * p * (i + 1) / (n + 1))
    sx = np.sin(np.pi * q * (j + 1) / (n + 1))
    cy, cx = np.cos(np.pi * p / (n + 1)), np.cos(np.pi * q / (n + 1))
    ey = {-1: cy, 0: 1.0, 1: cy}
    ex = {-1: cx, 0: 1.0, 1: cx}
    lam = sum(Wd[dy + 1, dx + 1] * ey[dy] * ex[dx] for dy in (-1, 0, 1) for dx in (-1, 0, 1))
    u0 = (sy * sx).astype(np.float32)
    _, _, got, info = _bench_plan_run("box9", n, T, u0=u0, W=W)
    want = lam ** T * (sy * sx)
    e = rel_l2(got, want)
    print(f"box9 sine-mode T=1000 relL2={e:.3e}")
    assert e <= 1e-5


def test_moderate_T1000_full_oracle(oracle):
    """1024^2, 1000 steps, whole grid against the FP64 oracle (the FP32 gate)."""
    for name in ("box9", "star13"):
        W = inputs.pattern_weights(name)
        u0 = inputs.field(512, 512) if name == "star13" else inputs.field(1024, 1024)
        T = 1000 if name == "box9" else 300
        ref = oracle.sweep_f64(u0, W, T)
        got, info = _gpu_run(u0, W, T)
        e2, ei = rel_l2(got, ref), rel_linf(got, ref)
        print(f"{name} T={T} relL2={e2:.3e} relLinf={ei:.3e}")
        assert e2 <= fp32_tol(T) and ei <= fp32_elem_tol(T, _taps(W))


@pytest.mark.parametrize("name", ["box9", "star13"])
def test_autotune_first_run(oracle, name):
    """opt.autotune times the candidate depths/CTA sizes on the first run and
    keeps one of them; the result still matches the oracle."""
    W = inputs.pattern_weights(name)
    u0 = inputs.field(300, 520)
    ref = oracle.sweep_f64(u0, W, 40)
    p = _plan(300, 520, W, autotune=True)
    x = torch.from_numpy(u0).cuda()
    y = p.run(x, 40)
    torch.cuda.synchronize()
    info = p.info()
    shape, r = inputs.PATTERNS[name]
    if info["kernel"] == 6:  # the cluster-resident kernel won: one launch per run
        assert info["tb_depth"] == 0 and 1 <= info["ctas"] <= 16
    else:
        assert info["tb_depth"] in DEPTHS[(r, shape)]
        assert info["threads"] % 32 == 0 and 32 <= info["threads"] <= 256
    assert rel_l2(y.cpu().numpy(), ref) <= fp32_tol(40)
    assert torch.equal(x, torch.from_numpy(u0).cuda())
    p.close()


@pytest.mark.parametrize("name", PATTERNS)
@pytest.mark.parametrize("boundary,shape", [("zero", (130, 257)), ("zero", (96, 256)),
                                            ("periodic", (96, 256)), ("periodic", (131, 260))])
def test_depth_does_not_change_bits(name, boundary, shape):
    """Every step is the same per-point arithmetic whatever the temporal-blocking
    depth or tiling, so all depths give the same bits.  (Periodic grids whose
    width is not a multiple of 4 are the exception: a wrapped column's image sits
    at another position of a thread's 4-column chunk and is summed in another
    order, so results there agree only to rounding; see test_periodic_unaligned_depths.)"""
    from paper_2605_07954_gb300 import Plan
    shp, r = inputs.PATTERNS[name]
    W = inputs.pattern_weights(name)
    x = torch.from_numpy(inputs.field(*shape)).cuda()
    outs = {}
    for k in DEPTHS[(r, shp)]:
        p = Plan(shape[0], shape[1], W, boundary=boundary, tb_depth=k)
        outs[k] = p.run(x, 12)
        torch.cuda.synchronize()
        p.close()
    ks = sorted(outs)
    bad = [k for k in ks if not torch.equal(outs[k], outs[ks[0]])]
    assert not bad, (name, boundary, shape, bad)


@pytest.mark.parametrize("name", ["heat5", "box9", "star13"])
@pytest.mark.parametrize("boundary", ["zero", "periodic"])
def test_tiling_does_not_change_bits(oracle, name, boundary):
    """CTA size and tile height change which CTA runs which tile (edge tiles are
    numbered first once there are at least 3 strips and 3 tile rows) and which
    tiles take the checked edge path, never the per-point arithmetic: every
    tiling gives the same bits, and they match the FP64 oracle."""
    from paper_2605_07954_gb300 import Plan
    W = inputs.pattern_weights(name)
    u0 = inputs.field(200, 704)
    x = torch.from_numpy(u0).cuda()
    T = 13
    outs = {}
    for threads, tile_rows in ((64, 20), (64, 0), (128, 33), (256, 0), (32, 9)):
        p = Plan(200, 704, W, boundary=boundary, kernel="stream", threads=threads, tile_rows=tile_rows)
        outs[(threads, tile_rows)] = (p.run(x, T), p.info())
        torch.cuda.synchronize()
        p.close()
    base_key = (64, 20)
    base, info = outs[base_key]
    assert info["ctas"] >= 9, info
    for key, (y, _) in outs.items():
        assert torch.equal(y, base), (name, boundary, key)
    ref = oracle.sweep_f64(u0, W, T, boundary)
    got = base.cpu().numpy()
    assert rel_l2(got, ref) <= fp32_tol(T) and rel_linf(got, ref) <= fp32_elem_tol(T, _taps(W))


@pytest.mark.parametrize("name", PATTERNS)
def test_periodic_unaligned_depths(oracle, name):
    """Periodic, width not a multiple of 4: every depth matches the oracle."""
    from paper_2605_07954_gb300 import Plan
    shp, r = inputs.PATTERNS[name]
    W = inputs.pattern_weights(name)
    u0 = inputs.field(130, 257)
    ref = oracle.sweep_f64(u0, W, 12, "periodic")
    x = torch.from_numpy(u0).cuda()
    for k in DEPTHS[(r, shp)]:
        p = Plan(130, 257, W, boundary="periodic", tb_depth=k)
        got = p.run(x, 12).cpu().numpy()
        p.close()
        assert rel_linf(got, ref) <= fp32_elem_tol(12, _taps(W)), k


def test_run_host_async_on_two_streams(oracle):
    """Two plans, each on its own stream, host buffers in and out without a
    synchronisation per call (stencil_run_host_async): both results match the
    FP64 oracle once the streams are done."""
    from paper_2605_07954_gb300 import Plan
    outs, refs = [], []
    streams = [torch.cuda.Stream(), torch.cuda.Stream()]
    plans = []
    for name, s in zip(("box9", "star13"), streams):
        W = inputs.pattern_weights(name)
        u0 = inputs.field(300, 400)
        hin = torch.from_numpy(u0).pin_memory()
        hout = torch.empty_like(hin).pin_memory()
        p = Plan(300, 400, W)
        p.run_host_async(hin.numpy(), 25, hout.numpy(), s.cuda_stream)
        plans.append((p, hin))
        outs.append(hout)
        refs.append(oracle.sweep_f64(u0, W, 25))
    for s in streams:
        s.synchronize()
    for (p, _), o, r in zip(plans, outs, refs):
        p.status()
        assert rel_l2(o.numpy(), r) <= fp32_tol(25)
        p.close()
