"""Pins for the CPU oracle, independent of the oracle's own code.

Each test checks oracle/ against something the mathematics or a library fixes:
a library correlation, a Kronecker-product matrix power, exact integer
arithmetic, Fourier / sine-mode closed forms, invariants, the adjoint dot test
and finite differences.  Asymmetric random weights are used wherever a flipped
index, a transposed operand or a wrong sign would otherwise cancel out.
"""
import os

import numpy as np
import pytest
import scipy.ndimage as ndi

from paper_2605_07954_gb300 import inputs

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _asym_weights(r, seed=7):
    rng = np.random.default_rng(seed)
    return rng.uniform(-1.0, 1.0, size=(2 * r + 1, 2 * r + 1))


# ---- generator ----------------------------------------------------------------------

def test_splitmix64_published_vector():
    want = []
    with open(os.path.join(GOLDEN, "splitmix64_state0.txt")) as f:
        for line in f:
            line = line.strip()
            if line and not line.startswith("#"):
                want.append(int(line, 16))
    got = [int(v) for v in inputs.splitmix64(0, 0, len(want))]
    assert got == want


def test_uniform_range_and_chunk_independence():
    a = inputs.uniform_f32(0, 0, 5_000_000)
    assert a.dtype == np.float32 and a.min() >= 0.0 and a.max() < 1.0
    b = inputs.uniform_f32(0, 0, 1000, first=4_194_000)
    assert np.array_equal(a[4_194_000:4_195_000], b)
    assert abs(float(a.mean()) - 0.5) < 1e-3


def test_weights_normalised():
    for name in ("box9", "star13", "box49"):
        w = inputs.pattern_weights(name)
        assert abs(float(w.astype(np.float64).sum()) - 1.0) < 1e-6
        shape, r = inputs.PATTERNS[name]
        assert np.all(w[~inputs.footprint(shape, r)] == 0)
        assert np.count_nonzero(w) == {"box9": 9, "star13": 13, "box49": 49}[name]


# ---- forward sweep ------------------------------------------------------------------

@pytest.mark.parametrize("r", [1, 2, 3])
@pytest.mark.parametrize("boundary,mode", [("zero", "constant"), ("periodic", "wrap")])
def test_sweep_matches_scipy_correlate(oracle, r, boundary, mode):
    """T steps equal T applications of scipy.ndimage.correlate (library routine)."""
    W = _asym_weights(r)
    u = np.random.default_rng(1).uniform(size=(13, 21))
    T = 5
    got = oracle.sweep_f64(u, W, T, boundary)
    ref = u.copy()
    for _ in range(T):
        ref = ndi.correlate(ref, W, mode=mode, cval=0.0)
    np.testing.assert_allclose(got, ref, rtol=1e-13, atol=1e-13)


def _shift_matrix(n, d, periodic):
    """S with (S v)[i] = v[i+d] (zero or wrapped outside)."""
    S = np.zeros((n, n))
    for i in range(n):
        k = i + d
        if periodic:
            S[i, k % n] = 1.0
        elif 0 <= k < n:
            S[i, k] = 1.0
    return S


@pytest.mark.parametrize("boundary", ["zero", "periodic"])
@pytest.mark.parametrize("r,ny,nx,T", [(1, 9, 12, 8), (3, 11, 8, 4), (2, 16, 16, 3)])
def test_dense_matrix_power(oracle, boundary, r, ny, nx, T):
    """Brute force: A = sum_w W[dy,dx] kron(S_y^dy, S_x^dx); u_T = A^T u_0."""
    per = boundary == "periodic"
    W = _asym_weights(r, seed=ny + nx)
    A = np.zeros((ny * nx, ny * nx))
    for dy in range(-r, r + 1):
        for dx in range(-r, r + 1):
            A += W[dy + r, dx + r] * np.kron(_shift_matrix(ny, dy, per), _shift_matrix(nx, dx, per))
    u0 = np.random.default_rng(2).uniform(size=(ny, nx))
    ref = (np.linalg.matrix_power(A, T) @ u0.reshape(-1)).reshape(ny, nx)
    got = oracle.sweep_f64(u0, W, T, boundary)
    np.testing.assert_allclose(got, ref, rtol=1e-12, atol=1e-12 * np.abs(ref).max())


def _int_sweep(u, Wi, T, r):
    """Exact integer T-step correlation with zero padding (Python ints)."""
    u = u.astype(object)
    ny, nx = u.shape
    for _ in range(T):
        p = np.zeros((ny + 2 * r, nx + 2 * r), dtype=object)
        p[r:r + ny, r:r + nx] = u
        v = np.zeros((ny, nx), dtype=object)
        for dy in range(-r, r + 1):
            for dx in range(-r, r + 1):
                v = v + int(Wi[dy + r, dx + r]) * p[r + dy:r + dy + ny, r + dx:r + dx + nx]
        u = v
    return u


@pytest.mark.parametrize("r,T", [(1, 10), (3, 5)])
def test_dyadic_exact(oracle, r, T):
    """Weights k/8 and inputs m/256: FP64 is exact; compare bit for bit to integers."""
    rng = np.random.default_rng(3)
    d = 2 * r + 1
    Wi = rng.integers(-2, 3, size=(d, d))  # |sum| <= 2(2r+1)^2 per step keeps < 2^53
    ui = rng.integers(0, 256, size=(10, 14))
    exact = _int_sweep(ui, Wi, T, r)
    scale = 8 ** T * 256
    want = np.array([[float(v) / scale for v in row] for row in exact])
    got = oracle.sweep_f64(ui / 256.0, Wi / 8.0, T)
    assert np.array_equal(got, want)
    # FP32 is exact while |numerator| <= (2 * 9)^T * 255 < 2^24, i.e. T <= 3 at r = 1.
    if r == 1:
        T3 = 3
        exact3 = _int_sweep(ui, Wi, T3, r)
        want3 = np.array([[float(v) / (8 ** T3 * 256) for v in row] for row in exact3])
        got32 = oracle.sweep_f32((ui / 256.0).astype(np.float32), (Wi / 8.0).astype(np.float32), T3)
        assert np.array_equal(got32.astype(np.float64), want3)


def _int_sweep_periodic(u, Wi, T, r):
    """Exact integer T-step correlation with wrapped indices (Python ints, np.roll)."""
    u = u.astype(object)
    for _ in range(T):
        v = np.zeros(u.shape, dtype=object)
        for dy in range(-r, r + 1):
            for dx in range(-r, r + 1):
                # v[i][j] += W[dy][dx] * u[(i+dy) mod ny][(j+dx) mod nx]
                v = v + int(Wi[dy + r, dx + r]) * np.roll(u, (-dy, -dx), axis=(0, 1))
        u = v
    return u


@pytest.mark.parametrize("r", [1, 2])
def test_dyadic_exact_periodic_fp32(oracle, r):
    """The FP32 oracle under the periodic rule: dyadic data, exact integer reference.

    Weights k/8 with |k| <= 2 and inputs m/256, m < 256: after T steps every
    value is an integer over 8^T * 256 of magnitude <= (2 (2r+1)^2)^T * 255,
    which needs at most 24 bits for T = 2 at r = 2 (50^2 * 255 < 2^20) and T = 3
    at r = 1 (18^3 * 255 < 2^21), so FP32 is exact and must agree bit for bit."""
    rng = np.random.default_rng(12 + r)
    d = 2 * r + 1
    Wi = rng.integers(-2, 3, size=(d, d))
    ui = rng.integers(0, 256, size=(9, 13))
    T = 3 if r == 1 else 2
    exact = _int_sweep_periodic(ui, Wi, T, r)
    want = np.array([[float(v) / (8 ** T * 256) for v in row] for row in exact])
    got32 = oracle.sweep_f32((ui / 256.0).astype(np.float32), (Wi / 8.0).astype(np.float32), T, "periodic")
    assert np.array_equal(got32.astype(np.float64), want)
    got64 = oracle.sweep_f64(ui / 256.0, Wi / 8.0, T, "periodic")
    assert np.array_equal(got64, want)


@pytest.mark.parametrize("name", ["heat5", "box9", "star13", "box49", "asym"])
def test_fourier_mode_periodic(oracle, name):
    """u_0 = cos(theta) decays as |lam|^T cos(theta + T arg lam), lam = sum W e^{i phase}."""
    if name == "asym":
        W = _asym_weights(2, seed=11) * 0.2
    else:
        W = inputs.pattern_weights(name).astype(np.float64)
    r = W.shape[0] // 2
    ny, nx, p, q, T = 24, 40, 3, 5, 7
    i, j = np.meshgrid(np.arange(ny), np.arange(nx), indexing="ij")
    theta = 2 * np.pi * (p * i / ny + q * j / nx)
    lam = 0j
    for dy in range(-r, r + 1):
        for dx in range(-r, r + 1):
            lam += W[dy + r, dx + r] * np.exp(2j * np.pi * (p * dy / ny + q * dx / nx))
    want = np.abs(lam) ** T * np.cos(theta + T * np.angle(lam))
    got = oracle.sweep_f64(np.cos(theta), W, T, "periodic")
    np.testing.assert_allclose(got, want, atol=1e-12)


def test_dirichlet_sine_mode_heat(oracle):
    """Zero boundary: sin modes are eigenvectors of the symmetric 5-point star."""
    c = float(np.float32(0.2))
    W = np.array([[0, c, 0], [c, 1 - 4 * c, c], [0, c, 0]])
    ny, nx, p, q, T = 30, 22, 2, 5, 40
    i, j = np.meshgrid(np.arange(ny), np.arange(nx), indexing="ij")
    u0 = np.sin(np.pi * p * (i + 1) / (ny + 1)) * np.sin(np.pi * q * (j + 1) / (nx + 1))
    lam = (1 - 4 * c) + 2 * c * np.cos(np.pi * p / (ny + 1)) + 2 * c * np.cos(np.pi * q / (nx + 1))
    got = oracle.sweep_f64(u0, W, T)
    np.testing.assert_allclose(got, lam ** T * u0, atol=1e-13)


def test_heat_literal_formula(oracle):
    """u + c(N+S+E+W-4u) equals the weight form with centre 1-4c, arms c (FP64)."""
    c = float(np.float32(0.2))
    W = np.array([[0, c, 0], [c, 1 - 4 * c, c], [0, c, 0]])
    u0 = inputs.field(64, 48).astype(np.float64)
    a = oracle.heat_literal_f64(u0, c, 30)
    b = oracle.sweep_f64(u0, W, 30)
    np.testing.assert_allclose(a, b, rtol=1e-13, atol=1e-15)
    # With every weight rounded to 0.2f (the library's Heat weight set) the
    # centre differs from 1-4c by ~1.2e-8: close, not equal.
    b32 = oracle.sweep_f64(u0, inputs.heat_weights(0.2), 30)
    rel = np.linalg.norm(b32 - a) / np.linalg.norm(a)
    assert 0 < rel < 1e-6


def test_worked_example_by_hand(oracle):
    """A unit impulse under the 5-point star with c = 1/8, two steps, worked by hand."""
    c = 0.125
    W = np.array([[0, c, 0], [c, 0.5, c], [0, c, 0]])
    u0 = np.zeros((5, 5)); u0[2, 2] = 1.0
    want = np.zeros((5, 5))
    # step 1: centre 1/2, arms 1/8.  step 2: centre 1/4+4/64, distance-1 arms 2*(1/2*1/8),
    # distance-2 arms 1/64, diagonals 2/64.
    want[2, 2] = 0.25 + 4 / 64
    for (a, b) in ((1, 2), (3, 2), (2, 1), (2, 3)):
        want[a, b] = 2 * 0.5 * 0.125
    for (a, b) in ((0, 2), (4, 2), (2, 0), (2, 4)):
        want[a, b] = 1 / 64
    for (a, b) in ((1, 1), (1, 3), (3, 1), (3, 3)):
        want[a, b] = 2 / 64
    assert np.array_equal(oracle.sweep_f64(u0, W, 2), want)


def test_constant_field(oracle):
    """Sum W = 1 (dyadic): periodic constants are preserved exactly; zero boundary
    preserves them beyond the light cone of the edge (Chebyshev distance r*T)."""
    rng = np.random.default_rng(5)
    Wi = rng.integers(1, 5, size=(7, 7)).astype(np.float64)
    W = Wi / Wi.sum()
    if not np.all((W * 2 ** 12) == np.round(W * 2 ** 12)):
        Wi = np.full((7, 7), 1.0); Wi[3, 3] = 16.0; W = Wi / 64.0
    u0 = np.full((40, 40), 0.75)
    assert np.array_equal(oracle.sweep_f64(u0, W, 4, "periodic"), u0)
    T, r = 3, 3
    got = oracle.sweep_f64(u0, W, T, "zero")
    m = r * T
    assert np.array_equal(got[m:-m, m:-m], u0[m:-m, m:-m])
    assert np.all(got[0, :] < 0.75)


def test_maximum_principle(oracle):
    """W >= 0, sum W <= 1: every output lies in [0, max u_0]."""
    for name in ("box9", "star13", "box49"):
        W = inputs.pattern_weights(name)
        u0 = inputs.field(50, 37)
        out = oracle.sweep_f64(u0, W, 20)
        assert out.min() >= 0.0 and out.max() <= u0.max() * (1 + 1e-12)


def test_light_cone(oracle):
    """The output on a window depends only on inputs within r*T of it."""
    W = _asym_weights(3, seed=9) * 0.3
    u0 = np.random.default_rng(6).uniform(size=(60, 70))
    T, r = 4, 3
    full = oracle.sweep_f64(u0, W, T)
    m = r * T
    y0, y1, x0, x1 = 20, 35, 25, 50
    sub = u0[y0 - m:y1 + m, x0 - m:x1 + m]
    win = oracle.sweep_f64(sub, W, T)[m:-m, m:-m]
    np.testing.assert_allclose(win, full[y0:y1, x0:x1], rtol=0, atol=1e-14)


@pytest.mark.parametrize("name,ny,nx,T,win,chunk", [
    ("box9", 120, 140, 37, 16, 5), ("star13", 200, 90, 23, 8, 7), ("box49", 60, 60, 9, 12, 4),
    ("asym", 80, 75, 11, 10, 3)])
def test_corner_window_is_the_light_cone(oracle, name, ny, nx, T, win, chunk):
    """corner_window_f64 (the shrinking light cone) equals the corner of a
    whole-grid sweep bit for bit, including grids narrower than the cone."""
    W = _asym_weights(2, seed=3) * 0.2 if name == "asym" else inputs.pattern_weights(name)
    u0 = inputs.field(ny, nx)
    full = oracle.sweep_f64(u0, W, T)[:win, :win]
    assert np.array_equal(oracle.corner_window_f64(u0, W, T, win, chunk), full)


def test_linearity_and_transpose(oracle):
    W = _asym_weights(2, seed=4) * 0.4
    rng = np.random.default_rng(8)
    x, y = rng.uniform(size=(2, 17, 23))
    a, b = 0.3, -1.7
    lhs = oracle.sweep_f64(a * x + b * y, W, 6)
    rhs = a * oracle.sweep_f64(x, W, 6) + b * oracle.sweep_f64(y, W, 6)
    np.testing.assert_allclose(lhs, rhs, rtol=1e-12, atol=1e-12)
    # transposing grid and weights transposes the output
    np.testing.assert_allclose(oracle.sweep_f64(x.T, W.T, 6), oracle.sweep_f64(x, W, 6).T,
                               rtol=1e-13, atol=1e-14)


def test_fp32_oracle_close_to_fp64(oracle):
    for name in ("heat5", "box9", "star13"):
        W = inputs.pattern_weights(name)
        u0 = inputs.field(96, 80)
        a = oracle.sweep_f64(u0, W, 100)
        b = oracle.sweep_f32(u0, W, 100).astype(np.float64)
        rel = np.linalg.norm(a - b) / np.linalg.norm(a)
        assert rel < 1e-6


# ---- adjoint ------------------------------------------------------------------------

@pytest.mark.parametrize("boundary", ["zero", "periodic"])
@pytest.mark.parametrize("r", [1, 3])
def test_adjoint_dot_test(oracle, boundary, r):
    """<A^T x, y> = <x, (A^T)' y>: the reverse sweep is the transpose of the forward."""
    W = _asym_weights(r, seed=12) * 0.3
    rng = np.random.default_rng(13)
    x = rng.normal(size=(19, 26))
    y = rng.normal(size=(19, 26))
    T = 9
    Ax = oracle.sweep_f64(x, W, T, boundary)
    ATy, _ = oracle.adjoint_f64(np.zeros_like(x), W, T, y, boundary)
    lhs, rhs = np.vdot(Ax, y), np.vdot(x, ATy)
    assert abs(lhs - rhs) <= 1e-13 * max(abs(lhs), 1.0)


def _loss(oracle, u0, W, T, target, boundary="zero"):
    uT = oracle.sweep_f64(u0, W, T, boundary)
    return 0.5 * float(np.sum((uT - target) ** 2))


@pytest.mark.parametrize("boundary", ["zero", "periodic"])
def test_adjoint_gradients_finite_differences(oracle, boundary):
    """dL/dW by central FD (h=1e-6) and dL/du0 along a direction (exact for a quadratic)."""
    ny = nx = 64
    T = 32
    u0 = inputs.field(ny, nx).astype(np.float64)
    target = inputs.field(ny, nx, stream=inputs.STREAM_TARGET).astype(np.float64)
    W = inputs.heat_weights(0.2).astype(np.float64)
    uT = oracle.sweep_f64(u0, W, T, boundary)
    g_u0, g_W = oracle.adjoint_f64(u0, W, T, uT - target, boundary)
    h = 1e-6
    for (a, b) in ((1, 1), (0, 1), (1, 0), (1, 2), (2, 1), (0, 0)):
        Wp, Wm = W.copy(), W.copy()
        Wp[a, b] += h
        Wm[a, b] -= h
        fd = (_loss(oracle, u0, Wp, T, target, boundary) -
              _loss(oracle, u0, Wm, T, target, boundary)) / (2 * h)
        assert abs(fd - g_W[a, b]) <= 1e-7 * max(1.0, abs(g_W[a, b])), (a, b, fd, g_W[a, b])
    v = np.random.default_rng(14).normal(size=u0.shape)
    hh = 1e-3
    fd = (_loss(oracle, u0 + hh * v, W, T, target, boundary) -
          _loss(oracle, u0 - hh * v, W, T, target, boundary)) / (2 * hh)
    an = float(np.vdot(g_u0, v))
    assert abs(fd - an) <= 1e-8 * max(1.0, abs(an))


def test_adjoint_weight_grad_single_step_brute(oracle):
    """T=1, tiny grid: dL/dW by differentiating the dense matrix form entry by entry."""
    r = 1
    W = _asym_weights(r, seed=21)
    rng = np.random.default_rng(22)
    u0 = rng.normal(size=(5, 6))
    g = rng.normal(size=(5, 6))
    _, gW = oracle.adjoint_f64(u0, W, 1, g)
    for dy in range(-r, r + 1):
        for dx in range(-r, r + 1):
            # dA/dW[dy,dx] = kron(S_y^dy, S_x^dx); dL/dW = g . (dA/dW u0)
            B = np.kron(_shift_matrix(5, dy, False), _shift_matrix(6, dx, False))
            want = float(g.reshape(-1) @ (B @ u0.reshape(-1)))
            assert abs(gW[dy + r, dx + r] - want) < 1e-12
