"""Parity at the benchmark's full sizes and launch configuration.

* The headline (Box-2D9P and Star-2D13P, 8192^2, 1000 steps, autotuned as
  bench.py runs it) and the Box-49 16384^2 x 200 variants against the FP64
  oracle windows stored by tests/golden/make_bench_windows.py.
* The weak-scaling sizes (16384^2, 32768^2 and Star-2D5P at 44800^2, which is
  2.0e9 points, near the int32 element range) on light-cone windows at the
  top-left corner, the bottom-right corner and the middle, T <= 8, against the
  FP64 oracle run on each window's light cone.
"""
import json
import os

import numpy as np
import pytest

from paper_2605_07954_gb300 import inputs
from _util import fp32_tol, rel_l2, rel_linf

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "bench_windows.json")


@pytest.fixture(scope="module")
def windows():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2605_07954_gb300 import build
    build.build()
    with open(GOLDEN) as f:
        return json.load(f)["workloads"]


def _plan(n, W, **kw):
    from paper_2605_07954_gb300 import Plan
    return Plan(n, n, W, **kw)


@pytest.mark.parametrize("name", ["box9", "star13"])
def test_headline_window(windows, name):
    rec = windows[f"{name}_8192_T1000"]
    W = inputs.pattern_weights(name)
    x = torch.from_numpy(inputs.field(8192, 8192)).cuda()
    p = _plan(8192, W, autotune=True)
    y = p.run(x, 1000)
    torch.cuda.synchronize()
    p.status()
    ref = np.asarray(rec["window"])
    got = y[:16, :16].cpu().numpy()
    assert rel_l2(got, ref) <= fp32_tol(1000), (name, p.info())
    # element-wise: the FP32 rounding of 1000 contracting steps of <= 13 taps
    assert rel_linf(got, ref) <= 1000 * 13 * 2.0 ** -24
    # maximum principle over the whole grid (non-negative weights summing to 1)
    assert float(y.min()) >= 0.0 and float(y.max()) <= float(x.max()) * (1 + 1e-6)
    p.close()


@pytest.mark.parametrize("dtype,compute,gate", [("f32", "fp32", 1e-5), ("bf16", "fp32", 1e-2),
                                                ("f32", "tc_tf32", 5e-2), ("bf16", "tc_bf16", 5e-2),
                                                ("f32", "tc_3xtf32", 1e-5)])
def test_box49_16384_window(windows, dtype, compute, gate):
    rec = windows["box49_16384_T200"]
    W = inputs.pattern_weights("box49")
    tdt = {"f32": torch.float32, "bf16": torch.bfloat16}[dtype]
    x = torch.from_numpy(inputs.field(16384, 16384)).to(tdt).cuda()
    p = _plan(16384, W, dtype=dtype, compute=compute)
    y = p.run(x, 200)
    torch.cuda.synchronize()
    p.status()
    err = rel_l2(y[:16, :16].float().cpu().numpy(), np.asarray(rec["window"]))
    assert err <= gate, (dtype, compute, err, p.info())
    p.close()


def _tiled(base: np.ndarray, n: int):
    """The n x n grid that repeats `base` (host) and the same grid on the device."""
    reps = -(-n // base.shape[0])
    dev = torch.from_numpy(base).cuda().repeat(reps, reps)[:n, :n].contiguous()
    return dev


def _host_block(base, y0, y1, x0, x1):
    """Rows [y0, y1) x columns [x0, x1) of the tiled grid, clipped to >= 0, on the host."""
    b = base.shape[0]
    rows = np.arange(max(0, y0), y1) % b
    cols = np.arange(max(0, x0), x1) % b
    return base[np.ix_(rows, cols)]


@pytest.mark.parametrize("name,n,T", [("box9", 16384, 8), ("star13", 16384, 6), ("box9", 32768, 8),
                                      ("star13", 32768, 4), ("heat5", 44800, 8)])
def test_large_grid_light_cone_windows(oracle, windows, name, n, T):
    W = inputs.pattern_weights(name)
    r = W.shape[0] // 2
    base = inputs.field(4096, 4096)
    x = _tiled(base, n)
    p = _plan(n, W)
    y = p.run(x, T)
    torch.cuda.synchronize()
    p.status()
    win, m = 24, r * T
    # top-left corner: the grid edge is the zero boundary
    ref = oracle.sweep_f64(_host_block(base, 0, win + m, 0, win + m), W, T)[:win, :win]
    got = y[:win, :win].cpu().numpy()
    assert rel_l2(got, ref) <= 1e-6 and rel_linf(got, ref) <= T * 13 * 2.0 ** -24, "top-left"
    # bottom-right corner (the last elements: flat index near n*n)
    blk = _host_block(base, n - win - m, n, n - win - m, n)
    ref = oracle.sweep_f64(blk, W, T)[-win:, -win:]
    got = y[-win:, -win:].cpu().numpy()
    assert rel_l2(got, ref) <= 1e-6 and rel_linf(got, ref) <= T * 13 * 2.0 ** -24, "bottom-right"
    # the middle: the window's light cone, its outer m rows and columns dropped
    c = n // 2
    blk = _host_block(base, c - m, c + win + m, c - m, c + win + m)
    ref = oracle.sweep_f64(blk, W, T)[m:m + win, m:m + win]
    got = y[c:c + win, c:c + win].cpu().numpy()
    assert rel_l2(got, ref) <= 1e-6 and rel_linf(got, ref) <= T * 13 * 2.0 ** -24, "middle"
    p.close()
    del x, y
    torch.cuda.empty_cache()


def test_batched_256_grids_windows(windows):
    """The 256-grid batched workload as bench.py runs it: the stored FP64 windows
    of its three smallest and three largest grids after 200 steps."""
    from paper_2605_07954_gb300 import Batch
    sides, kinds = inputs.batch_spec(256)
    grids = []
    for g, (sd, kind) in enumerate(zip(sides, kinds)):
        x = torch.from_numpy(inputs.field(int(sd), int(sd), stream=10000 + g)).cuda()
        grids.append(dict(x=x, out=torch.empty_like(x), weights=inputs.batch_grid_weights(kind, g), T=200))
    b = Batch(grids)
    b.run()
    torch.cuda.synchronize()
    b.status()
    checked = 0
    for g in range(256):
        rec = windows.get(f"batch_grid{g}")
        if rec is None:
            continue
        ref = np.asarray(rec["window"])
        got = grids[g]["out"][:16, :16].cpu().numpy()
        assert rel_l2(got, ref) <= 1e-5, (g, int(sides[g]))
        checked += 1
    assert checked == 6
    b.close()
