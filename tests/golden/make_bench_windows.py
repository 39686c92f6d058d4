#!/usr/bin/env python3
"""Write bench_windows.json: FP64 oracle windows of the benchmark workloads.

bench.py checks the output it times against these values (it may not run the
oracle itself), and the GPU tests use them for parity at the benchmark sizes.
Every value here comes from the oracle package only (oracle.corner_window_f64,
the light cone of a corner window, pinned against whole-grid sweeps in
tests/test_oracle_pins.py; oracle.sweep_f64 and oracle.adjoint_f64), on the
seeded inputs of paper_2605_07954_gb300.inputs that the benchmark draws.

Run from the repository root:  python tests/golden/make_bench_windows.py
(about a minute; the 13-point star's 1000-step light cone dominates).
"""
import json
import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import oracle  # noqa: E402
from paper_2605_07954_gb300 import inputs  # noqa: E402

WIN = 16


def field_corner(ny, nx, h, w, stream=inputs.STREAM_FIELD):
    """Rows [0, h) x columns [0, w) of inputs.field(ny, nx, stream=stream)."""
    h = min(h, ny)
    return inputs.uniform_f32(0, stream, h * nx).reshape(h, nx)[:, :min(w, nx)]


def window(ny, nx, W, T, stream=inputs.STREAM_FIELD):
    r = W.shape[0] // 2
    u = field_corner(ny, nx, WIN + r * T, WIN + r * T, stream)
    return oracle.corner_window_f64(u, W, T, WIN)


def main():
    oracle.build()
    out = {"_about": "FP64 oracle values of the top-left 16x16 window after T steps (zero rule) of the "
                     "benchmark workloads; written by tests/golden/make_bench_windows.py",
           "window": WIN, "workloads": {}}
    t0 = time.time()
    for name, n, T in (("box9", 8192, 1000), ("star13", 8192, 1000), ("box49", 16384, 200),
                       ("heat5", 512, 100)):
        W = inputs.pattern_weights(name)
        out["workloads"][f"{name}_{n}_T{T}"] = {
            "pattern": name, "ny": n, "nx": n, "T": T, "window": window(n, n, W, T).tolist()}
        print(f"{name} {n}^2 T={T}: {time.time() - t0:.1f} s", flush=True)
    # batched workload: the three smallest and three largest grids
    sides, kinds = inputs.batch_spec(256)
    order = np.argsort(sides, kind="stable")
    for g in [int(i) for i in list(order[:3]) + list(order[-3:])]:
        W = inputs.batch_grid_weights(kinds[g], g)
        n = int(sides[g])
        out["workloads"][f"batch_grid{g}"] = {
            "pattern": kinds[g], "grid": g, "ny": n, "nx": n, "T": 200,
            "window": window(n, n, W, 200, stream=10000 + g).tolist()}
    print(f"batched: {time.time() - t0:.1f} s", flush=True)
    # adjoint instance: Heat 0.2f, 64 x 64, 32 steps, L = 0.5 ||u_T - target||^2
    # (the weight gradient and the top-left window of the input gradient)
    n, T = 64, 32
    W = inputs.heat_weights(0.2)
    u0 = inputs.field(n, n)
    target = inputs.field(n, n, stream=inputs.STREAM_TARGET)
    uT = oracle.sweep_f64(u0, W, T)
    g_u0, g_w = oracle.adjoint_f64(u0, W, T, uT - target)
    out["workloads"]["adjoint_heat5_64_T32"] = {
        "pattern": "heat5", "ny": n, "nx": n, "T": T,
        "grad_u0_window": g_u0[:WIN, :WIN].tolist(), "grad_w": g_w.tolist()}
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "bench_windows.json")
    with open(path, "w") as f:
        json.dump(out, f, separators=(",", ":"))
        f.write("\n")
    print(f"wrote {path} in {time.time() - t0:.1f} s")


if __name__ == "__main__":
    main()
