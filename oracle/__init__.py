"""CPU oracle for iterated explicit 2D stencil sweeps (Jacobi update, Sec. II-C).

TEST INFRASTRUCTURE ONLY: tests/, ``__graft_entry__.smoke()`` and the CPU
baseline leg of ``bench.py`` are the only callers.  The product path never
imports this package, and this package imports nothing from the product.

The arithmetic lives in ``oracle.c`` (plain nested loops, FP64 and FP32);
this module compiles it with gcc and marshals numpy arrays through ctypes.

Conventions (shared with the library by definition, not by code):
  * grids are row-major ``(ny, nx)``; i = row (y), j = column (x);
  * ``W`` is ``(2r+1, 2r+1)``; ``W[dy+r, dx+r]`` multiplies ``u[i+dy, j+dx]``
    (cross-correlation, no flip);
  * boundary ``"zero"``: everything outside the grid is a frozen 0 (the
    paper's zero padding, Sec. IV-A); ``"periodic"``: indices wrap.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import sys

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lib = None

BOUNDARY = {"zero": 0, "periodic": 1}


def build(force: bool = False) -> str:
    """Compile oracle.c into liboracle.so beside it (gcc, OpenMP, no FMA contraction)."""
    if (not force and os.path.exists(_LIB)
            and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC)):
        return _LIB
    cmd = ["gcc", "-O2", "-std=c11", "-fopenmp", "-ffp-contract=off", "-fPIC",
           "-shared", "-o", _LIB + ".tmp", _SRC]
    subprocess.run(cmd, check=True)
    os.replace(_LIB + ".tmp", _LIB)
    return _LIB


def _load():
    global _lib
    if _lib is not None:
        return _lib
    build()
    lib = ctypes.CDLL(_LIB)
    i64, i32, dbl = ctypes.c_int64, ctypes.c_int, ctypes.c_double
    dp = ctypes.POINTER(ctypes.c_double)
    fp = ctypes.POINTER(ctypes.c_float)
    lib.oracle_sweep_f64.argtypes = [i64, i64, i32, dp, i32, i64, dp, dp]
    lib.oracle_sweep_f32.argtypes = [i64, i64, i32, fp, i32, i64, fp, fp]
    lib.oracle_heat_literal_f64.argtypes = [i64, i64, dbl, i64, dp, dp]
    lib.oracle_adjoint_f64.argtypes = [i64, i64, i32, dp, i32, i64, dp, dp, dp, dp]
    for f in (lib.oracle_sweep_f64, lib.oracle_sweep_f32, lib.oracle_heat_literal_f64,
              lib.oracle_adjoint_f64):
        f.restype = i32
    lib.oracle_num_threads.restype = i32
    lib.oracle_set_num_threads.argtypes = [i32]
    _lib = lib
    return lib


def _ptr(a: np.ndarray, ctype):
    return a.ctypes.data_as(ctypes.POINTER(ctype))


def _radius(W: np.ndarray) -> int:
    d = W.shape[0]
    if W.ndim != 2 or W.shape[1] != d or d % 2 != 1:
        raise ValueError(f"weights must be (2r+1, 2r+1), got {W.shape}")
    return d // 2


def _check(rc: int, what: str):
    if rc != 0:
        raise RuntimeError(f"{what} failed with oracle status {rc}")


def sweep_f64(u0, W, T: int, boundary: str = "zero") -> np.ndarray:
    """u_T in FP64 after T Jacobi steps from u0 (Sec. II-C); weights promoted exactly."""
    lib = _load()
    u0 = np.ascontiguousarray(u0, dtype=np.float64)
    W = np.ascontiguousarray(W, dtype=np.float64)
    r = _radius(W)
    out = np.empty_like(u0)
    ny, nx = u0.shape
    _check(lib.oracle_sweep_f64(ny, nx, r, _ptr(W, ctypes.c_double), BOUNDARY[boundary],
                                int(T), _ptr(u0, ctypes.c_double),
                                _ptr(out, ctypes.c_double)), "oracle_sweep_f64")
    return out


def sweep_f32(u0, W, T: int, boundary: str = "zero") -> np.ndarray:
    """u_T with FP32 arithmetic, dy-major then dx summation, no FMA contraction."""
    lib = _load()
    u0 = np.ascontiguousarray(u0, dtype=np.float32)
    W = np.ascontiguousarray(W, dtype=np.float32)
    r = _radius(W)
    out = np.empty_like(u0)
    ny, nx = u0.shape
    _check(lib.oracle_sweep_f32(ny, nx, r, _ptr(W, ctypes.c_float), BOUNDARY[boundary],
                                int(T), _ptr(u0, ctypes.c_float),
                                _ptr(out, ctypes.c_float)), "oracle_sweep_f32")
    return out


def heat_literal_f64(u0, c: float, T: int) -> np.ndarray:
    """u' = u + c(N+S+E+W-4u) written out, FP64, zero boundary."""
    lib = _load()
    u0 = np.ascontiguousarray(u0, dtype=np.float64)
    out = np.empty_like(u0)
    ny, nx = u0.shape
    _check(lib.oracle_heat_literal_f64(ny, nx, float(c), int(T), _ptr(u0, ctypes.c_double),
                                       _ptr(out, ctypes.c_double)), "oracle_heat_literal_f64")
    return out


def adjoint_f64(u0, W, T: int, gT, boundary: str = "zero"):
    """(dL/du0, dL/dW) in FP64 for a loss L(u_T) whose gradient at u_T is gT."""
    lib = _load()
    u0 = np.ascontiguousarray(u0, dtype=np.float64)
    gT = np.ascontiguousarray(gT, dtype=np.float64)
    W = np.ascontiguousarray(W, dtype=np.float64)
    r = _radius(W)
    g_u0 = np.empty_like(u0)
    g_W = np.empty_like(W)
    ny, nx = u0.shape
    _check(lib.oracle_adjoint_f64(ny, nx, r, _ptr(W, ctypes.c_double), BOUNDARY[boundary],
                                  int(T), _ptr(u0, ctypes.c_double), _ptr(gT, ctypes.c_double),
                                  _ptr(g_u0, ctypes.c_double), _ptr(g_W, ctypes.c_double)),
           "oracle_adjoint_f64")
    return g_u0, g_W


def corner_window_f64(u0, W, T: int, win: int = 16, chunk: int = 25) -> np.ndarray:
    """The top-left win x win window of u_T (zero rule, FP64), from the light cone only.

    A window of u_T depends only on inputs within r*T of it (P6, the light
    cone).  This runs sweep_f64 on the corner sub-grid and, after every chunk
    of s steps, drops the rows and columns beyond win + r*(T - t): exactly the
    ones the cut (which acts as a zero boundary) has made wrong.  Rows at the
    grid's own edges are exact throughout.  Each kept value is computed by the
    same operations as in a whole-grid sweep_f64, so the window is identical.
    """
    u0 = np.asarray(u0)
    r = _radius(np.asarray(W))
    ny, nx = u0.shape
    cur = np.asarray(u0[:min(ny, win + r * T), :min(nx, win + r * T)], dtype=np.float64)
    t = 0
    while t < T:
        s = min(chunk, T - t)
        cur = sweep_f64(cur, W, s, "zero")
        t += s
        cur = np.ascontiguousarray(cur[:min(ny, win + r * (T - t)), :min(nx, win + r * (T - t))])
    return cur[:win, :win].copy()


def num_threads() -> int:
    return int(_load().oracle_num_threads())


def set_num_threads(n: int) -> None:
    _load().oracle_set_num_threads(int(n))


if __name__ == "__main__":  # pragma: no cover
    print(build(force="--force" in sys.argv))
