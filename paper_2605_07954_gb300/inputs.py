"""Seeded synthetic inputs for the stencil library, its tests and its benchmark.

This module is the one piece shared between the CUDA path's callers and the
CPU oracle's callers.  It holds no stencil arithmetic: it only draws numbers
and builds the weight arrays of the four stencil patterns the paper studies
(Star2d-1r = Heat 5-point, Star2d-3r = 13-point, Box2d-1r = 9-point,
Box2d-3r = 49-point; shapes and radii as defined in Sec. II-B).

Generator
---------
A counter-based SplitMix64 (Steele, Lea and Flood, "Fast splittable
pseudorandom number generators", OOPSLA 2014):

    mix(z)   = z1 ^ (z1 >> 31) where
               z0 = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9
               z1 = (z0 ^ (z0 >> 27)) * 0x94D049BB133111EB   (mod 2**64)
    value(s, n) = mix(s + (n + 1) * 0x9E3779B97F4A7C15)       (mod 2**64)

``value(0, n)`` is the plain SplitMix64 sequence started from state 0.  A
(seed, stream) pair selects the start state ``s = mix((seed << 32) ^ stream)``.
A float in [0, 1) is ``(value >> 40) * 2**-24``: exact in FP32.

Streams: 0 = the field, 1 = the weights (grid g of a batch: 1000 + g),
2 = the adjoint target, 3 = batch sizes and pattern assignment.
"""
from __future__ import annotations

import numpy as np

_GAMMA = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)
_CHUNK = 1 << 22

STREAM_FIELD = 0
STREAM_WEIGHTS = 1
STREAM_TARGET = 2
STREAM_BATCH = 3


def _mix(z: np.ndarray) -> np.ndarray:
    with np.errstate(over="ignore"):
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        return z ^ (z >> np.uint64(31))


def start_state(seed: int, stream: int) -> int:
    """Start state of the (seed, stream) sequence."""
    z = np.array([((int(seed) << 32) ^ int(stream)) & 0xFFFFFFFFFFFFFFFF], dtype=np.uint64)
    return int(_mix(z)[0])


def splitmix64(state: int, first: int, count: int) -> np.ndarray:
    """Outputs ``first .. first+count-1`` of the SplitMix64 sequence from ``state``."""
    idx = np.arange(first + 1, first + 1 + count, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = np.uint64(state) + idx * _GAMMA
    return _mix(z)


def uniform_f32(seed: int, stream: int, count: int, first: int = 0) -> np.ndarray:
    """``count`` FP32 values in [0, 1) from the (seed, stream) sequence."""
    s = start_state(seed, stream)
    out = np.empty(count, dtype=np.float32)
    for lo in range(0, count, _CHUNK):
        n = min(_CHUNK, count - lo)
        v = splitmix64(s, first + lo, n) >> np.uint64(40)
        out[lo:lo + n] = v.astype(np.float32) * np.float32(2.0 ** -24)
    return out


def uniform_f64(seed: int, stream: int, count: int, first: int = 0) -> np.ndarray:
    """Same draws as :func:`uniform_f32`, returned as FP64 (exactly equal values)."""
    return uniform_f32(seed, stream, count, first).astype(np.float64)


def field(ny: int, nx: int, seed: int = 0, stream: int = STREAM_FIELD) -> np.ndarray:
    """A ``(ny, nx)`` FP32 field, uniform in [0, 1), row-major draw order."""
    return uniform_f32(seed, stream, ny * nx).reshape(ny, nx)


# ---- stencil footprints (Sec. II-B) ------------------------------------------------

def footprint(shape: str, r: int) -> np.ndarray:
    """Boolean ``(2r+1, 2r+1)`` mask: ``"box"`` = full square, ``"star"`` = the two axes."""
    d = 2 * r + 1
    if shape == "box":
        return np.ones((d, d), dtype=bool)
    if shape == "star":
        m = np.zeros((d, d), dtype=bool)
        m[r, :] = True
        m[:, r] = True
        return m
    raise ValueError(f"unknown shape {shape!r}")


def random_weights(shape: str, r: int, seed: int = 0, stream: int = STREAM_WEIGHTS) -> np.ndarray:
    """Weights uniform in [0, 1) on the footprint, normalised to sum 1.

    One draw per entry of the ``(2r+1)^2`` square in row-major order; entries
    off the footprint are zeroed; the sum is normalised in FP64 and the result
    rounded to FP32.  The FP32 array is the definitive weight set.
    """
    d = 2 * r + 1
    w = uniform_f64(seed, stream, d * d).reshape(d, d)
    w = np.where(footprint(shape, r), w, 0.0)
    return (w / w.sum()).astype(np.float32)


def heat_weights(c: float = 0.2) -> np.ndarray:
    """Heat-2D 5-point as weights: centre 1-4c, each arm c.  c=0.2 gives 0.2f everywhere."""
    w = np.zeros((3, 3), dtype=np.float32)
    w[1, 1] = np.float32(1.0 - 4.0 * c)
    w[0, 1] = w[2, 1] = w[1, 0] = w[1, 2] = np.float32(c)
    return w


PATTERNS = {
    # name: (shape, radius)
    "heat5": ("star", 1),
    "box9": ("box", 1),
    "star13": ("star", 3),
    "box49": ("box", 3),
}


def pattern_weights(name: str, seed: int = 0, stream: int = STREAM_WEIGHTS) -> np.ndarray:
    """Weights for a named pattern: Heat uses 0.2f, the others the random normalised rule."""
    if name == "heat5":
        return heat_weights(0.2)
    shape, r = PATTERNS[name]
    return random_weights(shape, r, seed, stream)


def batch_spec(n: int = 256, lo: int = 64, hi: int = 2048, seed: int = 0):
    """Sides log-uniform in [lo, hi] and a half/half Heat-5pt / Box-9pt assignment.

    side = round(exp(U ln hi + (1-U) ln lo)) clamped to [lo, hi] with U from
    stream 3 (draws 0..n-1); the pattern order is a Fisher-Yates shuffle of
    n/2 "heat5r" and n/2 "box9" driven by draws n..2n-2 of the same stream.
    "heat5r" is the 5-point star footprint with random normalised weights.
    """
    u = uniform_f64(seed, STREAM_BATCH, 2 * n)
    sides = np.rint(np.exp(u[:n] * np.log(hi) + (1.0 - u[:n]) * np.log(lo)))
    sides = np.clip(sides, lo, hi).astype(np.int64)
    kinds = ["heat5r"] * (n // 2) + ["box9"] * (n - n // 2)
    for k in range(n - 1, 0, -1):
        j = int(u[n + (n - 1 - k)] * (k + 1))
        kinds[k], kinds[j] = kinds[j], kinds[k]
    return sides, kinds


def batch_grid_weights(kind: str, g: int, seed: int = 0) -> np.ndarray:
    shape, r = {"heat5r": ("star", 1), "box9": ("box", 1)}[kind]
    return random_weights(shape, r, seed, 1000 + g)
