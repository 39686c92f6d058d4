"""Small helpers shared by the tests (error metrics, tolerances)."""
import numpy as np


def rel_l2(got, ref) -> float:
    got = np.asarray(got, dtype=np.float64)
    ref = np.asarray(ref, dtype=np.float64)
    den = np.linalg.norm(ref)
    return float(np.linalg.norm(got - ref) / (den if den > 0 else 1.0))


def rel_linf(got, ref) -> float:
    got = np.asarray(got, dtype=np.float64)
    ref = np.asarray(ref, dtype=np.float64)
    den = np.abs(ref).max()
    return float(np.abs(got - ref).max() / (den if den > 0 else 1.0))


def fp32_tol(T: int) -> float:
    """Relative-L2 gate for the FP32 path: 1e-5 per 1000 steps, never below 1e-5."""
    return 1e-5 * max(1.0, T / 1000.0)


# Element-wise gate: an FP32 sum of at most 49 products rounds each step by at
# most ~49 * 2^-24 of the sum of |terms|; with non-negative normalised weights
# that is <= 3e-6 of max|u| per step.  Errors of a contracting operator add
# up at most linearly in T.
def fp32_elem_tol(T: int, taps: int) -> float:
    return max(1, T) * taps * 2.0 ** -24 + 1e-7
