"""Shared helpers for the GPU tests (fixtures, tolerances)."""
import numpy as np

# Tolerances (relative). FP64 path: every step in double, so only summation order
# differs from the oracle: 1e-11 on ell, 1e-10 of max|grad| on the gradient.
# Mixed path: float32 pair terms (ex2.approx relative error ~2^-22, float32 rounding of
# distances), float32 sums over 256 columns, float64 beyond: 1e-6 on ell and on the
# gradient relative to max|grad|.
TOL_FP64_LL = 1e-11
TOL_FP64_G = 1e-10
TOL_MIXED_LL = 1e-6
TOL_MIXED_G = 1e-6


def rel(a, b):
    return abs(a - b) / max(abs(b), 1e-300)


def grad_err(g, ref):
    return float(np.max(np.abs(np.asarray(g) - np.asarray(ref))) / max(np.max(np.abs(ref)), 1e-300))
