"""Comparison helpers of the GPU parity tests: a state (or field) against the
oracle's, by relative L2 over all points and components and, beside it, by
the largest pointwise deviation relative to the largest value, so that a
wrong value at a few points (near the mask layer, in a ragged tile) cannot
hide under a small global norm."""
import numpy as np

# the pointwise bound is this many times the relative-L2 bound: an error
# spread over the field has max|d| / max|u| of the order of its relative L2
# norm; a factor 10 leaves room for errors that gather in the solid's layer
POINTWISE_FACTOR = 10.0


def rel_l2(a, b):
    a, b = np.asarray(a), np.asarray(b)
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def max_rel(a, b):
    a, b = np.asarray(a), np.asarray(b)
    return float(np.abs(a - b).max() / np.abs(b).max())


def check_state(a, b, tol, what=""):
    """rel L2 <= tol and max |a - b| <= POINTWISE_FACTOR tol max |b|."""
    l2, mx = rel_l2(a, b), max_rel(a, b)
    assert l2 <= tol, f"{what} relative L2 {l2:.3e} > {tol:.1e}"
    assert mx <= POINTWISE_FACTOR * tol, f"{what} pointwise {mx:.3e} > {POINTWISE_FACTOR * tol:.1e}"
    return l2, mx
