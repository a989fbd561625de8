"""Error metrics of the parity tests.

Every comparison of the GPU path with the oracle (or with the GPU's own FP64 path)
asserts two metrics: the relative l2 error over all outputs, and the element-wise
error max |y - ref| / max |ref| (the paper's errors are max-modulus ones, and a few
wrong targets can hide in an l2 norm over hundreds of thousands of values but not
in the maximum)."""
import numpy as np


def rel(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / np.linalg.norm(np.asarray(b)))


def rel_max(a, b):
    a, b = np.asarray(a), np.asarray(b)
    return float(np.abs(a - b).max() / np.abs(b).max())


def check(y, ref, tol, what=""):
    """Assert rel l2 <= tol and rel max <= tol; returns the l2 error."""
    e2, em = rel(y, ref), rel_max(y, ref)
    assert e2 <= tol, (what, "rel l2", e2, tol)
    assert em <= tol, (what, "rel max", em, tol)
    return e2
