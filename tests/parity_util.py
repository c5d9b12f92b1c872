"""Comparison helpers of the GPU parity tests (expected values always come from the oracle).

A block of outputs is (vectors, points): one right-hand side, sample or feature per row, one
point per column.  `close` checks it two ways: the relative Frobenius error over the whole
block (the bound each precision form is held to) and, point by point, the error of a point's
values against that point's own norm, so that one wrong point (a bad row of the product, a
wrongly indexed tile) fails even among many correct ones.  The point-wise bound is a small
multiple of the block bound: a point's relative error scatters around the block's."""
import numpy as np

POINT_FACTOR = 4.0


def rel(a, b):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


def pointwise_rel(a, b):
    """Largest over points (columns) of ||a[:, i] - b[:, i]|| / ||b[:, i]||.  A 1-D array is one
    value per point (a predictive mean or variance); its error is taken against the larger of
    |b_i| and the values' root mean square, since a single value can pass through zero."""
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    if a.ndim == 1:
        if not a.size:
            return 0.0
        den = np.maximum(np.abs(b), np.sqrt(np.mean(b * b)))
        return float(np.max(np.abs(a - b) / np.maximum(den, 1e-300)))
    num = np.linalg.norm(a - b, axis=0)
    den = np.maximum(np.linalg.norm(b, axis=0), 1e-300)
    return float(np.max(num / den)) if num.size else 0.0


def close(a, b, tol, point_factor=POINT_FACTOR):
    """True when the block error is below tol and every point's error below point_factor * tol."""
    e, p = rel(a, b), pointwise_rel(a, b)
    assert e < tol, "relative Frobenius error %.3g >= %.3g" % (e, tol)
    assert p < point_factor * tol, "worst point's relative error %.3g >= %.3g" % (p, point_factor * tol)
    return True
