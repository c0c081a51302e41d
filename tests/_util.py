"""Small helpers shared by the tests (no GP arithmetic here)."""
import numpy as np


def rel(a, b):
    """Norm-wise relative error ||a - b||_2 / ||b||_2 (the suite's error metric)."""
    a = np.asarray(a, dtype=np.float64).ravel()
    b = np.asarray(b, dtype=np.float64).ravel()
    nb = np.linalg.norm(b)
    return float(np.linalg.norm(a - b) / (nb if nb > 0 else 1.0))


def max_rel(a, b, floor=0.0):
    """Worst element-wise |a-b| / max(|b|, floor)."""
    a = np.asarray(a, dtype=np.float64).ravel()
    b = np.asarray(b, dtype=np.float64).ravel()
    return float(np.max(np.abs(a - b) / np.maximum(np.abs(b), floor))) if a.size else 0.0
