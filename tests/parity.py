"""Error measures of the GPU parity tests (test helper, no method arithmetic).

Every parity check compares the CUDA path's result a with the FP64 oracle's
b over ALL entries in two norms and takes the larger:

* the relative L2 error ||a - b||_2 / ||b||_2 over the whole state, and
* the element-wise error max_i |a_i - b_i| / max_i |b_i|,

so an error confined to a few entries (a rare hanging-node pattern among a
million cells) is not diluted by the sqrt(N) of the L2 norm.
"""
import numpy as np


def rel_l2(a, b):
    a = np.asarray(a, float)
    b = np.asarray(b, float)
    nb = np.linalg.norm(b)
    return float(np.linalg.norm(a - b) / nb) if nb > 0 else float(np.linalg.norm(a))


def rel_max(a, b):
    a = np.asarray(a, float)
    b = np.asarray(b, float)
    mb = np.abs(b).max() if b.size else 0.0
    d = np.abs(a - b).max() if a.size else 0.0
    return float(d / mb) if mb > 0 else float(d)


def rel(a, b):
    """max(relative L2 error, element-wise error relative to max |b|)."""
    return max(rel_l2(a, b), rel_max(a, b))


def rel_cols(a, b):
    """rel per column of two (n, B) arrays: a list of B errors."""
    return [rel(a[:, j], b[:, j]) for j in range(b.shape[1])]
