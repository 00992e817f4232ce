"""Line loads (Sec. 5.5's panel: forces distributed along lines).

A uniform line load of q per unit length along the segment [a, b], in a
fixed direction, enters the explicit step as consistent nodal forces of the
mesh nodes on the segment: with linear variation between neighbouring
nodes along the line, node i receives q (l_{i-1} + l_i) / 2, half the
lengths of the two node-to-node pieces it bounds.  The result is a list of
point loads in the ``Solver`` source format (one time function for all of
them), which ``set_load`` applies in the step kernels.
"""
from __future__ import annotations

import numpy as np


def nodes_on_segment(node_xyz, a, b, tol=1e-9):
    """Mesh nodes on the segment [a, b] and their positions t in [0, 1]
    along it, ascending."""
    a = np.asarray(a, float)
    b = np.asarray(b, float)
    d = b - a
    L2 = float(d @ d)
    if L2 <= 0.0:
        raise ValueError("degenerate segment")
    x = np.asarray(node_xyz, float)
    t = (x - a) @ d / L2
    off = x - a[None, :] - t[:, None] * d[None, :]
    scale = np.sqrt(L2)
    on = (np.linalg.norm(off, axis=1) <= tol * scale) & (t >= -tol) & (t <= 1 + tol)
    idx = np.nonzero(on)[0]
    order = np.argsort(t[idx], kind="stable")
    return idx[order], np.clip(t[idx][order], 0.0, 1.0)


def line_load(node_xyz, a, b, direction, q, t1, wavelet="ricker", rhs=0, n_cycles=5.0,
              tol=1e-9):
    """Point loads equivalent to q per unit length along [a, b]."""
    nodes, t = nodes_on_segment(node_xyz, a, b, tol)
    if len(nodes) < 2:
        raise ValueError("the segment holds fewer than two mesh nodes")
    length = float(np.linalg.norm(np.asarray(b, float) - np.asarray(a, float)))
    seg = np.diff(t) * length
    w = np.zeros(len(nodes))
    w[:-1] += 0.5 * seg
    w[1:] += 0.5 * seg
    d = np.asarray(direction, float)
    d = d / np.linalg.norm(d)
    return [{"node": int(n), "dir": d.tolist(), "t1": float(t1), "P0": float(q * wi),
             "wavelet": wavelet, "rhs": int(rhs), "n_cycles": float(n_cycles)}
            for n, wi in zip(nodes, w)]
