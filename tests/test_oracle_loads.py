"""Pins of the oracle's line loads (Sec. 5.5: forces along lines): the
consistent nodal forces of a uniform load q along a segment sum to q L, and
on a uniform mesh an interior node of the line carries q h, an end node
q h / 2; the product's helper (tributary lengths of the nodes on the line)
gives the same forces on refined meshes."""
import numpy as np
import pytest

import octree_gen as og
from oracle import cdm
from paper_2103_09100_gb300 import loads


def test_uniform_mesh_line_load():
    m = og.small_uniform(4, h=0.25)   # [0, 1]^3, h = 1 / 4
    f = cdm.line_load_forces(m, (0, 0.5, 1), (1, 0.5, 1), 3.0)
    x = m.node_xyz
    ends = [k for k in f if abs(x[k, 0]) < 1e-12 or abs(x[k, 0] - 1) < 1e-12]
    assert len(f) == 5 and len(ends) == 2
    for k, v in f.items():
        assert v == pytest.approx(3.0 * 0.25 * (0.5 if k in ends else 1.0), rel=1e-14)


@pytest.mark.parametrize("seg, q", [(((0, 0.5, 1), (1, 0.5, 1)), 2.0),
                                    (((0.5, 0, 1), (0.5, 1, 1)), 1.5),
                                    (((0.25, 0.25, 0.5), (0.25, 0.25, 1.0)), 4.0)])
def test_refined_mesh_total_and_product_helper(seg, q):
    m = og.config_corner_cube()
    a, b = seg
    f = cdm.line_load_forces(m, a, b, q)
    L = float(np.linalg.norm(np.subtract(b, a)))
    assert sum(f.values()) == pytest.approx(q * L, rel=1e-13)
    p = {s["node"]: s["P0"] for s in loads.line_load(m.node_xyz, a, b, (0, 0, 1), q, 1.0)}
    assert set(p) == set(f)
    assert max(abs(p[k] - f[k]) for k in f) <= 1e-14 * q
