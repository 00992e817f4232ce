"""The synthetic octrees obey the 2:1 rule across faces and edges (the
reading of Sec. 3.2.1's balance condition that makes every cell edge carry
at most one hanging node, so that a cell is described by a 12-bit mask of
mid-edge nodes): two cells that share a face or an edge differ by at most
one level.  Checked by brute force over all pairs of small meshes."""
import numpy as np
import pytest

import octree_gen as og


def _violations(m):
    size = (2 ** (m.lmax - m.level)).astype(np.int64)
    lo = m.anchor.astype(np.int64)
    hi = lo + size[:, None]
    bad = 0
    touching = 0
    for i in range(m.n_cells):
        ov = np.minimum(hi[i], hi) - np.maximum(lo[i], lo)      # (C, 3) overlap per axis
        dim = (ov > 0).sum(1)
        share = (ov >= 0).all(1) & (dim >= 1) & (dim <= 2)      # a face or an edge, not volume
        share[i] = False
        touching += int(share.sum())
        bad += int((share & (np.abs(m.level - m.level[i]) > 1)).sum())
    return bad, touching


@pytest.mark.parametrize("make", [og.config_corner_cube, lambda: og.tiny_refined(0),
                                  lambda: og.tiny_refined(3, lmax=3),
                                  lambda: og.cube_roller(4, refine_p=0.3)])
def test_face_and_edge_neighbours_differ_by_at_most_one_level(make):
    m = make()
    assert len(np.unique(m.level)) >= 2            # the mesh is graded
    bad, touching = _violations(m)
    assert touching > 0 and bad == 0


def test_no_two_cells_overlap():
    m = og.config_corner_cube()
    size = (2 ** (m.lmax - m.level)).astype(np.int64)
    lo = m.anchor.astype(np.int64)
    hi = lo + size[:, None]
    vol = int((size ** 3).sum())
    ext = hi.max(0) - lo.min(0)
    assert vol == int(np.prod(ext))                # the cells tile the domain
    for i in range(m.n_cells):
        ov = np.minimum(hi[i], hi) - np.maximum(lo[i], lo)
        inner = (ov > 0).all(1)
        inner[i] = False
        assert not inner.any()
