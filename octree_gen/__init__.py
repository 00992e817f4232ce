"""Seeded synthetic 2:1-balanced octree meshes (inputs only).

This module produces the *input mesh* of Algorithm 1 and nothing
else: cells, their hanging-node masks, node ids and coordinates, material
fields, fixed nodes and point loads.  It holds none of the method's
arithmetic (no stiffness, mass, pattern reduction or time stepping); both
the FP64 oracle and the GPU library consume its plain arrays.

Mesh format
-----------
Each cell carries 26 node slots (corner, mid-edge and face-centre nodes of
Sec. 3.2.1).  Slot positions on the doubled cube [-1, 1]^3:

* corners 0..7: c = i + 2j + 4k at (2i-1, 2j-1, 2k-1)
* mid-edges 8..19: 8 + 4a + r on the edge parallel to axis a, with the
  other axes (b, c) (increasing) at (2(r & 1) - 1, 2(r >> 1) - 1)
* face centres 20..25: 20 + 2a + side at coordinate a = 2 side - 1

``slot_node[cell, slot]`` is the global node id or -1 when the slot is
absent.  Mid-edge nodes exist where a finer neighbour puts a vertex (the
octree's hanging nodes, at most one per edge under the 2:1 rule, applied
across faces and edges).  A face carries a centre node when it has 1,
2 adjacent, 3 or 4 mid-edge nodes; with 0 or 2 opposite ones it has none.
This reading of the missing face-pattern figure is what makes the face
discretisation of two cells sharing a face identical.

Cells whose centre falls inside a removed region (cavity, trench) are
dropped after balancing; hanging-node masks come from the full balanced
tree so that faces shared with removed cells' siblings stay conforming.

Cells and nodes are numbered in Morton (Z-curve) order.
"""
from __future__ import annotations

import json
from dataclasses import dataclass, field
from typing import Callable, Optional

import numpy as np

# ---------------------------------------------------------------- geometry
_CORNER_POS = np.array([[2 * (c & 1) - 1, 2 * ((c >> 1) & 1) - 1, 2 * ((c >> 2) & 1) - 1]
                        for c in range(8)], dtype=np.int64)


def _edge_pos(e):
    a, r = divmod(e, 4)
    b, c = [x for x in range(3) if x != a]
    p = [0, 0, 0]
    p[b] = 2 * (r & 1) - 1
    p[c] = 2 * (r >> 1) - 1
    return p


def _face_pos(f):
    a, side = divmod(f, 2)
    p = [0, 0, 0]
    p[a] = 2 * side - 1
    return p


SLOT_POS = np.vstack([_CORNER_POS,
                      np.array([_edge_pos(e) for e in range(12)], dtype=np.int64),
                      np.array([_face_pos(f) for f in range(6)], dtype=np.int64)])

# For each face: the slots of its 4 boundary mid-edges in cyclic order.
_FACE_MIDS = []
for _f in range(6):
    _a, _side = divmod(_f, 2)
    _b, _c = [x for x in range(3) if x != _a]
    _mids = []
    for ub, uc in [(0, -1), (1, 0), (0, 1), (-1, 0)]:
        p = [0, 0, 0]
        p[_a] = 2 * _side - 1
        p[_b] = ub
        p[_c] = uc
        _mids.append(int(np.where((SLOT_POS == p).all(1))[0][0]))
    _FACE_MIDS.append(_mids)
FACE_MIDS = np.array(_FACE_MIDS, dtype=np.int64)   # (6, 4) slot ids 8..19


def morton3(x, y, z):
    """Interleave three non-negative int64 arrays (21 bits each)."""
    def spread(v):
        v = v.astype(np.uint64) & np.uint64(0x1FFFFF)
        v = (v | (v << np.uint64(32))) & np.uint64(0x1F00000000FFFF)
        v = (v | (v << np.uint64(16))) & np.uint64(0x1F0000FF0000FF)
        v = (v | (v << np.uint64(8))) & np.uint64(0x100F00F00F00F00F)
        v = (v | (v << np.uint64(4))) & np.uint64(0x10C30C30C30C30C3)
        v = (v | (v << np.uint64(2))) & np.uint64(0x1249249249249249)
        return v
    return spread(x) | (spread(y) << np.uint64(1)) | (spread(z) << np.uint64(2))


# ------------------------------------------------------------------ mesh
@dataclass
class OctreeMesh:
    name: str
    origin: np.ndarray          # (3,) physical position of the forest corner
    h_finest: float             # physical edge of a level-lmax cell
    lmax: int
    level: np.ndarray           # (C,) int8
    anchor: np.ndarray          # (C, 3) int64, finest-grid units
    h: np.ndarray               # (C,) float64 physical edge length
    mask: np.ndarray            # (C,) int32, 12-bit mid-edge mask
    slot_node: np.ndarray       # (C, 26) int32, -1 if absent
    node_xyz: np.ndarray        # (N, 3) float64
    E: np.ndarray               # (C,) Young's modulus
    rho: np.ndarray             # (C,) density
    nu: float                   # Poisson ratio (one value per mesh)
    fixed_nodes: np.ndarray     # nodes with all three DOFs fixed
    sources: list = field(default_factory=list)   # point loads (dicts)
    fixed_dof_list: np.ndarray = None   # further single DOFs held at zero (3 node + d)
    meta: dict = field(default_factory=dict)

    @property
    def n_cells(self):
        return int(self.level.shape[0])

    @property
    def n_nodes(self):
        return int(self.node_xyz.shape[0])

    @property
    def n_dof(self):
        return 3 * self.n_nodes

    def fixed_dofs(self):
        f = np.asarray(self.fixed_nodes, dtype=np.int64)
        extra = np.zeros(0, np.int64) if self.fixed_dof_list is None else \
            np.asarray(self.fixed_dof_list, np.int64)
        return np.unique(np.concatenate([3 * f, 3 * f + 1, 3 * f + 2, extra]))

    def nodes_per_cell(self):
        return (self.slot_node >= 0).sum(1)

    def summary(self):
        return {"name": self.name, "cells": self.n_cells, "nodes": self.n_nodes,
                "dof": self.n_dof, "levels": [int(self.level.min()), int(self.level.max())],
                "mean_nodes_per_cell": float(self.nodes_per_cell().mean()),
                "dof_per_cell": self.n_dof / max(1, self.n_cells)}


def _keys(q_coords, n_axis):
    """Key of level-q cells given integer level-q coordinates (k, 3)."""
    return (q_coords[:, 0] * n_axis[1] + q_coords[:, 1]) * n_axis[2] + q_coords[:, 2]


_DIRS18 = np.array([d for d in np.ndindex(3, 3, 3)
                    if 1 <= sum(abs(v - 1) for v in d) <= 2], dtype=np.int64) - 1


def build_octree(roots, lmin: int, lmax: int,
                 refine: Callable[[int, np.ndarray, float], np.ndarray],
                 h_root: float = 1.0):
    """Balanced octree over a forest of ``roots`` = (nx, ny, nz) root cubes.

    ``refine(q, centres, h_q)`` -> bool array: refine these level-q cells.
    Returns (internal sets per level, leaves (level, level-coords)).
    Levels below ``lmin`` are refined everywhere.  2:1 balance across faces
    and edges is enforced by requiring, for every refined cell X at level
    q >= 1, that the level-(q-1) cells containing X's 18 face/edge
    neighbour positions be refined too (and X's parent).
    """
    roots = np.asarray(roots, dtype=np.int64)
    internal = [np.zeros((0, 3), dtype=np.int64) for _ in range(lmax)]
    # top-down refinement
    cur = np.array([[i, j, k] for i in range(roots[0]) for j in range(roots[1])
                    for k in range(roots[2])], dtype=np.int64)
    for q in range(lmax):
        hq = h_root / 2 ** q
        centres = (cur + 0.5) * hq
        flag = np.ones(len(cur), bool) if q < lmin else np.asarray(refine(q, centres, hq), bool)
        internal[q] = cur[flag]
        kids = (internal[q][:, None, :] * 2 + _CORNER_POS[None, :, :].clip(0, 1)).reshape(-1, 3)
        cur = kids
    # bottom-up balance
    for q in range(lmax - 1, 0, -1):
        X = internal[q]
        if len(X) == 0:
            continue
        nq1 = roots * 2 ** (q - 1)
        need = [X // 2]
        for d in _DIRS18:
            nb = X + d
            nq = roots * 2 ** q
            ok = ((nb >= 0) & (nb < nq)).all(1)
            need.append(nb[ok] // 2)
        need = np.vstack(need + [internal[q - 1]])
        keys = _keys(need, nq1)
        _, idx = np.unique(keys, return_index=True)
        internal[q - 1] = need[idx]
    # leaves
    leaves = []
    all_roots = np.array([[i, j, k] for i in range(roots[0]) for j in range(roots[1])
                          for k in range(roots[2])], dtype=np.int64)
    prev = all_roots
    for q in range(lmax + 1):
        nq = roots * 2 ** q
        if q > 0:
            prev = (internal[q - 1][:, None, :] * 2 + _CORNER_POS[None, :, :].clip(0, 1)).reshape(-1, 3)
        if q < lmax:
            isin = np.isin(_keys(prev, nq), _keys(internal[q], nq))
            leaf = prev[~isin]
        else:
            leaf = prev
        leaves.append(leaf)
    return internal, leaves


def _edge_masks(q, coords, internal_q, roots):
    """12-bit mid-edge masks of level-q leaves: bit e is set when one of the
    three other level-q cells around edge e is refined."""
    nq = roots * 2 ** q
    ikeys = np.sort(_keys(internal_q, nq)) if len(internal_q) else np.zeros(0, np.int64)
    mask = np.zeros(len(coords), dtype=np.int64)
    for e in range(12):
        a, r = divmod(e, 4)
        b, c = [x for x in range(3) if x != a]
        sb, sc = 2 * (r & 1) - 1, 2 * (r >> 1) - 1
        hit = np.zeros(len(coords), bool)
        for db, dc in [(sb, 0), (0, sc), (sb, sc)]:
            d = np.zeros(3, dtype=np.int64)
            d[b] = db
            d[c] = dc
            nb = coords + d
            ok = ((nb >= 0) & (nb < nq)).all(1)
            if len(ikeys):
                k = _keys(np.where(ok[:, None], nb, 0), nq)
                pos = np.searchsorted(ikeys, k)
                pos = np.minimum(pos, len(ikeys) - 1)
                hit |= ok & (ikeys[pos] == k)
        mask |= hit.astype(np.int64) << e
    return mask


def _present_slots(mask):
    """(C, 26) bool: corners always, mid-edges from the mask, face centres
    on faces with 1, 2-adjacent, 3 or 4 mid-edge nodes."""
    C = len(mask)
    pres = np.zeros((C, 26), bool)
    pres[:, :8] = True
    for e in range(12):
        pres[:, 8 + e] = (mask >> e) & 1 == 1
    for f in range(6):
        has = pres[:, FACE_MIDS[f]]
        nh = has.sum(1)
        opposite = (nh == 2) & (has[:, 0] == has[:, 2])
        pres[:, 20 + f] = (nh >= 1) & ~opposite
    return pres


def make_mesh(name, roots, lmin, lmax, refine, h_root=1.0, origin=(0.0, 0.0, 0.0),
              remove: Optional[Callable[[np.ndarray], np.ndarray]] = None):
    roots = np.asarray(roots, dtype=np.int64)
    internal, leaves = build_octree(roots, lmin, lmax, refine, h_root)
    lv, anc, msk = [], [], []
    for q, coords in enumerate(leaves):
        if len(coords) == 0:
            continue
        m = _edge_masks(q, coords, internal[q] if q < lmax else np.zeros((0, 3), np.int64), roots)
        S = 2 ** (lmax - q)
        lv.append(np.full(len(coords), q, dtype=np.int8))
        anc.append(coords * S)
        msk.append(m)
    level = np.concatenate(lv)
    anchor = np.concatenate(anc)
    mask = np.concatenate(msk).astype(np.int32)
    h_finest = h_root / 2 ** lmax
    S = (2 ** (lmax - level.astype(np.int64)))
    h = S * h_finest
    centre = np.asarray(origin) + (anchor + 0.5 * S[:, None]) * h_finest
    if remove is not None:
        keep = ~np.asarray(remove(centre), bool)
        level, anchor, mask, S, h, centre = (level[keep], anchor[keep], mask[keep],
                                             S[keep], h[keep], centre[keep])
    # Morton order of cells
    order = np.argsort(morton3(anchor[:, 0], anchor[:, 1], anchor[:, 2]), kind="stable")
    level, anchor, mask, S, h, centre = (level[order], anchor[order], mask[order],
                                         S[order], h[order], centre[order])
    # node points on the doubled finest grid
    pres = _present_slots(mask)
    pts = (2 * anchor[:, None, :] + (SLOT_POS[None, :, :] + 1) * S[:, None, None])  # (C,26,3)
    mkey = morton3(pts[..., 0].ravel(), pts[..., 1].ravel(), pts[..., 2].ravel()).reshape(pts.shape[:2])
    uk, inv = np.unique(mkey[pres], return_inverse=True)
    slot_node = np.full(pres.shape, -1, dtype=np.int64)
    slot_node[pres] = inv
    node_pts = np.zeros((len(uk), 3), dtype=np.int64)
    node_pts[inv] = pts[pres]
    node_xyz = np.asarray(origin) + node_pts * (0.5 * h_finest)
    C = len(level)
    return OctreeMesh(name=name, origin=np.asarray(origin, float), h_finest=h_finest, lmax=lmax,
                      level=level, anchor=anchor, h=h.astype(np.float64), mask=mask,
                      slot_node=slot_node.astype(np.int32), node_xyz=node_xyz,
                      E=np.ones(C), rho=np.ones(C), nu=0.3,
                      fixed_nodes=np.zeros(0, np.int64))


# --------------------------------------------------------------- loads
def ricker_t1_for_mesh(mesh: OctreeMesh, cells_per_wavelength: float = 10.0):
    """t1 of a Ricker wavelet whose critical frequency f1 = 2.2 / t1 (Sec. 5)
    spans ``cells_per_wavelength`` of the coarsest cells at the slowest shear
    speed v_S = sqrt(E / (2 rho (1 + nu))) (Eq. wavespeed)."""
    vs = np.sqrt(mesh.E.min() / (2 * mesh.rho.max() * (1 + mesh.nu)))
    f1 = vs / (cells_per_wavelength * mesh.h.max())
    return 2.2 / f1


def nearest_node(mesh: OctreeMesh, p):
    d = np.linalg.norm(mesh.node_xyz - np.asarray(p)[None, :], axis=1)
    return int(np.argmin(d))


def point_source(node, direction, t1, P0=1.0, wavelet="ricker", rhs=0, n_cycles=5.0):
    d = np.asarray(direction, float)
    d = d / np.linalg.norm(d)
    return {"node": int(node), "dir": d.tolist(), "t1": float(t1), "P0": float(P0),
            "wavelet": wavelet, "rhs": int(rhs), "n_cycles": float(n_cycles)}


# --------------------------------------------------------------- configs
def config_corner_cube(seed=0, lmin=2, lmax=4, r0=0.65, p=0.15):
    """Unit cube, levels 2-4 refined toward corner 0 plus seeded random flags,
    z = 0 fixed, vertical Ricker point load at the top centre (~1.2k cells)."""
    rng = np.random.default_rng(seed)

    def refine(q, c, hq):
        d = np.linalg.norm(c, axis=1)
        return (d < r0 * (1.0 + 0.5 * (lmax - 1 - q))) | (rng.random(len(c)) < p)

    m = make_mesh("corner_cube_l2-4", (1, 1, 1), lmin, lmax, refine)
    m.fixed_nodes = np.where(np.abs(m.node_xyz[:, 2]) < 1e-12)[0]
    top = nearest_node(m, (0.5, 0.5, 1.0))
    m.sources = [point_source(top, (0, 0, -1), ricker_t1_for_mesh(m))]
    m.meta = {"seed": seed, "recipe": "corner refinement r0=%g p=%g" % (r0, p)}
    return m


def config_cavity_cube(seed=1, lmin=4, lmax=8, radius=0.2, band=0.072, sigma=0.3, p=0.002):
    """Cube minus a ball of radius 0.2 at the centre (staircase), levels 4-8
    refined in a band around the sphere plus seeded random flags with
    probability p per cell and level, E_e lognormal(sigma) per cell
    (~1M cells at the defaults), z = 0 fixed, Ricker at the top centre."""
    ctr = np.array([0.5, 0.5, 0.5])
    frng = np.random.default_rng(seed + 1000)

    def refine(q, c, hq):
        d = np.linalg.norm(c - ctr[None, :], axis=1)
        return (np.abs(d - radius) < band + 0.9 * hq) | (frng.random(len(c)) < p)

    def remove(c):
        return np.linalg.norm(c - ctr[None, :], axis=1) < radius

    m = make_mesh("cavity_cube_l4-8", (1, 1, 1), lmin, lmax, refine, remove=remove)
    rng = np.random.default_rng(seed)
    m.E = np.exp(sigma * rng.standard_normal(m.n_cells))
    m.fixed_nodes = np.where(np.abs(m.node_xyz[:, 2]) < 1e-12)[0]
    top = nearest_node(m, (0.5, 0.5, 1.0))
    m.sources = [point_source(top, (0, 0, -1), ricker_t1_for_mesh(m))]
    m.meta = {"seed": seed, "recipe": "sphere band=%g radius=%g sigma=%g" % (band, radius, sigma)}
    return m


def config_multi_point(seed=2, lmin=3, lmax=7, n_points=8, r0=0.118, n_rhs=64):
    """Cube, levels 3-7, refined around seeded random points (~200k cells);
    ``n_rhs`` load cases with random source node, direction and Ricker
    f1 scaled by U[0.5, 2]."""
    rng = np.random.default_rng(seed)
    pts = rng.random((n_points, 3))

    def refine(q, c, hq):
        d = np.min(np.linalg.norm(c[:, None, :] - pts[None, :, :], axis=2), axis=1)
        return d < r0 + 1.5 * hq

    m = make_mesh("multi_point_cube_l3-7", (1, 1, 1), lmin, lmax, refine)
    m.fixed_nodes = np.where(np.abs(m.node_xyz[:, 2]) < 1e-12)[0]
    free = np.setdiff1d(np.arange(m.n_nodes), m.fixed_nodes)
    t1_ref = ricker_t1_for_mesh(m)
    srcs = []
    for b in range(n_rhs):
        node = int(free[rng.integers(len(free))])
        v = rng.standard_normal(3)
        f_scale = rng.uniform(0.5, 2.0)
        srcs.append(point_source(node, v, t1_ref / f_scale, rhs=b))
    m.sources = srcs
    m.meta = {"seed": seed, "points": pts.tolist(), "n_rhs": n_rhs}
    return m


def _layer_z1(x, y):
    """Lower curved layer interface of the layered trench box."""
    return 2.0 / 3.0 + 0.15 * np.sin(np.pi * x / 2.0) * np.cos(np.pi * y / 2.0)


def _layer_z2(x, y):
    """Upper curved layer interface of the layered trench box."""
    return 4.0 / 3.0 + 0.10 * np.cos(np.pi * x) * np.sin(np.pi * y / 2.0)


def config_layered_trench(seed=3, lmin=5, lmax=10, band=0.02, half_len=1.0, layer_level=8,
                          p=0.002):
    """[0,4] x [0,4] x [0,2] as 2 x 2 x 1 roots of edge 2, levels 5-10:
    refined toward a free-surface trench of finite length (x in [1.9, 2.1],
    y in [1, 3], depth 0.2, removed; refinement by the 3-D distance to it),
    toward two curved layer interfaces (to level 8) and by seeded random
    flags with probability p per cell and level; three layers between the
    curved interfaces with E = 1 : 4 : 16 from top to bottom."""
    rng = np.random.default_rng(seed + 1000)

    def trench(c):
        return ((np.abs(c[:, 0] - 2.0) < 0.1) & (np.abs(c[:, 1] - 2.0) < half_len) &
                (c[:, 2] > 1.8))

    def refine(q, c, hq):
        dx = np.maximum(np.abs(c[:, 0] - 2.0) - 0.1, 0.0)
        dy = np.maximum(np.abs(c[:, 1] - 2.0) - half_len, 0.0)
        dz = np.maximum(1.8 - c[:, 2], 0.0)
        near_t = np.sqrt(dx * dx + dy * dy + dz * dz) < band + 1.2 * hq
        dl = np.minimum(np.abs(c[:, 2] - _layer_z1(c[:, 0], c[:, 1])),
                        np.abs(c[:, 2] - _layer_z2(c[:, 0], c[:, 1])))
        near_l = (dl < 0.9 * hq) & (q < layer_level)
        flags = (rng.random(len(c)) < p) & (q < lmax - 1)
        return near_t | near_l | flags

    m = make_mesh("layered_trench_l5-10", (2, 2, 1), lmin, lmax, refine, h_root=2.0, remove=trench)
    S = 2 ** (m.lmax - m.level.astype(np.int64))
    c = (m.anchor + 0.5 * S[:, None]) * m.h_finest + np.asarray(m.origin)[None, :]
    m.E = np.where(c[:, 2] > _layer_z2(c[:, 0], c[:, 1]), 1.0,
                   np.where(c[:, 2] > _layer_z1(c[:, 0], c[:, 1]), 4.0, 16.0))
    m.fixed_nodes = np.where(np.abs(m.node_xyz[:, 2]) < 1e-12)[0]
    top = nearest_node(m, (1.0, 2.0, 2.0))
    m.sources = [point_source(top, (0, 0, -1), ricker_t1_for_mesh(m))]
    m.meta = {"seed": seed, "layers_E": [1, 4, 16], "trench": "x in [1.9, 2.1], y in [1, 3], z > 1.8",
              "p": p}
    return m


def config_receiver_cube(seed=4, lmin=3, lmax=6, r0=0.5, p=0.15, n_recv_axis=16):
    """Cube, levels 3-6 (~100k cells at full size), 16 x 16 receivers at the
    top-surface nodes nearest to a regular grid; z = 0 fixed, Ricker source
    at the top centre."""
    rng = np.random.default_rng(seed)

    def refine(q, c, hq):
        d = np.linalg.norm(c - np.array([0.5, 0.5, 1.0])[None, :], axis=1)
        return (d < r0 + 2.0 * hq) | (rng.random(len(c)) < p)

    m = make_mesh("receiver_cube_l3-6", (1, 1, 1), lmin, lmax, refine)
    m.fixed_nodes = np.where(np.abs(m.node_xyz[:, 2]) < 1e-12)[0]
    top = nearest_node(m, (0.5, 0.5, 1.0))
    m.sources = [point_source(top, (0, 0, -1), ricker_t1_for_mesh(m))]
    g = (np.arange(n_recv_axis) + 0.5) / n_recv_axis
    rec = sorted({nearest_node(m, (x, y, 1.0)) for x in g for y in g})
    m.meta = {"seed": seed, "receivers": rec}
    return m


def small_uniform(n=2, lmax=None, h=1.0):
    """n x n x n uniform cells of edge h (no hanging nodes): level log2(n)."""
    L = int(round(np.log2(n)))
    return make_mesh("uniform_%d" % n, (1, 1, 1), L, L, lambda q, c, hq: np.zeros(len(c), bool),
                     h_root=h * n)


def tiny_refined(seed=0, lmax=2, p=0.3):
    """A 2-level cube with random refinement: a few dozen cells with hanging
    nodes of many patterns (for brute-force checks)."""
    rng = np.random.default_rng(seed)
    return make_mesh("tiny_refined_%d" % seed, (1, 1, 1), 1, lmax,
                     lambda q, c, hq: rng.random(len(c)) < p)


def cube_roller(n=8, L=8.0, E=1000.0, refine_p=0.0, seed=0):
    """[0, L]^3 cube of n^3 cells (n a power of two), E, nu = 0.3, rho = 1,
    roller supports on all six faces (the normal DOF of every face node held
    at zero), no load: the eigenfrequency benchmark of the paper's cube
    example.  refine_p > 0 refines a seeded random share of the cells once
    more (2:1-balanced, so hanging-node patterns appear)."""
    lv = int(round(np.log2(n)))
    rng = np.random.default_rng(seed)
    lmax = lv + (1 if refine_p > 0 else 0)
    m = make_mesh("cube_roller_%d_p%g" % (n, refine_p), (1, 1, 1), lv, lmax,
                  lambda q, c, hq: (rng.random(len(c)) < refine_p) if q == lv else np.zeros(len(c), bool),
                  h_root=L)
    m.E = np.full(m.n_cells, float(E))
    x = m.node_xyz
    tol = 1e-9 * L
    dofs = [3 * np.nonzero((np.abs(x[:, d]) < tol) | (np.abs(x[:, d] - L) < tol))[0] + d
            for d in range(3)]
    m.fixed_dof_list = np.sort(np.concatenate(dofs)).astype(np.int64)
    m.sources = []
    return m


CONFIGS = {
    "corner_cube": config_corner_cube,
    "cavity_cube": config_cavity_cube,
    "multi_point": config_multi_point,
    "layered_trench": config_layered_trench,
    "receiver_cube": config_receiver_cube,
}
