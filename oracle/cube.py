"""Reference octree cell, its 48 symmetry transforms and the 144 unique patterns.

Part of the FP64 oracle (test infrastructure; see ``oracle/__init__``).

Node slots of a cubic octree cell (Sec. 3.2.1, Fig. Octree_cell: corner,
mid-edge and centre nodes).  Positions are given on the doubled integer
cube [-1, 1]^3 so that every slot has integer coordinates:

* corners  0..7  : c = i + 2 j + 4 k,  position (2i-1, 2j-1, 2k-1)
* mid-edges 8..19: e = 4 a + r for an edge parallel to axis a; with (b, c) the
                   other two axes in increasing order, position[a] = 0,
                   position[b] = 2 (r & 1) - 1, position[c] = 2 (r >> 1) - 1
* face centres 20..25: f = 2 a + side, position[a] = 2 side - 1, others 0

This slot order is the octree mesh format's; the oracle derives every
position from the rule above on its own.

A hanging-node pattern is the 12-bit mask of present mid-edge nodes
(bit e <-> slot 8 + e); there are 2^12 = 4096 of them (Sec. 3.2.1).

Transforms (Sec. 3.2.2, Eqs. Rotate and Reflect): every product of the 90
degree rotations T_x, T_y, T_z and the mirrors R_x, R_y, R_z is a 3x3 matrix
with exactly one entry +-1 in each row and column; there are
3 x 2 x 1 x 2^3 = 48 of them.  They are enumerated here as
``op = 8 * perm_index + sign_bits`` with the permutations of (0, 1, 2) in
lexicographic order and sign bit r negating row r:  Q[r, perm[r]] = +-1.

Reading (Sec. 3.2.2 does not fix it): the canonical representative of an
orbit is its numerically smallest mask, and the transform of a cell is the
lowest-numbered op that maps its mask onto the canonical one.
"""
from __future__ import annotations

import itertools
from functools import lru_cache

import numpy as np

N_SLOTS = 26
N_CORNER, N_EDGE, N_FACE = 8, 12, 6


def slot_position(s: int) -> tuple[int, int, int]:
    """Doubled integer position of node slot ``s`` (see module docstring)."""
    if s < 8:
        return (2 * (s & 1) - 1, 2 * ((s >> 1) & 1) - 1, 2 * ((s >> 2) & 1) - 1)
    if s < 20:
        e = s - 8
        a, r = divmod(e, 4)
        b, c = [x for x in range(3) if x != a]
        p = [0, 0, 0]
        p[b] = 2 * (r & 1) - 1
        p[c] = 2 * (r >> 1) - 1
        return tuple(p)
    f = s - 20
    a, side = divmod(f, 2)
    p = [0, 0, 0]
    p[a] = 2 * side - 1
    return tuple(p)


SLOT_POS = np.array([slot_position(s) for s in range(N_SLOTS)], dtype=np.int64)
_POS_TO_SLOT = {tuple(p): s for s, p in enumerate(SLOT_POS.tolist())}


def pos_to_slot(p) -> int:
    return _POS_TO_SLOT[tuple(int(v) for v in p)]


# ---------------------------------------------------------------- transforms
# The generators of Eqs. (Rotate) and (Reflect), kept to show that the 48
# signed permutations are exactly the group they generate (a test checks it).
T_X = np.array([[1, 0, 0], [0, 0, 1], [0, -1, 0]])
T_Y = np.array([[0, 0, 1], [0, 1, 0], [-1, 0, 0]])
T_Z = np.array([[0, 1, 0], [-1, 0, 0], [0, 0, 1]])
R_X = np.diag([-1, 1, 1])
R_Y = np.diag([1, -1, 1])
R_Z = np.diag([1, 1, -1])


@lru_cache(maxsize=None)
def all_ops() -> tuple[np.ndarray, ...]:
    """The 48 signed permutation matrices in the fixed enumeration order."""
    ops = []
    for perm in itertools.permutations(range(3)):
        for bits in range(8):
            Q = np.zeros((3, 3), dtype=np.int64)
            for r in range(3):
                Q[r, perm[r]] = -1 if (bits >> r) & 1 else 1
            ops.append(Q)
    return tuple(ops)


@lru_cache(maxsize=None)
def slot_perm(op: int) -> tuple[int, ...]:
    """pi_g: the slot that slot s is carried to by x -> Q x."""
    Q = all_ops()[op]
    return tuple(pos_to_slot(Q @ SLOT_POS[s]) for s in range(N_SLOTS))


def apply_op_to_mask(op: int, mask: int) -> int:
    pi = slot_perm(op)
    out = 0
    for e in range(N_EDGE):
        if (mask >> e) & 1:
            out |= 1 << (pi[8 + e] - 8)
    return out


@lru_cache(maxsize=None)
def canonical_table() -> tuple[np.ndarray, np.ndarray]:
    """For all 4096 masks: (canonical mask, lowest op mapping mask onto it)."""
    canon = np.zeros(4096, dtype=np.int64)
    opof = np.zeros(4096, dtype=np.int64)
    for mask in range(4096):
        best, best_op = None, None
        for op in range(48):
            m2 = apply_op_to_mask(op, mask)
            if best is None or m2 < best:
                best, best_op = m2, op
        canon[mask] = best
        opof[mask] = best_op
    return canon, opof


def unique_patterns() -> list[int]:
    canon, _ = canonical_table()
    return sorted(set(canon.tolist()))


# -------------------------------------------------------- face discretisation
def face_slots(f: int):
    """(corner slots in cyclic order, mid slots between them, centre slot).

    The face with normal axis a lies in the plane spanned by (b, c); its
    boundary is walked (-,-) -> (+,-) -> (+,+) -> (-,+) in (b, c), with the
    mid-edge slot of each side between its two corners.
    """
    a, side = divmod(f, 2)
    b, c = [x for x in range(3) if x != a]

    def at(ub, uc):
        p = [0, 0, 0]
        p[a] = 2 * side - 1
        p[b] = ub
        p[c] = uc
        return pos_to_slot(p)

    corners = [at(-1, -1), at(1, -1), at(1, 1), at(-1, 1)]
    mids = [at(0, -1), at(1, 0), at(0, 1), at(-1, 0)]
    return corners, mids, at(0, 0)


def present_slots(mask: int) -> list[int]:
    """Slots present in a cell with mid-edge mask ``mask``.

    Reading of Sec. 3.2.1 / Fig. OctreeDist (the figure is missing): a face
    gets a centre node whenever it carries 1, 2 adjacent, 3 or 4 mid-edge
    nodes; a face with none or with 2 nodes on opposite edges has no centre.
    """
    slots = list(range(8)) + [8 + e for e in range(12) if (mask >> e) & 1]
    for f in range(6):
        _, mids, centre = face_slots(f)
        has = [((mask >> (m - 8)) & 1) == 1 for m in mids]
        nh = sum(has)
        opposite = nh == 2 and has[0] == has[2]
        if nh >= 1 and not opposite:
            slots.append(centre)
    return sorted(slots)


def face_elements(mask: int) -> list[list[int]]:
    """Surface elements of the cell boundary as lists of slots (cyclic order).

    Sec. 3.2.1: faces are polygons discretised into rectangles and isosceles
    triangles.  n_h = 0: one square.  n_h = 2 on opposite edges: two 1 x 1/2
    rectangles.  n_h = 4: four 1/2 x 1/2 squares around the centre.
    n_h = 1, 2 adjacent, 3: a fan of isosceles right triangles from the face
    centre to consecutive boundary nodes.  Orientation is fixed later so
    that every element sees the scaling centre on its inner side.
    """
    elems = []
    for f in range(6):
        corners, mids, centre = face_slots(f)
        has = [((mask >> (m - 8)) & 1) == 1 for m in mids]
        nh = sum(has)
        if nh == 0:
            elems.append(list(corners))
        elif nh == 4:
            for i in range(4):
                elems.append([corners[i], mids[i], centre, mids[(i + 3) % 4]])
        elif nh == 2 and has[0] == has[2]:
            if has[0]:   # mids on sides 0 and 2: split across side 0 / side 2
                elems.append([corners[0], mids[0], mids[2], corners[3]])
                elems.append([mids[0], corners[1], corners[2], mids[2]])
            else:        # mids on sides 1 and 3
                elems.append([corners[0], corners[1], mids[1], mids[3]])
                elems.append([mids[3], mids[1], corners[2], corners[3]])
        else:
            ring = []
            for i in range(4):
                ring.append(corners[i])
                if has[i]:
                    ring.append(mids[i])
            for i in range(len(ring)):
                elems.append([ring[i], ring[(i + 1) % len(ring)], centre])
    return elems
