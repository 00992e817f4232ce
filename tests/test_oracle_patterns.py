"""Pins of the oracle's pattern machinery (Sec. 3.2.1-3.2.2) against the paper."""
import itertools

import numpy as np
import pytest

from oracle import cube
from conftest import golden

G = golden("paper_values.json")


def test_generators_reproduce_printed_Q1_Q2():
    # Fig. OctTrans (c), (f): Q1 = T_x T_z and Q2 = R_x as printed.
    assert (cube.T_X @ cube.T_Z == np.array(G["Q1_TxTz"]["value"])).all()
    assert (cube.R_X == np.array(G["Q2_Rx"]["value"])).all()


def test_48_ops_are_the_group_generated_by_rotations_and_mirrors():
    ops = {tuple(Q.ravel()) for Q in cube.all_ops()}
    assert len(ops) == G["n_transforms"]["value"]
    # closure of {T_x, T_y, T_z, R_x, R_y, R_z} under multiplication
    gens = [cube.T_X, cube.T_Y, cube.T_Z, cube.R_X, cube.R_Y, cube.R_Z]
    group = {tuple(np.eye(3, dtype=int).ravel())}
    frontier = list(group)
    while frontier:
        nxt = []
        for g in frontier:
            Gm = np.array(g).reshape(3, 3)
            for h in gens:
                k = tuple((Gm @ h).ravel())
                if k not in group:
                    group.add(k)
                    nxt.append(k)
        frontier = nxt
    assert group == ops


def test_slot_permutations_are_bijections_preserving_slot_type():
    for op in range(48):
        pi = cube.slot_perm(op)
        assert sorted(pi) == list(range(26))
        for s in range(26):
            kind = 0 if s < 8 else (1 if s < 20 else 2)
            kind2 = 0 if pi[s] < 8 else (1 if pi[s] < 20 else 2)
            assert kind == kind2


def test_144_unique_patterns():
    assert len(cube.unique_patterns()) == G["n_unique_patterns"]["value"]


def test_burnside_count_independent_of_orbit_enumeration():
    # Burnside: #orbits = (1/|G|) sum_g 2^(cycles of g on the 12 edges).
    total = 0
    for op in range(48):
        pi = cube.slot_perm(op)
        seen, cycles = set(), 0
        for e in range(8, 20):
            if e in seen:
                continue
            cycles += 1
            x = e
            while x not in seen:
                seen.add(x)
                x = pi[x]
        total += 2 ** cycles
    assert total % 48 == 0 and total // 48 == G["n_unique_patterns"]["value"]


def test_canonical_op_maps_mask_onto_orbit_minimum():
    canon, opof = cube.canonical_table()
    rng = np.random.default_rng(0)
    for mask in rng.integers(0, 4096, 300):
        orbit = {cube.apply_op_to_mask(op, int(mask)) for op in range(48)}
        assert canon[mask] == min(orbit)
        assert cube.apply_op_to_mask(int(opof[mask]), int(mask)) == canon[mask]


def test_node_counts_match_paper():
    lo, hi = G["nodes_per_cell_range"]["value"]
    counts = {len(cube.present_slots(m)) for m in range(4096)}
    assert min(counts) == lo and max(counts) == hi
    for n in G["lumped_mass_figure_node_counts"]["value"]:
        assert n in counts
    # one hanging edge: 8 corners + 1 mid-edge + 2 face centres = 11 nodes
    assert len(cube.present_slots(1)) == 11


def test_face_elements_tile_each_face_exactly():
    # areas of the surface elements of every face sum to the face area (4 on
    # the doubled cube), and every present slot is used by some element
    for mask in [0, 1, 3, 5, 0x0F0, 0xFFF, 0b101010101010, 0b110011001100]:
        used = set()
        area = np.zeros(6)
        for el in cube.face_elements(mask):
            P = cube.SLOT_POS[el].astype(float)
            a = 0.0
            for i in range(1, len(el) - 1):
                a += 0.5 * np.linalg.norm(np.cross(P[i] - P[0], P[i + 1] - P[0]))
            axis = [a for a in range(3) if np.ptp(P[:, a]) == 0][0]
            side = int(P[0, axis] > 0)
            area[2 * axis + side] += a
            used.update(el)
        assert np.allclose(area, 4.0)
        assert used == set(cube.present_slots(mask))
