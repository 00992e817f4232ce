"""Invariance of the pattern matrices under the symmetries of their node sets.

A cube symmetry Q (one of the 48 signed permutations of Sec. 3.2.2) that
maps a pattern's set of mid-edge nodes onto itself maps the cell onto
itself, so the cell's stiffness and mass commute with the action of Q on
the cell's DOFs: with (P u) at the image slot of s equal to Q u_s,
P K P^T = K and P M P^T = M.  The check is geometric (node positions,
face triangulation, quadrature orientation and the elasticity matrix must
all respect the symmetry) and independent of how K was computed; an
anisotropy slipped into any of them, a mis-placed node or a face solved
with the wrong orientation breaks it.  Checked separately for the oracle's
pattern library and for the product's.
"""
import numpy as np
import pytest

from oracle import cube, sbfem
from paper_2103_09100_gb300 import patterns

# the 8-node cell, the 26-node cell, and patterns with large, small and
# trivial stabilisers (one, two, four and six mid-edge nodes)
MASKS = [0, 0xFFF, 0x001, 0x003, 0x005, 0x00F, 0x0F0, 0x111, 0x3C3, 0x555, 0x6A9]


def _oracle_action(mask, op):
    slots = cube.present_slots(mask)
    idx = {s: i for i, s in enumerate(slots)}
    pi = cube.slot_perm(op)
    Q = cube.all_ops()[op].astype(float)
    m = 3 * len(slots)
    P = np.zeros((m, m))
    for i, s in enumerate(slots):
        j = idx[pi[s]]
        P[3 * j:3 * j + 3, 3 * i:3 * i + 3] = Q
    return P


def _stabiliser(mask):
    return [op for op in range(48) if cube.apply_op_to_mask(op, mask) == mask]


@pytest.mark.parametrize("mask", MASKS)
def test_oracle_matrices_commute_with_stabiliser(mask):
    stab = _stabiliser(mask)
    # orbit-stabiliser: |orbit| |stab| = 48
    orbit = {cube.apply_op_to_mask(op, mask) for op in range(48)}
    assert len(orbit) * len(stab) == 48
    c = sbfem.solve_cell(mask)
    kmax, mmax = np.abs(c.K).max(), np.abs(c.M).max()
    for op in stab:
        P = _oracle_action(mask, op)
        assert np.allclose(P @ P.T, np.eye(len(P)))
        assert np.abs(P @ c.K @ P.T - c.K).max() < 1e-12 * kmax, (mask, op)
        assert np.abs(P @ c.M @ P.T - c.M).max() < 1e-12 * mmax, (mask, op)
        # the lumped mass is diagonal with equal entries on the three
        # components of a node only up to the symmetry: it is carried onto
        # itself by |P|
        assert np.abs(np.abs(P) @ c.M_lump - c.M_lump).max() < 1e-13, (mask, op)


def test_oracle_full_group_for_8_and_26_node_cells():
    assert len(_stabiliser(0)) == 48 and len(_stabiliser(0xFFF)) == 48


def _product_action(mask, op):
    slots = patterns.present(mask)
    idx = {s: i for i, s in enumerate(slots)}
    sm = patterns._slot_map(op)
    Q = patterns.op_matrix(op)
    m = 3 * len(slots)
    P = np.zeros((m, m))
    for i, s in enumerate(slots):
        j = idx[int(sm[s])]
        P[3 * j:3 * j + 3, 3 * i:3 * i + 3] = Q
    return P


def test_product_masters_commute_with_stabiliser():
    img = patterns._mask_images()
    masters = sorted({int(x) for x in patterns.classification_table()[0]})
    assert len(masters) == 144
    rng = np.random.default_rng(5)
    chosen = sorted(set(rng.choice(masters, 16, replace=False).tolist())
                    | {masters[0], masters[-1]})
    n_ops = 0
    for mk in chosen:
        stab = [op for op in range(48) if img[op, mk] == mk]
        assert 48 % len(stab) == 0
        _, K, lump, _ = patterns.master_matrices(mk)
        kmax = np.abs(K).max()
        for op in stab:
            P = _product_action(mk, op)
            assert np.abs(P @ K @ P.T - K).max() < 1e-12 * kmax, (mk, op)
            assert np.abs(np.abs(P) @ lump - lump).max() < 1e-13, (mk, op)
            n_ops += 1
    assert n_ops > len(chosen)
