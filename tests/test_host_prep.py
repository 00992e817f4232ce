"""Host-side set-up of the GPU library, checked on the CPU.

The product's classification (master, op, node order) and pattern matrices
are fed through a plain numpy restatement of what the force kernel computes
under the C ABI's conventions (u_m[r] = (-1)^{bit r} u[perm[r]] per node,
f = s_e T^T K_p u_m), and compared with the FP64 oracle's R_int.
"""
import ctypes
import itertools
import os

import numpy as np
import pytest

import octree_gen as og
from oracle import cdm
from paper_2103_09100_gb300 import patterns, _lib

PERMS = list(itertools.permutations(range(3)))


def emulate_force(slot_node, mask, h, E, nu, u):
    masters, cp, cs, ptr, nodes = patterns.classify_mesh(slot_node, mask)
    nn, K, Ml, _ = patterns.pattern_arrays(masters, nu)
    koff = np.concatenate([[0], np.cumsum(9 * nn.astype(np.int64) ** 2)])
    f = np.zeros_like(u)
    for e in range(len(cp)):
        p = cp[e]
        m = 3 * nn[p]
        Kp = K[koff[p]:koff[p + 1]].reshape(m, m)
        op = int(cs[e])
        perm = PERMS[op >> 3]
        sgn = np.array([-1.0 if (op >> r) & 1 else 1.0 for r in range(3)])
        nd = nodes[ptr[e]:ptr[e + 1]]
        ue = u.reshape(-1, 3)[nd][:, list(perm)] * sgn[None, :]
        fm = (E[e] * h[e]) * (Kp @ ue.ravel())
        fm = fm.reshape(-1, 3) * sgn[None, :]
        fc = np.zeros_like(fm)
        fc[:, list(perm)] = fm
        np.add.at(f.reshape(-1, 3), nd, fc)
    return f


@pytest.mark.parametrize("seed", [0, 1])
def test_product_setup_reproduces_oracle_force(seed):
    m = og.tiny_refined(seed, p=0.35)
    rng = np.random.default_rng(seed)
    m.E = np.exp(0.3 * rng.standard_normal(m.n_cells))
    P = cdm.make_problem(m, dt=0.01)
    u = rng.standard_normal(m.n_dof)
    f_or = cdm.apply_K(P, u)
    f_pr = emulate_force(m.slot_node, m.mask, m.h, m.E, m.nu, u)
    assert np.abs(f_pr - f_or).max() < 1e-13 * np.abs(f_or).max()


def test_corner_cube_force_and_mass():
    m = og.config_corner_cube()
    u = np.random.default_rng(3).standard_normal(m.n_dof)
    P = cdm.make_problem(m)
    f_or = cdm.apply_K(P, u)
    f_pr = emulate_force(m.slot_node, m.mask, m.h, m.E, m.nu, u)
    assert np.abs(f_pr - f_or).max() < 1e-13 * np.abs(f_or).max()


def test_product_patterns_match_oracle_all_144():
    from oracle import cube, sbfem
    master, op = patterns.classification_table()
    assert len(set(master.tolist())) == 144
    for p in sorted(set(master.tolist()))[::7]:
        slots, K, lump, dt = patterns.master_matrices(int(p))
        c = sbfem.master_cell(int(p))
        assert list(slots) == c.slots
        assert np.abs(K - c.K).max() < 1e-12 * np.abs(c.K).max()
        assert np.abs(lump - c.M_lump).max() < 1e-13
        assert abs(dt - sbfem.critical_dt(c.K, c.M_lump)) < 1e-12


def test_library_exports_every_declared_symbol():
    # the C-ABI library loads without a GPU and exports what include/sbx.h declares
    from paper_2103_09100_gb300 import build
    path = build.build()
    lib = ctypes.CDLL(path)
    hdr = open(os.path.join(os.path.dirname(__file__), "..", "include", "sbx.h")).read()
    import re
    declared = set(re.findall(r"^(?:int|const char \*)\s*(\w+)\(", hdr, re.M))
    assert declared == set(_lib.EXPORTS)
    for name in declared:
        assert hasattr(lib, name), name
