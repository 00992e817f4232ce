"""Pins of the oracle's assembly (Eqs. Rinte, KM_scale; Sec. 3.2.2) on tiny
meshes against brute force and mesh-level invariants."""
import numpy as np
import pytest

import octree_gen as og
from oracle import assembly, cdm


@pytest.fixture(scope="module", params=[0, 1, 2])
def tiny(request):
    m = og.tiny_refined(request.param)
    rng = np.random.default_rng(request.param)
    m.E = np.exp(0.3 * rng.standard_normal(m.n_cells))
    return m


def test_mesh_slots_follow_face_rule(tiny):
    assert assembly.check_mesh_slots(tiny)


def test_ebe_sum_equals_bruteforce_global_K(tiny):
    P = cdm.make_problem(tiny, dt=0.01)
    K = assembly.global_K_bruteforce(tiny)
    rng = np.random.default_rng(5)
    for _ in range(3):
        u = rng.standard_normal(tiny.n_dof)
        f_ebe = cdm.apply_K(P, u)
        f_bf = K @ u
        assert np.abs(f_ebe - f_bf).max() < 1e-13 * np.abs(f_bf).max()


def test_global_K_symmetric_six_rigid_modes(tiny):
    K = assembly.global_K_bruteforce(tiny).toarray()
    assert np.abs(K - K.T).max() < 1e-13 * np.abs(K).max()
    ev = np.linalg.eigvalsh(K)
    assert np.sum(np.abs(ev) < 1e-10 * ev.max()) == 6


def test_global_patch_test_interior_nodes(tiny):
    # a linear displacement field gives zero force at every interior node,
    # hanging and face-centre nodes included (conformity across faces)
    m = tiny
    m.E[:] = 1.0
    K = assembly.global_K_bruteforce(m)
    x = m.node_xyz
    A = np.random.default_rng(2).standard_normal((3, 3))
    f = (K @ (x @ A.T).ravel()).reshape(-1, 3)
    bnd = np.any((np.abs(x) < 1e-12) | (np.abs(x - 1) < 1e-12), axis=1)
    assert (~bnd).sum() > 0
    assert np.abs(f[~bnd]).max() < 1e-12 * np.abs(f[bnd]).max()


def test_lumped_mass_total_is_rho_volume():
    m = og.config_corner_cube()
    m.rho = 1.0 + np.random.default_rng(0).random(m.n_cells)
    M = assembly.lumped_mass(m)
    mass = np.sum(m.rho * m.h ** 3)
    for d in range(3):
        assert abs(M[d::3].sum() - mass) < 1e-12 * mass
    assert (M > 0).all()


def test_dt_cr_scaling_and_bound():
    # Eq. (tcr_scale) + Eq. (tcr): dt = min_e sqrt(rho/E) h dt_cr(p); with a
    # lumped mass the element bound is safe: 2/omega_max(global) >= dt_cr
    m = og.tiny_refined(1)
    m.E = np.exp(0.3 * np.random.default_rng(1).standard_normal(m.n_cells))
    dt = assembly.critical_dt(m)
    K = assembly.global_K_bruteforce(m).toarray()
    M = assembly.lumped_mass(m)
    d = 1 / np.sqrt(M)
    wmax = np.sqrt(np.linalg.eigvalsh(d[:, None] * K * d[None, :]).max())
    assert 2.0 / wmax >= dt * (1 - 1e-12)


def test_cavity_removal_keeps_conformity():
    # staircase removal (cells dropped after balancing): patch test still holds
    ctr = np.array([0.5, 0.5, 0.5])
    rng = np.random.default_rng(4)
    m = og.make_mesh("cav", (1, 1, 1), 1, 3,
                     lambda q, c, hq: (np.abs(np.linalg.norm(c - ctr, axis=1) - 0.25) < 0.2)
                     & (rng.random(len(c)) < 0.8),
                     remove=lambda c: np.linalg.norm(c - ctr, axis=1) < 0.25)
    assert assembly.check_mesh_slots(m)
    K = assembly.global_K_bruteforce(m)
    x = m.node_xyz
    A = np.random.default_rng(2).standard_normal((3, 3))
    f = (K @ (x @ A.T).ravel()).reshape(-1, 3)
    # interior <=> away from the outer cube and not on a removed-cell face
    on_outer = np.any((np.abs(x) < 1e-12) | (np.abs(x - 1) < 1e-12), axis=1)
    r = np.linalg.norm(x - ctr, axis=1)
    interior = ~on_outer & (r > 0.25 + 0.3)
    assert interior.sum() > 0
    assert np.abs(f[interior]).max() < 1e-12 * np.abs(f).max()
