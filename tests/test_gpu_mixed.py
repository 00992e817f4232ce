"""GPU parity of the mixed-precision (TF32x3 tensor-core) step against the
FP64 oracle.  Bar: relative L2 error <= 1e-5 (after 2000 steps on the corner
cube; after 200 steps on the full cavity mesh)."""
import numpy as np
import pytest

import octree_gen as og
from oracle import cdm
from paper_2103_09100_gb300 import Solver, _lib as L, build
from parity import rel

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    build.build()
    L.load()




@pytest.mark.parametrize("seed", [0, 1, 2])
def test_mixed_single_force(seed):
    m = og.tiny_refined(seed, p=0.35)
    m.E = np.exp(0.3 * np.random.default_rng(seed).standard_normal(m.n_cells))
    P = cdm.make_problem(m)
    u0 = np.random.default_rng(seed).standard_normal(m.n_dof)
    S = Solver.from_mesh(m, precision="mixed", dt=P.dt)
    S.initial(u0)
    S.step(1)
    f = S.field(L.SBX_F_INT)
    ref = cdm.apply_K(P, u0) - cdm.external_force(P, 0)
    assert rel(f, ref) < 1e-5


def test_mixed_corner_cube_2000_steps():
    m = og.config_corner_cube()
    P = cdm.make_problem(m)
    S = Solver.from_mesh(m, precision="mixed", dt=P.dt)
    u, up = cdm.initial_state(P)
    S.initial()
    worst = 0.0
    for k in range(20):
        u, up, _, _ = cdm.run(P, 100, u, up, n0=100 * k, threads=4)
        S.step(100)
        worst = max(worst, rel(S.field(L.SBX_U_N), u))
    print("corner cube mixed max rel error over 2000 steps: %.3e" % worst)
    assert worst < 1e-5


def test_mixed_full_size_cavity_200_steps():
    m = og.config_cavity_cube()
    P = cdm.make_problem(m)
    S = Solver.from_mesh(m, precision="mixed", dt=P.dt)
    u0 = np.random.default_rng(3).standard_normal(m.n_dof) * 1e-3
    u0[P.fixed] = 0
    u, up = cdm.initial_state(P, u0)
    S.initial(u0)
    S.step(1)
    f = S.field(L.SBX_F_INT)
    ref = cdm.apply_K(P, u0) - cdm.external_force(P, 0)
    assert rel(f, ref) < 1e-5
    S.initial(u0)
    S.step(200)
    u, up, _, _ = cdm.run(P, 200, u, up, threads=16)
    e = rel(S.field(L.SBX_U_N), u)
    print("cavity mixed 200-step rel error %.3e" % e)
    assert e < 1e-5


def test_mixed_receiver_cube_force_and_100_steps():
    # ~100k cells: full 128-cell tiles of the 8-node cell (the unrolled
    # path) with a ragged last tile, and the general path for the rest
    m = og.config_receiver_cube()
    P = cdm.make_problem(m)
    S = Solver.from_mesh(m, precision="mixed", dt=P.dt)
    u0 = np.random.default_rng(5).standard_normal(m.n_dof)
    u0[P.fixed] = 0
    S.initial(u0)
    S.step(1)
    ref = cdm.apply_K(P, u0) - cdm.external_force(P, 0)
    assert rel(S.field(L.SBX_F_INT), ref) < 1e-5
    u, up = cdm.initial_state(P, u0)
    S.initial(u0)
    S.step(100)
    u, up, _, _ = cdm.run(P, 100, u, up, threads=16)
    e = rel(S.field(L.SBX_U_N), u)
    print("receiver cube mixed 100-step rel error %.3e" % e)
    assert e < 1e-5


@pytest.mark.parametrize("n", [16, 32])
def test_mixed_uniform_bricks(n):
    # n^3 uniform cells: every cell in a complete 4 x 4 x 8 brick tile
    m = og.small_uniform(n)
    m.E = np.exp(0.3 * np.random.default_rng(n).standard_normal(m.n_cells))
    m.fixed_nodes = np.where(np.abs(m.node_xyz[:, 2]) < 1e-12)[0]
    P = cdm.make_problem(m)
    S = Solver.from_mesh(m, precision="mixed", dt=P.dt)
    assert L.sbx_query(S.ctx, L.SBX_Q_BRICK_TILES) == n ** 3 // 128
    u0 = np.random.default_rng(n + 1).standard_normal(m.n_dof)
    u0[P.fixed] = 0
    S.initial(u0)
    S.step(1)
    ref = cdm.apply_K(P, u0) - cdm.external_force(P, 0)
    assert rel(S.field(L.SBX_F_INT), ref) < 1e-5
    u, up = cdm.initial_state(P, u0)
    S.initial(u0)
    S.step(100)
    u, up, _, _ = cdm.run(P, 100, u, up, threads=16)
    assert rel(S.field(L.SBX_U_N), u) < 1e-5


def test_mixed_brick_and_list_tiles_cavity_counts():
    m = og.config_receiver_cube()
    S = Solver.from_mesh(m, precision="mixed")
    nb = L.sbx_query(S.ctx, L.SBX_Q_BRICK_TILES)
    print("receiver cube: %d brick tiles of %d tensor-core + SIMT tiles" % (nb, L.sbx_query(S.ctx, L.SBX_Q_TILES)))
    assert nb > 0


def _mixed_vs_oracle(m, n_steps, alpha=0.0, u0=None, v0=None, threads=4):
    P = cdm.make_problem(m, alpha=alpha)
    S = Solver.from_mesh(m, precision="mixed", dt=P.dt, alpha=alpha)
    S.initial(u0, v0)
    S.step(n_steps)
    u, up = cdm.initial_state(P, u0, v0)
    u, up, _, _ = cdm.run(P, n_steps, u, up, threads=threads)
    e = (rel(S.field(L.SBX_U_N), u), rel(S.field(L.SBX_U_NM1), up))
    S.close()
    return e


def test_mixed_single_cell_no_loads():
    m = og.small_uniform(1)
    m.sources = []
    u0 = np.random.default_rng(21).standard_normal(m.n_dof)
    e = _mixed_vs_oracle(m, 40, u0=u0, threads=1)
    assert max(e) < 1e-5, e


def test_mixed_damped_with_initial_velocity():
    # damped update (alpha > 0) and the Eq. D0 start with U_0, V_0 != 0
    m = og.config_corner_cube()
    rng = np.random.default_rng(22)
    u0 = rng.standard_normal(m.n_dof) * 1e-3
    v0 = rng.standard_normal(m.n_dof) * 1e-3
    e = _mixed_vs_oracle(m, 300, alpha=0.3, u0=u0, v0=v0)
    print("corner cube mixed, alpha 0.3, U_0 and V_0 given, 300 steps: %.3e %.3e" % e)
    assert max(e) < 1e-5, e


@pytest.mark.parametrize("n_steps", [1, 31, 32, 33, 65])
def test_mixed_split_step_and_graphs_agree(n_steps):
    # step_n (graph replay for runs of 32) = sbx_force + sbx_update per step,
    # bit for bit up to the reduction order of the atomics
    m = og.config_corner_cube()
    A = Solver.from_mesh(m, precision="mixed")
    B = Solver.from_mesh(m, precision="mixed", dt=A.dt)
    A.initial()
    B.initial()
    A.step(n_steps)
    for _ in range(n_steps):
        L.sbx_force(B.ctx, B.dt)
        L.sbx_update(B.ctx, B.dt)
    ua, ub = A.field(), B.field()
    assert rel(ub, ua) < 1e-6
    assert L.sbx_get_step(A.ctx) == L.sbx_get_step(B.ctx) == n_steps
