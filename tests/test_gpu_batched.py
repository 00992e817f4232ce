"""GPU parity of the batched form (B load cases per launch, field layout
[node][3][B]) against the FP64 oracle run separately for each load case.
Bars: FP64 batched 1e-12; FP32-contraction batched 1e-5 (relative L2 per
load case, max over cases)."""
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


def _with_sources(m, B, seed, t1_scale=4.0):
    rng = np.random.default_rng(seed)
    free = np.setdiff1d(np.arange(m.n_nodes), m.fixed_nodes)
    t1 = og.ricker_t1_for_mesh(m, t1_scale)
    m.sources = [og.point_source(int(free[rng.integers(len(free))]), rng.standard_normal(3),
                                 t1 / rng.uniform(0.5, 2.0), rhs=b) for b in range(B)]
    return m


def _compare(m, B, precision, n_steps, tol, threads=4, hanging=None):
    P0 = cdm.make_problem(m, rhs=0)
    S = Solver.from_mesh(m, precision=precision, n_rhs=B, dt=P0.dt)
    if hanging is not None:
        L.sbx_set_launch(S.ctx, L.SBX_LAUNCH_HANGING_KERNEL, hanging)
    S.initial()
    S.step(n_steps)
    g = S.field(L.SBX_U_N).reshape(-1, B)
    worst = 0.0
    for b in range(B):
        P = cdm.make_problem(m, dt=P0.dt, rhs=b)
        u, up = cdm.initial_state(P)
        u, _, _, _ = cdm.run(P, n_steps, u, up, threads=threads)
        worst = max(worst, rel(g[:, b], u))
    S.close()
    assert worst < tol, worst
    return worst


def test_batched_fp64_tiny():
    m = og.tiny_refined(1, p=0.35)
    m.fixed_nodes = np.where(np.abs(m.node_xyz[:, 2]) < 1e-12)[0]
    m = _with_sources(m, 32, 5)
    w = _compare(m, 32, "fp64", 150, 1e-12, threads=1)
    print("batched fp64 tiny: max rel error over 32 cases %.3e" % w)


@pytest.mark.parametrize("hname, hanging", [("tensor cores", L.SBX_HANGING_TENSOR),
                                            ("FP32 SIMT", L.SBX_HANGING_SIMT)])
def test_batched_fp32_corner_cube_1000_steps(hname, hanging):
    # the hanging-node patterns on the tensor cores (the default) or FP32 SIMT
    m = _with_sources(og.config_corner_cube(), 32, 7, t1_scale=10.0)
    w = _compare(m, 32, "fp32", 1000, 1e-5, hanging=hanging)
    print("batched fp32 corner cube, hanging patterns on %s, 1000 steps: max rel error over "
          "32 cases %.3e" % (hname, w))


def test_batched_64_cases_and_initial_field():
    m = og.tiny_refined(2, p=0.35)
    m.fixed_nodes = np.where(np.abs(m.node_xyz[:, 2]) < 1e-12)[0]
    m = _with_sources(m, 64, 9)
    B = 64
    P0 = cdm.make_problem(m, rhs=0)
    rng = np.random.default_rng(3)
    u0 = rng.standard_normal((m.n_dof, B)) * 1e-2
    fixed = m.fixed_dofs()
    u0[fixed] = 0
    S = Solver.from_mesh(m, precision="fp64", n_rhs=B, dt=P0.dt)
    S.initial(np.ascontiguousarray(u0.ravel()))
    S.step(60)
    g = S.field(L.SBX_U_N).reshape(-1, B)
    for b in [0, 17, 40, 63]:
        P = cdm.make_problem(m, dt=P0.dt, rhs=b)
        u, up = cdm.initial_state(P, u0[:, b])
        u, _, _, _ = cdm.run(P, 60, u, up)
        assert rel(g[:, b], u) < 1e-12
    S.close()


def test_batched_full_size_multi_point():
    m = og.config_multi_point()
    B = 64
    P0 = cdm.make_problem(m, rhs=0)
    S = Solver.from_mesh(m, precision="fp32", n_rhs=B, dt=P0.dt)
    rng = np.random.default_rng(4)
    u0 = rng.standard_normal((m.n_dof, B)) * 1e-3
    u0[m.fixed_dofs()] = 0
    S.initial(np.ascontiguousarray(u0.ravel()))
    S.step(20)
    g = S.field(L.SBX_U_N).reshape(-1, B)
    worst = 0.0
    for b in [0, 31, 63]:
        P = cdm.make_problem(m, dt=P0.dt, rhs=b)
        u, up = cdm.initial_state(P, u0[:, b])
        u, _, _, _ = cdm.run(P, 20, u, up, threads=16)
        worst = max(worst, rel(g[:, b], u))
    print("batched fp32 multi-point (%d cells), 20 steps: %.3e" % (m.n_cells, worst))
    assert worst < 1e-6
    S.close()


def test_batched_rejects_bad_sizes():
    m = og.tiny_refined(0)
    with pytest.raises(L.SbxError):
        Solver.from_mesh(m, precision="fp32", n_rhs=20)
    with pytest.raises(L.SbxError):
        Solver.from_mesh(m, precision="mixed", n_rhs=32)


def test_batched_fp32_damped_and_force_readback():
    # damped batched FP32 update and the FP32 force read back as FP64
    m = _with_sources(og.config_corner_cube(), 32, 9, t1_scale=10.0)
    alpha = 0.4
    P0 = cdm.make_problem(m, rhs=0, alpha=alpha)
    S = Solver.from_mesh(m, precision="fp32", n_rhs=32, dt=P0.dt, alpha=alpha)
    S.initial()
    S.step(200)
    g = S.field(L.SBX_U_N).reshape(-1, 32)
    fg = S.field(L.SBX_F_INT).reshape(-1, 32)
    for b in (0, 13, 31):
        P = cdm.make_problem(m, dt=P0.dt, rhs=b, alpha=alpha)
        u, up = cdm.initial_state(P)
        u, up, _, f = cdm.run(P, 200, u, up, threads=4, want_force=True)
        assert rel(g[:, b], u) < 1e-5
        # the oracle returns R_ext - R_int of the last step, the library R_int - R_ext
        assert rel(-fg[:, b], f) < 1e-4
    S.close()


def test_batched_fp32_other_tile_shapes():
    # every class re-tiled (sbx_set_launch) on FP32 SIMT: only the
    # reductions' order changes
    m = _with_sources(og.config_corner_cube(), 32, 11, t1_scale=10.0)
    P0 = cdm.make_problem(m, rhs=0)
    S = Solver.from_mesh(m, precision="fp32", n_rhs=32, dt=P0.dt)
    L.sbx_set_launch(S.ctx, L.SBX_LAUNCH_HANGING_KERNEL, L.SBX_HANGING_SIMT)
    for c, (cells, kb) in enumerate([(64, 150), (8, 56), (16, 72)]):
        L.sbx_set_launch(S.ctx, L.SBX_LAUNCH_BATCH_TILE_CELLS + c, cells)
        L.sbx_set_launch(S.ctx, L.SBX_LAUNCH_BATCH_SMEM_KB + c, kb)
        assert L.sbx_get_launch(S.ctx, L.SBX_LAUNCH_BATCH_TILE_CELLS + c) == cells
        assert L.sbx_get_launch(S.ctx, L.SBX_LAUNCH_BATCH_SMEM_KB + c) == kb
    S.initial()
    S.step(500)
    g = S.field(L.SBX_U_N).reshape(-1, 32)
    for b in (0, 9, 31):
        P = cdm.make_problem(m, dt=P0.dt, rhs=b)
        u, up = cdm.initial_state(P)
        u, _, _, _ = cdm.run(P, 500, u, up, threads=4)
        assert rel(g[:, b], u) < 1e-5
    S.close()
