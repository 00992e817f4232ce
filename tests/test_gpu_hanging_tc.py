"""The mixed form's two kernels for the hanging-node patterns against the
FP64 oracle: the tensor cores (SBX_HANGING_TENSOR, the default: tiles of up
to 128 cells of one pattern, TF32 x 3 with FP32 accumulation in tensor
memory) and FP32 SIMT (SBX_HANGING_SIMT, sbx_set_launch).  Errors by ``parity.rel`` (the larger of
the relative L2 and the element-wise error); bar 1e-5 as for every
FP32-contraction form."""
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


def solver(m, regular=L.SBX_MIXED_WALSH, hanging=L.SBX_HANGING_TENSOR, **kw):
    S = Solver.from_mesh(m, precision="mixed", **kw)
    # the tensor-core kernel is the library's default for these patterns
    assert L.sbx_get_launch(S.ctx, L.SBX_LAUNCH_HANGING_KERNEL) == L.SBX_HANGING_TENSOR
    L.sbx_set_mixed_kernel(S.ctx, regular)
    L.sbx_set_launch(S.ctx, L.SBX_LAUNCH_HANGING_KERNEL, hanging)
    assert L.sbx_get_launch(S.ctx, L.SBX_LAUNCH_HANGING_KERNEL) == hanging
    return S


HANGING = [("tensor", L.SBX_HANGING_TENSOR), ("simt", L.SBX_HANGING_SIMT)]


@pytest.mark.parametrize("seed", [0, 1, 3, 4])
def test_force_and_steps_tiny(seed):
    # a few dozen cells: every pattern tile ragged (far below 128 cells)
    m = og.tiny_refined(seed, p=0.6)
    m.E = np.exp(0.3 * np.random.default_rng(seed).standard_normal(m.n_cells))
    m.fixed_nodes = np.where(np.abs(m.node_xyz[:, 2]) < 1e-12)[0]
    P = cdm.make_problem(m)
    u0 = np.random.default_rng(seed + 10).standard_normal(m.n_dof)
    u0[P.fixed] = 0
    S = solver(m, dt=P.dt)
    S.initial(u0)
    S.step(1)
    ref = cdm.apply_K(P, u0) - cdm.external_force(P, 0)
    assert rel(S.field(L.SBX_F_INT), ref) < 1e-5
    S.initial(u0)
    S.step(100)
    u, up = cdm.initial_state(P, u0)
    u, _, _, _ = cdm.run(P, 100, u, up)
    assert rel(S.field(L.SBX_U_N), u) < 1e-5


@pytest.mark.parametrize("hname, hanging", HANGING)
@pytest.mark.parametrize("regular", [L.SBX_MIXED_WALSH, L.SBX_MIXED_TENSOR])
def test_corner_cube_2000_steps(regular, hname, hanging):
    # 30 patterns up to 26 nodes (78 DOF: the widest tile, N = 80)
    m = og.config_corner_cube()
    P = cdm.make_problem(m)
    S = solver(m, regular, hanging, dt=P.dt)
    S.initial()
    u, up = cdm.initial_state(P)
    worst = 0.0
    for k in range(4):
        S.step(500)
        u, up, _, _ = cdm.run(P, 500, u, up, n0=500 * k, threads=16)
        worst = max(worst, rel(S.field(L.SBX_U_N), u))
    print("corner cube, hanging patterns on %s, 2000 steps: %.3e" % (hname, worst))
    assert worst < 1e-5


@pytest.mark.parametrize("hname, hanging", HANGING)
def test_cavity_force_and_200_steps(hname, hanging):
    # full size: 30k hanging cells in 26 patterns, the benchmark's launch shape
    m = og.config_cavity_cube()
    P = cdm.make_problem(m)
    S = solver(m, hanging=hanging, dt=P.dt)
    u0 = np.random.default_rng(3).standard_normal(m.n_dof) * 1e-3
    u0[P.fixed] = 0
    S.initial(u0)
    S.step(1)
    ref = cdm.apply_K(P, u0) - cdm.external_force(P, 0)
    ef = rel(S.field(L.SBX_F_INT), ref)
    S.initial(u0)
    S.step(200)
    u, up = cdm.initial_state(P, u0)
    u, _, _, _ = cdm.run(P, 200, u, up, threads=16)
    e = rel(S.field(L.SBX_U_N), u)
    print("cavity cube, hanging patterns on %s: force %.3e, 200 steps %.3e" % (hname, ef, e))
    assert ef < 1e-5 and e < 1e-5


def test_launch_parameters_are_checked():
    m = og.tiny_refined(0, p=0.6)
    S = Solver.from_mesh(m, precision="mixed")
    with pytest.raises(L.SbxError):
        L.sbx_set_launch(S.ctx, L.SBX_LAUNCH_HANGING_KERNEL, 7)
    with pytest.raises(L.SbxError):
        L.sbx_set_launch(S.ctx, L.SBX_LAUNCH_WALSH_CTAS_PER_SM, 9)
    with pytest.raises(L.SbxError):
        L.sbx_set_launch(S.ctx, 99, 0)
    L.sbx_set_launch(S.ctx, L.SBX_LAUNCH_WALSH_CTAS_PER_SM, 5)
    assert L.sbx_get_launch(S.ctx, L.SBX_LAUNCH_WALSH_CTAS_PER_SM) == 5
