"""The two kernels of the mixed form for the regular 8-node cells: the
Walsh-basis FP32 SIMT kernel (the default, also covered by every run of
test_gpu_mixed.py) and the TF32x3 tensor-core kernel
(sbx_set_mixed_kernel(SBX_MIXED_TENSOR)), each against the FP64 oracle with
the bars of test_gpu_mixed.py (relative L2 error <= 1e-5)."""
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




def solver(m, kind, **kw):
    S = Solver.from_mesh(m, precision="mixed", **kw)
    L.sbx_set_mixed_kernel(S.ctx, kind)
    return S


KINDS = [("walsh", L.SBX_MIXED_WALSH), ("tensor", L.SBX_MIXED_TENSOR)]


@pytest.mark.parametrize("name, kind", KINDS)
@pytest.mark.parametrize("n", [16, 32])
def test_uniform_force_and_steps(n, name, kind):
    m = og.small_uniform(n)
    m.E = np.exp(0.3 * np.random.default_rng(n).standard_normal(m.n_cells))
    m.fixed_nodes = np.where(np.abs(m.node_xyz[:, 2]) < 1e-12)[0]
    P = cdm.make_problem(m)
    S = solver(m, kind, dt=P.dt)
    assert L.sbx_query(S.ctx, L.SBX_Q_WALSH_CELLS) == (m.n_cells if name == "walsh" else 0)
    u0 = np.random.default_rng(n + 1).standard_normal(m.n_dof)
    u0[P.fixed] = 0
    S.initial(u0)
    S.step(1)
    ref = cdm.apply_K(P, u0) - cdm.external_force(P, 0)
    e1 = rel(S.field(L.SBX_F_INT), ref)
    u, up = cdm.initial_state(P, u0)
    S.initial(u0)
    S.step(100)
    u, up, _, _ = cdm.run(P, 100, u, up, threads=16)
    e2 = rel(S.field(L.SBX_U_N), u)
    print("uniform %d^3, %s kernel: force %.3e, 100 steps %.3e" % (n, name, e1, e2))
    assert e1 < 1e-5 and e2 < 1e-5


@pytest.mark.parametrize("name, kind", KINDS)
def test_corner_cube_2000_steps(name, kind):
    m = og.config_corner_cube()
    P = cdm.make_problem(m)
    S = solver(m, kind, dt=P.dt)
    S.initial()
    S.step(2000)
    u, up = cdm.initial_state(P)
    u, up, _, _ = cdm.run(P, 2000, u, up, threads=16)
    e = rel(S.field(L.SBX_U_N), u)
    print("corner cube, %s kernel, 2000 steps: %.3e" % (name, e))
    assert e < 1e-5
