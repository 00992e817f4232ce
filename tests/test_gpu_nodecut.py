"""Node-cut stepping on the GPU: the parts of a partition, each a library
context with sbx_force / interface sum / sbx_update, held by one process
(the parts take turns on one device), against the single-domain oracle."""
import numpy as np
import pytest

import octree_gen as og
from oracle import cdm
from paper_2103_09100_gb300 import _lib as L, build, nodecut
from paper_2103_09100_gb300.partition import partition

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    build.build()
    L.load()


def _run(m, n_parts, precision, n_steps, u0=None, v0=None):
    parts = partition(m.slot_node, n_parts, fixed_nodes=m.fixed_nodes, sources=m.sources,
                      weight=((m.slot_node >= 0).sum(1) ** 2))
    eng = [nodecut.NodeCutSolver(p, m.mask, m.h, m.E, m.rho, m.nu, precision=precision)
           for p in parts]
    dt = nodecut.setup_together(eng, 0.5, u0=u0, v0=v0)
    nodecut.step_together(eng, n_steps)
    out = [(e.part.nodes, e.field(L.SBX_U_N).reshape(-1, 3)) for e in eng]
    for e in eng:
        e.close()
    return dt, out


@pytest.mark.parametrize("n_parts", [2, 3])
def test_nodecut_fp64_equals_oracle(n_parts):
    m = og.config_corner_cube()
    m.E = np.exp(0.3 * np.random.default_rng(4).standard_normal(m.n_cells))
    rng = np.random.default_rng(5)
    u0 = rng.standard_normal(m.n_dof) * 1e-3
    v0 = rng.standard_normal(m.n_dof) * 1e-3
    dt, out = _run(m, n_parts, "fp64", 200, u0, v0)
    P = cdm.make_problem(m, dt=dt)
    u, up = cdm.initial_state(P, u0, v0)
    u, _, _, _ = cdm.run(P, 200, u, up, threads=4)
    ug = u.reshape(-1, 3)
    for nodes, ul in out:
        assert np.abs(ul - ug[nodes]).max() <= 1e-11 * np.abs(ug).max()


def test_nodecut_mixed_receiver_cube():
    m = og.config_receiver_cube()
    dt, out = _run(m, 2, "mixed", 300)
    P = cdm.make_problem(m, dt=dt)
    u, up = cdm.initial_state(P)
    u, _, _, _ = cdm.run(P, 300, u, up, threads=16)
    ug = u.reshape(-1, 3)
    num = sum(float(np.sum((ul - ug[nodes]) ** 2)) for nodes, ul in out)
    den = sum(float(np.sum(ug[nodes] ** 2)) for nodes, _ in out)
    e = (num / den) ** 0.5
    print("node-cut mixed, 2 parts, 300 steps: rel error %.3e" % e)
    assert e < 1e-5


def test_split_step_equals_step_n():
    from paper_2103_09100_gb300 import Solver
    m = og.config_corner_cube()
    A = Solver.from_mesh(m, precision="fp64")
    B = Solver.from_mesh(m, precision="fp64", dt=A.dt)
    A.initial()
    B.initial()
    A.step(57)
    for _ in range(57):
        L.sbx_force(B.ctx, B.dt)
        L.sbx_update(B.ctx, B.dt)
    assert np.abs(A.field() - B.field()).max() <= 1e-13 * np.abs(A.field()).max()
    with pytest.raises(L.SbxError):
        L.sbx_update(B.ctx, B.dt)
    L.sbx_force(B.ctx, B.dt)
    with pytest.raises(L.SbxError):
        L.sbx_force(B.ctx, B.dt)
