"""Edge cases of the force paths: a mesh with no regular 8-node cell at all
(every cell has hanging nodes, so the Walsh and tensor-core kernels get no
tiles and only the pattern kernels run) and a mesh of one regular cell,
each in the FP64, mixed and batched forms, against the FP64 oracle's
K u - f_ext on the same random field."""
import copy

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


def _subset(mesh, keep):
    """The cells `keep` with their nodes renumbered (no loads, no supports)."""
    sn = mesh.slot_node[keep]
    used = np.unique(sn[sn >= 0])
    m = copy.copy(mesh)
    m.level, m.anchor, m.h, m.mask = mesh.level[keep], mesh.anchor[keep], mesh.h[keep], mesh.mask[keep]
    m.E, m.rho = mesh.E[keep], mesh.rho[keep]
    m.slot_node = np.where(sn >= 0, np.searchsorted(used, np.maximum(sn, 0)), -1).astype(np.int32)
    m.node_xyz = mesh.node_xyz[used]
    m.fixed_nodes = np.zeros(0, np.int64)
    m.fixed_dof_list = None
    m.sources = []
    return m


def _meshes():
    base = og.config_corner_cube()
    npn = (base.slot_node >= 0).sum(1)
    hanging = _subset(base, np.nonzero(npn > 8)[0])
    single = _subset(og.small_uniform(2), np.array([0]))
    return {"hanging_only": hanging, "single_regular": single}


@pytest.mark.parametrize("name", ["hanging_only", "single_regular"])
@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_force_on_edge_meshes(name, precision):
    m = _meshes()[name]
    P = cdm.make_problem(m)
    S = Solver.from_mesh(m, precision=precision, dt=P.dt)
    if name == "hanging_only":
        assert L.sbx_query(S.ctx, L.SBX_Q_WALSH_CELLS) == 0
    u0 = np.random.default_rng(7).standard_normal(m.n_dof)
    S.initial(u0)
    S.step(1)
    ref = cdm.apply_K(P, u0)
    e = rel(S.field(L.SBX_F_INT), ref)
    print("%s (%d cells), %s: force rel error %.3e" % (name, m.n_cells, precision, e))
    assert e < (1e-12 if precision == "fp64" else 1e-5)


@pytest.mark.parametrize("name", ["hanging_only", "single_regular"])
def test_batched_force_on_edge_meshes(name):
    m = _meshes()[name]
    P = cdm.make_problem(m)
    B = 32
    u0 = np.random.default_rng(8).standard_normal((m.n_dof, B))
    S = Solver.from_mesh(m, precision="fp32", n_rhs=B, dt=P.dt)
    S.initial(u0.ravel())
    S.step(1)
    f = S.field(L.SBX_F_INT).reshape(m.n_dof, B)
    worst = 0.0
    for b in (0, 13, 31):
        ref = cdm.apply_K(P, u0[:, b])
        worst = max(worst, rel(f[:, b], ref))
    print("%s batched: force rel error %.3e" % (name, worst))
    assert worst < 1e-5
