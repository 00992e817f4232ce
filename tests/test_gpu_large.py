"""Full-size layered-trench octree (~7.7M cells, ~30M DOF, 42 patterns;
levels 5-10 refined toward a free-surface trench of finite length, two
curved layer interfaces and seeded random flags; three layers E = 1 : 4 :
16): the mixed form's force
at sampled nodes against the FP64 oracle (each sampled node's force depends
only on its incident cells, so the oracle runs on those cells alone), and
500 mixed steps against 500 FP64 steps on the GPU (the FP64 path is itself
pinned to the oracle at smaller sizes)."""
import copy

import numpy as np
import pytest

import octree_gen as og
from oracle import cdm
from paper_2103_09100_gb300 import Solver, _lib as L, build
from parity import rel

pytestmark = [pytest.mark.gpu, pytest.mark.slow]


@pytest.fixture(scope="module", autouse=True)
def _built():
    build.build()
    L.load()


@pytest.fixture(scope="module")
def trench():
    return og.config_layered_trench()


def _around(mesh, nodes):
    """Sub-mesh of the cells incident to `nodes` (local numbering) and the
    local ids of `nodes`."""
    sel = np.nonzero(np.isin(mesh.slot_node, nodes).any(1))[0]
    sn = mesh.slot_node[sel]
    used = np.unique(sn[sn >= 0])
    m = copy.copy(mesh)
    m.level, m.anchor, m.h, m.mask = mesh.level[sel], mesh.anchor[sel], mesh.h[sel], mesh.mask[sel]
    m.E, m.rho = mesh.E[sel], mesh.rho[sel]
    m.slot_node = np.where(sn >= 0, np.searchsorted(used, np.maximum(sn, 0)), -1)
    m.node_xyz = mesh.node_xyz[used]
    m.fixed_nodes = np.zeros(0, np.int64)
    m.sources = []
    return m, used, np.searchsorted(used, nodes)


def test_trench_force_at_sampled_nodes(trench):
    import torch
    m = copy.copy(trench)
    m.sources = []
    m.fixed_nodes = np.zeros(0, np.int64)
    free0, total = torch.cuda.mem_get_info()
    S = Solver.from_mesh(m, precision="mixed")
    free1, _ = torch.cuda.mem_get_info()
    print("layered trench: %d cells, %d DOF, %d patterns, device memory %.2f GB"
          % (m.n_cells, m.n_dof, len(S.masters), (free0 - free1) / 1e9))
    assert len(S.masters) >= 30   # many hanging-node patterns at scale
    rng = np.random.default_rng(11)
    u0 = rng.standard_normal(m.n_dof)
    S.initial(u0)
    S.step(1)
    f = S.field(L.SBX_F_INT).reshape(-1, 3)
    S.close()
    samples = np.unique(rng.choice(m.n_nodes, 2000, replace=False))
    sub, used, loc = _around(m, samples)
    P = cdm.make_problem(sub)
    ref = cdm.apply_K(P, u0.reshape(-1, 3)[used].ravel()).reshape(-1, 3)[loc]
    err = rel(f[samples], ref)
    print("layered trench: force at %d sampled nodes, rel error %.3e" % (len(samples), err))
    assert err < 1e-5


def test_trench_500_steps_mixed_vs_fp64(trench):
    m = trench
    A = Solver.from_mesh(m, precision="fp64")
    B = Solver.from_mesh(m, precision="mixed", dt=A.dt)
    A.initial()
    B.initial()
    A.step(500)
    B.step(500)
    ua, ub = A.field(), B.field()
    e = rel(ub, ua)
    print("layered trench: 500 steps, mixed vs FP64 rel error %.3e (|u| %.3e)"
          % (e, np.linalg.norm(ua)))
    assert np.linalg.norm(ua) > 0
    assert e < 1e-5
