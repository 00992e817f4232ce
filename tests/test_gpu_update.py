"""The mixed form's two update kernels (Eq. DnMdiag): rows streamed through
shared memory by 1-D bulk copies in chunks of 128 nodes (SBX_UPDATE_BULK,
the default) and per-thread loads (SBX_UPDATE_THREAD).  Same arithmetic,
so on a mesh whose forces do not depend on the order of the reductions the
states agree bit for bit, undamped and damped, with an odd node count (the
last chunk's odd node is read directly) and many chunks per CTA; and both
agree with the FP64 oracle."""
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


def _run(m, kernel, steps, u0, **kw):
    S = Solver.from_mesh(m, precision="mixed", **kw)
    assert L.sbx_get_launch(S.ctx, L.SBX_LAUNCH_UPDATE_KERNEL) == L.SBX_UPDATE_BULK
    L.sbx_set_launch(S.ctx, L.SBX_LAUNCH_UPDATE_KERNEL, kernel)
    assert L.sbx_get_launch(S.ctx, L.SBX_LAUNCH_UPDATE_KERNEL) == kernel
    S.initial(u0)
    S.step(steps)
    out = (S.field(L.SBX_U_N), S.field(L.SBX_U_NM1))
    S.close()
    return out


def corner_pairs(n_pairs, seed=0):
    """Pairs of unit cells that share one corner node (cell A's corner
    (1, 1, 1) is cell B's corner (0, 0, 0)), 15 nodes per pair: every node
    receives at most two force contributions, and a sum of two FP32 terms
    does not depend on their order, so the force (and every state) is the
    same from run to run."""
    C, N = 2 * n_pairs, 15 * n_pairs
    j = np.arange(n_pairs)
    slot = -np.ones((C, 26), np.int32)
    slot[0::2, :8] = 15 * j[:, None] + np.arange(8)
    slot[1::2, 0] = 15 * j + 7
    slot[1::2, 1:8] = 15 * j[:, None] + np.arange(8, 15)
    k = np.arange(8)
    cor = np.stack([k & 1, (k >> 1) & 1, k >> 2], 1).astype(float)
    xyz = np.zeros((N, 3))
    off = np.stack([3.0 * j, 0.0 * j, 0.0 * j], 1)
    xyz[(15 * j[:, None] + k).ravel()] = (off[:, None, :] + cor[None]).reshape(-1, 3)
    xyz[(15 * j[:, None] + 7 + k[1:]).ravel()] = (off[:, None, :] + 1 + cor[None, 1:]).reshape(-1, 3)
    rng = np.random.default_rng(seed)
    return og.OctreeMesh(name="corner_pairs_%d" % n_pairs, origin=np.zeros(3), h_finest=1.0,
                         lmax=0, level=np.zeros(C, np.int8), anchor=np.zeros((C, 3), np.int64),
                         h=np.ones(C), mask=np.zeros(C, np.int32), slot_node=slot, node_xyz=xyz,
                         E=np.exp(0.2 * rng.standard_normal(C)), rho=np.ones(C), nu=0.3,
                         fixed_nodes=np.zeros(0, np.int64))


@pytest.mark.parametrize("alpha", [0.0, 0.3])
def test_bulk_and_thread_updates_agree_bitwise(alpha):
    # 900,015 nodes (odd): 7032 chunks of 128, several per CTA and stage
    m = corner_pairs(60001)
    assert m.n_nodes % 2 == 1
    P = cdm.make_problem(m, alpha=alpha)
    u0 = np.random.default_rng(7).standard_normal(m.n_dof) * 1e-3
    ub, ubm = _run(m, L.SBX_UPDATE_BULK, 60, u0, dt=P.dt, alpha=alpha)
    ut, utm = _run(m, L.SBX_UPDATE_THREAD, 60, u0, dt=P.dt, alpha=alpha)
    assert np.array_equal(ub, ut) and np.array_equal(ubm, utm)
    u, up = cdm.initial_state(P, u0)
    u, _, _, _ = cdm.run(P, 60, u, up, threads=16)
    assert rel(ub, u) < 1e-5


def test_bulk_update_cavity_cube():
    # the benchmark mesh (1,146,297 nodes), both kernels against the oracle
    m = og.config_cavity_cube()
    P = cdm.make_problem(m)
    u0 = np.random.default_rng(7).standard_normal(m.n_dof) * 1e-3
    u0[P.fixed] = 0
    u, up = cdm.initial_state(P, u0)
    u, _, _, _ = cdm.run(P, 60, u, up, threads=16)
    for kernel in (L.SBX_UPDATE_BULK, L.SBX_UPDATE_THREAD):
        ug, _ = _run(m, kernel, 60, u0, dt=P.dt)
        assert rel(ug, u) < 1e-5


@pytest.mark.parametrize("n_pairs", [5, 8])
def test_bulk_update_fewer_nodes_than_a_chunk(n_pairs):
    # 75 (odd) and 120 nodes: one ragged chunk
    m = corner_pairs(n_pairs, seed=n_pairs)
    P = cdm.make_problem(m)
    u0 = np.random.default_rng(n_pairs).standard_normal(m.n_dof)
    ub, _ = _run(m, L.SBX_UPDATE_BULK, 50, u0, dt=P.dt)
    ut, _ = _run(m, L.SBX_UPDATE_THREAD, 50, u0, dt=P.dt)
    assert np.array_equal(ub, ut)
    u, up = cdm.initial_state(P, u0)
    u, _, _, _ = cdm.run(P, 50, u, up)
    assert rel(ub, u) < 1e-5


@pytest.mark.parametrize("seed", [0, 2])
def test_bulk_update_hanging_nodes_small(seed):
    m = og.tiny_refined(seed, p=0.6)
    m.fixed_nodes = np.where(np.abs(m.node_xyz[:, 2]) < 1e-12)[0]
    P = cdm.make_problem(m)
    u0 = np.random.default_rng(seed).standard_normal(m.n_dof)
    u0[P.fixed] = 0
    ub, _ = _run(m, L.SBX_UPDATE_BULK, 50, u0, dt=P.dt)
    u, up = cdm.initial_state(P, u0)
    u, _, _, _ = cdm.run(P, 50, u, up)
    assert rel(ub, u) < 1e-5


def test_update_kernel_parameter_checked():
    m = og.tiny_refined(0, p=0.6)
    S = Solver.from_mesh(m, precision="mixed")
    with pytest.raises(L.SbxError):
        L.sbx_set_launch(S.ctx, L.SBX_LAUNCH_UPDATE_KERNEL, 2)
    S.close()
