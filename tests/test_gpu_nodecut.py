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


def _run_neighbours(m, n_parts, precision, n_steps, overlap=True, u0=None):
    parts = partition(m.slot_node, n_parts, fixed_nodes=m.fixed_nodes, sources=m.sources,
                      weight=((m.slot_node >= 0).sum(1) ** 2))
    eng = [nodecut.NodeCutSolver(p, m.mask, m.h, m.E, m.rho, m.nu, precision=precision,
                                 overlap=overlap) for p in parts]
    assert all(e.G is not None for e in eng) == overlap
    dt = nodecut.setup_together(eng, 0.5, u0=u0)
    nodecut.step_neighbours_together(eng, n_steps)
    out = [(e.part.nodes, e.part.cut_local, e.field(L.SBX_U_N).reshape(-1, 3)) for e in eng]
    nb = [len(e.plan.neighbours) for e in eng]
    for e in eng:
        e.close()
    return dt, out, nb


@pytest.mark.parametrize("n_parts", [3, 4])
def test_neighbour_exchange_with_overlap_fp64(n_parts):
    # interface cells (owner context) and interior cells (guest on the same
    # state), shared rows packed and summed by the library's kernels
    m = og.config_corner_cube()
    m.E = np.exp(0.3 * np.random.default_rng(4).standard_normal(m.n_cells))
    u0 = np.random.default_rng(5).standard_normal(m.n_dof) * 1e-3
    dt, out, nb = _run_neighbours(m, n_parts, "fp64", 200, u0=u0)
    if n_parts == 4:
        assert max(nb) >= 3
    P = cdm.make_problem(m, dt=dt)
    u, up = cdm.initial_state(P, u0)
    u, _, _, _ = cdm.run(P, 200, u, up, threads=4)
    ug = u.reshape(-1, 3)
    seen = {}
    for nodes, cut, ul in out:
        assert np.abs(ul - ug[nodes]).max() <= 1e-11 * np.abs(ug).max()
        for v in cut:   # identical histories of a cut node on all its parts
            g = int(nodes[v])
            if g in seen:
                assert np.array_equal(seen[g], ul[v])
            else:
                seen[g] = ul[v].copy()


def test_neighbour_exchange_with_overlap_mixed_receiver_cube():
    m = og.config_receiver_cube()
    dt, out, _ = _run_neighbours(m, 3, "mixed", 300)
    P = cdm.make_problem(m, dt=dt)
    u, up = cdm.initial_state(P)
    u, _, _, _ = cdm.run(P, 300, u, up, threads=16)
    ug = u.reshape(-1, 3)
    num = sum(float(np.sum((ul - ug[nodes]) ** 2)) for nodes, _, ul in out)
    den = sum(float(np.sum(ug[nodes] ** 2)) for nodes, _, _ in out)
    mx = max(float(np.abs(ul - ug[nodes]).max()) for nodes, _, ul in out) / np.abs(ug).max()
    e = max((num / den) ** 0.5, mx)
    print("node-cut mixed, 3 parts, neighbour exchange with overlap, 300 steps: %.3e" % e)
    assert e < 1e-5


def test_shared_state_rules():
    from paper_2103_09100_gb300 import Solver
    import torch
    m = og.config_corner_cube()
    m.sources = []
    st = torch.cuda.Stream()
    A = Solver.from_mesh(m, precision="fp64", stream=st.cuda_stream)
    B = Solver.from_mesh(m, precision="fp64", stream=st.cuda_stream, dt=A.dt)
    C = Solver.from_mesh(m, precision="fp64", dt=A.dt)   # its own stream
    with pytest.raises(L.SbxError):
        L.sbx_share_state(C.ctx, A.ctx)
    L.sbx_share_state(B.ctx, A.ctx)
    assert np.array_equal(B.field(L.SBX_MASS), A.field(L.SBX_MASS))   # its own mass
    for call in (lambda: B.step(1), lambda: B.field(), lambda: L.sbx_update(B.ctx, B.dt)):
        with pytest.raises(L.SbxError) as e:
            call()
        assert e.value.code == L.SBX_ESTATE
    with pytest.raises(L.SbxError) as e:
        L.sbx_destroy(A.ctx)
    assert e.value.code == L.SBX_ESTATE
    # the guest adds the same cells' forces into the owner's accumulator:
    # owner + guest = twice the owner's force
    u0 = np.random.default_rng(1).standard_normal(m.n_dof)
    A.initial(u0)
    L.sbx_force(A.ctx, A.dt)
    f1 = L.read_field(A.ctx, L.SBX_F_INT, np.empty(m.n_dof)).copy()
    A.initial(u0)
    L.sbx_force(A.ctx, A.dt)
    L.sbx_force(B.ctx, A.dt)
    f2 = L.read_field(A.ctx, L.SBX_F_INT, np.empty(m.n_dof))
    assert np.abs(f2 - 2 * f1).max() <= 1e-12 * np.abs(f1).max()
    B.close()
    C.close()
    A.close()


def test_bench_nodecut_mode():
    # bench.py's node-cut line: the cavity mesh in 3 parts on this GPU
    import json
    import os
    import subprocess
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    out = subprocess.run([sys.executable, os.path.join(root, "bench.py"), "--nodecut", "3",
                          "--steps", "20", "--warmup", "3"], capture_output=True, text=True,
                         cwd=root, timeout=900)
    assert out.returncode == 0, out.stderr[-2000:]
    d = json.loads(out.stdout.strip().splitlines()[-1])
    assert d["form"] == "nodecut" and d["parts"] == 3 and d["steps"] == 20
    assert d["ms_per_step"] > 0 and d["t_C_ms"] > 0 and d["t_W_ms"] > 0
    assert len(d["neighbours"]) == 3 and min(d["cut_nodes"]) > 0
    assert d["rel_err_vs_single_domain"] < 1e-6
