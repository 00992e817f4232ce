"""Node-cut partition and interface sum (host logic, CPU).

The product's partition, HaloExchange and the torch.distributed step
driver run here with the FP64 oracle as each part's local force engine
(the GPU engine is tested in test_gpu_nodecut.py): the parts' stepped
states must equal the single-domain oracle run at every node."""
import copy
import os
import socket
import tempfile

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import octree_gen as og
from oracle import assembly, cdm
from paper_2103_09100_gb300 import nodecut
from paper_2103_09100_gb300.partition import (HaloExchange, halo_pack_host, halo_plan,
                                               halo_sum_host, partition, split_ranges)


def sub_mesh(mesh, part):
    m = copy.copy(mesh)
    c = part.cells
    m.level, m.anchor, m.h, m.mask = mesh.level[c], mesh.anchor[c], mesh.h[c], mesh.mask[c]
    m.E, m.rho = mesh.E[c], mesh.rho[c]
    m.slot_node = part.slot_node
    m.node_xyz = mesh.node_xyz[part.nodes]
    m.fixed_nodes = part.fixed_nodes
    m.sources = part.sources
    return m


class OracleEngine:
    """One part stepped by the FP64 oracle (test double of the GPU engine)."""

    def __init__(self, mesh, part, alpha=0.0):
        self.part, self.halo, self.alpha = part, HaloExchange(part), alpha
        self.sub = sub_mesh(mesh, part)
        self.P = cdm.make_problem(self.sub)
        self.dt_cr_local = assembly.critical_dt(self.sub)
        self.M = self.P.M_diag.copy()
        self.pending = False

    def pack_mass(self):
        return self.halo.pack(torch.from_numpy(self.M.reshape(-1, 3).copy()))

    def unpack_mass(self, buf):
        m = torch.from_numpy(self.M.reshape(-1, 3).copy())
        self.halo.unpack(m, buf)
        self.M = m.numpy().ravel().copy()

    def set_dt(self, dt):
        self.dt = dt
        self.P = cdm.make_problem(self.sub, dt=dt, alpha=self.alpha)

    def initial_local(self, u0=None, v0=None):
        n = self.P.n_dof
        self.u = np.zeros(n) if u0 is None else np.array(u0, float)
        self.v0 = np.zeros(n) if v0 is None else np.array(v0, float)
        self.u[self.P.fixed] = 0.0
        self.v0[self.P.fixed] = 0.0
        self.n = 0
        self.f = cdm.apply_K(self.P, self.u) - cdm.external_force(self.P, 0)
        self.pending = True

    def pack_force(self):
        return self.halo.pack(torch.from_numpy(self.f.reshape(-1, 3)))

    def unpack_force(self, buf):
        self.halo.unpack(torch.from_numpy(self.f.reshape(-1, 3)), buf)

    def finish_initial(self):
        minv = 1.0 / self.M
        minv[self.P.fixed] = 0.0
        acc = -minv * self.f - self.alpha * self.v0
        self.up = self.u - self.dt * self.v0 + 0.5 * self.dt ** 2 * acc
        self.up[self.P.fixed] = 0.0

    def force(self):
        if self.pending:
            return False
        self.f = cdm.apply_K(self.P, self.u) - cdm.external_force(self.P, self.n)
        self.pending = True
        return True

    def update(self):
        w = self.dt ** 2 / self.M / (1 + 0.5 * self.alpha * self.dt)
        w[self.P.fixed] = 0.0
        a, b = 2.0 / (1 + 0.5 * self.alpha * self.dt), (1 - 0.5 * self.alpha * self.dt) / (1 + 0.5 * self.alpha * self.dt)
        un = a * self.u - b * self.up - w * self.f
        self.up, self.u = self.u, un
        self.n += 1
        self.pending = False


class OracleNeighbourEngine(OracleEngine):
    """The oracle engine with the neighbour-only exchange: the part's cells
    split into interface cells (touching a cut node) and interior cells,
    the shared rows packed, the canonical sum on the host."""

    def __init__(self, mesh, part, alpha=0.0):
        super().__init__(mesh, part, alpha)
        self.torch = torch
        self.plan = halo_plan(part)
        self.recv = torch.zeros((max(1, self.plan.n_rows), 3), dtype=torch.float64)
        sn = part.slot_node
        cut = np.zeros(part.n_nodes, bool)
        cut[part.cut_local] = True
        self.inter = (cut[np.maximum(sn, 0)] & (sn >= 0)).any(1)

    def _problem(self, sel):
        m = copy.copy(self.sub)
        m.level, m.anchor, m.h, m.mask = (a[sel] for a in (m.level, m.anchor, m.h, m.mask))
        m.E, m.rho, m.slot_node = m.E[sel], m.rho[sel], m.slot_node[sel]
        with np.errstate(divide="ignore"):
            return cdm.make_problem(m, dt=self.dt, alpha=self.alpha)

    def set_dt(self, dt):
        super().set_dt(dt)
        self.P_I = self._problem(np.nonzero(self.inter)[0])
        self.P_R = self._problem(np.nonzero(~self.inter)[0]) if (~self.inter).any() else None

    def force_interface(self):
        if self.pending:
            return False
        self.f = cdm.apply_K(self.P_I, self.u) - cdm.external_force(self.P, self.n)
        self.pending = True
        return True

    def force_interior(self):
        if self.P_R is not None:
            self.f = self.f + cdm.apply_K(self.P_R, self.u)

    def pack(self):
        return torch.from_numpy(np.ascontiguousarray(halo_pack_host(self.plan, self.f.reshape(-1, 3))))

    def sum(self, recv):
        halo_sum_host(self.plan, self.f.reshape(-1, 3), recv.numpy())


def _mesh():
    m = og.config_corner_cube()
    m.E = np.exp(0.3 * np.random.default_rng(7).standard_normal(m.n_cells))
    return m


def test_split_ranges():
    b = split_ranges(10, 3)
    assert b[0] == 0 and b[-1] == 10 and np.all(np.diff(b) > 0)
    w = np.ones(100); w[:10] = 10.0
    b = split_ranges(100, 2, w)
    assert abs(w[:b[1]].sum() - w[b[1]:].sum()) <= 10.0
    with pytest.raises(ValueError):
        split_ranges(3, 4)


@pytest.mark.parametrize("P", [1, 2, 3, 5])
def test_partition_invariants(P):
    m = _mesh()
    parts = partition(m.slot_node, P, fixed_nodes=m.fixed_nodes, sources=m.sources)
    cells = np.concatenate([p.cells for p in parts])
    assert np.array_equal(cells, np.arange(m.n_cells))
    held = np.zeros(m.n_nodes, int)
    for p in parts:
        sn = m.slot_node[p.cells]
        assert np.array_equal(p.nodes, np.unique(sn[sn >= 0]))
        back = np.where(p.slot_node >= 0, p.nodes[np.maximum(p.slot_node, 0)], -1)
        assert np.array_equal(back, sn)
        held[p.nodes] += 1
        assert np.array_equal(np.sort(p.nodes[p.cut_local]), p.nodes[p.cut_local])
    cut = np.nonzero(held >= 2)[0]
    assert held.min() >= 1
    for p in parts:
        assert p.n_cut == len(cut)
        assert np.array_equal(cut[p.cut_pos], p.nodes[p.cut_local])
        assert np.array_equal(np.isin(p.nodes, cut), np.isin(np.arange(p.n_nodes), p.cut_local))
    # every source in exactly one part; every fixed node wherever it is held
    assert sum(len(p.sources) for p in parts) == len(m.sources)
    for p in parts:
        assert set(p.nodes[p.fixed_nodes]) == set(m.fixed_nodes) & set(p.nodes)


@pytest.mark.parametrize("P", [2, 4])
def test_interface_sum_gives_global_force(P):
    m = _mesh()
    Pg = cdm.make_problem(m)
    u = np.random.default_rng(1).standard_normal(m.n_dof)
    fg = cdm.apply_K(Pg, u).reshape(-1, 3)
    parts = partition(m.slot_node, P)
    halos = [HaloExchange(p) for p in parts]
    fl = []
    for p in parts:
        Pl = cdm.make_problem(sub_mesh(m, p))
        fl.append(torch.from_numpy(cdm.apply_K(Pl, u.reshape(-1, 3)[p.nodes].ravel()).reshape(-1, 3)))
    total = sum(h.pack(f) for h, f in zip(halos, fl))
    for h, f, p in zip(halos, fl, parts):
        h.unpack(f, total)
        assert np.abs(f.numpy() - fg[p.nodes]).max() <= 1e-12 * np.abs(fg).max()


def test_steps_together_equal_global_oracle():
    m = _mesh()
    parts = partition(m.slot_node, 3, fixed_nodes=m.fixed_nodes, sources=m.sources)
    eng = [OracleEngine(m, p) for p in parts]
    rng = np.random.default_rng(2)
    u0 = rng.standard_normal(m.n_dof) * 1e-3
    v0 = rng.standard_normal(m.n_dof) * 1e-3
    dt = nodecut.setup_together(eng, 0.5, u0=u0, v0=v0)
    nodecut.step_together(eng, 40)
    Pg = cdm.make_problem(m, dt=dt)
    u, up = cdm.initial_state(Pg, u0, v0)
    u, _, _, _ = cdm.run(Pg, 40, u, up)
    ug = u.reshape(-1, 3)
    for e in eng:
        assert np.abs(e.u.reshape(-1, 3) - ug[e.part.nodes]).max() <= 1e-12 * np.abs(ug).max()


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _rank_main(rank, world, port, out_dir, n_steps):
    import torch.distributed as dist
    dist.init_process_group("gloo", init_method="tcp://127.0.0.1:%d" % port, rank=rank,
                            world_size=world)
    try:
        m = _mesh()
        parts = partition(m.slot_node, world, fixed_nodes=m.fixed_nodes, sources=m.sources)
        e = OracleEngine(m, parts[rank])
        u0 = np.random.default_rng(2).standard_normal(m.n_dof) * 1e-3
        dt = nodecut.setup_distributed(e, 0.5, u0=u0)
        times = {}
        nodecut.step_distributed(e, n_steps, times=times)
        np.savez(os.path.join(out_dir, "r%d.npz" % rank), u=e.u, nodes=e.part.nodes, dt=dt,
                 t_C=times["t_C"], t_W=times["t_W"])
    finally:
        dist.destroy_process_group()


def test_gloo_two_ranks_equal_global_oracle():
    mp = pytest.importorskip("torch.multiprocessing")
    n_steps = 30
    with tempfile.TemporaryDirectory() as d:
        mp.spawn(_rank_main, args=(2, _free_port(), d, n_steps), nprocs=2, join=True)
        res = [np.load(os.path.join(d, "r%d.npz" % r)) for r in range(2)]
    m = _mesh()
    dt = float(res[0]["dt"])
    assert dt == float(res[1]["dt"])
    Pg = cdm.make_problem(m, dt=dt)
    u0 = np.random.default_rng(2).standard_normal(m.n_dof) * 1e-3
    u, up = cdm.initial_state(Pg, u0)
    u, _, _, _ = cdm.run(Pg, n_steps, u, up)
    ug = u.reshape(-1, 3)
    for r in res:
        assert np.abs(r["u"].reshape(-1, 3) - ug[r["nodes"]]).max() <= 1e-12 * np.abs(ug).max()
        # the per-rank split of the step time (Sec. 4): own work and interface sum
        assert float(r["t_C"]) > 0.0 and float(r["t_W"]) > 0.0


def _rank_leaves(rank, world, port, out_dir):
    # rank 1 leaves after set-up (between steps, nothing in flight); rank 0's
    # next interface sum must fail with an error instead of hanging
    import datetime
    import torch.distributed as dist
    dist.init_process_group("gloo", init_method="tcp://127.0.0.1:%d" % port, rank=rank,
                            world_size=world, timeout=datetime.timedelta(seconds=5))
    m = _mesh()
    parts = partition(m.slot_node, world, fixed_nodes=m.fixed_nodes, sources=m.sources)
    e = OracleEngine(m, parts[rank])
    nodecut.setup_distributed(e, 0.5)
    status = "stepped"
    if rank == 1:
        status = "left"
    else:
        try:
            nodecut.step_distributed(e, 5)
        except Exception as exc:   # the peer is gone
            status = "detected: %s" % type(exc).__name__
    with open(os.path.join(out_dir, "r%d.txt" % rank), "w") as f:
        f.write(status)
    if rank == 0:
        dist.destroy_process_group()


def test_gloo_rank_leaving_is_detected():
    mp = pytest.importorskip("torch.multiprocessing")
    with tempfile.TemporaryDirectory() as d:
        mp.spawn(_rank_leaves, args=(2, _free_port(), d), nprocs=2, join=True)
        s0 = open(os.path.join(d, "r0.txt")).read()
        s1 = open(os.path.join(d, "r1.txt")).read()
    assert s1 == "left"
    assert s0.startswith("detected"), s0


@pytest.mark.parametrize("P", [3, 4, 6])
def test_halo_plan_neighbour_lists(P):
    m = _mesh()
    parts = partition(m.slot_node, P)
    byr = {p.rank: p for p in parts}
    n_nb = []
    for p in parts:
        pl = halo_plan(p)
        n_nb.append(len(pl.neighbours))
        for q, loc in p.shared.items():
            other = byr[q]
            # the shared nodes, the same on both sides and in the same order
            assert np.array_equal(p.nodes[loc], other.nodes[other.shared[p.rank]])
            assert np.array_equal(p.nodes[loc], np.intersect1d(p.nodes, other.nodes))
        # each cut node: one contribution per holding part, own one once
        for j, v in enumerate(pl.cut_nodes):
            src = pl.contrib_src[pl.contrib_ptr[j]:pl.contrib_ptr[j + 1]]
            assert len(src) == len(p.holders[j]) >= 2
            assert (src < 0).sum() == 1
            assert list(p.holders[j]) == sorted(p.holders[j])
    # the mesh gives every part of a 4+-part partition several neighbours
    if P >= 4:
        assert max(n_nb) >= 3


@pytest.mark.parametrize("P", [3, 5])
def test_neighbour_sum_gives_global_force_on_every_holder(P):
    m = _mesh()
    Pg = cdm.make_problem(m)
    u = np.random.default_rng(1).standard_normal(m.n_dof)
    fg = cdm.apply_K(Pg, u).reshape(-1, 3)
    parts = partition(m.slot_node, P)
    plans = [halo_plan(p) for p in parts]
    fl = [cdm.apply_K(cdm.make_problem(sub_mesh(m, p)), u.reshape(-1, 3)[p.nodes].ravel()).reshape(-1, 3)
          for p in parts]
    sends = [halo_pack_host(pl, f) for pl, f in zip(plans, fl)]
    byr = {p.rank: (p, pl, snd) for p, pl, snd in zip(parts, plans, sends)}
    for p, pl, f in zip(parts, plans, fl):
        recv = np.zeros_like(sends[p.rank])
        for i, q in enumerate(pl.neighbours):
            op, opl, osnd = byr[int(q)]
            j = int(np.nonzero(opl.neighbours == p.rank)[0][0])
            recv[pl.send_ptr[i]:pl.send_ptr[i + 1]] = osnd[opl.send_ptr[j]:opl.send_ptr[j + 1]]
        halo_sum_host(pl, f, recv)
        assert np.abs(f - fg[p.nodes]).max() <= 1e-12 * np.abs(fg).max()
    # every holder of a cut node computed the same sum, bit for bit
    seen = {}
    for p, f in zip(parts, fl):
        for v in p.cut_local:
            g = int(p.nodes[v])
            if g in seen:
                assert np.array_equal(seen[g], f[v])
            else:
                seen[g] = f[v].copy()


def _rank_neighbours(rank, world, port, out_dir, n_steps):
    import torch.distributed as dist
    dist.init_process_group("gloo", init_method="tcp://127.0.0.1:%d" % port, rank=rank,
                            world_size=world)
    try:
        m = _mesh()
        parts = partition(m.slot_node, world, fixed_nodes=m.fixed_nodes, sources=m.sources)
        e = OracleNeighbourEngine(m, parts[rank])
        u0 = np.random.default_rng(2).standard_normal(m.n_dof) * 1e-3
        dt = nodecut.setup_distributed(e, 0.5, u0=u0)
        times = {}
        nodecut.step_neighbours(e, n_steps, times=times)
        np.savez(os.path.join(out_dir, "r%d.npz" % rank), u=e.u, nodes=e.part.nodes, dt=dt,
                 cut=e.part.nodes[e.part.cut_local], nb=e.plan.neighbours,
                 n_inter=int((~e.inter).sum()), t_C=times["t_C"], t_W=times["t_W"])
    finally:
        dist.destroy_process_group()


def test_gloo_four_ranks_neighbour_exchange_equal_global_oracle():
    mp = pytest.importorskip("torch.multiprocessing")
    n_steps, world = 30, 4
    with tempfile.TemporaryDirectory() as d:
        mp.spawn(_rank_neighbours, args=(world, _free_port(), d, n_steps), nprocs=world, join=True)
        res = [np.load(os.path.join(d, "r%d.npz" % r)) for r in range(world)]
    m = _mesh()
    dt = float(res[0]["dt"])
    Pg = cdm.make_problem(m, dt=dt)
    u0 = np.random.default_rng(2).standard_normal(m.n_dof) * 1e-3
    u, up = cdm.initial_state(Pg, u0)
    u, _, _, _ = cdm.run(Pg, n_steps, u, up)
    ug = u.reshape(-1, 3)
    assert max(len(r["nb"]) for r in res) >= 3          # a part with three neighbours
    assert all(int(r["n_inter"]) > 0 for r in res)      # interior cells overlap the exchange
    seen = {}
    for r in res:
        ul = r["u"].reshape(-1, 3)
        assert float(r["dt"]) == dt
        assert np.abs(ul - ug[r["nodes"]]).max() <= 1e-12 * np.abs(ug).max()
        assert float(r["t_C"]) > 0.0 and float(r["t_W"]) > 0.0
        # the cut nodes' histories are identical on every rank that holds them
        pos = {int(g): i for i, g in enumerate(r["nodes"])}
        for g in r["cut"]:
            row = ul[pos[int(g)]]
            if int(g) in seen:
                assert np.array_equal(seen[int(g)], row)
            else:
                seen[int(g)] = row
