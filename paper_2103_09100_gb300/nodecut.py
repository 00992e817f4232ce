"""Node-cut multi-GPU stepping (Sec. 4): one ``Solver`` per part, the
partial internal forces of the cut nodes summed every step.

``NodeCutSolver`` is one part on one GPU (one rank).  It splits every step
into ``sbx_force`` -> interface sum -> ``sbx_update`` through the C ABI and
reaches the library's force buffer in place (``sbx_field_ptr``), so the sum
runs on the device on the library's stream (NCCL ``all_reduce`` under
``torch.distributed``).  ``step_distributed`` drives any engine with the
same four methods (``force`` -> True when it computed a new partial force,
``pack_force``, ``unpack_force``, ``update``) over ``torch.distributed``;
``step_together`` drives several engines held by one process (the parts
then take turns on one device).

Per step the interface sum is neighbour to neighbour (``HaloPlan``): with
``overlap`` a part is two library contexts sharing one state
(``sbx_share_state``): the cells that touch a cut node (owner) and the
interior cells (guest).  ``step_neighbours`` then orders each step as the
paper's Sec. 4.2 does: interface force, pack of the shared rows
(``sbx_halo_pack``), the point-to-point exchange started, the interior
force while it runs, the canonical sum (``sbx_halo_sum``), the update.

Set-up: the lumped mass of the cut nodes is summed once (``sbx_set_mass``),
dt is the minimum of the parts' critical steps times ``dt_factor``, and the
start-up of Eq. D0 uses the summed initial force: after ``set_initial`` the
part evaluates f_0 = K U_0 - R_ext(0), sums it, rewrites U_-1 = U_0 - dt V_0
+ dt^2/2 (-M^-1 f_0 - alpha V_0) and keeps f_0 for the first update.
"""
from __future__ import annotations

import numpy as np

from . import _lib as L
from .partition import HaloExchange, Part, halo_exchange_p2p, halo_plan
from .solver import Solver


class _DeviceArray:
    """A device buffer of the library exposed through the CUDA array interface."""

    def __init__(self, ptr, shape, typestr):
        self.__cuda_array_interface__ = {"shape": shape, "typestr": typestr,
                                         "data": (int(ptr), False), "version": 3,
                                         "strides": None}


def field_view(ctx, which, torch):
    """(N, 3) float64 or (N, 4) float32 torch view of a library field (one load case)."""
    ptr, n, lay = L.sbx_field_ptr(ctx, which)
    if lay == L.SBX_LAYOUT_F32_NODE4:
        return torch.as_tensor(_DeviceArray(ptr, (n // 4, 4), "<f4"), device="cuda")
    return torch.as_tensor(_DeviceArray(ptr, (n // 3, 3), "<f8"), device="cuda")


class NodeCutSolver:
    """One part of a node-cut partition on one GPU.

    overlap=True splits the part's cells into the interface cells (touching
    a cut node; the owner context, which holds the loads and steps) and the
    interior cells (a guest context on the owner's state), so that the
    neighbour exchange runs while the interior force is computed."""

    def __init__(self, part: Part, mask, h, E, rho, nu, precision="fp64", device=0,
                 dt=None, alpha=0.0, overlap=False):
        import torch
        self.torch = torch
        self.part = part
        self.halo = HaloExchange(part)
        self.plan = halo_plan(part)
        self.stream = torch.cuda.Stream(device=device)
        self.device = device
        c = part.cells
        mask, h, E, rho = (np.asarray(a)[c] for a in (mask, h, E, rho))
        sn = part.slot_node
        inter = np.ones(len(c), bool)
        if overlap and len(part.cut_local):
            cut = np.zeros(part.n_nodes, bool)
            cut[part.cut_local] = True
            inter = (cut[np.maximum(sn, 0)] & (sn >= 0)).any(1)
            if inter.all() or not inter.any():
                inter = np.ones(len(c), bool)
        kw = dict(precision=precision, device=device, stream=self.stream.cuda_stream, dt=dt,
                  alpha=alpha)
        sel = np.nonzero(inter)[0]
        self.S = Solver(sn[sel], mask[sel], h[sel], E[sel], rho[sel], nu, part.n_nodes,
                        fixed_nodes=part.fixed_nodes, sources=part.sources, **kw)
        self.G = None   # guest: the interior cells
        self.dt_cr_local = self.S.dt_cr
        if not inter.all():
            rest = np.nonzero(~inter)[0]
            self.G = Solver(sn[rest], mask[rest], h[rest], E[rest], rho[rest], nu, part.n_nodes,
                            fixed_nodes=part.fixed_nodes, **kw)
            L.sbx_share_state(self.G.ctx, self.S.ctx)
            self.dt_cr_local = min(self.dt_cr_local, self.G.dt_cr)
        self.n_interface_cells = int(len(sel))
        L.sbx_halo_plan(self.S.ctx, self.plan.send_idx, self.plan.cut_nodes,
                        self.plan.contrib_ptr, self.plan.contrib_src)
        width, dtype = (4, torch.float32) if precision == "mixed" else (3, torch.float64)
        n = max(1, self.plan.n_rows)
        self.send = torch.zeros((n, width), dtype=dtype, device="cuda:%d" % device)
        self.recv = torch.zeros_like(self.send)
        self.dt = self.S.dt
        self.alpha = float(alpha)
        self.pending = False

    def _local_mass(self):
        m = self.S.field(L.SBX_MASS)
        if self.G is not None:
            m = m + self.G.field(L.SBX_MASS)
        return m.reshape(-1, 3)

    # ---- set-up
    def pack_mass(self):
        return self.halo.pack(self.torch.from_numpy(self._local_mass()))

    def unpack_mass(self, buf):
        m = self.torch.from_numpy(self._local_mass().copy())
        self.halo.unpack(m, buf.cpu())
        L.sbx_set_mass(self.S.ctx, np.ascontiguousarray(m.numpy().ravel()))

    def set_dt(self, dt):
        self.dt = float(dt)
        self.S.dt = self.dt

    def initial_local(self, u0=None, v0=None):
        """set_initial on the part, then f_0 (local part) into the force buffer."""
        self.u0, self.v0 = u0, v0
        self.S.initial(u0, v0)
        L.sbx_force(self.S.ctx, self.dt)
        if self.G is not None:
            L.sbx_force(self.G.ctx, self.dt)
        self.pending = True

    def finish_initial(self):
        """U_-1 from the summed f_0 (Eq. D0 with the interface sum)."""
        t = self.torch
        with t.cuda.stream(self.stream):
            f0 = field_view(self.S.ctx, L.SBX_F_INT, t)[:, :3].double()
            mass = field_view(self.S.ctx, L.SBX_MASS, t)
            minv = 1.0 / mass
            if len(self.part.fixed_nodes):
                minv[t.as_tensor(self.part.fixed_nodes, device=minv.device)] = 0.0
            u0 = field_view(self.S.ctx, L.SBX_U_N, t)
            um1 = field_view(self.S.ctx, L.SBX_U_NM1, t)
            v0 = (t.as_tensor(np.asarray(self.v0, np.float64).reshape(-1, 3), device=u0.device)
                  if self.v0 is not None else t.zeros_like(u0))
            acc = -minv * f0 - self.alpha * v0
            um1.copy_(u0 - self.dt * v0 + 0.5 * self.dt * self.dt * acc)
            if len(self.part.fixed_nodes):
                um1[t.as_tensor(self.part.fixed_nodes, device=um1.device)] = 0.0

    # ---- one step: force -> interface sum -> update
    def force(self):
        """Partial force of this part's cells; False when the force buffer
        already holds the summed force (the start-up's f_0)."""
        if self.pending:
            return False
        L.sbx_force(self.S.ctx, self.dt)
        if self.G is not None:
            L.sbx_force(self.G.ctx, self.dt)
        self.pending = True
        return True

    # ---- one step with the neighbour exchange (step_neighbours)
    def force_interface(self):
        """Partial force of the interface cells (all cells without overlap);
        False when the force buffer already holds the summed force."""
        if self.pending:
            return False
        L.sbx_force(self.S.ctx, self.dt)
        self.pending = True
        return True

    def force_interior(self):
        if self.G is not None:
            L.sbx_force(self.G.ctx, self.dt)

    def pack(self):
        """The rows this part sends, packed on the library's stream."""
        L.sbx_halo_pack(self.S.ctx, self.send)
        return self.send

    def sum(self, recv):
        """Canonical interface sum once recv holds the neighbours' rows (the
        library's stream waits for the stream recv was filled on)."""
        self.stream.wait_stream(self.torch.cuda.current_stream(self.device))
        L.sbx_halo_sum(self.S.ctx, recv)

    def pack_force(self):
        t = self.torch
        with t.cuda.stream(self.stream):
            buf = self.halo.pack(field_view(self.S.ctx, L.SBX_F_INT, t))
        t.cuda.current_stream().wait_stream(self.stream)   # the collective runs there
        return buf

    def unpack_force(self, buf):
        t = self.torch
        self.stream.wait_stream(t.cuda.current_stream())
        with t.cuda.stream(self.stream):
            self.halo.unpack(field_view(self.S.ctx, L.SBX_F_INT, t), buf)

    def update(self):
        L.sbx_update(self.S.ctx, self.dt, self.alpha)
        self.pending = False

    def field(self, which=L.SBX_U_N):
        self.stream.synchronize()
        return self.S.field(which)

    def sync(self):
        """Wait for this part's work on the device (library and sum streams)."""
        self.torch.cuda.synchronize()

    def close(self):
        if self.G is not None:
            self.G.close()
        self.S.close()


def step_distributed(engine, n, group=None, times=None):
    """n steps of one rank's engine; the interface sum is an all_reduce.

    times: optional dict in which the split of the step time that Sec. 4's
    timing study reports per rank accumulates, in seconds on the host
    clock: 't_C' the rank's own work (force and update), 't_W' the
    interface sum (pack, all_reduce, unpack, including the wait for the
    slowest rank).  The engine is then synchronised between the phases
    (its ``sync()``, if it has one), which gives up their overlap; without
    ``times`` nothing is synchronised."""
    import torch.distributed as dist
    if times is None:
        for _ in range(n):
            if engine.force():
                buf = engine.pack_force()
                dist.all_reduce(buf, op=dist.ReduceOp.SUM, group=group)
                engine.unpack_force(buf)
            engine.update()
        return
    import time
    sync = getattr(engine, "sync", None) or (lambda: None)
    times.setdefault("t_C", 0.0)
    times.setdefault("t_W", 0.0)
    for _ in range(n):
        t0 = time.perf_counter()
        fresh = engine.force()
        sync()
        t1 = time.perf_counter()
        if fresh:
            buf = engine.pack_force()
            dist.all_reduce(buf, op=dist.ReduceOp.SUM, group=group)
            engine.unpack_force(buf)
            sync()
        t2 = time.perf_counter()
        engine.update()
        sync()
        t3 = time.perf_counter()
        times["t_C"] += (t1 - t0) + (t3 - t2)
        times["t_W"] += t2 - t1


def step_neighbours(engine, n, group=None, times=None):
    """n steps of one rank's engine with the neighbour-only exchange:
    interface force, pack, point-to-point exchange started (NCCL on the
    library's stream order; gloo through host buffers), interior force while
    it runs, canonical sum, update.  ``times`` as in ``step_distributed``
    (t_C own work, t_W exchange and sum; the phases are then synchronised)."""
    import time
    import torch.distributed as dist
    torch = engine.torch
    sync = getattr(engine, "sync", None) or (lambda: None)
    on_gpu = dist.get_backend(group) == "nccl"
    host = None
    if times is not None:
        times.setdefault("t_C", 0.0)
        times.setdefault("t_W", 0.0)
    for _ in range(n):
        t0 = time.perf_counter()
        fresh = engine.force_interface()
        if fresh:
            send = engine.pack()
            if on_gpu:
                with torch.cuda.stream(engine.stream):
                    ops = _p2p_ops(engine.plan, send, engine.recv, group)
                    works = dist.batch_isend_irecv(ops) if ops else []
                engine.force_interior()
                t1 = time.perf_counter()
                with torch.cuda.stream(engine.stream):
                    for w in works:
                        w.wait()
                    engine.sum(engine.recv)
            else:
                if host is None:
                    host = (torch.empty(send.shape, dtype=send.dtype).pin_memory()
                            if send.is_cuda else torch.empty_like(send),
                            torch.empty(send.shape, dtype=send.dtype).pin_memory()
                            if send.is_cuda else torch.empty_like(send))
                if send.is_cuda:   # the pack ran on the library's stream
                    engine.stream.synchronize()
                host[0].copy_(send)
                ops = _p2p_ops(engine.plan, host[0], host[1], group)
                works = dist.batch_isend_irecv(ops) if ops else []
                engine.force_interior()
                t1 = time.perf_counter()
                for w in works:
                    w.wait()
                engine.recv.copy_(host[1])
                engine.sum(engine.recv)
            if times is not None:
                sync()
        else:
            t1 = time.perf_counter()
        t2 = time.perf_counter()
        engine.update()
        if times is not None:
            sync()
            t3 = time.perf_counter()
            times["t_C"] += (t1 - t0) + (t3 - t2)
            times["t_W"] += t2 - t1


def _p2p_ops(plan, send, recv, group):
    import torch.distributed as dist
    ops = []
    for i, q in enumerate(plan.neighbours):
        a, b = int(plan.send_ptr[i]), int(plan.send_ptr[i + 1])
        ops.append(dist.P2POp(dist.isend, send[a:b], int(q), group=group))
        ops.append(dist.P2POp(dist.irecv, recv[a:b], int(q), group=group))
    return ops


def exchange_together(engines):
    """The neighbour exchange of parts held by one process: part k's receive
    block from neighbour q is q's send block for k."""
    by_rank = {e.part.rank: e for e in engines}
    for e in engines:
        pl = e.plan
        for i, q in enumerate(pl.neighbours):
            o = by_rank[int(q)]
            j = int(np.nonzero(o.plan.neighbours == e.part.rank)[0][0])
            a, b = int(pl.send_ptr[i]), int(pl.send_ptr[i + 1])
            c, d = int(o.plan.send_ptr[j]), int(o.plan.send_ptr[j + 1])
            e.recv[a:b].copy_(o.send[c:d].to(e.recv.device))


def step_neighbours_together(engines, n):
    """step_neighbours for several parts held by one process."""
    for _ in range(n):
        fresh = [e.force_interface() for e in engines]
        if all(fresh):
            for e in engines:
                e.pack()
            for e in engines:
                e.stream.synchronize()
            exchange_together(engines)
            for e in engines:
                e.force_interior()
                e.sum(e.recv)
        for e in engines:
            e.update()


def step_together(engines, n):
    """n steps of several parts held by one process (summed in place)."""
    for _ in range(n):
        fresh = [e.force() for e in engines]
        if all(fresh):
            bufs = [e.pack_force() for e in engines]
            total = bufs[0].clone()
            for b in bufs[1:]:
                total += b.to(total.device)
            for e in engines:
                e.unpack_force(total)
        for e in engines:
            e.update()


def setup_together(engines, dt_factor=0.5, u0=None, v0=None):
    """Mass sum, common dt and start-up for parts held by one process;
    u0 / v0 are global (N, 3) arrays or None."""
    total = None
    for e in engines:
        b = e.pack_mass()
        total = b if total is None else total + b
    for e in engines:
        e.unpack_mass(total)
    dt = dt_factor * min(e.dt_cr_local for e in engines)
    for e in engines:
        e.set_dt(dt)
        nodes = e.part.nodes
        e.initial_local(None if u0 is None else np.ascontiguousarray(np.asarray(u0).reshape(-1, 3)[nodes].ravel()),
                        None if v0 is None else np.ascontiguousarray(np.asarray(v0).reshape(-1, 3)[nodes].ravel()))
    bufs = [e.pack_force() for e in engines]
    tot = bufs[0].clone()
    for b in bufs[1:]:
        tot += b
    for e in engines:
        e.unpack_force(tot)
        e.finish_initial()
    return dt


def setup_distributed(engine, dt_factor=0.5, u0=None, v0=None, group=None):
    """The same set-up for one rank of a torch.distributed job."""
    import torch
    import torch.distributed as dist
    b = engine.pack_mass()
    dev = "cuda" if dist.get_backend(group) == "nccl" else "cpu"
    b = b.to(dev)
    dist.all_reduce(b, op=dist.ReduceOp.SUM, group=group)
    engine.unpack_mass(b)
    t = torch.tensor([engine.dt_cr_local], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MIN, group=group)
    dt = dt_factor * float(t.item())
    engine.set_dt(dt)
    nodes = engine.part.nodes
    engine.initial_local(None if u0 is None else np.ascontiguousarray(np.asarray(u0).reshape(-1, 3)[nodes].ravel()),
                         None if v0 is None else np.ascontiguousarray(np.asarray(v0).reshape(-1, 3)[nodes].ravel()))
    buf = engine.pack_force()
    dist.all_reduce(buf, op=dist.ReduceOp.SUM, group=group)
    engine.unpack_force(buf)
    engine.finish_initial()
    return dt
