"""Node-cut partition of an octree mesh over several GPUs (Sec. 4) and the
interface sum of the partial internal forces.

Each part holds a contiguous range of cells in the mesh's Morton order (a
space-filling-curve partition) and every node its cells touch.  Nodes
touched by more than one part lie on a cut.  Per step every part computes
the internal force of its own cells (the library's ``sbx_force``), the
partial forces of the cut nodes are summed over the parts, and every part
runs the update (``sbx_update``) on all of its nodes; a cut node then has
the same force, mass and history on every part that holds it, so its
displacement stays identical everywhere without further exchange.

Two forms of the sum:

* ``HaloExchange``: one collective over a vector that holds every cut node
  of the whole partition once (each part writes its partial forces into the
  positions of its cut nodes, ``all_reduce``, read back).  Simple; every
  rank ships every interface.  Used once at set-up for the lumped mass.
* ``HaloPlan`` (per step): each part exchanges with each neighbouring part
  only the nodes the two share (Sec. 4.2: the interface DOFs of neighbouring
  subdomains), by point-to-point send / receive; every part then sums each
  cut node's partial forces in one canonical order -- the holding parts in
  ascending rank -- so that all holders of a node compute bit-identical
  sums and its history stays identical everywhere.

Point loads on a cut node are applied by the lowest part that holds the
node, so they are counted once.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np


@dataclass
class Part:
    """One part: cells ``cells`` (global ids, ascending), nodes ``nodes``
    (global ids, ascending; local node id = position), ``slot_node`` in
    local ids, the cut nodes ``cut_local`` (local ids) and their positions
    ``cut_pos`` in the global cut vector."""
    rank: int
    cells: np.ndarray
    nodes: np.ndarray
    slot_node: np.ndarray
    cut_local: np.ndarray
    cut_pos: np.ndarray
    n_cut: int
    fixed_nodes: np.ndarray = field(default_factory=lambda: np.zeros(0, np.int64))
    sources: list = field(default_factory=list)
    # neighbour rank -> local ids of the nodes shared with it, ascending by
    # global id (the same order on both sides)
    shared: dict = field(default_factory=dict)
    # per local cut node (order of cut_local): the ranks holding it, ascending
    holders: list = field(default_factory=list)

    @property
    def n_nodes(self):
        return int(len(self.nodes))

    def local(self, global_nodes):
        """Local ids of global node ids that this part holds (-1 otherwise)."""
        g = np.asarray(global_nodes, np.int64)
        i = np.searchsorted(self.nodes, g)
        i = np.minimum(i, len(self.nodes) - 1)
        return np.where(self.nodes[i] == g, i, -1)


def split_ranges(n_cells, n_parts, weight=None):
    """Contiguous cell ranges with near-equal total weight (default: equal
    counts).  Returns the n_parts + 1 boundaries."""
    if n_parts < 1 or n_parts > max(1, n_cells):
        raise ValueError("need 1 <= n_parts <= n_cells")
    if weight is None:
        return np.round(np.linspace(0, n_cells, n_parts + 1)).astype(np.int64)
    c = np.concatenate([[0.0], np.cumsum(np.asarray(weight, np.float64))])
    targets = c[-1] * np.arange(1, n_parts) / n_parts
    inner = np.searchsorted(c, targets)
    b = np.concatenate([[0], inner, [n_cells]]).astype(np.int64)
    for k in range(1, n_parts + 1):   # keep every part non-empty
        b[k] = max(b[k], b[k - 1] + 1)
    for k in range(n_parts - 1, -1, -1):
        b[k] = min(b[k], b[k + 1] - 1)
    return b


def partition(slot_node, n_parts, fixed_nodes=(), sources=(), weight=None):
    """Split the cells (rows of ``slot_node``, in Morton order) into
    ``n_parts`` contiguous ranges and build each part's local numbering and
    cut lists.  ``weight`` (per cell, optional) balances the ranges, e.g. by
    the contraction cost m_p^2."""
    slot_node = np.asarray(slot_node)
    C = slot_node.shape[0]
    b = split_ranges(C, n_parts, weight)
    node_sets = []
    for k in range(n_parts):
        sn = slot_node[b[k]:b[k + 1]]
        node_sets.append(np.unique(sn[sn >= 0]))
    # cut nodes: held by >= 2 parts
    allnodes = np.concatenate(node_sets)
    uniq, counts = np.unique(allnodes, return_counts=True)
    cut = uniq[counts >= 2]
    # lowest part holding each node (point loads go there)
    owner = {}
    for k in range(n_parts - 1, -1, -1):
        for q in node_sets[k]:
            owner[int(q)] = k
    # holders of every cut node, ascending rank
    holders = {int(q): [] for q in cut}
    for k in range(n_parts):
        for q in np.intersect1d(node_sets[k], cut, assume_unique=True):
            holders[int(q)].append(k)
    fixed_nodes = np.asarray(fixed_nodes, np.int64)
    parts = []
    for k in range(n_parts):
        nodes = node_sets[k]
        sn = slot_node[b[k]:b[k + 1]]
        loc = np.full(sn.shape, -1, np.int64)
        m = sn >= 0
        loc[m] = np.searchsorted(nodes, sn[m])
        in_cut = np.isin(nodes, cut)
        cut_local = np.nonzero(in_cut)[0].astype(np.int64)
        cut_pos = np.searchsorted(cut, nodes[cut_local]).astype(np.int64)
        P = Part(rank=k, cells=np.arange(b[k], b[k + 1], dtype=np.int64), nodes=nodes,
                 slot_node=loc.astype(slot_node.dtype), cut_local=cut_local, cut_pos=cut_pos,
                 n_cut=int(len(cut)))
        P.holders = [holders[int(q)] for q in nodes[cut_local]]
        for q in range(n_parts):
            if q == k:
                continue
            common = np.intersect1d(nodes, node_sets[q], assume_unique=True)
            if len(common):
                P.shared[q] = np.searchsorted(nodes, common).astype(np.int64)
        fl = P.local(fixed_nodes) if len(fixed_nodes) else np.zeros(0, np.int64)
        P.fixed_nodes = fl[fl >= 0]
        for s in sources:
            if owner.get(int(s["node"])) == k:
                t = dict(s)
                t["node"] = int(P.local([s["node"]])[0])
                P.sources.append(t)
        parts.append(P)
    return parts


class HaloExchange:
    """Sum of the cut nodes' values over the parts.

    ``pack(v)`` copies this part's cut-node rows of ``v`` (a (N_local, k)
    tensor or array) into a zeroed global cut vector (n_cut, k);
    ``unpack(v, buf)`` writes the summed rows back.  ``exchange(v)`` does
    both around one ``all_reduce`` (``torch.distributed``, default group)."""

    def __init__(self, part: Part):
        self.part = part

    def pack(self, v):
        import torch
        t = v if isinstance(v, torch.Tensor) else torch.from_numpy(np.asarray(v))
        idx = torch.as_tensor(self.part.cut_local, device=t.device)
        pos = torch.as_tensor(self.part.cut_pos, device=t.device)
        buf = torch.zeros((self.part.n_cut,) + tuple(t.shape[1:]), dtype=t.dtype, device=t.device)
        buf.index_copy_(0, pos, t.index_select(0, idx))
        return buf

    def unpack(self, v, buf):
        import torch
        t = v if isinstance(v, torch.Tensor) else torch.from_numpy(v)
        idx = torch.as_tensor(self.part.cut_local, device=t.device)
        pos = torch.as_tensor(self.part.cut_pos, device=t.device)
        t.index_copy_(0, idx, buf.index_select(0, pos))

    def exchange(self, v, group=None):
        import torch.distributed as dist
        buf = self.pack(v)
        dist.all_reduce(buf, op=dist.ReduceOp.SUM, group=group)
        self.unpack(v, buf)
        return v


@dataclass
class HaloPlan:
    """Neighbour-only interface sum of one part.

    Send buffer: rows f[send_idx] (the nodes shared with each neighbour,
    neighbours in ascending rank, each block ascending by global id);
    ``send_ptr[i]:send_ptr[i + 1]`` is the block of ``neighbours[i]``.  The
    receive buffer has the same blocks, filled by the neighbours.  For cut
    node ``cut_nodes[j]`` (local id) the contributions are
    ``contrib_src[contrib_ptr[j]:contrib_ptr[j + 1]]`` in ascending rank of
    the holding part: -1 for this part's own partial force, else a row of
    the receive buffer."""
    neighbours: np.ndarray
    send_idx: np.ndarray
    send_ptr: np.ndarray
    cut_nodes: np.ndarray
    contrib_ptr: np.ndarray
    contrib_src: np.ndarray

    @property
    def n_rows(self):
        return int(len(self.send_idx))


def halo_plan(part: Part) -> HaloPlan:
    nb = np.array(sorted(part.shared), np.int64)
    blocks = [part.shared[int(q)] for q in nb]
    send_ptr = np.concatenate([[0], np.cumsum([len(b) for b in blocks])]).astype(np.int64)
    send_idx = np.concatenate(blocks).astype(np.int64) if blocks else np.zeros(0, np.int64)
    row_of = {}   # (neighbour, local node) -> receive row
    for i, q in enumerate(nb):
        for r, v in enumerate(blocks[i]):
            row_of[(int(q), int(v))] = int(send_ptr[i] + r)
    ptr, src = [0], []
    for v, hs in zip(part.cut_local, part.holders):
        for h in hs:
            src.append(-1 if h == part.rank else row_of[(h, int(v))])
        ptr.append(len(src))
    return HaloPlan(nb, send_idx, send_ptr, np.asarray(part.cut_local, np.int64),
                    np.array(ptr, np.int64), np.array(src, np.int64))


def halo_pack_host(plan: HaloPlan, f):
    """Host form of the pack (tests and CPU engines): rows f[send_idx]."""
    return f[plan.send_idx]


def halo_sum_host(plan: HaloPlan, f, recv):
    """Host form of the canonical interface sum, in place: for every cut
    node, its contributions added in ascending rank of the holding part,
    starting from zero."""
    for j, v in enumerate(plan.cut_nodes):
        acc = 0.0 * f[v]
        for s in plan.contrib_src[plan.contrib_ptr[j]:plan.contrib_ptr[j + 1]]:
            acc = acc + (f[v] if s < 0 else recv[s])
        f[v] = acc
    return f


def halo_exchange_p2p(plan: HaloPlan, send, recv, group=None):
    """Send each neighbour its block and receive its block of the same
    nodes (torch.distributed point-to-point: NCCL between GPUs, gloo on
    CPU); returns when the receive buffer is filled."""
    import torch.distributed as dist
    ops = []
    for i, q in enumerate(plan.neighbours):
        a, b = int(plan.send_ptr[i]), int(plan.send_ptr[i + 1])
        ops.append(dist.P2POp(dist.isend, send[a:b], int(q), group=group))
        ops.append(dist.P2POp(dist.irecv, recv[a:b], int(q), group=group))
    if ops:
        for w in dist.batch_isend_irecv(ops):
            w.wait()
    return recv
