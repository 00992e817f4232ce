"""Test helper: a mesh in the ORACLE's pattern classification (its canonical
masks, ops and master matrices), ready for the library's set_patterns and
mesh_upload.  Running the GPU kernels on the oracle's own master matrices
compares the kernels with the oracle's stepper on identical matrices; the
product's independently computed pattern library agrees with the oracle's
to ~3e-15, a difference that long runs amplify."""
import numpy as np

from oracle import cube, sbfem
from paper_2103_09100_gb300 import _lib as L


def oracle_mesh_arrays(m, patterns):
    """(n_nodes per pattern, packed K, packed lumped mass, cell_pattern,
    cell_sym, cell_ptr, cell_nodes) with `patterns` the oracle's canonical
    masks in its pattern-table order."""
    canon_tab, op_tab = cube.canonical_table()
    mask = np.asarray(m.mask, np.int64)
    canon = canon_tab[mask]
    op = op_tab[mask]
    pidx = {int(p): i for i, p in enumerate(patterns)}
    slots = [np.array(cube.present_slots(int(p)), np.int64) for p in patterns]
    nn = np.array([len(s) for s in slots], np.int32)
    cell_pat = np.array([pidx[int(c)] for c in canon], np.int32)
    npc = nn[cell_pat].astype(np.int64)
    ptr = np.concatenate([[0], np.cumsum(npc)]).astype(np.int64)
    nodes = np.empty(int(ptr[-1]), np.int32)
    for key in np.unique(canon * 64 + op):
        c, g = int(key // 64), int(key % 64)
        cells = np.nonzero((canon == c) & (op == g))[0]
        pi = cube.slot_perm(g)
        inv = np.empty(26, np.int64)
        inv[np.array(pi)] = np.arange(26)
        t = slots[pidx[c]]
        rows = m.slot_node[cells][:, inv[t]]
        pos = ptr[cells][:, None] + np.arange(len(t))[None, :]
        nodes[pos.ravel()] = rows.ravel()
    K = np.concatenate([sbfem.master_cell(int(p), m.nu).K.ravel() for p in patterns])
    Ml = np.concatenate([sbfem.master_cell(int(p), m.nu).M_lump for p in patterns])
    return nn, K, Ml, cell_pat, op.astype(np.uint8), ptr, nodes


def oracle_context(m, P, precision=L.SBX_PREC_FP64):
    """A library context on the oracle's matrices, with the mesh's loads."""
    nn, K, Ml, cp, cs, ptr, nodes = oracle_mesh_arrays(m, P.tables["patterns"])
    ctx = L.sbx_create(0)
    try:
        L.set_patterns(ctx, nn, K, Ml)
        L.mesh_upload(ctx, m.n_nodes, cp, cs, ptr, nodes, m.h, m.E, m.rho,
                      np.ascontiguousarray(P.fixed, np.int64), 1, precision)
        if len(m.sources):
            from paper_2103_09100_gb300.solver import WAVES
            src = m.sources
            L.set_load(ctx, np.array([s["node"] for s in src], np.int64),
                       np.ascontiguousarray(np.array([s["dir"] for s in src], float).ravel()),
                       np.array([s.get("rhs", 0) for s in src], np.int32),
                       WAVES[src[0]["wavelet"]], np.array([s["t1"] for s in src], float),
                       np.array([s["P0"] for s in src], float),
                       np.array([s.get("n_cycles", 5.0) for s in src], float))
    except Exception:
        L.sbx_destroy(ctx)
        raise
    return ctx


class OracleMatrixSolver:
    """A library context on the oracle's master matrices, stepped like a
    Solver (initial / step / field / close)."""

    def __init__(self, m, P, precision=L.SBX_PREC_FP64):
        self.ctx = oracle_context(m, P, precision)
        self.dt, self.n_dof = P.dt, m.n_dof

    def initial(self, u0=None, v0=None):
        L.set_initial(self.ctx, u0, v0, self.dt)

    def step(self, n):
        L.step_n(self.ctx, n, self.dt)

    def field(self, which=L.SBX_U_N):
        import numpy as np
        return L.read_field(self.ctx, which, np.empty(self.n_dof))

    def close(self):
        L.sbx_destroy(self.ctx)
