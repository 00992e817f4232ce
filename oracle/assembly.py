"""Element matrices of real cells, global assembly and the critical step.

Part of the FP64 oracle (test infrastructure; see ``oracle/__init__``).

* Eq. (KM_scale): a cell of edge h and modulus E has K = E h K_1 and
  M = rho h^3 M_1, where K_1, M_1 belong to the unit master cell of its
  pattern and Poisson ratio.
* Sec. 3.2.2: a cell whose mask is carried onto the master's mask by the
  transform Q has u_master = Q u_cell node by node (nodes carried by the
  same transform) and f_cell = Q^-1 f_master, i.e. K_cell = T^T K_p T with
  T the 3n x 3n signed permutation built from Q and the node map.
* Eqs. (tcr), (tcr_scale): dt_cr of a cell = sqrt(rho/E) h dt_cr of its
  master; the mesh step is the minimum over cells.
* Brute force: the global sparse K assembled from matrices computed by the
  SBFEM directly in every cell's own frame (no pattern reduction).
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp

from . import cube, sbfem


def transform_matrix(mask: int):
    """(canonical mask, op, T) with u_master = T u_cell for a cell of ``mask``.

    DOF order on both sides: present slots in increasing order, xyz inside.
    """
    canon_tab, op_tab = cube.canonical_table()
    canon = int(canon_tab[mask])
    op = int(op_tab[mask])
    Q = cube.all_ops()[op]
    pi = cube.slot_perm(op)
    cs = cube.present_slots(mask)
    ms = cube.present_slots(canon)
    assert sorted(pi[s] for s in cs) == ms
    mloc = {s: j for j, s in enumerate(ms)}
    n = len(cs)
    T = np.zeros((3 * n, 3 * n))
    for i, s in enumerate(cs):
        j = mloc[pi[s]]
        T[3 * j:3 * j + 3, 3 * i:3 * i + 3] = Q
    return canon, op, T


def cell_matrices_from_master(mask: int, h: float, E: float, rho: float, nu: float):
    """K_cell = E h T^T K_p T and the lumped mass rho h^3 diag(T^T M_p T)."""
    canon, op, T = transform_matrix(mask)
    mc = sbfem.master_cell(canon, nu)
    K = (E * h) * (T.T @ mc.K @ T)
    ML = (rho * h ** 3) * np.diag(T.T @ np.diag(mc.M_lump) @ T)
    return K, ML


def cell_dofs(mesh, c):
    nodes = mesh.slot_node[c][np.array(cube.present_slots(int(mesh.mask[c])))]
    assert (nodes >= 0).all()
    return (3 * nodes[:, None] + np.arange(3)[None, :]).ravel()


def check_mesh_slots(mesh):
    """The mesh's present slots agree with the face-centre rule of ``cube``."""
    for c in range(mesh.n_cells):
        pres = np.where(mesh.slot_node[c] >= 0)[0].tolist()
        if pres != cube.present_slots(int(mesh.mask[c])):
            return False
    return True


def global_K_bruteforce(mesh) -> sp.csr_matrix:
    """Global K from SBFEM matrices computed in each cell's own frame."""
    rows, cols, vals = [], [], []
    cache = {}
    for c in range(mesh.n_cells):
        mask = int(mesh.mask[c])
        if mask not in cache:
            cache[mask] = sbfem.solve_cell(mask, 1.0, 1.0, mesh.nu, 1.0).K
        Ke = mesh.E[c] * mesh.h[c] * cache[mask]
        d = cell_dofs(mesh, c)
        rows.append(np.repeat(d, len(d)))
        cols.append(np.tile(d, len(d)))
        vals.append(Ke.ravel())
    n = mesh.n_dof
    return sp.csr_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                         shape=(n, n))


def _mask_groups(mesh):
    """Cells grouped by hanging-node mask: {mask: cell indices}."""
    masks = np.asarray(mesh.mask, np.int64)
    order = np.argsort(masks, kind="stable")
    uniq, first = np.unique(masks[order], return_index=True)
    bounds = list(first) + [len(order)]
    return {int(u): order[bounds[i]:bounds[i + 1]] for i, u in enumerate(uniq)}


def lumped_mass(mesh) -> np.ndarray:
    """Global diagonal mass M_diag (Algorithm 1, set-up): sum over cells of
    rho_e h_e^3 diag(T^T M_lump,p T), added in through each cell's DOFs."""
    M = np.zeros(mesh.n_dof)
    for mask, cells in _mask_groups(mesh).items():
        _, ML = cell_matrices_from_master(mask, 1.0, 1.0, 1.0, mesh.nu)
        slots = np.array(cube.present_slots(mask))
        nodes = mesh.slot_node[cells][:, slots].astype(np.int64)
        dofs = (3 * nodes[:, :, None] + np.arange(3)[None, None, :]).reshape(len(cells), -1)
        w = (mesh.rho[cells] * mesh.h[cells] ** 3)[:, None] * ML[None, :]
        np.add.at(M, dofs.ravel(), w.ravel())
    return M


def critical_dt(mesh) -> float:
    """min over cells of sqrt(rho/E) h dt_cr(master) (Eqs. tcr, tcr_scale)."""
    canon_tab, _ = cube.canonical_table()
    best = np.inf
    for mask, cells in _mask_groups(mesh).items():
        mc = sbfem.master_cell(int(canon_tab[mask]), mesh.nu)
        dtp = sbfem.critical_dt(mc.K, mc.M_lump)
        best = min(best, float(np.min(np.sqrt(mesh.rho[cells] / mesh.E[cells]) * mesh.h[cells])) * dtp)
    return float(best)


def pattern_tables(mesh):
    """Per-cell inputs of the explicit-K stepper in ``cdm``.

    Returns dict with: canonical pattern list, per-cell pattern index,
    scale s_e = E_e h_e, cell DOFs (own slot order), and for every cell node
    i the master node tmap[i] plus per-component (master component, sign),
    which together spell out K_cell = s_e T^T K_p T entry by entry.
    """
    canon_tab, op_tab = cube.canonical_table()
    masks = np.asarray(mesh.mask, np.int64)
    pats = sorted(set(int(canon_tab[m]) for m in np.unique(masks)))
    pidx = {p: i for i, p in enumerate(pats)}
    C = mesh.n_cells
    nper = np.array([len(cube.present_slots(int(m))) for m in range(4096)])[masks]
    ptr = np.zeros(C + 1, np.int64)
    np.cumsum(nper, out=ptr[1:])
    cell_pat = np.zeros(C, np.int64)
    tmap = np.zeros(ptr[-1], np.int64)
    nodes_all = np.zeros(ptr[-1], np.int64)
    comp = np.zeros((C, 3), np.int64)
    sign = np.zeros((C, 3), np.int64)
    for mask, cells in _mask_groups(mesh).items():
        canon, op = int(canon_tab[mask]), int(op_tab[mask])
        cell_pat[cells] = pidx[canon]
        Q = cube.all_ops()[op]
        pi = cube.slot_perm(op)
        cs = cube.present_slots(mask)
        ms = cube.present_slots(canon)
        mloc = {s: j for j, s in enumerate(ms)}
        tm = np.array([mloc[pi[s]] for s in cs], np.int64)
        # (T u)[3j + r] = sum_a Q[r, a] u[3i + a]  =>  cell component a maps to
        # master component r = the row where column a of Q is nonzero.
        cr = [int(np.nonzero(Q[:, a])[0][0]) for a in range(3)]
        comp[cells] = cr
        sign[cells] = [int(Q[cr[a], a]) for a in range(3)]
        idx = (ptr[cells][:, None] + np.arange(len(cs))[None, :]).ravel()
        tmap[idx] = np.tile(tm, len(cells))
        nodes = mesh.slot_node[cells][:, np.array(cs)]
        if (nodes < 0).any():
            raise ValueError("mesh slot table disagrees with the face-centre rule")
        nodes_all[idx] = nodes.ravel()
    dofs = (3 * nodes_all[:, None] + np.arange(3)[None, :]).ravel()
    Ks = [sbfem.master_cell(p, mesh.nu).K for p in pats]
    MLs = [sbfem.master_cell(p, mesh.nu).M_lump for p in pats]
    return {"patterns": pats, "cell_pat": cell_pat, "scale": mesh.E * mesh.h,
            "node_ptr": ptr, "dofs": dofs.astype(np.int64), "tmap": tmap,
            "comp": comp, "sign": sign, "K": Ks, "M_lump": MLs}
