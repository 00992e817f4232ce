"""Master-cell pattern library: classification and SBFEM pattern matrices.

Host-side set-up for the GPU solver (untimed, like the paper's initialisation
stage, Sec. 4.2).  Produces what ``set_patterns`` and ``mesh_upload`` take.

Classification (Sec. 3.2.2).  A cell's hanging-node pattern is its 12-bit
mask of present mid-edge nodes.  The 48 signed permutations Q act on it;
cells whose masks share an orbit share one master cell.  This library takes
the *largest* mask of each orbit as master.  ``sym`` follows the library's
op convention (see include/sbx.h): op = 8 * perm_index + sign_bits, with the
permutations of (0, 1, 2) in lexicographic order, and
u_master[r] = (-1)^{bit r} u_cell[perm[r]] node by node.

Pattern matrices (Sec. 2): the scaled boundary finite element of the unit
cube [0, 1]^3 with scaling centre at its middle.  The SBFE equation is solved
through the stable invariant subspace of the Hamiltonian coefficient matrix
(real Schur form with the left-half-plane block first) rather than explicit
eigenvectors; K = Q_q Q_u^-1 is the same matrix as Phi_q1 Phi_u1^-1 (Eq. K)
because both bases span the bounded-mode subspace.  The radial mass
integral of Sec. 2.2 becomes the Lyapunov equation
(S + 3/2 I)^T W + W (S + 3/2 I) = Q_u^T M0 Q_u with S the block's exponent
matrix, and M = Q_u^-T W Q_u^-1.  Lumping and the critical step follow
Sec. 3.3 and Eq. (tcr).
"""
from __future__ import annotations

import itertools
from functools import lru_cache

import numpy as np
import scipy.linalg as sla

# ------------------------------------------------------------ slot geometry
# Slot positions of the octree mesh format, on the unit cube [0, 1]^3.
def _slot_xyz():
    P = np.zeros((26, 3))
    for c in range(8):
        P[c] = [c & 1, (c >> 1) & 1, (c >> 2) & 1]
    for e in range(12):
        a = e // 4
        r = e % 4
        oth = [x for x in (0, 1, 2) if x != a]
        P[8 + e, a] = 0.5
        P[8 + e, oth[0]] = r & 1
        P[8 + e, oth[1]] = r >> 1
    for f in range(6):
        P[20 + f] = 0.5
        P[20 + f, f // 2] = f % 2
    return P


SLOT_XYZ = _slot_xyz()
_KEY = {tuple((2 * p).astype(int)): s for s, p in enumerate(SLOT_XYZ)}

# ------------------------------------------------------------------- ops
PERMS = list(itertools.permutations((0, 1, 2)))


def op_matrix(op: int) -> np.ndarray:
    perm = PERMS[op // 8]
    Q = np.zeros((3, 3))
    for r in range(3):
        Q[r, perm[r]] = -1.0 if (op >> r) & 1 else 1.0
    return Q


@lru_cache(maxsize=None)
def _slot_map(op: int) -> np.ndarray:
    Q = op_matrix(op)
    out = np.zeros(26, np.int64)
    for s in range(26):
        p = Q @ (SLOT_XYZ[s] - 0.5) + 0.5
        out[s] = _KEY[tuple(np.rint(2 * p).astype(int))]
    return out


@lru_cache(maxsize=None)
def _mask_images() -> np.ndarray:
    """img[op, mask] = mask carried by op."""
    masks = np.arange(4096)
    img = np.zeros((48, 4096), np.int64)
    for op in range(48):
        sm = _slot_map(op)
        for e in range(12):
            img[op] |= ((masks >> e) & 1) << (sm[8 + e] - 8)
    return img


@lru_cache(maxsize=None)
def classification_table():
    """(master mask, op) for every mask; master = largest mask of the orbit,
    op = smallest op number carrying the mask onto it."""
    img = _mask_images()
    master = img.max(0)
    op = np.argmax(img == master[None, :], axis=0)
    return master, op


# ------------------------------------------------------- node sets and faces
def present(mask: int) -> list[int]:
    """Present slots: corners, mask mid-edges, face centres of faces with
    1, 2-adjacent, 3 or 4 mid-edge nodes (the mesh format's rule)."""
    out = list(range(8))
    out += [8 + e for e in range(12) if mask >> e & 1]
    for f in range(6):
        mids = _face_ring(f)[1]
        on = [bool(mask >> (m - 8) & 1) for m in mids]
        if sum(on) >= 1 and not (sum(on) == 2 and on[0] == on[2]):
            out.append(20 + f)
    return sorted(out)


@lru_cache(maxsize=None)
def _face_ring(f: int):
    """Boundary slots of face f ordered by angle about its centre, and the
    four mid-edge slots in the same angular order."""
    a = f // 2
    ctr = SLOT_XYZ[20 + f]
    cand = [s for s in range(20) if abs(SLOT_XYZ[s, a] - ctr[a]) < 1e-12]
    u, v = [x for x in (0, 1, 2) if x != a]
    ang = {s: np.arctan2(SLOT_XYZ[s, v] - 0.5, SLOT_XYZ[s, u] - 0.5) for s in cand}
    ring = sorted(cand, key=lambda s: ang[s])
    mids = [s for s in ring if s >= 8]
    return ring, mids


def surface_mesh(mask: int) -> list[list[int]]:
    """Surface elements (Sec. 3.2.1): squares, 1 x 1/2 rectangles, 1/2 x 1/2
    squares or a triangle fan about the face centre."""
    elems = []
    for f in range(6):
        ring, mids = _face_ring(f)
        live = [s for s in ring if s < 8 or mask >> (s - 8) & 1]
        on = [bool(mask >> (m - 8) & 1) for m in mids]
        nh = sum(on)
        c = 20 + f
        if nh == 0:
            elems.append(live)
        elif nh == 4:
            for i in range(0, 8, 2):          # corners sit at even ring positions
                elems.append([live[i - 1], live[i], live[i + 1], c])
        elif nh == 2 and on[0] == on[2]:
            k0 = live.index([m for m, o in zip(mids, on) if o][0])
            rot = live[k0:] + live[:k0]       # starts at a live mid-edge node
            elems.append(rot[0:4])
            elems.append(rot[3:6] + rot[0:1])
        else:
            for i in range(len(live)):
                elems.append([live[i], live[(i + 1) % len(live)], c])
    return elems


# -------------------------------------------------------------- integration
_G3 = np.polynomial.legendre.leggauss(3)
# 6-point degree-4 triangle rule (Dunavant), area-normalised weights
_TA, _TB = 0.445948490915965, 0.091576213509771
_TW1, _TW2 = 0.223381589678011, 0.109951743655322
_TRI = np.array([[_TA, _TA], [1 - 2 * _TA, _TA], [_TA, 1 - 2 * _TA],
                 [_TB, _TB], [1 - 2 * _TB, _TB], [_TB, 1 - 2 * _TB]])
_TRIW = 0.5 * np.array([_TW1] * 3 + [_TW2] * 3)


def _rules(nn):
    if nn == 4:
        x, w = _G3
        return [(a, b, wa * wb) for a, wa in zip(x, w) for b, wb in zip(x, w)]
    return [(p[0], p[1], w) for p, w in zip(_TRI, _TRIW)]


def _shape(nn, r, s):
    if nn == 4:
        sr = np.array([-1, 1, 1, -1.0])
        ss = np.array([-1, -1, 1, 1.0])
        return (1 + sr * r) * (1 + ss * s) / 4, sr * (1 + ss * s) / 4, ss * (1 + sr * r) / 4
    return np.array([1 - r - s, r, s]), np.array([-1.0, 1, 0]), np.array([-1.0, 0, 1])


def _hooke(nu):
    lam = nu / ((1 + nu) * (1 - 2 * nu))
    mu = 1 / (2 * (1 + nu))
    D = np.diag([2 * mu] * 3 + [mu] * 3)
    D[:3, :3] += lam
    return D


# strain rows: xx yy zz yz xz xy ; column = derivative axis * 3 + component
_GRAD2VOIGT = np.zeros((6, 9))
for _row, pairs in enumerate([[(0, 0)], [(1, 1)], [(2, 2)], [(1, 2), (2, 1)],
                              [(0, 2), (2, 0)], [(0, 1), (1, 0)]]):
    for d, c in pairs:
        _GRAD2VOIGT[_row, 3 * d + c] = 1.0


def _coefficients(mask: int, nu: float):
    slots = present(mask)
    idx = {s: i for i, s in enumerate(slots)}
    m = 3 * len(slots)
    D = _hooke(nu)
    E0 = np.zeros((m, m)); E1 = np.zeros((m, m)); E2 = np.zeros((m, m)); M0 = np.zeros((m, m))
    for el in surface_mesh(mask):
        X = SLOT_XYZ[el] - 0.5
        nn = len(el)
        # outward orientation: (x_r x x_s) . x > 0 at the element centroid
        N, Nr, Ns = _shape(nn, 0.0 if nn == 4 else 1 / 3, 0.0 if nn == 4 else 1 / 3)
        if np.dot(np.cross(Nr @ X, Ns @ X), N @ X) < 0:
            el = el[::-1]
            X = X[::-1]
        dof = np.array([3 * idx[s] + c for s in el for c in range(3)])
        for r, s, w in _rules(nn):
            N, Nr, Ns = _shape(nn, r, s)
            J = np.array([N @ X, Nr @ X, Ns @ X])
            det = np.linalg.det(J)
            G = np.linalg.inv(J)          # rows: d/dx_i = sum_k G[i,k] d/dhat_k
            # B(k) maps nodal u to strains for the hat-derivative k
            def Bk(k, coef):
                out = np.zeros((6, 3 * nn))
                for a in range(nn):
                    grad = np.zeros((9, 3))
                    for i in range(3):
                        for c in range(3):
                            grad[3 * i + c, c] = G[i, k] * coef[a]
                    out[:, 3 * a:3 * a + 3] = _GRAD2VOIGT @ grad
                return out
            B1 = Bk(0, N)
            B2 = Bk(1, Nr) + Bk(2, Ns)
            ix = np.ix_(dof, dof)
            E0[ix] += w * det * B1.T @ D @ B1
            E1[ix] += w * det * B2.T @ D @ B1
            E2[ix] += w * det * B2.T @ D @ B2
            Nu = np.kron(N[None, :], np.eye(3))
            M0[ix] += w * det * Nu.T @ Nu
    return slots, E0, E1, E2, M0


@lru_cache(maxsize=None)
def master_matrices(mask: int, nu: float = 0.3):
    """(slots, K, lumped mass, dt_cr) of the unit master cell, E = rho = 1."""
    slots, E0, E1, E2, M0 = _coefficients(mask, nu)
    m = E0.shape[0]
    A = np.linalg.solve(E0, E1.T)              # E0^-1 E1^T
    Bm = np.linalg.inv(E0)
    Z = np.block([[A - 0.5 * np.eye(m), -Bm],
                  [E1 @ A - E2, -(E1 @ Bm) + 0.5 * np.eye(m)]])
    T, Qs, sdim = sla.schur(Z, output="real", sort="lhp")
    if sdim != m:
        raise RuntimeError("stable subspace has dimension %d, expected %d" % (sdim, m))
    Qu, Qq = Qs[:m, :m], Qs[m:, :m]
    K = np.linalg.solve(Qu.T, Qq.T).T
    K = 0.5 * (K + K.T)
    S = -T[:m, :m] - 0.5 * np.eye(m)           # displacement-exponent matrix
    m0 = Qu.T @ M0 @ Qu
    Aly = S + 1.5 * np.eye(m)
    W = sla.solve_sylvester(Aly.T, Aly, m0)
    Qi = np.linalg.inv(Qu)
    M = Qi.T @ W @ Qi
    M = 0.5 * (M + M.T)
    n = m // 3
    lump = np.einsum("idjd->id", M.reshape(n, 3, n, 3)).ravel()
    w2 = sla.eigh(K, np.diag(lump), eigvals_only=True)
    dt = 2.0 / np.sqrt(w2.max())
    return tuple(slots), K, lump, float(dt)


# ------------------------------------------------------------ mesh prep
def classify_mesh(slot_node: np.ndarray, mask: np.ndarray):
    """Per cell: master mask, op, and node ids in master-slot order.

    Returns (masters (sorted list), cell_pattern (index into masters),
    cell_sym (uint8), cell_ptr (int64), cell_nodes (int32)).
    """
    master_tab, op_tab = classification_table()
    mask = np.asarray(mask, np.int64)
    cm = master_tab[mask]
    cop = op_tab[mask]
    masters = sorted(set(cm.tolist()))
    pidx = {p: i for i, p in enumerate(masters)}
    cell_pattern = np.array([pidx[p] for p in cm.tolist()], np.int32)
    npat = np.array([len(present(p)) for p in masters], np.int64)
    counts = npat[cell_pattern]
    cell_ptr = np.zeros(len(mask) + 1, np.int64)
    np.cumsum(counts, out=cell_ptr[1:])
    cell_nodes = np.empty(cell_ptr[-1], np.int32)
    # group cells by (mask, op) and fill vectorised
    key = mask * 64 + cop
    for k in np.unique(key):
        sel = np.where(key == k)[0]
        mk, op = int(k // 64), int(k % 64)
        sm = _slot_map(op)
        inv = np.empty(26, np.int64)
        inv[sm] = np.arange(26)
        mslots = present(int(master_tab[mk]))
        cslots = inv[mslots]                     # cell slot for each master node
        nodes = slot_node[sel][:, cslots]
        if (nodes < 0).any():
            raise ValueError("cell node missing for its pattern")
        base = cell_ptr[sel]
        cell_nodes[(base[:, None] + np.arange(len(mslots))[None, :]).ravel()] = nodes.ravel()
    return masters, cell_pattern, cop.astype(np.uint8), cell_ptr, cell_nodes


def pattern_arrays(masters, nu=0.3):
    """n_nodes, packed K (row-major), packed lumped mass, dt_cr per master."""
    nn, Ks, Ms, dts = [], [], [], []
    for p in masters:
        slots, K, lump, dt = master_matrices(int(p), nu)
        nn.append(len(slots))
        Ks.append(K.ravel())
        Ms.append(lump)
        dts.append(dt)
    return (np.array(nn, np.int32), np.ascontiguousarray(np.concatenate(Ks)),
            np.ascontiguousarray(np.concatenate(Ms)), np.array(dts))
