"""Scaled boundary finite element of one cubic octree cell, in FP64.

Part of the FP64 oracle (test infrastructure; see ``oracle/__init__``).

Follows Sec. 2 of the paper step by step:

1. The cell boundary is discretised into 4-node quadrilaterals and 3-node
   triangles (Sec. 2.1; the face patterns of Sec. 3.2.1 are read in
   ``cube.face_elements``).  The scaling centre O is the cell centre.
2. Boundary geometry x(eta, zeta) = N x (Eq. xyz_hat) and the boundary
   Jacobian J (Eq. J_bd).
3. The strain operator L = b1 d/dxi + (b2 d/deta + b3 d/dzeta) / xi (Eq. L)
   with B1 = b1 N^u, B2 = b2 N^u_,eta + b3 N^u_,zeta (Eq. B1B2).  The paper
   leaves b1, b2, b3 to the SBFEM monograph; they follow from the chain
   rule: with x^ = xi x(eta, zeta), [d/dx^, d/dy^, d/dz^]^T =
   J^-1 [d/dxi, d/deta / xi, d/dzeta / xi]^T, so b_k = sum_i L_i (J^-1)_{i,k}
   where L = L_1 d/dx + L_2 d/dy + L_3 d/dz.
4. E0, E1, E2 (Eq. E0E1E2) and M0^e by Gauss quadrature, assembled over the
   surface elements.  On the planar faces of a cube |J| is constant and the
   integrands are polynomials, so the rules used here are exact.
5. The SBFE equation (Eq. SBFE) with the internal force q (Eq. q_E0E1) is
   reduced to first order by X = [xi^0.5 u ; xi^-0.5 q], giving
   xi X_,xi = -Z X with
       Z = [[E0^-1 E1^T - I/2,        -E0^-1        ],
            [E1 E0^-1 E1^T - E2,   -E1 E0^-1 + I/2  ]].
   An eigenvector of Z with eigenvalue lam gives u = Phi_u xi^(-lam-1/2)
   (Eq. u_q_phixic).  The m modes with bounded displacement at the scaling
   centre (displacement exponent s = -lam - 1/2 with Re(s) > -1/2) form
   Phi_u1, Phi_q1, and K = Phi_q1 Phi_u1^-1 (Eq. K).
6. M0 = sum_e int N^u^T rho N^u |J|, m0 = Phi_u1^T M0 Phi_u1,
   m_ij = m0_ij / (s_i + s_j + 3), M = Phi_u1^-T m Phi_u1^-1 (Sec. 2.2).
   Reading: the exponents written lambda_i in the radial integral are the
   displacement exponents s_i (the integrand is xi^s_i xi^s_j xi^2).
7. Lumping (Sec. 3.3): for each node and direction d, sum the row entries
   of M that belong to direction d; cross-direction entries are dropped.
8. Element critical time step dt_cr = 2 / omega_max (Eq. tcr), with
   omega_max^2 the largest eigenvalue of the pencil (K, M_lump).
   Reading: the lumped mass is used, as it is the mass the solver steps with.

Node and DOF order of a cell: its present slots in increasing slot order;
DOF = 3 * local_node + direction (x, y, z).
"""
from __future__ import annotations

from dataclasses import dataclass
from functools import lru_cache

import numpy as np

from . import cube

# ------------------------------------------------------------ quadrature
_GL_PTS, _GL_WTS = np.polynomial.legendre.leggauss(4)


def quad_rule():
    """4x4 Gauss-Legendre on [-1, 1]^2 (exact to degree 7 per variable)."""
    pts, wts = [], []
    for i, a in enumerate(_GL_PTS):
        for j, b in enumerate(_GL_PTS):
            pts.append((a, b))
            wts.append(_GL_WTS[i] * _GL_WTS[j])
    return np.array(pts), np.array(wts)


def tri_rule():
    """Collapsed 4x4 Gauss rule on the triangle {eta, zeta >= 0, eta + zeta <= 1}.

    eta = (1 + a) / 2, zeta = (1 - eta)(1 + b) / 2, weight factor (1 - eta) / 4.
    Exact for polynomials of total degree <= 7.
    """
    pts, wts = [], []
    for i, a in enumerate(_GL_PTS):
        for j, b in enumerate(_GL_PTS):
            eta = 0.5 * (1.0 + a)
            zeta = 0.5 * (1.0 - eta) * (1.0 + b)
            pts.append((eta, zeta))
            wts.append(_GL_WTS[i] * _GL_WTS[j] * 0.25 * (1.0 - eta))
    return np.array(pts), np.array(wts)


def shape_functions(nn: int, eta: float, zeta: float):
    """N, dN/deta, dN/dzeta of the 4-node quadrilateral or 3-node triangle."""
    if nn == 4:
        ce = np.array([-1.0, 1.0, 1.0, -1.0])
        cz = np.array([-1.0, -1.0, 1.0, 1.0])
        N = 0.25 * (1 + ce * eta) * (1 + cz * zeta)
        dNe = 0.25 * ce * (1 + cz * zeta)
        dNz = 0.25 * cz * (1 + ce * eta)
        return N, dNe, dNz
    if nn == 3:
        N = np.array([1.0 - eta - zeta, eta, zeta])
        dNe = np.array([-1.0, 1.0, 0.0])
        dNz = np.array([-1.0, 0.0, 1.0])
        return N, dNe, dNz
    raise ValueError(nn)


# ------------------------------------------------------- elasticity operators
def elasticity_D(E: float, nu: float) -> np.ndarray:
    """Isotropic elasticity matrix, Voigt order (xx, yy, zz, yz, xz, xy),
    engineering shear strains."""
    c = E / ((1 + nu) * (1 - 2 * nu))
    D = np.zeros((6, 6))
    D[:3, :3] = c * nu
    for i in range(3):
        D[i, i] = c * (1 - nu)
        D[3 + i, 3 + i] = c * (1 - 2 * nu) / 2
    return D


def strain_L() -> list[np.ndarray]:
    """L_1, L_2, L_3 with eps = (L_1 d/dx + L_2 d/dy + L_3 d/dz) u."""
    L1 = np.zeros((6, 3))
    L2 = np.zeros((6, 3))
    L3 = np.zeros((6, 3))
    L1[0, 0] = 1; L1[4, 2] = 1; L1[5, 1] = 1   # eps_xx, gamma_xz, gamma_xy
    L2[1, 1] = 1; L2[3, 2] = 1; L2[5, 0] = 1   # eps_yy, gamma_yz, gamma_xy
    L3[2, 2] = 1; L3[3, 1] = 1; L3[4, 0] = 1   # eps_zz, gamma_yz, gamma_xz
    return [L1, L2, L3]


def _Nu(N):
    """N^u = [N_1 I3, N_2 I3, ...] (3 x 3n)."""
    nn = len(N)
    out = np.zeros((3, 3 * nn))
    for a in range(nn):
        out[:, 3 * a:3 * a + 3] = N[a] * np.eye(3)
    return out


def surface_element_matrices(X: np.ndarray, D: np.ndarray, rho: float):
    """E0^e, E1^e, E2^e, M0^e of one surface element with node coords X (nn x 3).

    X is ordered so that det J > 0 (scaling centre O at the origin).
    """
    nn = X.shape[0]
    pts, wts = quad_rule() if nn == 4 else tri_rule()
    L = strain_L()
    m = 3 * nn
    E0 = np.zeros((m, m)); E1 = np.zeros((m, m)); E2 = np.zeros((m, m)); M0 = np.zeros((m, m))
    for (eta, zeta), w in zip(pts, wts):
        N, dNe, dNz = shape_functions(nn, eta, zeta)
        J = np.vstack([N @ X, dNe @ X, dNz @ X])          # Eq. (J_bd)
        detJ = np.linalg.det(J)
        if detJ <= 0:
            raise ValueError("surface element oriented inwards")
        Ji = np.linalg.inv(J)
        b = [sum(L[i] * Ji[i, k] for i in range(3)) for k in range(3)]  # b1, b2, b3
        B1 = b[0] @ _Nu(N)                                  # Eq. (B1)
        B2 = b[1] @ _Nu(dNe) + b[2] @ _Nu(dNz)              # Eq. (B2)
        E0 += w * detJ * (B1.T @ D @ B1)
        E1 += w * detJ * (B2.T @ D @ B1)
        E2 += w * detJ * (B2.T @ D @ B2)
        Nu = _Nu(N)
        M0 += w * detJ * rho * (Nu.T @ Nu)
    return E0, E1, E2, M0


def cell_coefficients(mask: int, h: float = 1.0, E: float = 1.0, nu: float = 0.3,
                      rho: float = 1.0):
    """Assembled E0, E1, E2, M0 of the cell (edge length h, centre at 0)."""
    slots = cube.present_slots(mask)
    loc = {s: i for i, s in enumerate(slots)}
    m = 3 * len(slots)
    D = elasticity_D(E, nu)
    E0 = np.zeros((m, m)); E1 = np.zeros((m, m)); E2 = np.zeros((m, m)); M0 = np.zeros((m, m))
    for el in cube.face_elements(mask):
        X = cube.SLOT_POS[el].astype(float) * (h / 2.0)
        # orient so that the outward normal points away from O (det J > 0)
        N, dNe, dNz = shape_functions(len(el), 1 / 3 if len(el) == 3 else 0.0,
                                      1 / 3 if len(el) == 3 else 0.0)
        J = np.vstack([N @ X, dNe @ X, dNz @ X])
        if np.linalg.det(J) < 0:
            el = el[::-1]
            X = X[::-1]
        e0, e1, e2, m0 = surface_element_matrices(X, D, rho)
        dofs = np.concatenate([[3 * loc[s] + d for d in range(3)] for s in el])
        ix = np.ix_(dofs, dofs)
        E0[ix] += e0; E1[ix] += e1; E2[ix] += e2; M0[ix] += m0
    return slots, E0, E1, E2, M0


@dataclass
class CellMatrices:
    slots: list
    K: np.ndarray           # stiffness (Eq. K), symmetrised
    M: np.ndarray           # consistent mass (Sec. 2.2)
    M_lump: np.ndarray      # diagonal of the lumped mass (Sec. 3.3)
    s: np.ndarray           # displacement exponents of the bounded modes
    K_asym: float           # ||K - K^T|| / ||K|| before symmetrising
    K_imag: float           # max |Im K| / ||K|| before taking the real part


def solve_cell(mask: int, h: float = 1.0, E: float = 1.0, nu: float = 0.3,
               rho: float = 1.0) -> CellMatrices:
    """Stiffness, consistent mass and lumped mass of one cell (Sec. 2.2, 3.3)."""
    slots, E0, E1, E2, M0 = cell_coefficients(mask, h, E, nu, rho)
    m = E0.shape[0]
    E0i = np.linalg.inv(E0)
    I = np.eye(m)
    Z = np.block([[E0i @ E1.T - 0.5 * I, -E0i],
                  [E1 @ E0i @ E1.T - E2, -E1 @ E0i + 0.5 * I]])
    lam, V = np.linalg.eig(Z)
    order = np.argsort(lam.real)
    sel = order[:m]                       # Re(lam) < 0  <=>  Re(s) > -1/2
    if not (lam.real[sel].max() < 0 < lam.real[order[m:]].min()):
        raise ValueError("eigenvalues of Z do not split into bounded/unbounded halves")
    s = -lam[sel] - 0.5
    Phi_u = V[:m, sel]
    Phi_q = V[m:, sel]
    Phi_u_inv = np.linalg.inv(Phi_u)
    Kc = Phi_q @ Phi_u_inv                                  # Eq. (K)
    normK = np.linalg.norm(Kc)
    K_imag = float(np.abs(Kc.imag).max() / normK)
    K = Kc.real
    K_asym = float(np.linalg.norm(K - K.T) / np.linalg.norm(K))
    K = 0.5 * (K + K.T)
    m0 = Phi_u.T @ M0 @ Phi_u                               # m0 = Phi^T M0 Phi
    mm = m0 / (s[:, None] + s[None, :] + 3.0)               # radial integral
    Mc = Phi_u_inv.T @ mm @ Phi_u_inv                       # M = Phi^-T m Phi^-1
    M = Mc.real
    M = 0.5 * (M + M.T)
    return CellMatrices(slots, K, M, lump_mass(M), s, K_asym, K_imag)


def lump_mass(M: np.ndarray) -> np.ndarray:
    """Sec. 3.3: per node and direction, sum the same-direction row entries."""
    m = M.shape[0]
    out = np.zeros(m)
    for i in range(m):
        d = i % 3
        out[i] = sum(M[i, j] for j in range(d, m, 3))
    return out


def critical_dt(K: np.ndarray, M_lump: np.ndarray) -> float:
    """Eq. (tcr): dt_cr = 2 / omega_max of the element with its lumped mass."""
    d = 1.0 / np.sqrt(M_lump)
    w2 = np.linalg.eigvalsh(d[:, None] * K * d[None, :])
    return 2.0 / np.sqrt(w2.max())


@lru_cache(maxsize=None)
def master_cell(mask: int, nu: float = 0.3) -> CellMatrices:
    """Master element of a pattern: unit edge length, E = 1, rho = 1 (Sec. 3.2.3)."""
    return solve_cell(mask, 1.0, 1.0, nu, 1.0)
