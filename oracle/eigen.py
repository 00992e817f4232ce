"""Free vibration of the lumped-mass system: K x = omega^2 M_diag x on the
free DOFs (the cube example of Sec. 5: eigenfrequencies of a cube on roller
supports, computed with the same K and lumped M the explicit solver steps
with).  TEST INFRASTRUCTURE ONLY (see the package header).

* ``cube_frequencies`` -- the exact frequencies of the continuum cube
  [0, L]^3 with roller supports on all faces.  Separation of variables with
  u_x ~ sin(l pi x / L) cos(m pi y / L) cos(n pi z / L) (and cyclically)
  turns Navier's equation into the 3x3 problem
  (lambda + mu) k (k . a) + mu |k|^2 a = rho omega^2 a,  k = (pi / L)(l, m, n):
  one P branch omega = |k| v_P along k and two S branches omega = |k| v_S
  across it, with v_P^2 = E (1 - nu) / (rho (1 + nu) (1 - 2 nu)) and
  v_S^2 = E / (2 rho (1 + nu)) (the 3-D wave speeds of Eq. wavespeed; the
  paper's Eq. Cube_f writes the plane-stress speed for the first branch).
  An index equal to 0 removes the displacement component that carries the
  sine in that direction, so the polarisation a must have that component
  0: a wave vector with one zero index keeps P and one S branch, with two
  zero indices only P.
* ``frequencies`` -- the lowest discrete frequencies of a mesh: the global
  K assembled cell by cell (``assembly.global_K_bruteforce``), the lumped
  mass (``assembly.lumped_mass``), the fixed DOFs removed, then a dense
  symmetric-definite eigensolver (scipy.linalg.eigh) -- a library routine
  used as one step.
"""
from __future__ import annotations

import numpy as np
import scipy.linalg as sla

from . import assembly


def cube_frequencies(E: float, nu: float, rho: float, L: float, count: int, kmax: int = 6):
    """The `count` lowest exact frequencies (rad/s) with multiplicity."""
    vp = np.sqrt(E * (1 - nu) / (rho * (1 + nu) * (1 - 2 * nu)))
    vs = np.sqrt(E / (2 * rho * (1 + nu)))
    out = []
    for l in range(kmax + 1):
        for m in range(kmax + 1):
            for n in range(kmax + 1):
                idx = (l, m, n)
                nz = sum(1 for i in idx if i == 0)
                if nz == 3:
                    continue
                k = np.pi / L * np.sqrt(l * l + m * m + n * n)
                out.append(k * vp)                       # P, always allowed
                out.extend([k * vs] * (2 - nz))          # S: 2, 1 or 0 branches
    return np.sort(np.array(out))[:count]


def free_dofs(mesh) -> np.ndarray:
    mask = np.ones(mesh.n_dof, bool)
    mask[mesh.fixed_dofs()] = False
    return np.nonzero(mask)[0]


def frequencies(mesh, count: int | None = None) -> np.ndarray:
    """Ascending omega of K x = omega^2 M x on the free DOFs (all of them
    when count is None)."""
    K = assembly.global_K_bruteforce(mesh)
    M = assembly.lumped_mass(mesh)
    f = free_dofs(mesh)
    Kf = K[f][:, f].toarray()
    w2 = sla.eigh(Kf, np.diag(M[f]), eigvals_only=True)
    w = np.sqrt(np.maximum(w2, 0.0))
    return w if count is None else w[:count]
