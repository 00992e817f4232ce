"""Eigenfrequencies of the lumped-mass system K x = omega^2 M x (the cube
example of Sec. 5) from the library's Lanczos iteration (``sbx_lanczos``:
k steps on the GPU with full reorthogonalisation, K applied by the FP64
element-by-element kernel of the explicit step).  The k x k tridiagonal
matrix it returns is diagonalised here on the host (numpy; k is at most a
few hundred, against 3N unknowns on the GPU)."""
from __future__ import annotations

import numpy as np

from . import _lib as L


def ritz_frequencies(alpha: np.ndarray, beta: np.ndarray, rel_breakdown: float = 1e-12):
    """Ascending sqrt of the eigenvalues of the tridiagonal (alpha, beta),
    cut where the Krylov space was exhausted (beta ~ 0)."""
    k = len(alpha)
    scale = max(float(np.abs(alpha).max()), 1e-300)
    m = k
    for j in range(k - 1):
        if beta[j] <= rel_breakdown * scale:
            m = j + 1
            break
    T = np.diag(alpha[:m]) + np.diag(beta[:m - 1], 1) + np.diag(beta[:m - 1], -1)
    return np.sqrt(np.maximum(np.linalg.eigvalsh(T), 0.0))


def lanczos_frequencies(solver, k: int, seed: int = 0, v0=None) -> np.ndarray:
    """Ritz frequencies (rad / time unit) after k Lanczos steps from a seeded
    random start; each distinct eigenvalue appears once."""
    if v0 is None:
        v0 = np.random.default_rng(seed).standard_normal(solver.n_dof)
    alpha, beta = L.sbx_lanczos(solver.ctx, k, v0)
    return ritz_frequencies(alpha, beta)
