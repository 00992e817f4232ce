"""FP64 discrete adjoint of the explicit step and the per-cell modulus gradient.

Part of the FP64 oracle (test infrastructure; see ``oracle/__init__``).

Forward (Eq. DnMdiag, undamped), from rest (U_0 = 0, Udot_0 = 0, so by
Eq. D0 U_-1 = W R_ext(0) / 2 does not depend on the moduli):
    U_{n+1} = 2 U_n - U_{n-1} - W (K(E) U_n - R_ext(t_n)),   W = dt^2 M^-1
with W = 0 on fixed DOFs.  Misfit at receiver DOFs r over n = 1..N:
    J = 1/2 sum_n sum_r (U_n[r] - d_n[r])^2.
Adjoint (lambda_n = total derivative of J with respect to U_n):
    lambda_n = g_n + (2 I - K W) lambda_{n+1} - lambda_{n+2},
    g_n = dJ/dU_n (partial),  lambda_{N+1} = lambda_{N+2} = 0,
using (W K)^T = K W (K symmetric, W diagonal).  K depends on E_e only
through K_e = E_e h_e T_e^T K_p T_e (Eq. KM_scale), hence
    dJ/dE_e = - sum_{n=0}^{N-1} (W lambda_{n+1})_e^T (K_e / E_e) U_{n,e}.
Every quantity here is plain FP64; the K applications use the oracle's
element-by-element sum.

``gradient`` keeps every state; ``gradient_checkpointed`` computes the same
sums for long runs, keeping the state pair (U_{s-1}, U_s) only at every k-th
step s and stepping each segment forward again, from its pair, just before
the reverse sweep needs it.  Both sum the same terms in the same order.
"""
from __future__ import annotations

import numpy as np

from . import assembly, cdm


def forward_states(P, n_steps):
    """All states U_{-1}, U_0, ..., U_N (rows), from rest."""
    u, up = cdm.initial_state(P)
    out = np.zeros((n_steps + 2, P.n_dof))
    out[0] = up
    out[1] = u
    for n in range(n_steps):
        u, up, _, _ = cdm.run(P, 1, u, up, n0=n)
        out[n + 2] = u
    return out


def misfit(states, rec, data):
    """J = 1/2 sum_{n=1..N} sum_r (U_n[r] - d_n[r])^2; data[n-1, r] = d_n[r]."""
    N = data.shape[0]
    r = states[2:N + 2][:, rec] - data
    return 0.5 * float(np.sum(r * r))


def cell_energy_terms(P, a, b):
    """Per cell e: a_e^T (K_e / E_e) b_e with K_e from the explicit
    pattern tables (same entries as the stepper uses)."""
    t = P.tables
    out = np.zeros(P.mesh.n_cells)
    Ks = t["K"]
    for c in range(P.mesh.n_cells):
        n0, n1 = t["node_ptr"][c], t["node_ptr"][c + 1]
        nn = n1 - n0
        dofs = t["dofs"][3 * n0:3 * n1]
        tm = t["tmap"][n0:n1]
        comp, sign = t["comp"][c], t["sign"][c]
        Kp = Ks[t["cell_pat"][c]]
        rows = (3 * tm[:, None] + comp[None, :]).ravel()
        sg = np.tile(sign, nn).astype(float)
        Ke = P.mesh.h[c] * sg[:, None] * Kp[np.ix_(rows, rows)] * sg[None, :]
        out[c] = a[dofs] @ Ke @ b[dofs]
    return out


def gradient(P, n_steps, rec, data):
    """(J, dJ/dE) by the discrete adjoint (requires alpha = 0)."""
    if P.alpha != 0.0:
        raise ValueError("the adjoint is written for the undamped recurrence")
    S = forward_states(P, n_steps)
    J = misfit(S, rec, data)
    W = P.dt2minv
    lam1 = np.zeros(P.n_dof)      # lambda_{n+1}
    lam2 = np.zeros(P.n_dof)      # lambda_{n+2}
    grad = np.zeros(P.mesh.n_cells)
    for n in range(n_steps, 0, -1):
        g = np.zeros(P.n_dof)
        np.add.at(g, rec, S[n + 1][rec] - data[n - 1])
        lam = g + 2.0 * lam1 - cdm.apply_K(P, W * lam1) - lam2
        # the pair (lambda_n, U_{n-1}) enters dJ/dE through U_n = ... - W K U_{n-1}
        grad -= cell_energy_terms(P, W * lam, S[n])      # S[n] = U_{n-1}
        lam2, lam1 = lam1, lam
    return J, grad


def misfit_of_moduli(mesh, E, dt, n_steps, rec, data, sources=None):
    """J(E) by a fresh forward run (for finite differences)."""
    E0 = mesh.E
    try:
        mesh.E = np.asarray(E, float)
        P = cdm.make_problem(mesh, dt=dt, sources=sources)
        return misfit(forward_states(P, n_steps), rec, data)
    finally:
        mesh.E = E0


def traces(P, n_steps, rec, threads=1):
    """U_n[rec] for n = 1..N (rows), forward from rest."""
    u, up = cdm.initial_state(P)
    _, _, tr, _ = cdm.run(P, n_steps, u, up, receivers=rec, threads=threads)
    return tr


def gradient_checkpointed(P, n_steps, rec, data, every=64, threads=1):
    """(J, dJ/dE) as ``gradient``, holding k + 2 states at a time (k = every).

    Forward: from rest, the misfit terms of U_1..U_N and the pairs
    (U_{s-1}, U_s) for s = 0, k, 2k, ...  Reverse, segment by segment from
    the last: U_{s0+1}..U_{s0+k} are stepped again from the pair at s0, then
    for n = s0+k down to s0+1
        lambda_n = g_n + 2 lambda_{n+1} - K W lambda_{n+1} - lambda_{n+2}
        dJ/dE   -= (W lambda_n)^T (K_e / E_e) U_{n-1}   (per cell).
    """
    if P.alpha != 0.0:
        raise ValueError("the adjoint is written for the undamped recurrence")
    rec = np.asarray(rec, np.int64)
    u, up = cdm.initial_state(P)
    pairs = {0: (up.copy(), u.copy())}
    J = 0.0
    for s0 in range(0, n_steps, every):
        k = min(every, n_steps - s0)
        u, up, tr, _ = cdm.run(P, k, u, up, n0=s0, receivers=rec, threads=threads)
        r = tr - data[s0:s0 + k]
        J += 0.5 * float(np.sum(r * r))
        pairs[s0 + k] = (up.copy(), u.copy())
    W = P.dt2minv
    everything = np.arange(P.n_dof, dtype=np.int64)
    lam1 = np.zeros(P.n_dof)
    lam2 = np.zeros(P.n_dof)
    grad = np.zeros(P.mesh.n_cells)
    for s0 in reversed(range(0, n_steps, every)):
        k = min(every, n_steps - s0)
        up, u = pairs[s0]
        # seg[j] = U_{s0 + j - 1}, j = 0..k+1
        _, _, later, _ = cdm.run(P, k, u, up, n0=s0, receivers=everything, threads=threads)
        seg = np.concatenate([up[None, :], u[None, :], later], axis=0)
        for n in range(s0 + k, s0, -1):
            Un, Unm1 = seg[n - s0 + 1], seg[n - s0]
            g = np.zeros(P.n_dof)
            np.add.at(g, rec, Un[rec] - data[n - 1])
            lam = g + 2.0 * lam1 - cdm.apply_K(P, W * lam1, threads=threads) - lam2
            grad -= cdm.cell_energy(P, W * lam, Unm1, threads=threads)
            lam2, lam1 = lam1, lam
    return J, grad
