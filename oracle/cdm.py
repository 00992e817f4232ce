"""Oracle time stepping: Algorithm 1 with Eqs. (D0), (DnMdiag), loads of Sec. 5.

Part of the FP64 oracle (test infrastructure; see ``oracle/__init__``).

``build()`` compiles ``cdm.c`` with gcc into ``oracle/_build/libcdm.so``.
``Problem`` gathers what the set-up stage of Algorithm 1 prepares: per-cell pattern,
scale s_e = E_e h_e, DOF lists, the transform tables, the global diagonal
mass, dt^2 M^-1 with zeros on fixed DOFs (reading: Dirichlet DOFs are held
at zero), and the point loads.  ``run`` steps the C solver.  ``run_sparse``
is a second, independent stepper on the brute-force global K.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
from dataclasses import dataclass

import numpy as np

from . import assembly

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "cdm.c")
_LIB = os.path.join(_HERE, "_build", "libcdm.so")
_lib = None

WAVELETS = {"ricker": 0, "triangle": 1, "sine_burst": 2}


def build(force: bool = False) -> str:
    os.makedirs(os.path.dirname(_LIB), exist_ok=True)
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + ".tmp%d" % os.getpid()
        subprocess.check_call(["gcc", "-O2", "-fopenmp", "-fPIC", "-shared", "-std=c99",
                               "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    if _lib is None:
        _lib = C.CDLL(build())
        _lib.oracle_load_amplitude.restype = C.c_double
        _lib.oracle_load_amplitude.argtypes = [C.c_int, C.c_double, C.c_double, C.c_double]
    return _lib


def _p(a, ct):
    return a.ctypes.data_as(C.POINTER(ct))


def load_amplitude(kind: str, t: float, t1: float, ncyc: float = 5.0) -> float:
    return _load().oracle_load_amplitude(WAVELETS[kind], t, t1, ncyc)


@dataclass
class Problem:
    mesh: object
    tables: dict
    M_diag: np.ndarray
    dt: float
    alpha: float
    dt2minv: np.ndarray
    fixed: np.ndarray
    load_dof: np.ndarray
    load_amp: np.ndarray
    load_wave: np.ndarray
    wave_kind: np.ndarray
    wave_t1: np.ndarray
    wave_ncyc: np.ndarray
    # flattened pattern matrices
    pat_m: np.ndarray
    pat_off: np.ndarray
    kp: np.ndarray

    @property
    def n_dof(self):
        return self.M_diag.shape[0]


def make_problem(mesh, dt=None, dt_factor=0.5, alpha=0.0, sources=None, rhs=0) -> Problem:
    """The set-up stage of Algorithm 1 for ``mesh``.  ``dt`` defaults to
    dt_factor * dt_cr (Eqs. tcr, tcr_scale).  Only sources of load case
    ``rhs`` are applied."""
    tab = assembly.pattern_tables(mesh)
    M = assembly.lumped_mass(mesh)
    if dt is None:
        dt = dt_factor * assembly.critical_dt(mesh)
    fixed = mesh.fixed_dofs()
    dt2minv = dt * dt / M
    dt2minv[fixed] = 0.0
    srcs = mesh.sources if sources is None else sources
    srcs = [s for s in srcs if s.get("rhs", 0) == rhs]
    ld, la, lw, wk, wt, wn = [], [], [], [], [], []
    for w, s in enumerate(srcs):
        wk.append(WAVELETS[s["wavelet"]]); wt.append(s["t1"]); wn.append(s.get("n_cycles", 5.0))
        for d in range(3):
            if s["dir"][d] != 0.0:
                ld.append(3 * s["node"] + d)
                la.append(s["dir"][d] * s["P0"])
                lw.append(w)
    pat_m = np.array([k.shape[0] for k in tab["K"]], np.int64)
    pat_off = np.concatenate([[0], np.cumsum(pat_m ** 2)[:-1]]).astype(np.int64)
    kp = np.concatenate([k.ravel() for k in tab["K"]])
    return Problem(mesh, tab, M, float(dt), float(alpha), dt2minv, fixed,
                   np.array(ld, np.int64), np.array(la, float), np.array(lw, np.int64),
                   np.array(wk, np.int64), np.array(wt, float), np.array(wn, float),
                   pat_m, pat_off, np.ascontiguousarray(kp))


def _mesh_args(P: Problem):
    t = P.tables
    keep = [P.pat_m, P.pat_off, P.kp, t["cell_pat"], np.ascontiguousarray(t["scale"], float),
            t["node_ptr"], t["dofs"], t["tmap"], np.ascontiguousarray(t["comp"].ravel()),
            np.ascontiguousarray(t["sign"].ravel())]
    args = [_p(keep[0], C.c_int64), _p(keep[1], C.c_int64), _p(keep[2], C.c_double),
            _p(keep[3], C.c_int64), _p(keep[4], C.c_double), _p(keep[5], C.c_int64),
            _p(keep[6], C.c_int64), _p(keep[7], C.c_int64), _p(keep[8], C.c_int64),
            _p(keep[9], C.c_int64)]
    return keep, args


def apply_K(P: Problem, u: np.ndarray, threads: int = 1) -> np.ndarray:
    """R_int = sum_e K_e u_e (Eq. Rinte); threads > 1 splits the cells over
    OpenMP threads (per-thread sums added in thread order)."""
    lib = _load()
    u = np.ascontiguousarray(u, float)
    f = np.zeros(P.n_dof)
    keep, args = _mesh_args(P)
    if threads > 1:
        rc = lib.oracle_apply_K_threads(C.c_int64(P.n_dof), C.c_int64(P.mesh.n_cells), *args,
                                        _p(u, C.c_double), _p(f, C.c_double), C.c_int(threads))
        if rc != 0:
            raise RuntimeError("oracle_apply_K_threads failed: %d" % rc)
    else:
        lib.oracle_apply_K(C.c_int64(P.n_dof), C.c_int64(P.mesh.n_cells), *args,
                           _p(u, C.c_double), _p(f, C.c_double))
    return f


def cell_energy(P: Problem, a: np.ndarray, b: np.ndarray, threads: int = 1) -> np.ndarray:
    """Per cell e: a_e^T (K_e / E_e) b_e, K_e / E_e = h_e T_e^T K_p T_e
    (Eq. KM_scale), built entry by entry in C."""
    lib = _load()
    a = np.ascontiguousarray(a, float)
    b = np.ascontiguousarray(b, float)
    h = np.ascontiguousarray(P.mesh.h, float)
    out = np.zeros(P.mesh.n_cells)
    keep, args = _mesh_args(P)
    args[4] = _p(h, C.c_double)
    lib.oracle_cell_energy(C.c_int64(P.n_dof), C.c_int64(P.mesh.n_cells), *args,
                           _p(a, C.c_double), _p(b, C.c_double), _p(out, C.c_double),
                           C.c_int(threads))
    return out


def external_force(P: Problem, n: int) -> np.ndarray:
    f = np.zeros(P.n_dof)
    t = n * P.dt
    for k in range(len(P.load_dof)):
        w = P.load_wave[k]
        kind = [k_ for k_, v in WAVELETS.items() if v == P.wave_kind[w]][0]
        f[P.load_dof[k]] += P.load_amp[k] * load_amplitude(kind, t, P.wave_t1[w], P.wave_ncyc[w])
    return f


def initial_state(P: Problem, u0=None, v0=None):
    """(U_0, U_-1) by Eq. (D0).  Reading: the starting acceleration is
    Udd_0 = M^-1 (R_ext(t=0) - K U_0 - alpha M Ud_0)."""
    n = P.n_dof
    u0 = np.zeros(n) if u0 is None else np.array(u0, float)
    v0 = np.zeros(n) if v0 is None else np.array(v0, float)
    u0[P.fixed] = 0.0
    v0[P.fixed] = 0.0
    r = external_force(P, 0) - apply_K(P, u0)
    acc = r / P.M_diag - P.alpha * v0
    acc[P.fixed] = 0.0
    um1 = u0 - P.dt * v0 + 0.5 * P.dt ** 2 * acc
    um1[P.fixed] = 0.0
    return u0, um1


def run(P: Problem, n_steps: int, u_c: np.ndarray, u_p: np.ndarray, n0: int = 0,
        receivers=None, threads: int = 1, want_force: bool = False):
    """Advance n_steps from (U_n0, U_n0-1).  Returns (U_N, U_N-1, rec, f_last)."""
    lib = _load()
    u_c = np.array(u_c, float, copy=True)
    u_p = np.array(u_p, float, copy=True)
    rec = np.zeros(0, np.int64) if receivers is None else np.asarray(receivers, np.int64)
    rec_out = np.zeros((n_steps, len(rec)))
    f_last = np.zeros(P.n_dof) if want_force else None
    keep, args = _mesh_args(P)
    rc = lib.oracle_cdm_run(
        C.c_int64(P.n_dof), C.c_int64(P.mesh.n_cells), *args,
        _p(P.dt2minv, C.c_double),
        C.c_int64(len(P.load_dof)), _p(P.load_dof, C.c_int64), _p(P.load_amp, C.c_double),
        _p(P.load_wave, C.c_int64), _p(P.wave_kind, C.c_int64), _p(P.wave_t1, C.c_double),
        _p(P.wave_ncyc, C.c_double),
        C.c_double(P.dt), C.c_double(P.alpha), C.c_int64(n0), C.c_int64(n_steps),
        _p(u_c, C.c_double), _p(u_p, C.c_double),
        C.c_int64(len(rec)), _p(rec, C.c_int64), _p(rec_out, C.c_double),
        _p(f_last, C.c_double) if want_force else None, C.c_int(threads))
    if rc != 0:
        raise RuntimeError("oracle_cdm_run failed: %d" % rc)
    return u_c, u_p, rec_out, f_last


def run_sparse(K, M_diag, dt, alpha, fixed, n_steps, u_c, u_p, fext=None, n0=0):
    """Independent stepper on an assembled sparse K (Eq. DnMdiag verbatim)."""
    dt2minv = dt * dt / M_diag
    dt2minv[fixed] = 0.0
    u_c = np.array(u_c, float)
    u_p = np.array(u_p, float)
    for s in range(n_steps):
        r = -(K @ u_c)
        if fext is not None:
            r = r + fext(n0 + s)
        u_n = (dt2minv * r + 2 * u_c - (1 - 0.5 * alpha * dt) * u_p) / (1 + 0.5 * alpha * dt)
        u_p, u_c = u_c, u_n
    return u_c, u_p


def line_load_forces(mesh, a, b, q, tol=1e-9):
    """Consistent nodal forces (magnitudes) of a uniform line load q along
    the segment [a, b]: every cell edge piece between two consecutive nodes
    of the edge that lies on the segment contributes q * length / 2 to each
    of its two nodes, each physical piece once.  Returns {node: force}."""
    from . import cube
    a = np.asarray(a, float)
    b = np.asarray(b, float)
    d = b - a
    L = float(np.linalg.norm(d))
    x = np.asarray(mesh.node_xyz, float)

    def on(pt):
        t = float((pt - a) @ d) / (L * L)
        return (np.linalg.norm(pt - a - t * d) <= tol * L) and -tol <= t <= 1 + tol

    ends = []   # the two corner slots of each edge: the mid-edge's position with
    for e in range(12):   # its coordinate along the edge set to -1 and +1
        p = cube.SLOT_POS[8 + e].copy()
        ax = e // 4
        p0, p1 = p.copy(), p.copy()
        p0[ax], p1[ax] = -1, 1
        ends.append((cube.pos_to_slot(p0), cube.pos_to_slot(p1)))
    pieces = set()
    for c in range(mesh.n_cells):
        for e in range(12):
            c0, c1 = ends[e]
            mid = 8 + e
            seq = [mesh.slot_node[c, c0]]
            if mesh.slot_node[c, mid] >= 0:
                seq.append(mesh.slot_node[c, mid])
            seq.append(mesh.slot_node[c, c1])
            for u, v in zip(seq[:-1], seq[1:]):
                if on(x[u]) and on(x[v]):
                    pieces.add((min(u, v), max(u, v)))
    out = {}
    for u, v in sorted(pieces):
        half = 0.5 * q * float(np.linalg.norm(x[u] - x[v]))
        out[u] = out.get(u, 0.0) + half
        out[v] = out.get(v, 0.0) + half
    return out
