"""Pins of the oracle's time stepping (Sec. 3.1, Algorithm 1, Sec. 5 loads)
against closed forms, an independent sparse stepper and invariants."""
import ctypes as C

import numpy as np
import pytest

import octree_gen as og
from oracle import assembly, cdm
from conftest import golden

G = golden("paper_values.json")


def _sdof_run(k, m, dt, alpha, u0, v0, n):
    """Drive the C stepper on a one-node 'mesh' whose K_p = k I3."""
    lib = cdm._load()
    i64 = lambda a: np.asarray(a, np.int64)
    pat_m, pat_off, kp = i64([3]), i64([0]), np.ascontiguousarray(k * np.eye(3).ravel())
    cell_pat, scale = i64([0]), np.array([1.0])
    node_ptr, dofs, tmap = i64([0, 1]), i64([0, 1, 2]), i64([0])
    comp, sign = i64([0, 1, 2]), i64([1, 1, 1])
    dt2minv = np.full(3, dt * dt / m)
    # Eq. (D0) with Udd_0 = -(k/m) u0 - alpha v0
    acc = -(k / m) * u0 - alpha * v0
    uc = np.full(3, float(u0))
    up = np.full(3, u0 - dt * v0 + 0.5 * dt * dt * acc)
    z = np.zeros(1, np.int64)
    hist = np.zeros((n, 1))
    rec = i64([0])
    P = lambda a, t: a.ctypes.data_as(C.POINTER(t))
    rc = lib.oracle_cdm_run(C.c_int64(3), C.c_int64(1), P(pat_m, C.c_int64), P(pat_off, C.c_int64),
                            P(kp, C.c_double), P(cell_pat, C.c_int64), P(scale, C.c_double),
                            P(node_ptr, C.c_int64), P(dofs, C.c_int64), P(tmap, C.c_int64),
                            P(comp, C.c_int64), P(sign, C.c_int64), P(dt2minv, C.c_double),
                            C.c_int64(0), P(z, C.c_int64), P(np.zeros(1), C.c_double),
                            P(z, C.c_int64), P(z, C.c_int64), P(np.ones(1), C.c_double),
                            P(np.ones(1), C.c_double), C.c_double(dt), C.c_double(alpha),
                            C.c_int64(0), C.c_int64(n), P(uc, C.c_double), P(up, C.c_double),
                            C.c_int64(1), P(rec, C.c_int64), P(hist, C.c_double), None, C.c_int(1))
    assert rc == 0
    return np.concatenate([[u0], hist[:, 0]])


def test_sdof_closed_form_cos_n_theta():
    # m u'' + k u = 0, u0 = 1, v0 = 0: CDM with the D0 start gives exactly
    # u_n = cos(n theta), cos(theta) = 1 - omega^2 dt^2 / 2
    k, m = 4.0, 1.0
    w = np.sqrt(k / m)
    for dt in [0.1, 0.5, 0.99 * 2 / w]:
        u = _sdof_run(k, m, dt, 0.0, 1.0, 0.0, 400)
        th = np.arccos(1 - 0.5 * (w * dt) ** 2)
        assert np.abs(u - np.cos(th * np.arange(401))).max() < 1e-11


def test_sdof_damped_two_root_recurrence():
    # with C = alpha M (Eq. DnM) the recurrence is
    # (1 + a dt/2) u_{n+1} - (2 - w^2 dt^2) u_n + (1 - a dt/2) u_{n-1} = 0
    k, m, alpha, dt = 9.0, 1.0, 0.7, 0.05
    w2 = k / m
    u = _sdof_run(k, m, dt, alpha, 1.0, 0.3, 300)
    r = np.roots([1 + 0.5 * alpha * dt, -(2 - w2 * dt * dt), 1 - 0.5 * alpha * dt])
    um1 = 1.0 - dt * 0.3 + 0.5 * dt * dt * (-w2 * 1.0 - alpha * 0.3)
    # u_n = A r1^n + B r2^n with u_0 = 1, u_-1 = um1
    Mx = np.array([[1, 1], [1 / r[0], 1 / r[1]]])
    A, B = np.linalg.solve(Mx, [1.0, um1])
    n = np.arange(301)
    exact = (A * r[0] ** n + B * r[1] ** n).real
    assert np.abs(u - exact).max() < 1e-10


def test_sdof_stability_limit():
    # Eq. (tcr): bounded for dt < 2/omega, exponential growth above
    k = 1.0
    ok = _sdof_run(k, 1.0, 1.99, 0.0, 1.0, 0.0, 2000)
    bad = _sdof_run(k, 1.0, 2.01, 0.0, 1.0, 0.0, 2000)
    assert np.abs(ok).max() < 20
    assert np.abs(bad).max() > 1e6


@pytest.mark.parametrize("alpha", [0.0, 0.8])
def test_rigid_motion_from_eq_d0_start(alpha):
    # A free mesh moving as a rigid translation c + t b: K annihilates it, so
    # every DOF follows the SDOF recurrence without stiffness,
    # (1 + a dt/2) u_{n+1} - 2 u_n + (1 - a dt/2) u_{n-1} = 0, from the
    # Eq. (D0) start u_-1 = c - dt b + dt^2/2 (-a b).  Undamped that is
    # exact linear motion u_n = c + n dt b; damped, u_n = A + B r^n with
    # r = (1 - a dt/2) / (1 + a dt/2).  Pins initial_state's velocity and
    # damping terms and their signs.
    m = og.tiny_refined(4)
    m.fixed_nodes = np.zeros(0, np.int64)
    m.sources = []
    P = cdm.make_problem(m, dt_factor=0.5, alpha=alpha)
    assert len(P.fixed) == 0
    c = np.array([0.3, -0.2, 0.5])
    b = np.array([1.0, 0.4, -0.7])
    nn = m.n_dof // 3
    u0, um1 = cdm.initial_state(P, np.tile(c, nn), np.tile(b, nn))
    n = 60
    uN, uNm1, _, _ = cdm.run(P, n, u0, um1)
    dt = P.dt
    if alpha == 0.0:
        exact_n, exact_nm1 = c + n * dt * b, c + (n - 1) * dt * b
    else:
        r = (1 - 0.5 * alpha * dt) / (1 + 0.5 * alpha * dt)
        cm1 = c - dt * b - 0.5 * dt * dt * alpha * b
        # A + B = c, A + B / r = cm1
        B = (c - cm1) / (1 - 1 / r)
        A = c - B
        exact_n, exact_nm1 = A + B * r ** n, A + B * r ** (n - 1)
    scale = np.abs(exact_n).max()
    assert np.abs(uN.reshape(-1, 3) - exact_n[None, :]).max() < 1e-10 * scale
    assert np.abs(uNm1.reshape(-1, 3) - exact_nm1[None, :]).max() < 1e-10 * scale


@pytest.fixture(scope="module")
def tiny_problem():
    m = og.tiny_refined(2)
    m.E = np.exp(0.3 * np.random.default_rng(2).standard_normal(m.n_cells))
    m.fixed_nodes = np.where(np.abs(m.node_xyz[:, 2]) < 1e-12)[0]
    top = og.nearest_node(m, (0.5, 0.5, 1.0))
    m.sources = [og.point_source(top, (0.3, 0.1, -1), og.ricker_t1_for_mesh(m, 4.0))]
    return cdm.make_problem(m, dt_factor=0.5)


def test_c_stepper_equals_sparse_stepper_with_load(tiny_problem):
    P = tiny_problem
    K = assembly.global_K_bruteforce(P.mesh)
    u0, um1 = cdm.initial_state(P)
    uc, up, _, _ = cdm.run(P, 300, u0, um1)
    vc, vp = cdm.run_sparse(K, P.M_diag, P.dt, 0.0, P.fixed, 300, u0, um1,
                            fext=lambda n: cdm.external_force(P, n))
    assert np.linalg.norm(uc - vc) < 1e-12 * np.linalg.norm(vc)
    assert np.abs(uc[P.fixed]).max() == 0.0


def test_discrete_energy_conserved(tiny_problem):
    # f = 0, alpha = 0: E_n = 1/2 |u_{n+1} - u_n|_M^2 / dt^2 + 1/2 u_{n+1}^T K u_n
    # is an exact invariant of the recurrence (up to round-off)
    P = tiny_problem
    K = assembly.global_K_bruteforce(P.mesh)
    Pz = cdm.make_problem(P.mesh, dt=P.dt, sources=[])
    rng = np.random.default_rng(0)
    u0 = rng.standard_normal(P.n_dof)
    u0[P.fixed] = 0
    uc, up = u0, u0.copy()
    energies = []
    for _ in range(20):
        nc, npv, _, _ = cdm.run(Pz, 25, uc, up)
        du = nc - npv
        energies.append(0.5 * du @ (P.M_diag * du) / P.dt ** 2 + 0.5 * nc @ (K @ npv))
        uc, up = nc, npv
    e = np.array(energies)
    assert np.abs(e - e[0]).max() < 1e-11 * abs(e[0])


def test_global_stability_limit(tiny_problem):
    # bounded just below 2/omega_max(global), blows up just above it
    P = tiny_problem
    K = assembly.global_K_bruteforce(P.mesh).toarray()
    free = np.setdiff1d(np.arange(P.n_dof), P.fixed)
    d = 1 / np.sqrt(P.M_diag[free])
    wmax = np.sqrt(np.linalg.eigvalsh(d[:, None] * K[np.ix_(free, free)] * d[None, :]).max())
    rng = np.random.default_rng(1)
    u0 = rng.standard_normal(P.n_dof)
    u0[P.fixed] = 0
    for fac, bounded in [(0.99, True), (1.02, False)]:
        Pz = cdm.make_problem(P.mesh, dt=fac * 2 / wmax, sources=[])
        uc, _, _, _ = cdm.run(Pz, 3000, u0, u0)
        grew = (not np.isfinite(uc).all()) or np.abs(uc).max() > 1e3 * np.abs(u0).max()
        assert grew != bounded


def test_openmp_split_matches_sequential():
    m = og.config_corner_cube()
    P = cdm.make_problem(m)
    u0, um1 = cdm.initial_state(P)
    a, _, _, _ = cdm.run(P, 200, u0, um1)
    b, _, _, _ = cdm.run(P, 200, u0, um1, threads=4)
    assert np.linalg.norm(a - b) < 1e-12 * np.linalg.norm(a)


# ------------------------------------------------------------------ loads
def _spectrum(kind, t1, ncyc=5.0, n=1 << 16, T=None):
    T = T or 40 * t1
    t = np.linspace(0, T, n, endpoint=False)
    p = np.array([cdm.load_amplitude(kind, ti, t1, ncyc) for ti in t])
    A = np.abs(np.fft.rfft(p)) * (T / n)
    f = np.fft.rfftfreq(n, T / n)
    return f, A, t, p


def test_ricker_shape_and_central_frequency():
    t1 = 0.8
    assert abs(cdm.load_amplitude("ricker", t1, t1) - 1.0) < 1e-15
    assert abs(cdm.load_amplitude("ricker", t1 + t1 / 5, t1)) < 1e-15
    f, A, _, _ = _spectrum("ricker", t1, n=1 << 14)
    fm = f[np.argmax(A)]
    want = G["ricker_fm_times_t1"]["value"] / t1          # Eq. (Ricker_fm)
    assert abs(fm - want) < 2 * (f[1] - f[0])
    # Eq. (Ricker_A): normalised amplitude spectrum shape
    x = f / want
    shape = (2 / np.sqrt(np.pi)) * x ** 2 * np.exp(-x ** 2)
    assert np.abs(A / A.max() - shape / shape.max()).max() < 1e-3
    # Sec. 5: f1 ~ 2.2 / t1 bounds ~95 % of the area of A(f)
    cum = np.cumsum(A) / A.sum()
    f1 = f[np.searchsorted(cum, G["ricker_f1_times_t1"]["energy_fraction"])]
    assert abs(f1 * t1 - G["ricker_f1_times_t1"]["value"]) < 0.1


def test_triangle_pulse_spectrum():
    t1 = 0.5
    assert cdm.load_amplitude("triangle", t1, t1) == 1.0
    assert cdm.load_amplitude("triangle", 2.5 * t1, t1) == 0.0
    f, A, _, _ = _spectrum("triangle", t1, n=1 << 14)
    shape = np.sinc(f * t1) ** 2                          # Eq. (Triangle_A)
    assert np.abs(A / A.max() - shape).max() < 1e-3
    cum = np.cumsum(shape) / shape.sum()
    f1 = f[np.searchsorted(cum, 0.95)]
    assert abs(f1 * t1 - G["triangle_f1_times_t1"]["value"]) < 0.1


def test_sine_burst_central_frequency():
    t1, n = 1.0, 5.0
    f, A, _, _ = _spectrum("sine_burst", t1, n, n=1 << 14)
    assert abs(f[np.argmax(A)] - n / t1) < 2 * (f[1] - f[0])   # f_m = n / t1
    assert cdm.load_amplitude("sine_burst", 1.2, t1, n) == 0.0
