"""Pins of the oracle's SBFEM cell matrices (Sec. 2, 3.2.3, 3.3) against
closed forms and invariants that do not come from the oracle itself."""
import numpy as np
import pytest

from oracle import cube, sbfem
from conftest import golden

G = golden("paper_values.json")
MASKS = [0, 1, 3, 5, 0x021, 0x0F0, 0xFFF, 0b101010101010, 0b110011001100, 2049]


def _nodes(mask, h=1.0):
    return cube.SLOT_POS[cube.present_slots(mask)].astype(float) * (h / 2.0)


def _linear_field(X, A, b=None):
    u = X @ A.T
    if b is not None:
        u = u + b[None, :]
    return u.ravel()


def _strain(A):
    e = 0.5 * (A + A.T)
    return np.array([e[0, 0], e[1, 1], e[2, 2], 2 * e[1, 2], 2 * e[0, 2], 2 * e[0, 1]])


def _D_closed(E, nu):
    # Lame form of isotropic Hooke's law: sigma = lam tr(eps) I + 2 mu eps
    lam = E * nu / ((1 + nu) * (1 - 2 * nu))
    mu = E / (2 * (1 + nu))
    D = np.zeros((6, 6))
    D[:3, :3] = lam
    D[np.arange(3), np.arange(3)] += 2 * mu
    D[np.arange(3, 6), np.arange(3, 6)] = mu
    return D


@pytest.mark.parametrize("mask", MASKS)
def test_K_symmetric_real_six_rigid_modes(mask):
    c = sbfem.master_cell(mask)
    assert c.K_asym < 1e-12 and c.K_imag < 1e-12
    ev = np.linalg.eigvalsh(c.K)
    tol = 1e-10 * ev.max()
    assert np.sum(np.abs(ev) < tol) == 6
    assert ev[6] > 1e-3 * ev.max() * 0.01


def test_all_144_patterns_sound():
    for p in cube.unique_patterns():
        c = sbfem.master_cell(p)
        assert c.K_asym < 1e-12 and c.K_imag < 1e-12, p
        ev = np.linalg.eigvalsh(c.K)
        assert np.sum(np.abs(ev) < 1e-10 * ev.max()) == 6, p
        assert (c.M_lump > 0).all(), p
        assert np.allclose([c.M_lump[d::3].sum() for d in range(3)], 1.0, atol=1e-12), p
        assert np.linalg.eigvalsh(c.M).min() > 0, p


@pytest.mark.parametrize("mask", MASKS)
@pytest.mark.parametrize("E,nu,h", [(1.0, 0.3, 1.0), (3.7, 0.2, 0.37), (1.0, 0.0, 2.0)])
def test_linear_fields_energy_is_exact(mask, E, nu, h):
    # For u = A x (+ b), the SBFEM solution is exact, so for any two linear
    # fields v^T K u = V eps(v)^T D eps(u) with V = h^3 (Sec. 2.2, patch test).
    c = sbfem.solve_cell(mask, h=h, E=E, nu=nu)
    X = _nodes(mask, h)
    rng = np.random.default_rng(mask)
    D = _D_closed(E, nu)
    for _ in range(4):
        A = rng.standard_normal((3, 3))
        B = rng.standard_normal((3, 3))
        u = _linear_field(X, A, rng.standard_normal(3))
        v = _linear_field(X, B, rng.standard_normal(3))
        lhs = v @ c.K @ u
        rhs = h ** 3 * _strain(B) @ D @ _strain(A)
        assert abs(lhs - rhs) <= 1e-11 * (abs(rhs) + E * h ** 3)


@pytest.mark.parametrize("mask", MASKS)
def test_linear_field_force_is_equilibrated(mask):
    # K u for u linear is a self-equilibrated nodal load: zero resultant and
    # zero resultant moment about the centre.
    c = sbfem.master_cell(mask)
    X = _nodes(mask)
    A = np.random.default_rng(7).standard_normal((3, 3))
    f = (c.K @ _linear_field(X, A)).reshape(-1, 3)
    assert np.abs(f.sum(0)).max() < 1e-12
    assert np.abs(np.cross(X, f).sum(0)).max() < 1e-12


@pytest.mark.parametrize("mask", MASKS[:5])
def test_scaling_law_K_and_M(mask):
    # Eq. (KM_scale): K ~ E h, M ~ rho h^3, computed from scratch at another size
    c1 = sbfem.solve_cell(mask, h=1.0, E=1.0, rho=1.0)
    c2 = sbfem.solve_cell(mask, h=0.3, E=2.5, rho=7.0)
    assert np.allclose(c2.K, 2.5 * 0.3 * c1.K, rtol=0, atol=1e-12 * np.abs(c2.K).max())
    assert np.allclose(c2.M, 7.0 * 0.3 ** 3 * c1.M, rtol=0, atol=1e-12 * np.abs(c2.M).max())


@pytest.mark.parametrize("mask", MASKS)
def test_consistent_mass_exact_for_linear_fields(mask):
    # u = b + A x on the cube [-h/2, h/2]^3: kinetic form
    # u^T M u = rho (|b|^2 h^3 + ||A||_F^2 h^5 / 12)  (the radial integral
    # 1/(s_i + s_j + 3) of Sec. 2.2 with s = 0 and 1)
    h, rho = 0.8, 2.0
    c = sbfem.solve_cell(mask, h=h, rho=rho)
    X = _nodes(mask, h)
    rng = np.random.default_rng(3)
    A = rng.standard_normal((3, 3))
    b = rng.standard_normal(3)
    u = _linear_field(X, A, b)
    exact = rho * (b @ b * h ** 3 + np.sum(A * A) * h ** 5 / 12.0)
    assert abs(u @ c.M @ u - exact) < 1e-12 * exact


def test_lumped_mass_8_node_cube_is_one_eighth():
    c = sbfem.master_cell(0)
    assert np.allclose(c.M_lump, 1.0 / 8.0, atol=1e-14)


@pytest.mark.parametrize("mask", MASKS)
def test_lumping_conserves_mass_per_direction(mask):
    # Sec. 3.3: the total mass of each direction is conserved
    c = sbfem.solve_cell(mask, h=0.5, rho=3.0)
    for d in range(3):
        assert abs(c.M_lump[d::3].sum() - 3.0 * 0.125) < 1e-13


@pytest.mark.parametrize("mask", MASKS)
def test_lumped_mass_first_moment_is_the_centroid(mask):
    # With the direction-wise row sums of Sec. 3.3, sum_i m_i,d x_i equals the
    # kinetic cross term of the constant and the linear field d, i.e.
    # rho * integral of x over the cell: rho h^3 (x_c + shift) for the cube
    # [-h/2, h/2]^3 moved by `shift`.  Catches lumped masses handed to the
    # wrong node, which the conservation check above does not.
    h, rho = 0.5, 3.0
    c = sbfem.solve_cell(mask, h=h, rho=rho)
    shift = np.array([0.3, -0.7, 1.1])
    X = _nodes(mask, h) + shift[None, :]
    for d in range(3):
        mom = c.M_lump[d::3] @ X
        assert np.abs(mom - rho * h ** 3 * shift).max() < 1e-13


def test_displacement_exponents():
    # three translations (s = 0) and nine linear fields (s = 1) are among the
    # bounded modes of every pattern
    for mask in MASKS:
        s = np.sort(sbfem.master_cell(mask).s.real)
        assert np.allclose(s[:3], 0, atol=1e-10)
        assert np.allclose(s[3:12], 1, atol=1e-9)
        assert s[12] > 1 + 1e-6


def test_transform_consistency_direct_vs_master():
    # Sec. 3.2.2: K of a cell computed directly in its own frame equals
    # T^T K_p T of its master cell
    from oracle import assembly
    rng = np.random.default_rng(11)
    for mask in list(rng.integers(1, 4096, 24)) + [1, 2, 4, 2048, 4095]:
        mask = int(mask)
        direct = sbfem.solve_cell(mask)
        canon, op, T = assembly.transform_matrix(mask)
        via = T.T @ sbfem.master_cell(canon).K @ T
        assert np.abs(direct.K - via).max() < 1e-12 * np.abs(direct.K).max()
        Mvia = np.diag(T.T @ np.diag(sbfem.master_cell(canon).M_lump) @ T)
        assert np.abs(direct.M_lump - Mvia).max() < 1e-13


def test_beam_time_steps_below_critical_soft():
    # Sec. 5.2 prints dt for three beam meshes (nu = 0, h = 0.0625, v_P = 100);
    # in units of h / v_P they are 0.9435, 0.5026, 0.5408.  Soft check: each is
    # below the element critical step of the uniform cell (the paper chose them
    # below the stability limit); the hanging-node values are only logged.
    g = G["beam_dt_ms"]
    ratios = [v * 1e-3 * g["vP_m_per_s"] / g["h_m"] for v in g["value"]]
    c0 = sbfem.solve_cell(0, nu=0.0)
    dt0 = sbfem.critical_dt(c0.K, c0.M_lump)
    assert ratios[0] <= dt0 + 1e-12
    hang = [sbfem.critical_dt(sbfem.solve_cell(m, nu=0.0).K, sbfem.solve_cell(m, nu=0.0).M_lump)
            for m in (1, 0xFFF)]
    print("dt_cr v/h: uniform %.4f, one hanging edge %.4f, all edges %.4f; paper %s"
          % (dt0, hang[0], hang[1], ["%.4f" % r for r in ratios]))
