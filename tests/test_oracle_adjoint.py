"""Pin of the oracle's discrete adjoint: dJ/dE_e against central finite
differences of the misfit (FP64), and linearity checks."""
import numpy as np
import pytest

import octree_gen as og
from oracle import adjoint, cdm


@pytest.fixture(scope="module")
def case():
    m = og.tiny_refined(3, p=0.35)
    rng = np.random.default_rng(3)
    m.E = np.exp(0.3 * rng.standard_normal(m.n_cells))
    m.fixed_nodes = np.where(np.abs(m.node_xyz[:, 2]) < 1e-12)[0]
    top = og.nearest_node(m, (0.5, 0.5, 1.0))
    m.sources = [og.point_source(top, (0.1, 0.2, -1.0), og.ricker_t1_for_mesh(m, 3.0))]
    P = cdm.make_problem(m, dt_factor=0.5)
    n_steps = 120
    top_nodes = np.where(np.abs(m.node_xyz[:, 2] - 1.0) < 1e-12)[0][:6]
    rec = 3 * top_nodes + 2
    # data from perturbed moduli
    m2E = m.E * (1 + 0.1 * rng.standard_normal(m.n_cells))
    data_states = None
    E0 = m.E
    m.E = m2E
    P2 = cdm.make_problem(m, dt=P.dt)
    data_states = adjoint.forward_states(P2, n_steps)
    m.E = E0
    data = data_states[2:n_steps + 2][:, rec]
    return m, P, n_steps, rec, data


def test_adjoint_gradient_matches_central_differences(case):
    m, P, N, rec, data = case
    J, g = adjoint.gradient(P, N, rec, data)
    assert J > 0
    rng = np.random.default_rng(0)
    for c in rng.choice(m.n_cells, 6, replace=False):
        eps = 1e-6 * m.E[c]
        Ep = m.E.copy(); Ep[c] += eps
        Em = m.E.copy(); Em[c] -= eps
        fd = (adjoint.misfit_of_moduli(m, Ep, P.dt, N, rec, data)
              - adjoint.misfit_of_moduli(m, Em, P.dt, N, rec, data)) / (2 * eps)
        assert abs(g[c] - fd) <= 1e-6 * max(abs(fd), 1e-3 * np.abs(g).max()), (c, g[c], fd)


def test_adjoint_directional_derivative(case):
    # dJ along a random direction of all moduli, against central differences
    m, P, N, rec, data = case
    _, g = adjoint.gradient(P, N, rec, data)
    v = np.random.default_rng(1).standard_normal(m.n_cells) * m.E
    eps = 1e-7
    fd = (adjoint.misfit_of_moduli(m, m.E + eps * v, P.dt, N, rec, data)
          - adjoint.misfit_of_moduli(m, m.E - eps * v, P.dt, N, rec, data)) / (2 * eps)
    assert abs(g @ v - fd) <= 1e-6 * abs(fd)


def test_zero_residual_gives_zero_gradient(case):
    # data equal to the model's own response: J = 0 and dJ/dE = 0
    m, P, N, rec, _ = case
    S = adjoint.forward_states(P, N)
    J, g = adjoint.gradient(P, N, rec, S[2:N + 2][:, rec])
    assert J == 0.0 and np.abs(g).max() == 0.0


@pytest.mark.parametrize("every", [1, 7, 64, 120, 500])
@pytest.mark.parametrize("threads", [1, 3])
def test_checkpointed_adjoint_equals_store_all(case, every, threads):
    # the long-run form (pairs every k steps, segments stepped again, C
    # energy terms, threaded K) sums the same terms as the store-all form,
    # which the central differences above pin
    m, P, N, rec, data = case
    J0, g0 = adjoint.gradient(P, N, rec, data)
    J1, g1 = adjoint.gradient_checkpointed(P, N, rec, data, every=every, threads=threads)
    assert abs(J1 - J0) <= 1e-12 * J0
    assert np.abs(g1 - g0).max() <= 1e-11 * np.abs(g0).max()


def test_c_energy_terms_and_threaded_K(case):
    m, P, N, rec, data = case
    rng = np.random.default_rng(5)
    a = rng.standard_normal(P.n_dof)
    b = rng.standard_normal(P.n_dof)
    e_py = adjoint.cell_energy_terms(P, a, b)
    e_c = cdm.cell_energy(P, a, b, threads=2)
    assert np.abs(e_c - e_py).max() <= 1e-13 * np.abs(e_py).max()
    # a^T K b summed over cells equals a^T (K b)
    assert abs(np.sum(e_c * m.E) - a @ cdm.apply_K(P, b)) <= 1e-12 * np.abs(e_c * m.E).sum()
    assert np.abs(cdm.apply_K(P, b, threads=4) - cdm.apply_K(P, b)).max() <= \
        1e-13 * np.abs(cdm.apply_K(P, b)).max()


def test_traces_are_the_states_at_the_receivers(case):
    m, P, N, rec, data = case
    S = adjoint.forward_states(P, N)
    assert np.abs(adjoint.traces(P, N, rec, threads=2) - S[2:N + 2][:, rec]).max() <= \
        1e-13 * np.abs(S).max()
