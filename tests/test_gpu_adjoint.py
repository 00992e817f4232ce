"""GPU discrete adjoint (sbx_adjoint) against the FP64 oracle adjoint and
against central finite differences of the misfit."""
import numpy as np
import pytest

import octree_gen as og
from oracle import adjoint as oadj, cdm
from paper_2103_09100_gb300 import Solver, _lib as L, build
from parity import rel

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    build.build()
    L.load()


@pytest.fixture(scope="module")
def tiny():
    m = og.tiny_refined(3, p=0.35)
    rng = np.random.default_rng(3)
    m.E = np.exp(0.3 * rng.standard_normal(m.n_cells))
    m.fixed_nodes = np.where(np.abs(m.node_xyz[:, 2]) < 1e-12)[0]
    top = og.nearest_node(m, (0.5, 0.5, 1.0))
    m.sources = [og.point_source(top, (0.1, 0.2, -1.0), og.ricker_t1_for_mesh(m, 3.0))]
    P = cdm.make_problem(m)
    N = 150
    top_nodes = np.where(np.abs(m.node_xyz[:, 2] - 1.0) < 1e-12)[0][:8]
    rec = 3 * top_nodes + 2
    E0 = m.E
    m.E = E0 * (1 + 0.1 * rng.standard_normal(m.n_cells))
    data = oadj.forward_states(cdm.make_problem(m, dt=P.dt), N)[2:N + 2][:, rec]
    m.E = E0
    return m, P, N, rec, data


def test_adjoint_matches_oracle_fp64(tiny):
    m, P, N, rec, data = tiny
    J0, g0 = oadj.gradient(P, N, rec, data)
    S = Solver.from_mesh(m, precision="fp64", dt=P.dt)
    S.initial()
    J, g = S.adjoint(N, rec, data, ckpt_every=16)
    assert abs(J - J0) <= 1e-10 * J0
    assert rel(g, g0) <= 1e-9


@pytest.mark.parametrize("k", [1, 7, 150, 1000])
def test_checkpoint_interval_does_not_change_the_result(tiny, k):
    m, P, N, rec, data = tiny
    S = Solver.from_mesh(m, precision="fp64", dt=P.dt)
    S.initial()
    J1, g1 = S.adjoint(N, rec, data, ckpt_every=16)
    S.initial()
    J2, g2 = S.adjoint(N, rec, data, ckpt_every=k)
    assert abs(J2 - J1) <= 1e-12 * J1
    assert rel(g2, g1) <= 1e-12
    # the state is back at rest afterwards
    assert np.abs(S.field(L.SBX_U_N)).max() == 0.0


def test_adjoint_central_differences_gpu(tiny):
    m, P, N, rec, data = tiny
    S = Solver.from_mesh(m, precision="fp64", dt=P.dt)
    S.initial()
    _, g = S.adjoint(N, rec, data)

    def J_of(E):
        S.set_modulus(E)
        S.initial()
        J, _ = S.adjoint(N, rec, data, ckpt_every=N)
        return J

    for c in np.random.default_rng(1).choice(m.n_cells, 5, replace=False):
        eps = 1e-6 * m.E[c]
        Ep = m.E.copy(); Ep[c] += eps
        Em = m.E.copy(); Em[c] -= eps
        fd = (J_of(Ep) - J_of(Em)) / (2 * eps)
        assert abs(g[c] - fd) <= 1e-6 * max(abs(fd), 1e-3 * np.abs(g).max()), (c, g[c], fd)


def test_autograd_function(tiny):
    torch = pytest.importorskip("torch")
    from paper_2103_09100_gb300 import adjoint as gadj
    m, P, N, rec, data = tiny
    S = Solver.from_mesh(m, precision="fp64", dt=P.dt)
    E = torch.tensor(m.E, dtype=torch.float64, requires_grad=True)
    J = gadj.misfit(E, S, N, rec, data, ckpt_every=32)
    (2.0 * J).backward()
    _, g0 = oadj.gradient(P, N, rec, data)
    assert rel(E.grad.numpy(), 2 * g0) <= 1e-9
