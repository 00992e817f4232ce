"""Receiver time histories recorded on the GPU during step_n (one row per
step, U after that step at the chosen state-array entries) against the FP64
oracle's receiver output of the same run: bit-for-bit up to FP64 rounding in
the FP64 form (1e-12 of the largest recorded value), 1e-5 in the mixed form,
and per load case in the batched form."""
import numpy as np
import pytest

import octree_gen as og
from oracle import cdm
from paper_2103_09100_gb300 import Solver, _lib as L, build

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    build.build()
    L.load()


def _receivers(m, k=12, seed=4):
    rng = np.random.default_rng(seed)
    src = m.sources[0]["node"]
    nodes = np.unique(np.concatenate([[src], rng.choice(m.n_nodes, k, replace=False)]))
    return np.sort(np.concatenate([3 * nodes + 2, 3 * nodes[:4]]))


@pytest.mark.parametrize("precision, tol", [("fp64", 1e-12), ("mixed", 1e-5)])
def test_history_matches_oracle(precision, tol):
    m = og.config_corner_cube()
    P = cdm.make_problem(m)
    rec = _receivers(m)
    S = Solver.from_mesh(m, precision=precision, dt=P.dt)
    S.initial()
    S.set_receivers(rec, 100)
    for n in (40, 1, 24):      # a graph-captured run, a single step, more
        S.step(n)
    h = S.history()
    assert h.shape == (65, len(rec))
    u, up = cdm.initial_state(P)
    _, _, ref, _ = cdm.run(P, 65, u, up, receivers=rec)
    scale = np.abs(ref).max()
    assert scale > 0
    e = np.abs(h - ref).max() / scale
    print("corner cube %s: receiver history, 65 steps x %d receivers, max error %.3e"
          % (precision, len(rec), e))
    assert e < tol
    # the last row is the state read back
    assert np.array_equal(h[-1], S.field()[rec])


def test_history_capacity_and_off():
    m = og.config_corner_cube()
    S = Solver.from_mesh(m, precision="fp64")
    S.initial()
    rec = _receivers(m)
    S.set_receivers(rec, 10)
    S.step(25)
    h = S.history()
    assert h.shape == (10, len(rec))          # rows past the capacity are dropped
    S.set_receivers([], 1)                    # off
    S.step(3)
    with pytest.raises(L.SbxError):
        S.history()


def test_history_batched_cases():
    m = og.config_corner_cube()
    B = 32
    P = cdm.make_problem(m)
    rng = np.random.default_rng(9)
    u0 = 1e-3 * rng.standard_normal((m.n_dof, B))
    u0[P.fixed] = 0.0
    S = Solver.from_mesh(m, precision="fp32", n_rhs=B, dt=P.dt)
    S.initial(u0.ravel())
    dofs = _receivers(m)
    cases = np.array([0, 7, 31])
    rec = (dofs[:, None] * B + cases[None, :]).ravel()
    S.set_receivers(rec, 50)
    S.step(30)
    h = S.history().reshape(30, len(dofs), len(cases))
    worst = 0.0
    for j, b in enumerate(cases):
        P0 = cdm.make_problem(m, dt=P.dt)
        if b != 0:
            P0.load_dof = P0.load_dof[:0]   # the source drives load case 0 only
        u, up = cdm.initial_state(P0, u0[:, b])
        _, _, ref, _ = cdm.run(P0, 30, u, up, receivers=dofs)
        worst = max(worst, np.abs(h[:, :, j] - ref).max() / np.abs(ref).max())
    print("corner cube batched (B = %d): receiver history max error %.3e" % (B, worst))
    assert worst < 1e-5
