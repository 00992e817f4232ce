"""The launch-configuration autotuner (batched tile shapes per pattern
class; the mixed form's kernel choices): the tuned table is no slower than
the library's defaults as measured in the same run, applying it to a fresh
solver of the same mesh reproduces the configuration, it survives a save /
load round trip, and the tuned solver's results equal the oracle's with the
usual bars (a tile shape only reorders the reductions)."""
import os
import tempfile

import numpy as np
import pytest

import octree_gen as og
from oracle import cdm
from paper_2103_09100_gb300 import Solver, _lib as L, autotune, build
from parity import rel

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    build.build()
    L.load()


def _sources(m, B, seed):
    rng = np.random.default_rng(seed)
    free = np.setdiff1d(np.arange(m.n_nodes), m.fixed_nodes)
    t1 = og.ricker_t1_for_mesh(m, 10.0)
    m.sources = [og.point_source(int(free[rng.integers(len(free))]), rng.standard_normal(3),
                                 t1 / rng.uniform(0.5, 2.0), rhs=b) for b in range(B)]
    return m


def test_batched_autotune_table_reproduces():
    m = _sources(og.config_corner_cube(), 32, 3)
    P0 = cdm.make_problem(m, rhs=0)
    S = Solver.from_mesh(m, precision="fp32", n_rhs=32, dt=P0.dt)
    S.initial()
    table = autotune.tune(S, steps=5, repeats=3)
    print("batched autotune: default %.4f ms, tuned %.4f ms, params %s"
          % (table["force_ms_default"], table["force_ms_tuned"], table["params"]))
    assert table["force_ms_tuned"] <= table["force_ms_default"]
    assert set(table["params"]) == {w for w, _ in autotune.search_space(S)}
    with tempfile.TemporaryDirectory() as d:
        path = os.path.join(d, "table.json")
        autotune.save(table, path)
        back = autotune.load(path)
    assert back["params"] == table["params"] and back["mesh"] == table["mesh"]
    # a fresh solver of the same mesh takes the same configuration
    T = Solver.from_mesh(m, precision="fp32", n_rhs=32, dt=P0.dt)
    autotune.apply(T, back)
    for w, v in back["params"].items():
        assert L.sbx_get_launch(T.ctx, w) == v
    # and steps to the oracle's states
    T.initial()
    T.step(300)
    g = T.field(L.SBX_U_N).reshape(-1, 32)
    for b in (0, 21):
        P = cdm.make_problem(m, dt=P0.dt, rhs=b)
        u, up = cdm.initial_state(P)
        u, _, _, _ = cdm.run(P, 300, u, up, threads=8)
        assert rel(g[:, b], u) < 1e-5
    # another mesh is refused
    other = Solver.from_mesh(_sources(og.config_corner_cube(seed=5), 32, 3), precision="fp32",
                             n_rhs=32)
    with pytest.raises(ValueError):
        autotune.apply(other, back)


def test_mixed_autotune():
    m = og.config_receiver_cube()
    P = cdm.make_problem(m)
    S = Solver.from_mesh(m, precision="mixed", dt=P.dt)
    S.initial()
    table = autotune.tune(S, steps=10, repeats=3)
    print("mixed autotune: default %.4f ms, tuned %.4f ms, params %s"
          % (table["force_ms_default"], table["force_ms_tuned"], table["params"]))
    assert table["force_ms_tuned"] <= table["force_ms_default"]
    S.initial()
    S.step(100)
    u, up = cdm.initial_state(P)
    u, _, _, _ = cdm.run(P, 100, u, up, threads=16)
    assert rel(S.field(L.SBX_U_N), u) < 1e-5
