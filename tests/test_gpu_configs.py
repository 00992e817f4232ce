"""Parity of the benchmark configurations at their full size and step count,
each against the FP64 oracle (errors by ``parity.rel``: the larger of the
relative L2 error and the element-wise error relative to max |u_ref|).

* cavity cube (1.02M cells, 3.44M DOF, lognormal E, Ricker at the top
  centre), 2000 steps from rest: the FP64 kernels on the oracle's master
  matrices (bar 1e-12 through step 1000, then 1e-15 per step), the FP64
  form through the product's own pattern library (bar 5e-12, derived in
  the test) and the mixed form with either kernel for the regular cells
  (bar 1e-5), checked every 500 steps;
* multi-point cube (200k cells), 64 load cases (random source nodes,
  directions and Ricker frequencies), FP32 contraction, 1000 steps: 8
  seeded cases against the oracle run case by case (bar 1e-5);
* receiver cube (110k cells), adjoint over 4000 steps with 256 receivers
  and a checkpoint every 64 steps: the GPU FP64 and FP32-contraction
  gradients dJ/dE (FP64 also on the oracle's master matrices) against the
  oracle's FP64 checkpointed adjoint, and the
  FP64 gradient against central differences (eps = 1e-6 E_e) on 20 seeded
  random cells.
"""
import os

import numpy as np
import pytest

import octree_gen as og
from oracle import adjoint as oadj, cdm
from paper_2103_09100_gb300 import Solver, _lib as L, build
from oracle_upload import oracle_context
from parity import rel, rel_l2, rel_max

pytestmark = pytest.mark.gpu

THREADS = os.cpu_count() or 1


@pytest.fixture(scope="module", autouse=True)
def _built():
    build.build()
    L.load()


class _Ctx:
    """A bare library context stepped like a Solver."""
    def __init__(self, ctx, dt, n_dof):
        self.ctx, self.dt, self.n_dof = ctx, dt, n_dof

    def initial(self):
        L.set_initial(self.ctx, None, None, self.dt)

    def step(self, n):
        L.step_n(self.ctx, n, self.dt)

    def field(self, which=L.SBX_U_N):
        return L.read_field(self.ctx, which, np.empty(self.n_dof))

    def close(self):
        L.sbx_destroy(self.ctx)


def test_cavity_cube_2000_steps_fp64_and_mixed():
    m = og.config_cavity_cube()
    P = cdm.make_problem(m)
    # FP64 kernels on the oracle's own master matrices: the same arithmetic
    # up to rounding: bar 1e-12 through step 1000; each step's FP64
    # rounding (a few units of 2^-52 in a different order on either side)
    # compounds linearly in the undamped recurrence, so later the bar is
    # 1e-15 per step (2e-12 at step 2000).  FP64 through the product's own pattern
    # library: its K_p agree with the oracle's to within 7e-15 of the
    # largest entry (all 144 masters; a few 1e-15 for the common ones).  A
    # relative stiffness difference d shifts every frequency by d / 2, and
    # the fastest modes turn by up to ~2 radians per step at dt = dt_cr / 2,
    # so after N steps the states may differ by ~N d = 2000 * 2.5e-15: bar
    # 5e-12.
    forms = {"fp64 (oracle matrices)": (_Ctx(oracle_context(m, P), P.dt, m.n_dof),
                                        lambda n: max(1e-12, 1e-15 * n)),
             "fp64": (Solver.from_mesh(m, precision="fp64", dt=P.dt), lambda n: 5e-12)}
    for name, kind in (("mixed walsh", L.SBX_MIXED_WALSH), ("mixed tensor", L.SBX_MIXED_TENSOR)):
        S = Solver.from_mesh(m, precision="mixed", dt=P.dt)
        L.sbx_set_mixed_kernel(S.ctx, kind)
        forms[name] = (S, lambda n: 1e-5)
    for S, _ in forms.values():
        S.initial()
    u, up = cdm.initial_state(P)
    done = 0
    for chunk in (500, 500, 500, 500):
        u, up, _, _ = cdm.run(P, chunk, u, up, n0=done, threads=THREADS)
        done += chunk
        assert np.linalg.norm(u) > 0
        for name, (S, bar) in forms.items():
            S.step(chunk)
            g = S.field(L.SBX_U_N)
            print("cavity cube, %s, step %d: rel L2 %.3e, element-wise %.3e (bar %.1e)"
                  % (name, done, rel_l2(g, u), rel_max(g, u), bar(done)))
            assert rel(g, u) < bar(done), (name, done)
    for name, (S, _) in forms.items():
        assert L.sbx_get_step(S.ctx) == 2000
        S.close()


def test_multi_point_64_cases_1000_steps():
    m = og.config_multi_point()
    B = 64
    n_steps = 1000
    P0 = cdm.make_problem(m, rhs=0)
    S = Solver.from_mesh(m, precision="fp32", n_rhs=B, dt=P0.dt)
    S.initial()
    S.step(n_steps)
    g = S.field(L.SBX_U_N).reshape(-1, B)
    S.close()
    cases = np.sort(np.random.default_rng(11).choice(B, 8, replace=False))
    worst = 0.0
    for b in cases:
        P = cdm.make_problem(m, dt=P0.dt, rhs=int(b))
        u, up = cdm.initial_state(P)
        u, _, _, _ = cdm.run(P, n_steps, u, up, threads=THREADS)
        e = rel(g[:, b], u)
        print("multi-point, case %d, %d steps: rel L2 %.3e, element-wise %.3e"
              % (b, n_steps, rel_l2(g[:, b], u), rel_max(g[:, b], u)))
        assert np.linalg.norm(u) > 0
        worst = max(worst, e)
    assert worst < 1e-5, worst


def _blob_moduli(m):
    """Moduli with a +10 % Gaussian blob under the source (the true model the
    observed traces come from)."""
    S = 2 ** (m.lmax - m.level.astype(np.int64))
    c = (m.anchor + 0.5 * S[:, None]) * m.h_finest
    blob = np.exp(-np.sum((c - np.array([0.5, 0.5, 0.7])) ** 2, 1) / (2 * 0.15 ** 2))
    return m.E * (1 + 0.1 * blob)


def test_receiver_cube_adjoint_4000_steps():
    m = og.config_receiver_cube()
    N, every = 4000, 64
    rec = 3 * np.array(m.meta["receivers"], np.int64) + 2
    assert len(rec) == 256
    P = cdm.make_problem(m)
    # observed traces: the oracle's forward run with the blob moduli
    E0 = m.E
    m.E = _blob_moduli(m)
    data = oadj.traces(cdm.make_problem(m, dt=P.dt), N, rec, threads=THREADS)
    m.E = E0
    J_ref, g_ref = oadj.gradient_checkpointed(P, N, rec, data, every=every, threads=THREADS)
    assert J_ref > 0

    # the FP64 adjoint kernels on the oracle's own master matrices
    O = oracle_context(m, P)
    L.set_initial(O, None, None, P.dt)
    go = np.empty(m.n_cells)
    Jo = L.sbx_adjoint(O, N, P.dt, rec, np.ascontiguousarray(data.ravel()), every, go)
    L.sbx_destroy(O)
    S64 = Solver.from_mesh(m, precision="fp64", dt=P.dt)
    S64.initial()
    J64, g64 = S64.adjoint(N, rec, data, ckpt_every=every)
    S32 = Solver.from_mesh(m, precision="fp32", dt=P.dt)
    S32.initial()
    J32, g32 = S32.adjoint(N, rec, data, ckpt_every=every)
    S32.close()
    print("receiver cube, %d steps: J oracle %.9e, FP64 (oracle matrices) %.9e, FP64 %.9e, "
          "FP32 %.9e" % (N, J_ref, Jo, J64, J32))
    for name, g in (("FP64 (oracle matrices)", go), ("FP64", g64), ("FP32", g32)):
        print("dJ/dE vs oracle, %s: rel L2 %.3e, element-wise %.3e"
              % (name, rel_l2(g, g_ref), rel_max(g, g_ref)))
    assert abs(Jo - J_ref) <= 1e-10 * J_ref
    assert rel(go, g_ref) < 1e-9
    # through the product's own pattern library, whose K_p differ from the
    # oracle's by up to 7e-15: the states drift apart by ~N * 2.5e-15 = 1e-11
    # over 4000 steps, and J, a sum of squared residuals ~10x smaller than
    # the states, by ~2 * 10 * 1e-11: bars 1e-8
    assert abs(J64 - J_ref) <= 1e-8 * J_ref
    assert rel(g64, g_ref) < 1e-8
    # FP32 contraction: a relative rounding of ~2^-24 per step, growing at
    # most linearly over 4000 steps (4000 * 6e-8 = 2.4e-4), bar 1e-3
    assert abs(J32 - J_ref) <= 1e-4 * J_ref
    assert rel(g32, g_ref) < 1e-3

    # central differences of the GPU FP64 misfit on 20 seeded random cells.
    # J is summed with FP64 atomics in a varying order, so each evaluation
    # carries a noise of ~1e-13 J; divided by 2 eps that floor is
    # 5e-8 J / E_e, below which a difference says nothing.
    def J_of(E):
        S64.set_modulus(E)
        S64.initial()
        J, _ = S64.adjoint(N, rec, data, ckpt_every=every)
        return J

    cells = np.random.default_rng(20).choice(m.n_cells, 20, replace=False)
    for c in cells:
        eps = 1e-6 * m.E[c]
        Ep = m.E.copy(); Ep[c] += eps
        Em = m.E.copy(); Em[c] -= eps
        fd = (J_of(Ep) - J_of(Em)) / (2 * eps)
        floor = 5e-8 * J64 / m.E[c]
        print("cell %d: adjoint %.9e, central difference %.9e (floor %.1e)" % (c, g64[c], fd, floor))
        assert abs(g64[c] - fd) <= 1e-4 * abs(fd) + floor, (c, g64[c], fd)
    S64.close()
