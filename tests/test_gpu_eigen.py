"""GPU Lanczos (sbx_lanczos: K applied by the explicit step's FP64 force
kernel, full reorthogonalisation on the device) against the FP64 oracle's
dense eigen-solution of the same K and lumped M, on roller-supported cubes
(the paper's cube example): a refined cube with hanging nodes run to the
full Krylov space, a uniform 8^3 cube's lowest distinct frequencies, and a
64^3 cube timed and compared with the continuum frequency."""
import time

import numpy as np
import pytest

import octree_gen as og
from oracle import eigen as oeig
from paper_2103_09100_gb300 import Solver, _lib as L, build, eigen

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    build.build()
    L.load()


def distinct(w, rtol=1e-7):
    out = [w[0]]
    for x in w[1:]:
        if x > out[-1] * (1 + rtol):
            out.append(x)
    return np.array(out)


def test_refined_cube_full_krylov_space():
    m = og.cube_roller(4, refine_p=0.3)
    ref = oeig.frequencies(m)
    S = Solver.from_mesh(m, precision="fp64")
    nf = len(oeig.free_dofs(m))
    w = eigen.lanczos_frequencies(S, nf)
    want = distinct(ref)[:12]
    got = np.array([w[np.argmin(np.abs(w - x))] for x in want])
    e = np.abs(got - want) / want
    print("refined cube (%d free DOF): lowest 12 distinct frequencies, max rel error %.2e"
          % (nf, e.max()))
    assert e.max() < 1e-9


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_uniform_cube_lowest_frequencies(precision):
    m = og.cube_roller(8)
    ref = distinct(oeig.frequencies(m, 12))[:3]
    S = Solver.from_mesh(m, precision=precision)   # the mixed context still applies K in FP64
    w = distinct(eigen.lanczos_frequencies(S, 200))[:3]
    e = np.abs(w - ref) / ref
    print("uniform 8^3 cube (%s context): lowest distinct frequencies %s, rel error %.2e"
          % (precision, np.round(w / (np.pi / 8), 4), e.max()))
    assert e.max() < 1e-9


def test_large_cube_timing_and_continuum():
    import torch
    m = og.cube_roller(64)
    S = Solver.from_mesh(m, precision="fp64")
    k = 300
    v0 = np.random.default_rng(1).standard_normal(m.n_dof)
    L.sbx_lanczos(S.ctx, 4, v0)                      # warm-up
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    alpha, beta = L.sbx_lanczos(S.ctx, k, v0)
    dt = time.perf_counter() - t0
    w = eigen.ritz_frequencies(alpha, beta)
    ex = oeig.cube_frequencies(1000.0, 0.3, 1.0, 8.0, 1)[0]
    e = abs(w[0] - ex) / ex
    print("64^3 cube (%d DOF): %d Lanczos steps in %.3f s (%.2f ms per step), lowest frequency "
          "%.6f vs continuum %.6f (rel %.2e)" % (m.n_dof, k, dt, 1e3 * dt / k, w[0], ex, e))
    assert e < 2e-3
